"""The paper's literal QP iteration: OSQP's ADMM on the full KKT system.

Paper: Sec. III-B, Eq. (kkt_system), Eqs. (ldl), (backsolve_1)-(backsolve_2)
and Alg. 1 (f_init, one factorisation, then N_QP times a solve and the ADMM
update f_ADMM); the update steps are OSQP's (Stellato et al. 2020, Sec. 3,
their Algorithm 1), to which the paper defers after Eq. (backsolve_2).

The horizon QP of qp.py in OSQP's form

    minimise 1/2 x^T P x + q^T x   subject to   l <= A x <= u

with x the stacked horizon z = [u_0, x_1, u_1, ..., u_{N-1}, x_N] and A the
dynamics rows (l = u = e) stacked over the stage inequality rows (C, lo, hi).
Rows free on both sides never bind and are left out.  Step size per row:
rho_eq = 1e3 rho on the rows with l = u (the dynamics and the wrench of a
swing foot), rho on every other row.

One iteration, from (x, z, y) (rho a diagonal matrix):

    [[P + sigma I, A^T], [A, -rho^-1]] [x~; nu] = [sigma x - q; z - rho^-1 y]
    z~  = z + rho^-1 (nu - y)
    x+  = alpha x~ + (1 - alpha) x
    zr  = alpha z~ + (1 - alpha) z
    z+  = clip(zr + rho^-1 y, l, u)
    y+  = y + rho (zr - z+)

The KKT matrix is factored once per solve (rho fixed, as in the paper's fixed
N_QP mode) by a dense LU factorisation (scipy) and every iteration reuses it.
Starting point (f_init, Alg. 1): x^0 = the current base pose and the nominal
joint angles repeated over the horizon, every other entry zero; z^0 = the
projection of A x^0 onto [l, u]; y^0 = 0.

Scaling (f_Ruiz, Alg. 1): OSQP's modified Ruiz equilibration (Stellato et al.
2020, Sec. 5.1).  Each of its iterations divides every column of the KKT
matrix [[P, A^T], [A, 0]] by the square root of its inf-norm (variables:
D, rows: E; norms below 1e-4 count as 1, above 1e4 as 1e4), then scales the
cost by c = 1 / max(mean of the columns' inf-norms of P, |q|_inf) (same
limits).  The scaled problem is (c D P D, c D q, E A D, E l, E u); the ADMM
runs on it from the scaled start (D^-1 x^0, E z^0, 0) and its iterate maps
back as x = D x_s, z = E^-1 z_s, y = E y_s / c.

Oracle code: test infrastructure only.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from . import qp as qpmod
from . import torque

RHO_EQ_FACTOR = 1e3


@dataclass
class LiteralQP:
    P: np.ndarray
    q: np.ndarray
    A: np.ndarray
    l: np.ndarray
    u: np.ndarray
    rho: np.ndarray      # per-row step size
    n_dyn: int           # the first n_dyn rows of A are the dynamics


def literal_form(qp, rho: float = 0.1) -> LiteralQP:
    """OSQP data (P, q, A, l, u, rho per row) of a DenseQP."""
    keep = np.isfinite(qp.lo) | np.isfinite(qp.hi)
    C, lo, hi = qp.C[keep], qp.lo[keep], qp.hi[keep]
    A = np.vstack([qp.E, C])
    l = np.concatenate([qp.e, lo])
    u = np.concatenate([qp.e, hi])
    rv = np.where(l == u, RHO_EQ_FACTOR * rho, rho)
    return LiteralQP(qp.P, qp.q, A, l, u, rv, qp.E.shape[0])


def start_point(lq: LiteralQP, qp, x0, q_nom):
    """(x^0, z^0, y^0): f_init's z_init (every x_k, k >= 1, is the current
    base position and orientation with the nominal joints q_nom; velocities,
    wrenches and joint rates zero), its row values projected onto [l, u],
    zero multipliers."""
    x = np.zeros(60 * qp.N)
    xk = np.zeros(30)
    xk[0:6] = np.asarray(x0, float)[0:6]
    xk[12:30] = q_nom
    for k in range(1, qp.N + 1):
        x[60 * (k - 1) + 30:60 * (k - 1) + 60] = xk
    return x, np.clip(lq.A @ x, lq.l, lq.u), np.zeros(len(lq.l))


def _limit(v, lo=1e-4, hi=1e4):
    v = np.asarray(v, dtype=float)
    return np.where(v < lo, 1.0, np.minimum(v, hi))


def ruiz(lq: LiteralQP, iters: int = 10):
    """(scaled LiteralQP, D, E, c) after `iters` equilibration iterations."""
    P, q, A = lq.P.copy(), lq.q.copy(), lq.A.copy()
    n, m = P.shape[0], A.shape[0]
    D, E, c = np.ones(n), np.ones(m), 1.0
    for _ in range(iters):
        col = np.maximum(np.abs(P).max(axis=0), np.abs(A).max(axis=0))
        row = np.abs(A).max(axis=1)
        dt = 1.0 / np.sqrt(_limit(col))
        et = 1.0 / np.sqrt(_limit(row))
        P = dt[:, None] * P * dt[None, :]
        q = dt * q
        A = et[:, None] * A * dt[None, :]
        D, E = D * dt, E * et
        g = 1.0 / float(_limit(max(np.abs(P).max(axis=0).mean(), np.abs(q).max())))
        P, q, c = g * P, g * q, g * c
    return LiteralQP(P, q, A, E * lq.l, E * lq.u, lq.rho, lq.n_dyn), D, E, c


def kkt_matrix(lq: LiteralQP, sigma: float) -> np.ndarray:
    """A_K of Eq. (kkt_system) with a per-row rho."""
    n, m = lq.P.shape[0], lq.A.shape[0]
    K = np.zeros((n + m, n + m))
    K[:n, :n] = lq.P + sigma * np.eye(n)
    K[:n, n:] = lq.A.T
    K[n:, :n] = lq.A
    K[n:, n:] = -np.diag(1.0 / lq.rho)
    return K


def iterate(lq: LiteralQP, x, z, y, iters: int, *, sigma: float = 1e-6, alpha: float = 1.6,
            lu=None, trace=None):
    """`iters` OSQP iterations from (x, z, y); returns (x, z, y).  trace, if a
    list, receives (x~, z~, x, z, y) of every iteration."""
    n = lq.P.shape[0]
    if lu is None:
        lu = sla.lu_factor(kkt_matrix(lq, sigma))
    rho = lq.rho
    for _ in range(iters):
        rhs = np.concatenate([sigma * x - lq.q, z - y / rho])
        sol = sla.lu_solve(lu, rhs)
        xt, nu = sol[:n], sol[n:]
        zt = z + (nu - y) / rho
        x = alpha * xt + (1.0 - alpha) * x
        zr = alpha * zt + (1.0 - alpha) * z
        zn = np.clip(zr + y / rho, lq.l, lq.u)
        y = y + rho * (zr - zn)
        z = zn
        if trace is not None:
            trace.append((xt, zt, x, z, y))
    return x, z, y


def residuals(lq: LiteralQP, x, z, y):
    """OSQP's primal and dual residuals (inf-norms) and their scales."""
    Ax = lq.A @ x
    Px = lq.P @ x
    Aty = lq.A.T @ y
    rp = np.max(np.abs(Ax - z)) if len(z) else 0.0
    rd = np.max(np.abs(Px + lq.q + Aty))
    sp = max(np.max(np.abs(Ax)), np.max(np.abs(z)))
    sd = max(np.max(np.abs(Px)), np.max(np.abs(Aty)), np.max(np.abs(lq.q)))
    return rp, rd, sp, sd


def solve_until(lq: LiteralQP, x, z, y, *, eps_abs=1e-5, eps_rel=1e-5, max_iter=4000, check_every=10,
                sigma=1e-6, alpha=1.6, scaling=0):
    """Iterate until OSQP's stopping test (mixed absolute / relative form, on
    the unscaled iterate) holds at a check, or max_iter; with `scaling` Ruiz
    iterations the ADMM runs on the scaled problem.  Returns the unscaled
    (x, z, y, iterations)."""
    if scaling:
        sq, D, E, c = ruiz(lq, scaling)
        xs, zs, ys = x / D, E * z, c * y / E
    else:
        sq, D, E, c = lq, np.ones(len(x)), np.ones(len(z)), 1.0
        xs, zs, ys = x, z, y
    lu = sla.lu_factor(kkt_matrix(sq, sigma))
    it = 0
    while it < max_iter:
        step = min(check_every, max_iter - it)
        xs, zs, ys = iterate(sq, xs, zs, ys, step, sigma=sigma, alpha=alpha, lu=lu)
        it += step
        rp, rd, sp, sd = residuals(lq, D * xs, zs / E, E * ys / c)
        if rp <= eps_abs + eps_rel * sp and rd <= eps_abs + eps_rel * sd:
            break
    return D * xs, zs / E, E * ys / c, it


def literal_agent(m: dict, x0, cmd, phase, qd_meas, iters: int, *, rho: float = 0.1, sigma: float = 1e-6,
                  alpha: float = 1.6, scaling: int = 0, kin=None):
    """Alg. 1 for one agent with a fixed N_QP = iters: f_init, f_param, the
    KKT system, `scaling` Ruiz iterations (f_Ruiz), one factorisation, iters
    OSQP iterations, the torque map of the last iterate (line search
    alpha = 1).  kin: the kinematic rows' parameters (qp.agent_qp), or None."""
    x0 = np.asarray(x0, float)
    qp, ex = qpmod.agent_qp(m, x0, cmd, phase, kin=kin)
    lq = literal_form(qp, rho)
    x, z, y = start_point(lq, qp, x0, np.asarray(m["q_nom"], float))
    if scaling:
        sq, D, E, c = ruiz(lq, scaling)
        xs, zs, ys = iterate(sq, x / D, E * z, np.zeros_like(y), iters, sigma=sigma, alpha=alpha)
        x, z, y = D * xs, zs / E, E * ys / c
    else:
        x, z, y = iterate(lq, x, z, y, iters, sigma=sigma, alpha=alpha)
    N = qp.N
    u = np.stack([qp.u(x, k) for k in range(N)])
    xs = np.vstack([x0[None, :]] + [qp.x(x, k)[None, :] for k in range(1, N + 1)])
    tau, q_set, qd_set = torque.torque_map(m, x0, qd_meas, u[0], u[1], x1=xs[1])
    return dict(tau=tau, q_set=q_set, qd_set=qd_set, x=xs, u=u, z=z, y=y, qp=qp, lq=lq)
