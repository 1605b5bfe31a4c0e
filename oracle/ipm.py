"""Dense primal-dual interior-point QP solver (Mehrotra predictor-corrector).

Solves   min 1/2 z^T P z + q^T z   s.t.  E z = e,  lo <= C z <= hi
with P positive definite.  This is the oracle's exact solve of the horizon
QP; the paper's own solver (Sec. III-B, OSQP's ADMM) is only a faster way to
the same unique optimum.

Method (Mehrotra 1992; Nocedal & Wright, Numerical Optimization, 2nd ed.,
Sec. 16.6, predictor-corrector for inequality-constrained QPs):
  * rows with lo == hi join the equalities; infinite bounds are dropped; the
    rest become one-sided rows G z <= h with slacks s >= 0 and duals lam >= 0;
  * Newton step on the perturbed KKT system, eliminating s and lam:
      (P + G^T diag(lam/s) G) dz + E^T dnu = r,  E dz = -r_e,
    by a dense Cholesky of H = P + G^T D G and of the Schur complement
    E H^-1 E^T;
    when that Cholesky breaks down (H numerically singular as lam/s grows on
    the active rows near a vertex), the same Newton step is taken from the
    equivalent augmented system [[P, E^T, G^T], [E, 0, 0], [G, 0, -S/Lam]]
    by an LU factorisation instead;
  * affine predictor, centring sigma = (mu_aff/mu)^3, corrector;
  * step to 0.99 of the boundary.
Stops when mu <= tol_mu and the scaled residuals are <= tol_res.

Oracle code: test infrastructure only.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla


@dataclass
class IPMResult:
    z: np.ndarray
    nu: np.ndarray          # multipliers of E z = e
    y: np.ndarray           # per-row multipliers of lo <= C z <= hi (y > 0: upper)
    iters: int
    mu: float
    res_dual: float
    res_eq: float
    res_ineq: float
    converged: bool


def _split_rows(C, lo, hi):
    eq = np.isfinite(lo) & np.isfinite(hi) & (lo == hi)
    up = np.isfinite(hi) & ~eq
    dn = np.isfinite(lo) & ~eq
    return eq, up, dn


def solve_qp(P, q, E, e, C, lo, hi, *, tol_mu=1e-13, tol_res=1e-11, max_iter=200):
    n = P.shape[0]
    eq, up, dn = _split_rows(C, lo, hi)
    Ea = np.vstack([E, C[eq]]) if eq.any() else E
    ea = np.concatenate([e, lo[eq]]) if eq.any() else e
    G = np.vstack([C[up], -C[dn]])
    h = np.concatenate([hi[up], -lo[dn]])
    m = G.shape[0]
    p = Ea.shape[0]

    scale_d = 1.0 + np.max(np.abs(q), initial=0.0)
    scale_p = 1.0 + max(np.max(np.abs(h), initial=0.0), np.max(np.abs(ea), initial=0.0))

    # start: equality-constrained minimiser of 1/2 z^T (P + G^T G) z + (q - G^T h)^T z
    H0 = P + G.T @ G
    K0 = np.block([[H0, Ea.T], [Ea, np.zeros((p, p))]])
    sol = np.linalg.solve(K0, np.concatenate([-q + G.T @ h, ea]))
    z = sol[:n]
    nu = sol[n:]
    s = np.maximum(h - G @ z, 1.0)
    lam = np.ones(m)

    def newton(rd, re, ri, rc, chol, Hinv_EaT, Schol):
        # P dz + Ea^T dnu + G^T dlam = -rd ; Ea dz = -re ; G dz + ds = -ri ;
        # lam*ds + s*dlam = rc
        rhs = -rd - G.T @ ((rc + lam * ri) / s)
        Hinv_rhs = sla.cho_solve(chol, rhs)
        dnu = sla.cho_solve(Schol, Ea @ Hinv_rhs + re)
        dz = Hinv_rhs - Hinv_EaT @ dnu
        ds = -ri - G @ dz
        dlam = (rc - lam * ds) / s
        return dz, dnu, ds, dlam

    def newton_aug(rd, re, ri, rc, lu):
        sol = sla.lu_solve(lu, np.concatenate([-rd, -re, -ri - rc / lam]))
        dz, dnu, dlam = sol[:n], sol[n:n + p], sol[n + p:]
        ds = (rc - s * dlam) / lam
        return dz, dnu, ds, dlam

    def max_step(v, dv):
        neg = dv < 0
        if not neg.any():
            return 1.0
        return min(1.0, float(np.min(-v[neg] / dv[neg])))

    it = 0
    converged = False
    for it in range(1, max_iter + 1):
        rd = P @ z + q + Ea.T @ nu + G.T @ lam
        re = Ea @ z - ea
        ri = G @ z + s - h
        mu = float(s @ lam) / max(m, 1)
        if (mu <= tol_mu and np.max(np.abs(rd)) <= tol_res * scale_d
                and np.max(np.abs(re), initial=0.0) <= tol_res * scale_p
                and np.max(np.abs(ri), initial=0.0) <= tol_res * scale_p):
            converged = True
            break
        D = lam / s
        H = P + G.T @ (D[:, None] * G)
        try:
            chol = sla.cho_factor(H, lower=True, check_finite=False)
            Hinv_EaT = sla.cho_solve(chol, Ea.T)
            Schol = sla.cho_factor(Ea @ Hinv_EaT, lower=True, check_finite=False)

            def step(rc):
                return newton(rd, re, ri, rc, chol, Hinv_EaT, Schol)
        except np.linalg.LinAlgError:
            K = np.block([[P, Ea.T, G.T],
                          [Ea, np.zeros((p, p)), np.zeros((p, m))],
                          [G, np.zeros((m, p)), -np.diag(s / lam)]])
            lu = sla.lu_factor(K, check_finite=False)

            def step(rc):
                return newton_aug(rd, re, ri, rc, lu)
        # predictor
        dz_a, _, ds_a, dl_a = step(-s * lam)
        a_aff = min(max_step(s, ds_a), max_step(lam, dl_a))
        mu_aff = float((s + a_aff * ds_a) @ (lam + a_aff * dl_a)) / max(m, 1)
        sigma = (mu_aff / mu) ** 3 if mu > 0 else 0.0
        # corrector
        rc = -s * lam - ds_a * dl_a + sigma * mu
        dz, dnu, ds, dl = step(rc)
        a = min(0.99 * min(max_step(s, ds), max_step(lam, dl)), 1.0)
        z = z + a * dz
        nu = nu + a * dnu
        s = s + a * ds
        lam = lam + a * dl

    rd = P @ z + q + Ea.T @ nu + G.T @ lam
    re = Ea @ z - ea
    ri = G @ z + s - h
    mu = float(s @ lam) / max(m, 1)
    # per-row multipliers of the two-sided form: P z + q + E^T nu + C^T y = 0
    y = np.zeros(C.shape[0])
    nup, ndn = int(up.sum()), int(dn.sum())
    y[up] += lam[:nup]
    y[dn] -= lam[nup:nup + ndn]
    y[eq] = nu[E.shape[0]:]
    return IPMResult(z=z, nu=nu[:E.shape[0]], y=y, iters=it, mu=mu,
                     res_dual=float(np.max(np.abs(rd))),
                     res_eq=float(np.max(np.abs(re), initial=0.0)),
                     res_ineq=float(np.max(np.abs(ri), initial=0.0)),
                     converged=converged)
