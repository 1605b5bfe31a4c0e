"""ADMM with the dynamics kept exact in the x-update: the iteration the
Riccati forms run (their ADMM and the paper's fixed-N_QP mode).

Paper: Alg. 1 and Sec. III-B (OSQP's update, to which the paper defers after
Eq. backsolve_2).  Reading used: the stage rows (C, lo, hi of qp.py) are the
ADMM rows; the dynamics E z = e are not split but imposed exactly in every
x-update, so the KKT system of the x-update is

    [[P + sigma I + C^T diag(rho_r) C, E^T], [E, 0]] [z~; nu] =
        [sigma z - q + C^T (diag(rho_r) w - y); e]

with rho_r = 1e3 rho on rows with lo = hi, rho on the other constrained rows
and no row where both bounds are infinite (a free row is left out).  Then,
with w~ = C z~ (OSQP's z~ for an exact solve):

    z  <- alpha z~ + (1 - alpha) z
    wh  = alpha w~ + (1 - alpha) w
    w  <- clip(wh + y / rho_r, lo, hi)
    y  <- y + rho_r (wh - w)

Start (f_init): z^0 the current base pose and nominal joints repeated, every
other entry zero; w^0 = clip(C z^0); y^0 = 0.  rho fixed.

Oracle code: test infrastructure only.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

RHO_EQ_FACTOR = 1e3


def row_steps(qp, rho: float):
    """(keep mask, rho_r of the kept rows)."""
    keep = np.isfinite(qp.lo) | np.isfinite(qp.hi)
    lo, hi = qp.lo[keep], qp.hi[keep]
    return keep, np.where(lo == hi, RHO_EQ_FACTOR * rho, rho)


def iterate(qp, z, w, y, iters: int, *, rho: float = 0.1, sigma: float = 1e-6, alpha: float = 1.6,
            trace=None):
    """`iters` iterations from (z, w, y) (w, y over the kept rows); returns
    (z, w, y).  trace, if a list, receives (z~, w~, z, w, y) per iteration."""
    keep, rr = row_steps(qp, rho)
    C, lo, hi = qp.C[keep], qp.lo[keep], qp.hi[keep]
    n, m = qp.P.shape[0], qp.E.shape[0]
    K = np.zeros((n + m, n + m))
    K[:n, :n] = qp.P + sigma * np.eye(n) + C.T @ (rr[:, None] * C)
    K[:n, n:] = qp.E.T
    K[n:, :n] = qp.E
    lu = sla.lu_factor(K)
    z, w, y = (np.array(v, dtype=float) for v in (z, w, y))
    for _ in range(iters):
        rhs = np.concatenate([sigma * z - qp.q + C.T @ (rr * w - y), qp.e])
        zt = sla.lu_solve(lu, rhs)[:n]
        wt = C @ zt
        z = alpha * zt + (1.0 - alpha) * z
        wh = alpha * wt + (1.0 - alpha) * w
        w = np.clip(wh + y / rr, lo, hi)
        y = y + rr * (wh - w)
        if trace is not None:
            trace.append((zt.copy(), wt.copy(), z.copy(), w.copy(), y.copy()))
    return z, w, y


def start_point(qp, x0, q_nom, rho: float = 0.1):
    """(z^0, w^0, y^0) of f_init."""
    keep, _ = row_steps(qp, rho)
    z = np.zeros(60 * qp.N)
    xk = np.zeros(30)
    xk[0:6] = np.asarray(x0, float)[0:6]
    xk[12:30] = q_nom
    for k in range(1, qp.N + 1):
        z[60 * (k - 1) + 30:60 * (k - 1) + 60] = xk
    w = np.clip(qp.C[keep] @ z, qp.lo[keep], qp.hi[keep])
    return z, w, np.zeros(int(keep.sum()))
