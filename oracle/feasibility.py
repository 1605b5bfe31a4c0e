"""Primal feasibility of an agent's horizon QP (OSQP's infeasibility status).

The constraint set {z : E z = e, lo <= C z <= hi} of the dense QP
(qp.DenseQP) is empty exactly when the linear program
    min 0   s.t.  E z = e,  C z <= hi,  -C z <= -lo   (finite bounds only)
has no feasible point.  The LP is handed to scipy's HiGHS solver (a library
primitive); its status 2 means infeasible.  For the joint limits of this
problem there is also a closed form, used as this function's pin in
tests/test_oracle_solver.py: joint j is reachable in the first stage only if
|q0_j| <= q_lim + dt qd_max (q_1 = q0 + dt qd_0, |qd_0| <= qd_max,
|q_1| <= q_lim), and every other row admits u = 0.

Oracle code: test infrastructure only.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import linprog


def is_feasible(qp) -> bool:
    C, lo, hi = np.asarray(qp.C, float), np.asarray(qp.lo, float), np.asarray(qp.hi, float)
    up, dn = np.isfinite(hi), np.isfinite(lo)
    A_ub = np.vstack([C[up], -C[dn]])
    b_ub = np.concatenate([hi[up], -lo[dn]])
    n = C.shape[1]
    res = linprog(np.zeros(n), A_ub=A_ub, b_ub=b_ub, A_eq=qp.E, b_eq=qp.e, bounds=[(None, None)] * n,
                  method="highs")
    if res.status == 2:
        return False
    if res.status != 0:
        raise RuntimeError(f"feasibility LP did not finish: {res.message}")
    return True


def joint_limits_reachable(model, x0) -> bool:
    """Closed form: every joint can reach its box in the first stage."""
    q0 = np.asarray(x0, float)[12:30]
    lim = float(model["q_lim"]) + float(model["dt"]) * float(model["qd_max"])
    return bool(np.all(np.abs(q0) <= lim))
