"""Brute-force active-set enumeration for small QPs (a pin for the IPM).

For  min 1/2 z^T P z + q^T z  s.t.  E z = e,  lo <= C z <= hi  (P > 0) the
optimum is the unique point satisfying the KKT conditions.  Every pattern of
{inactive, at lower, at upper} over the rows is tried: the equality-
constrained QP of that pattern is solved through its KKT matrix, and the
pattern is kept when the point is primal feasible and every multiplier has
the right sign (y <= 0 at a lower bound, y >= 0 at an upper bound, with
stationarity P z + q + E^T nu + C^T y = 0).  3^m solves: toy sizes only.

Oracle code: test infrastructure only.
"""
from __future__ import annotations

import itertools

import numpy as np


def brute_force_qp(P, q, E, e, C, lo, hi, tol=1e-9):
    n = P.shape[0]
    m = C.shape[0]
    options = []
    for i in range(m):
        if np.isfinite(lo[i]) and lo[i] == hi[i]:
            options.append((1,))                 # equality: always active
            continue
        o = [0]
        if np.isfinite(lo[i]):
            o.append(1)
        if np.isfinite(hi[i]):
            o.append(2)
        options.append(tuple(o))
    best = None
    for pat in itertools.product(*options):
        act = [i for i in range(m) if pat[i] != 0]
        Ca = C[act]
        ba = np.array([lo[i] if pat[i] == 1 else hi[i] for i in act])
        Aeq = np.vstack([E, Ca]) if act else E
        beq = np.concatenate([e, ba]) if act else e
        p = Aeq.shape[0]
        K = np.block([[P, Aeq.T], [Aeq, np.zeros((p, p))]])
        rhs = np.concatenate([-q, beq])
        if np.linalg.matrix_rank(K) < n + p:
            continue
        sol = np.linalg.solve(K, rhs)
        z = sol[:n]
        mult = sol[n + E.shape[0]:]
        Cz = C @ z
        if np.any(Cz < lo - tol) or np.any(Cz > hi + tol):
            continue
        ok = True
        y = np.zeros(m)
        for j, i in enumerate(act):
            y[i] = mult[j]
            if np.isfinite(lo[i]) and lo[i] == hi[i]:
                continue
            if pat[i] == 1 and mult[j] > tol:
                ok = False
            if pat[i] == 2 and mult[j] < -tol:
                ok = False
        if ok:
            best = (z, y, pat)
            break
    return best
