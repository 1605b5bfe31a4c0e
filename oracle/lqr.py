"""Closed-form affine finite-horizon LQR by dynamic programming (a pin).

Used only to pin the interior-point oracle: when no inequality constraint of
the horizon QP is active, its optimum is the LQR optimum below, which is
computed by an independent method (the textbook backward Riccati recursion
of the value function V_k(x) = 1/2 x^T P_k x + p_k^T x, e.g. Anderson & Moore,
Optimal Control, ch. 2, extended with the affine term c_k and references).

  minimise sum_k 1/2 |x_k - xr_k|^2_Qb + 1/2 |u_k - ur_k|^2_Rb + 1/2 |x_N - xr_N|^2_Qb
  s.t. x_{k+1} = A_k x_k + B_k u_k + c_k, x_0 given,
       u_k[j] = 0 for every j with fixed[k, j] (swing-foot wrench).

Oracle code: test infrastructure only.
"""
from __future__ import annotations

import numpy as np


def affine_lqr(A, B, c, Qb, Rb, x0, x_ref, u_ref, fixed=None):
    N = len(A)
    nu = B[0].shape[1]
    if fixed is None:
        fixed = np.zeros((N, nu), dtype=bool)
    P = np.diag(Qb)
    p = -Qb * x_ref[N]
    gains = [None] * N
    for k in range(N - 1, -1, -1):
        free = ~fixed[k]
        Bf = B[k][:, free]
        Rf = np.diag(Rb[free])
        s = P @ c[k] + p
        Quu = Rf + Bf.T @ P @ Bf
        Qux = Bf.T @ P @ A[k]
        qu = -Rf @ u_ref[k][free] + Bf.T @ s
        Qxx = np.diag(Qb) + A[k].T @ P @ A[k]
        qx = -Qb * x_ref[k] + A[k].T @ s
        K = -np.linalg.solve(Quu, Qux)
        d = -np.linalg.solve(Quu, qu)
        P = Qxx + Qux.T @ K
        P = 0.5 * (P + P.T)
        p = qx + Qux.T @ d
        gains[k] = (free, K, d)
    x = np.zeros((N + 1, A[0].shape[0]))
    u = np.zeros((N, nu))
    x[0] = x0
    for k in range(N):
        free, K, d = gains[k]
        u[k, free] = K @ x[k] + d
        x[k + 1] = A[k] @ x[k] + B[k] @ u[k] + c[k]
    return x, u
