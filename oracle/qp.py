"""Dense horizon QP of one agent (paper Eq. (mpc_formulation), linearised).

  minimise  sum_{k=0}^{N-1} dt [(x_k - xr_k)^T Q (x_k - xr_k) + (u_k - ur_k)^T R (u_k - ur_k)]
            + dt (x_N - xr_N)^T Q (x_N - xr_N)
  s.t.      x_{k+1} = A_k x_k + B_k u_k + c_k,   x_0 = x0 (fixed)
            lo_k <= C_u u_k + C_x x_{k+1} <= hi_k,   k = 0..N-1
            (56 rows per stage, refs.stage_rows; 64 with the kinematic rows)

The stage cost is weighted by dt (Eq. mpc_formulation); there is no 1/2, so
the Hessian is 2 dt diag(Q), 2 dt diag(R).

Variables are interleaved z = [u_0, x_1, u_1, x_2, ..., u_{N-1}, x_N]; block k
(60 wide) is (u_k, x_{k+1}).  In standard form:
  min 1/2 z^T P z + q^T z + const   s.t.  E z = e,  lo <= C z <= hi.

Oracle code: test infrastructure only.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import model as mdl
from . import refs


@dataclass
class DenseQP:
    P: np.ndarray
    q: np.ndarray
    const: float
    E: np.ndarray
    e: np.ndarray
    C: np.ndarray
    lo: np.ndarray
    hi: np.ndarray
    N: int

    def u(self, z, k):
        return z[60 * k:60 * k + 30]

    def x(self, z, k):
        """x_k for k >= 1 (x_0 is not a variable)."""
        return z[60 * (k - 1) + 30:60 * (k - 1) + 60]

    def objective(self, z):
        return 0.5 * z @ self.P @ z + self.q @ z + self.const


def build_qp(A, B, c, Q, R, dt, x0, x_ref, u_ref, rows):
    """Assemble the dense QP.

    A, B, c: per-stage affine model; Q, R: diagonal weights (30,);
    rows: list of (C_u, C_x, lo, hi) per stage.
    """
    N = len(A)
    n = 60 * N
    P = np.zeros((n, n))
    qv = np.zeros(n)
    const = dt * (x0 - x_ref[0]) @ (Q * (x0 - x_ref[0]))
    for k in range(N):
        iu = slice(60 * k, 60 * k + 30)
        ix = slice(60 * k + 30, 60 * k + 60)
        wx = dt * Q
        P[iu, iu] = np.diag(2.0 * dt * R)
        P[ix, ix] = np.diag(2.0 * wx)
        qv[iu] = -2.0 * dt * R * u_ref[k]
        qv[ix] = -2.0 * wx * x_ref[k + 1]
        const += dt * u_ref[k] @ (R * u_ref[k]) + wx @ (x_ref[k + 1] ** 2)
    E = np.zeros((30 * N, n))
    e = np.zeros(30 * N)
    for k in range(N):
        r = slice(30 * k, 30 * k + 30)
        E[r, 60 * k + 30:60 * k + 60] = np.eye(30)      # x_{k+1}
        E[r, 60 * k:60 * k + 30] = -B[k]                 # u_k
        if k == 0:
            e[r] = c[0] + A[0] @ x0
        else:
            E[r, 60 * (k - 1) + 30:60 * (k - 1) + 60] = -A[k]   # x_k
            e[r] = c[k]
    nr = rows[0][0].shape[0]
    C = np.zeros((nr * N, n))
    lo = np.zeros(nr * N)
    hi = np.zeros(nr * N)
    for k in range(N):
        Cu, Cx, l_k, h_k = rows[k]
        r = slice(nr * k, nr * k + nr)
        C[r, 60 * k:60 * k + 30] = Cu
        C[r, 60 * k + 30:60 * k + 60] = Cx
        lo[r] = l_k
        hi[r] = h_k
    return DenseQP(P, qv, float(const), E, e, C, lo, hi, N)


def agent_qp(model, x0, cmd, phase0, kin=None):
    """Everything of f_init/f_param/f_KKT for one agent: (qp, extras).

    kin: None, or dict(z_swing, v_to, v_td) to append each stage's eight
    kinematic rows (no-slip, swing height; refs.kin_rows) as rows 56-63."""
    stance = refs.contact_schedule(model, phase0)
    x_ref, u_ref = refs.references(model, x0, cmd, stance)
    A, B, c = mdl.linearise(model, x0, u_ref)
    rows = [refs.stage_rows(model, stance[k]) for k in range(int(model["N"]))]
    if kin is not None:
        for k in range(len(rows)):
            ek = refs.kin_rows(model, cmd, phase0, k, kin)
            rows[k] = tuple(np.concatenate([a, b]) for a, b in zip(rows[k], ek))
    qp = build_qp(A, B, c, np.asarray(model["Q"], float), np.asarray(model["R"], float),
                  float(model["dt"]), np.asarray(x0, float), x_ref, u_ref, rows)
    extras = dict(stance=stance, x_ref=x_ref, u_ref=u_ref, A=A, B=B, c=c, rows=rows)
    return qp, extras
