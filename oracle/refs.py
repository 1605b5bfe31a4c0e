"""Contact schedule, desired trajectory, input references and bounds.

Paper: Sec. III-A.
  * Contact schedule: a phase per contact is integrated along the horizon and
    each node is stance or swing by comparing the phase with the switch value;
    the two feet are offset by half a period.  Reading used: period T_gait,
    per-foot duty d_i and offset o_i;  phi_k = frac(phi_0 + k dt/T_gait),
    stance_{k,i} = frac(phi_k + o_i) < d_i.  The decision is taken in IEEE
    double arithmetic in exactly this operation order (no fused multiply-add).
  * Desired trajectory, Eqs. (des_traj_1)..(des_traj_5): height = c_h, yaw
    integrated with c_wz, linear velocity (c_vx, c_vy) in the yaw frame,
    yaw rate c_wz; nominal joints; every other reference 0.  The yaw of node k
    is yaw_0 + k dt c_wz.
  * Desired vertical force = weight / number of feet in stance (0 in swing).
  * Constraints of Eq. (mpc_formulation), reading used: per stage and foot, a
    4-sided friction pyramid and 0 <= f_z <= fz_max in stance, the whole
    6-D wrench = 0 in swing; |qdot| <= qd_max; |q(k+1)| <= q_lim.

Row layout of one stage's 56 inequality rows (shared convention of the API):
  0-11  wrench box on u[0:12]     (foot L: f 0-2, m 3-5; foot R: f 6-8, m 9-11)
  12-19 pyramid, 4 per foot:  f_x - mu f_z, -f_x - mu f_z, f_y - mu f_z, -f_y - mu f_z
  20-37 qdot box on u[12:30]
  38-55 joint box on x_{k+1}[12:30]

Oracle code: test infrastructure only.
"""
from __future__ import annotations

import math

import numpy as np

from .model import GRAVITY

INF = math.inf


def contact_schedule(model, phase0):
    """stance[k, i] (bool) for k = 0..N-1, i = 0 (left), 1 (right)."""
    N = int(model["N"])
    step = float(model["dt"]) / float(model["period"])
    out = np.zeros((N, 2), dtype=bool)
    for k in range(N):
        ph = float(phase0) + float(k) * step
        ph = ph - math.floor(ph)
        for i in range(2):
            s = ph + float(model["offset"][i])
            s = s - math.floor(s)
            out[k, i] = s < float(model["duty"][i])
    return out


def references(model, x0, cmd, stance):
    """x_ref (N+1, 30) and u_ref (N, 30)."""
    N = int(model["N"])
    dt = float(model["dt"])
    c_h, c_vx, c_vy, c_wz = (float(c) for c in cmd)
    x_ref = np.zeros((N + 1, 30))
    for k in range(N + 1):
        yaw = float(x0[5]) + k * dt * c_wz
        x_ref[k, 2] = c_h
        x_ref[k, 5] = yaw
        x_ref[k, 6] = math.cos(yaw) * c_vx - math.sin(yaw) * c_vy
        x_ref[k, 7] = math.sin(yaw) * c_vx + math.cos(yaw) * c_vy
        x_ref[k, 11] = c_wz
        x_ref[k, 12:30] = model["q_nom"]
    u_ref = np.zeros((N, 30))
    weight = float(model["mass"]) * GRAVITY
    for k in range(N):
        n_st = int(stance[k].sum())
        for i in range(2):
            if stance[k, i]:
                u_ref[k, 6 * i + 2] = weight / n_st
    return x_ref, u_ref


def stage_rows(model, stance_k):
    """(C_u (56,30), C_x (56,30), lo (56,), hi (56,)) for one stage.

    Row r reads C_u[r] @ u_k + C_x[r] @ x_{k+1}.
    """
    mu = float(model["mu"])
    Cu = np.zeros((56, 30))
    Cx = np.zeros((56, 30))
    lo = np.full(56, -INF)
    hi = np.full(56, INF)
    for r in range(12):
        Cu[r, r] = 1.0
    for i in range(2):
        b = 6 * i
        if stance_k[i]:
            lo[b + 2], hi[b + 2] = 0.0, float(model["fz_max"])
        else:
            lo[b:b + 6] = 0.0
            hi[b:b + 6] = 0.0
        p = 12 + 4 * i
        Cu[p + 0, b + 0], Cu[p + 0, b + 2] = 1.0, -mu
        Cu[p + 1, b + 0], Cu[p + 1, b + 2] = -1.0, -mu
        Cu[p + 2, b + 1], Cu[p + 2, b + 2] = 1.0, -mu
        Cu[p + 3, b + 1], Cu[p + 3, b + 2] = -1.0, -mu
        if stance_k[i]:
            hi[p:p + 4] = 0.0
    for j in range(18):
        Cu[20 + j, 12 + j] = 1.0
        lo[20 + j], hi[20 + j] = -float(model["qd_max"]), float(model["qd_max"])
        Cx[38 + j, 12 + j] = 1.0
        lo[38 + j], hi[38 + j] = -float(model["q_lim"]), float(model["q_lim"])
    return Cu, Cx, lo, hi
