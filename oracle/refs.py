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


# ---------------------------------------------------------------- kinematic rows
# The no-slip and swing-height rows of Eq. (mpc_formulation) (Contact: the
# stance foot's velocity J(q) qdot is zero; Swing: the foot height equals
# h_des, a fifth-order Bezier curve over the swing, Eqs. bezier_1..5).
#
# Readings used:
#  * Node n's generalised velocity is (v_n, w_n, u_{n-1} joint rates): the
#    joint rates that carry q_{n-1} to q_n, as in the semi-implicit step
#    q_{i+1} = q_i + dt qdot_{i+1} of Eq. (mpc_formulation).  So the rows of
#    node k+1 read (u_k, x_{k+1}), the API's stage-row form.  Node 0 is data
#    and has none.
#  * Foot position p + r_i(q) with the model's lever r_i(q) (model.py); its
#    velocity is v + J_leg_i[0:3] qdot_leg_i and its height p_z + r_i(q)_z.
#  * Ground level: the height of the foot at the nominal joint angles with the
#    base at the commanded height c_h, i.e. the row p_z + J_z (q_leg - q_nom)
#    equals c_h + B(t_sw) (the lever's own z cancels).
#  * The quintic has six control points and Eqs. bezier_1..5 fix five; the
#    sixth condition is dB/dt(0.5) = 0 (the apex of the swing at mid-swing).
#  * Contact state and swing progress of node n from the same phase as the
#    schedule: s = frac(frac(phi_0 + n dt / T) + o_i), stance if s < d_i,
#    else t_sw = (s - d_i) / (1 - d_i).
#
# Row layout of the eight kinematic rows of stage k (rows 56-63 when enabled):
#   56 + 3i + r  no-slip of foot i, component r (x, y, z), node k+1 in stance
#   62 + i       swing height of foot i, node k+1 in swing
# Rows whose foot is in the other contact state are free.

def bezier_points(z_swing, v_to, v_td):
    """Control points b_0..b_5 of the swing-height quintic
    B(t) = sum_j C(5, j) t^j (1 - t)^(5 - j) b_j with B(0) = B(1) = 0,
    B(0.5) = z_swing, dB/dt(0) = v_to, dB/dt(1) = v_td, dB/dt(0.5) = 0."""
    b0 = b5 = 0.0
    b1 = float(v_to) / 5.0                 # dB/dt(0) = 5 (b1 - b0)
    b4 = -float(v_td) / 5.0                # dB/dt(1) = 5 (b5 - b4)
    # B(0.5) = (b0 + 5 b1 + 10 b2 + 10 b3 + 5 b4 + b5) / 32
    s = (32.0 * float(z_swing) - b0 - 5.0 * b1 - 5.0 * b4 - b5) / 10.0      # b2 + b3
    # dB/dt(0.5) = 5/16 (-b0 - 3 b1 - 2 b2 + 2 b3 + 3 b4 + b5)
    d = (b0 + 3.0 * b1 - 3.0 * b4 - b5) / 2.0                                # b3 - b2
    return np.array([b0, b1, 0.5 * (s - d), 0.5 * (s + d), b4, b5])


def bezier(t, b):
    """B(t) for control points b (Bernstein form)."""
    t = float(t)
    return sum(math.comb(5, j) * t ** j * (1.0 - t) ** (5 - j) * b[j] for j in range(6))


def node_contact(model, phase0, n):
    """(stance (2,) bool, t_sw (2,)) of node n; t_sw is 0 in stance."""
    step = float(model["dt"]) / float(model["period"])
    ph = float(phase0) + float(n) * step
    ph = ph - math.floor(ph)
    st = np.zeros(2, dtype=bool)
    tsw = np.zeros(2)
    for i in range(2):
        s = ph + float(model["offset"][i])
        s = s - math.floor(s)
        d = float(model["duty"][i])
        st[i] = s < d
        if not st[i]:
            tsw[i] = (s - d) / (1.0 - d)
    return st, tsw


def kin_rows(model, cmd, phase0, k, kin):
    """(C_u (8,30), C_x (8,30), lo (8,), hi (8,)) of stage k's kinematic rows
    (node k+1); kin = dict(z_swing, v_to, v_td)."""
    Cu = np.zeros((8, 30))
    Cx = np.zeros((8, 30))
    lo = np.full(8, -INF)
    hi = np.full(8, INF)
    st, tsw = node_contact(model, phase0, k + 1)
    b = bezier_points(kin["z_swing"], kin["v_to"], kin["v_td"])
    for i in range(2):
        J = np.asarray(model["J_leg"][i], float)
        legs = slice(12 + 5 * i, 17 + 5 * i)
        for r in range(3):
            Cu[3 * i + r, legs] = J[r]
            Cx[3 * i + r, 6 + r] = 1.0
            if st[i]:
                lo[3 * i + r] = hi[3 * i + r] = 0.0
        Cx[6 + i, 2] = 1.0
        Cx[6 + i, legs] = J[2]
        if not st[i]:
            h = float(cmd[0]) + bezier(tsw[i], b) + J[2] @ np.asarray(model["q_nom"][5 * i:5 * i + 5], float)
            lo[6 + i] = hi[6 + i] = h
    return Cu, Cx, lo, hi
