"""First-stage solution -> joint torques (paper Sec. III-C, Eqs. (rnea), (mpc_torque)).

  q_MPC    = q*[0] = x0.q          (the initial-state constraint fixes it)
  qdot_MPC = qdot*[0] = u_0.qdot
  qddot    = (u_1.qdot - u_0.qdot) / dt         (Eq. mpc_formulation, qddot_i)
  W_i      = u_0 wrench of foot i (f_i, m_i)
  tau_RNEA,j = [M(q) qddot + h(q, qdot)]_j - [J_leg^T W]_j     (Eq. rnea)
    with a kinematic tree (model keys tree_*): M qddot + h by the spatial
    recursive Newton-Euler algorithm (rnea.py) over the tree, the floating
    base moving as the MPC predicts: orientation Theta_0, angular velocity
    w_0, base acceleration (x_1 - x_0)/dt of the twist (v, w);
    without one: a synthetic diagonal joint model M_j qddot_j + h_j;
    the contact term uses the model's 6x5 leg Jacobian per foot in both
    cases (the MPC's own contact model); the arms carry none
  tau_MPC  = K_p (q_MPC - q) + K_d (qdot_MPC - qdot) + tau_RNEA   (Eq. mpc_torque)

q is the measured joint position (= x0.q) and qdot the measured joint rate.

Oracle code: test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from workload import TREE_CHAINS

from . import model as mdl
from . import rnea


def torque_map(model, x0, qd_meas, u0, u1, x1=None):
    dt = float(model["dt"])
    x0 = np.asarray(x0, float)
    q_mpc = np.array(x0[12:30], dtype=float)
    qd_mpc = np.array(u0[12:30], dtype=float)
    qdd = (np.asarray(u1[12:30], float) - qd_mpc) / dt
    if "tree_axis" in model:
        x1 = np.asarray(x1, float)
        inv = rnea.rnea(rnea.chain_parents(TREE_CHAINS, 18), model["tree_axis"], model["tree_offset"],
                        model["tree_mass"], model["tree_com"], model["tree_inertia"], q_mpc, qd_mpc, qdd,
                        base_R=mdl.rotation(x0[3:6]), base_w=x0[9:12], base_v=x0[6:9],
                        base_dw=(x1[9:12] - x0[9:12]) / dt, base_a=(x1[6:9] - x0[6:9]) / dt)
    else:
        inv = np.asarray(model["M_j"], float) * qdd + np.asarray(model["h_j"], float)
    tau = np.zeros(18)
    for j in range(18):
        tau[j] = (model["Kp"][j] * (q_mpc[j] - x0[12 + j])
                  + model["Kd"][j] * (qd_mpc[j] - qd_meas[j])
                  + inv[j])
    for foot in range(2):
        W = np.asarray(u0[6 * foot:6 * foot + 6], float)
        for jj in range(5):
            j = 5 * foot + jj
            tau[j] -= sum(model["J_leg"][foot][r][jj] * W[r] for r in range(6))
    return tau, q_mpc, qd_mpc
