"""First-stage solution -> joint torques (paper Sec. III-C, Eqs. (rnea), (mpc_torque)).

  q_MPC    = q*[0] = x0.q          (the initial-state constraint fixes it)
  qdot_MPC = qdot*[0] = u_0.qdot
  qddot    = (u_1.qdot - u_0.qdot) / dt         (Eq. mpc_formulation, qddot_i)
  W_i      = u_0 wrench of foot i (f_i, m_i)
  tau_RNEA,j = M_j qddot_j + h_j - [J_leg^T W]_j     (Eq. rnea; synthetic joint
               model: diagonal M, bias h, 6x5 leg Jacobian per foot; arms carry
               no contact term)
  tau_MPC  = K_p (q_MPC - q) + K_d (qdot_MPC - qdot) + tau_RNEA   (Eq. mpc_torque)

q is the measured joint position (= x0.q) and qdot the measured joint rate.

Oracle code: test infrastructure only.
"""
from __future__ import annotations

import numpy as np


def torque_map(model, x0, qd_meas, u0, u1):
    dt = float(model["dt"])
    q_mpc = np.array(x0[12:30], dtype=float)
    qd_mpc = np.array(u0[12:30], dtype=float)
    qdd = (np.asarray(u1[12:30], float) - qd_mpc) / dt
    tau = np.zeros(18)
    for j in range(18):
        tau[j] = (model["Kp"][j] * (q_mpc[j] - x0[12 + j])
                  + model["Kd"][j] * (qd_mpc[j] - qd_meas[j])
                  + model["M_j"][j] * qdd[j] + model["h_j"][j])
    for foot in range(2):
        W = np.asarray(u0[6 * foot:6 * foot + 6], float)
        for jj in range(5):
            j = 5 * foot + jj
            tau[j] -= sum(model["J_leg"][foot][r][jj] * W[r] for r in range(6))
    return tau, q_mpc, qd_mpc
