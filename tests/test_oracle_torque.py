"""Pins for the oracle's torque map (paper Sec. III-C, Eqs. rnea and
mpc_torque) on a case worked by hand with a nonzero joint acceleration."""
import numpy as np

from oracle.torque import torque_map


def test_torque_with_joint_acceleration_by_hand():
    # dt = 0.02, K_d = 1, M_j = 0.1, h_j = 2 (legs) and -1 (arms).
    # u_0 joint rates 0.2, u_1 joint rates 0.5 (legs) and -0.2 (arms), measured
    # rates 0.1:
    #   K_d term   = 1 * (0.2 - 0.1) = 0.1
    #   legs:  qdd = (0.5 - 0.2) / 0.02 = 15,  M qdd = 1.5
    #   arms:  qdd = (-0.2 - 0.2) / 0.02 = -20, M qdd = -2.0
    # leg Jacobians: J_L[2][0] = 0.3 (f_z -> joint 0), J_L[3][1] = 0.5 (m_x ->
    # joint 1), J_R[0][0] = -0.4 (f_x -> joint 5); W_L = (0, 0, 200, 4, 0, 0),
    # W_R = (50, 0, 150, 0, 0, 0):
    #   tau_0  = 0.1 + 1.5 + 2 - 0.3*200   = -56.4
    #   tau_1  = 0.1 + 1.5 + 2 - 0.5*4     = 1.6
    #   tau_2  = 0.1 + 1.5 + 2             = 3.6   (likewise 3, 4, 6..9)
    #   tau_5  = 0.1 + 1.5 + 2 + 0.4*50    = 23.6
    #   tau_12 = 0.1 - 2.0 - 1             = -2.9  (every arm joint)
    # K_p (q_MPC - q) is 0: q_MPC is the measured x0.q.
    J = np.zeros((2, 6, 5))
    J[0, 2, 0], J[0, 3, 1], J[1, 0, 0] = 0.3, 0.5, -0.4
    h = np.r_[np.full(10, 2.0), np.full(8, -1.0)]
    m = dict(dt=0.02, Kp=np.full(18, 30.0), Kd=np.ones(18), M_j=np.full(18, 0.1), h_j=h, J_leg=J)
    x0 = np.zeros(30)
    x0[12:30] = np.linspace(-0.4, 0.4, 18)
    u0 = np.zeros(30)
    u0[0:6] = (0, 0, 200, 4, 0, 0)
    u0[6:12] = (50, 0, 150, 0, 0, 0)
    u0[12:30] = 0.2
    u1 = np.zeros(30)
    u1[12:22] = 0.5
    u1[22:30] = -0.2
    tau, q_set, qd_set = torque_map(m, x0, np.full(18, 0.1), u0, u1)
    want = np.r_[-56.4, 1.6, 3.6, 3.6, 3.6, 23.6, 3.6, 3.6, 3.6, 3.6, np.full(8, -2.9)]
    assert np.allclose(tau, want, atol=1e-12)
    assert np.allclose(q_set, x0[12:30])
    assert np.allclose(qd_set, 0.2)
