"""Pins for the oracle's model and linearisation (paper Sec. III-A, Eq. base_dynamics)."""
import numpy as np
import pytest

from oracle import model as mdl
from oracle.solve import agent_params
from workload import make_agents


def _agent(i=0, name="small"):
    m, inp = make_agents(name, [i])
    return agent_params(m, 0), {k: v[0] for k, v in inp.items()}


def _skew_inv(S):
    return np.array([S[2, 1], S[0, 2], S[1, 0]])


@pytest.mark.parametrize("seed", range(5))
def test_euler_rate_map_matches_rotation_derivative(seed):
    # dR/dt R^T = [w]x for R = Rz Ry Rx; central differences of R along
    # Theta(t) = Theta + t Theta_dot give w, compare with E(Theta) Theta_dot.
    rng = np.random.default_rng(seed)
    th = rng.uniform(-1.0, 1.0, 3)
    thd = rng.normal(size=3)
    h = 1e-6
    Rd = (mdl.rotation(th + h * thd) - mdl.rotation(th - h * thd)) / (2 * h)
    w = _skew_inv(Rd @ mdl.rotation(th).T)
    assert np.allclose(mdl.euler_rate_matrix(th) @ thd, w, atol=1e-8)


def test_euler_rate_identity_at_zero():
    assert np.allclose(mdl.euler_rate_matrix(np.zeros(3)), np.eye(3))


@pytest.mark.parametrize("i", range(4))
def test_complex_step_matches_central_differences(i):
    m, inp = _agent(i)
    x0 = inp["x0"]
    u = np.zeros(30)
    u[2], u[8] = 110.0, 130.0
    u[0], u[7], u[3] = 5.0, -3.0, 0.4
    u[12:] = np.linspace(-1, 1, 18)
    Iw = mdl.world_inertia(m, x0[3:6])
    f0, fx, fu = mdl.jacobians(m, x0, u, Iw)
    h = 1e-6
    for j in range(30):
        e = np.zeros(30)
        e[j] = h
        dx = (mdl.dynamics(m, x0 + e, u, Iw) - mdl.dynamics(m, x0 - e, u, Iw)) / (2 * h)
        du = (mdl.dynamics(m, x0, u + e, Iw) - mdl.dynamics(m, x0, u - e, Iw)) / (2 * h)
        assert np.allclose(fx[:, j], dx, rtol=1e-6, atol=1e-7)
        assert np.allclose(fu[:, j], du, rtol=1e-6, atol=1e-7)


def test_torque_free_rigid_body_invariants():
    # With no wrench, the frozen-inertia body keeps |I_w w| and w^T I_w w:
    # d/dt |I w|^2 = 2 (I w).(-w x I w) = 0 and d/dt w^T I w = 0.
    m, inp = _agent(1)
    x = inp["x0"].copy()
    x[9:12] = (0.7, -1.1, 0.4)
    Iw = mdl.world_inertia(m, x[3:6])
    f = mdl.dynamics(m, x, np.zeros(30), Iw)
    w, wd = x[9:12], f[9:12]
    assert abs((Iw @ w) @ (Iw @ wd)) < 1e-12
    assert abs(w @ Iw @ wd) < 1e-12
    # free fall: v_dot = g, joints follow their rates
    assert np.allclose(f[6:9], [0, 0, -9.81])
    assert np.allclose(f[0:3], x[6:9])


def test_linearisation_structure():
    m, inp = _agent(2)
    x0 = inp["x0"]
    dt = m["dt"]
    u_st = np.zeros((2, 30))
    u_st[0, 2], u_st[0, 8] = 120.0, 120.0       # both feet loaded
    A, B, c = mdl.linearise(m, x0, u_st)
    # flight stage: no force, so the joints do not move the angular rate
    assert np.allclose(A[1][9:12, 12:30], 0.0)
    assert not np.allclose(A[0][9:12, 12:22], 0.0)
    # forces enter the linear velocity as dt/m, joint rates the joints as dt
    assert np.allclose(B[0][6:9, 0:3], dt / m["mass"] * np.eye(3))
    assert np.allclose(B[0][12:30, 12:30], dt * np.eye(18))
    # the affine model reproduces one Euler step at the linearisation point
    Iw = mdl.world_inertia(m, x0[3:6])
    for k in range(2):
        step = x0 + dt * mdl.dynamics(m, x0, u_st[k], Iw)
        assert np.allclose(A[k] @ x0 + B[k] @ u_st[k] + c[k], step, atol=1e-12)


def test_world_angular_momentum_conserved_by_true_rotation():
    # Torque free, the world angular momentum L = R I_b R^T w is constant while
    # R turns with w.  The model's w_dot (inertia frozen at the current
    # attitude) must give dL/dt = 0; the gyroscopic term with the wrong sign
    # would give 2 w x I_w w instead.
    from scipy.linalg import expm
    m, inp = _agent(3)
    x = inp["x0"].copy()
    x[9:12] = (0.9, -0.6, 1.3)
    R0 = mdl.rotation(x[3:6])
    Ib = np.diag(m["inertia"])
    Iw = R0 @ Ib @ R0.T
    w = x[9:12]
    wd = mdl.dynamics(m, x, np.zeros(30), Iw)[9:12]
    W = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])

    def L(t):
        R = expm(W * t) @ R0
        return R @ Ib @ R.T @ (w + t * wd)

    h = 1e-5
    dL = (L(h) - L(-h)) / (2 * h)
    assert np.abs(dL).max() < 1e-8 * (1 + np.abs(Iw @ w).max())


def _hand_model():
    """A model with every number chosen by hand: level attitude (so the world
    inertia is diag(2, 3, 4)), mass 25 kg, left lever (0.1, 0.05, -0.6) m,
    right lever (-0.1, -0.05, -0.6) m, and a left-leg Jacobian whose first
    three rows are 0.2 e_0, 0.3 e_1 and 0.1 e_3 (everything else zero)."""
    J = np.zeros((2, 6, 5))
    J[0, 0, 0], J[0, 1, 1], J[0, 2, 3] = 0.2, 0.3, 0.1
    return dict(mass=25.0, inertia=np.array([2.0, 3.0, 4.0]),
                lever=np.array([[0.1, 0.05, -0.6], [-0.1, -0.05, -0.6]]),
                J_leg=J, q_nom=np.zeros(18), dt=0.02)


def test_single_stance_contact_moment_by_hand():
    # Left foot alone, f = (10, 0, 200) N, m = (1, 2, 3) N m, lever
    # r = (0.1, 0.05, -0.6) m, at rest and level (Eq. base_dynamics):
    #   r x f = (0.05*200 - (-0.6)*0, (-0.6)*10 - 0.1*200, 0.1*0 - 0.05*10)
    #         = (10, -26, -0.5);   + m = (11, -24, 2.5)
    #   w_dot = diag(2, 3, 4)^-1 (11, -24, 2.5) = (5.5, -8, 0.625)
    #   v_dot = f / 25 + g = (0.4, 0, 8 - 9.81) = (0.4, 0, -1.81)
    # (f x r in place of r x f would give w_dot = (-4.5, 9.333, 0.875).)
    m = _hand_model()
    x = np.zeros(30)
    x[2] = 0.6
    u = np.zeros(30)
    u[0:3] = (10.0, 0.0, 200.0)
    u[3:6] = (1.0, 2.0, 3.0)
    f = mdl.dynamics(m, x, u, mdl.world_inertia(m, x[3:6]))
    assert np.allclose(f[9:12], [5.5, -8.0, 0.625], atol=1e-12)
    assert np.allclose(f[6:9], [0.4, 0.0, -1.81], atol=1e-12)
    assert np.allclose(f[3:6], 0.0)
    # the right foot's lever enters with its own force only
    u2 = np.zeros(30)
    u2[6:9] = (0.0, 0.0, 100.0)
    # r_R x (0, 0, 100) = (-0.05*100, 0.1*100, 0) = (-5, 10, 0)
    f2 = mdl.dynamics(m, x, u2, mdl.world_inertia(m, x[3:6]))
    assert np.allclose(f2[9:12], [-2.5, 10.0 / 3.0, 0.0], atol=1e-12)


def test_lever_follows_the_leg_joints_by_hand():
    # q_leg,L - q_nom = (0.5, -1.0, 0, 2.0, 0):
    #   J_r (q - q_nom) = (0.2*0.5, 0.3*(-1.0), 0.1*2.0) = (0.1, -0.3, 0.2)
    #   r_L = (0.1, 0.05, -0.6) + (0.1, -0.3, 0.2) = (0.2, -0.25, -0.4)
    # with f_L = (0, 0, 100):  r x f = (-0.25*100, -0.2*100, 0) = (-25, -20, 0)
    #   w_dot = (-25/2, -20/3, 0)
    m = _hand_model()
    x = np.zeros(30)
    x[12:17] = (0.5, -1.0, 0.0, 2.0, 0.0)
    x[17:22] = (0.3, 0.3, 0.3, 0.3, 0.3)      # right leg: its Jacobian is zero
    assert np.allclose(mdl.foot_lever(m, x[12:30], 0), [0.2, -0.25, -0.4], atol=1e-15)
    assert np.allclose(mdl.foot_lever(m, x[12:30], 1), [-0.1, -0.05, -0.6], atol=1e-15)
    u = np.zeros(30)
    u[2] = 100.0
    f = mdl.dynamics(m, x, u, mdl.world_inertia(m, x[3:6]))
    assert np.allclose(f[9:12], [-12.5, -20.0 / 3.0, 0.0], atol=1e-12)


def test_joint_column_of_the_angular_rate_block_by_hand():
    # d w_dot / d q_leg,j = I_w^-1 ((J_r e_j) x f) at the linearisation input,
    # times dt in A_k.  f_L = (0, 0, 100), dt = 0.02, I_w = diag(2, 3, 4):
    #   j = 0: (0.2, 0, 0) x f = (0, -20, 0)  -> dt (0, -20/3, 0) = (0, -0.13333, 0)
    #   j = 1: (0, 0.3, 0) x f = (30, 0, 0)   -> dt (15, 0, 0)    = (0.3, 0, 0)
    #   j = 3: (0, 0, 0.1) x f = 0            -> 0
    #   j = 2, 4 and the right leg (no force, zero Jacobian): 0
    m = _hand_model()
    x0 = np.zeros(30)
    x0[2] = 0.6
    u_ref = np.zeros((2, 30))
    u_ref[0, 2] = 100.0
    A, B, c = mdl.linearise(m, x0, u_ref)
    col = A[0][9:12, 12:30]
    want = np.zeros((3, 18))
    want[:, 0] = (0.0, -0.02 * 20.0 / 3.0, 0.0)
    want[:, 1] = (0.02 * 15.0, 0.0, 0.0)
    assert np.allclose(col, want, atol=1e-13)
    # second stage: no force, so no joint coupling
    assert np.allclose(A[1][9:12, 12:30], 0.0, atol=1e-15)
    # the force column of the same block: dt I_w^-1 [r_L]x, e.g. d w_dot / d f_x
    # = I_w^-1 (r x e_x) = I_w^-1 (0, -0.6, -0.05) -> dt (0, -0.2, -0.0125)
    assert np.allclose(B[0][9:12, 0], [0.0, -0.02 * 0.2, -0.02 * 0.0125], atol=1e-15)
