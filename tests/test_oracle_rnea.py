"""Pins for the oracle's spatial recursive Newton-Euler inverse dynamics
(paper Eq. rnea): textbook closed forms (pendulum, double pendulum), the
structure of the joint-space dynamics (symmetric positive-definite mass
matrix, the power identity qdot^T C qdot = 1/2 qdot^T Mdot qdot), and
physical invariances (gravity as an upward base acceleration, the base's
linear velocity, a rotation about the vertical)."""
import numpy as np
import pytest

from oracle import model as mdl
from oracle.rnea import chain_parents, rnea, rot_axis
from workload import TREE_CHAINS, make_trees

G = mdl.GRAVITY


def _tree(i=0):
    t = make_trees("uneven", np.arange(i + 1))
    return (chain_parents(TREE_CHAINS, 18), t["tree_axis"][i], t["tree_offset"][i], t["tree_mass"][i],
            t["tree_com"][i], t["tree_inertia"][i])


def _state(seed, n=18):
    g = np.random.default_rng(seed)
    return g.uniform(-1, 1, n), g.uniform(-2, 2, n), g.uniform(-5, 5, n)


@pytest.mark.parametrize("q,qdd", [(0.3, 0.0), (-1.1, 2.5), (2.0, -4.0)])
def test_pendulum(q, qdd):
    # point mass m at distance l below a horizontal axis: tau = m l^2 qdd + m g l sin q
    m, l = 2.3, 0.7
    tau = rnea([-1], [(1.0, 0.0, 0.0)], [np.zeros(3)], [m], [(0.0, 0.0, -l)], [np.zeros(3)],
               [q], [0.4], [qdd])
    assert tau[0] == pytest.approx(m * l * l * qdd + m * G * l * np.sin(q), rel=1e-12, abs=1e-12)


def test_double_pendulum_textbook():
    m1, m2, l1, l2 = 1.5, 0.8, 0.6, 0.45
    for seed in range(5):
        (t1, t2), (d1, d2), (a1, a2) = _state(seed, 2)
        tau = rnea([-1, 0], [(1.0, 0, 0), (1.0, 0, 0)], [np.zeros(3), (0.0, 0.0, -l1)], [m1, m2],
                   [(0.0, 0.0, -l1), (0.0, 0.0, -l2)], [np.zeros(3), np.zeros(3)], [t1, t2], [d1, d2], [a1, a2])
        c2, s2 = np.cos(t2), np.sin(t2)
        M11 = m1 * l1 ** 2 + m2 * (l1 ** 2 + l2 ** 2 + 2 * l1 * l2 * c2)
        M12 = m2 * (l2 ** 2 + l1 * l2 * c2)
        M22 = m2 * l2 ** 2
        h1 = -m2 * l1 * l2 * s2 * (2 * d1 * d2 + d2 ** 2) + (m1 + m2) * G * l1 * np.sin(t1) \
            + m2 * G * l2 * np.sin(t1 + t2)
        h2 = m2 * l1 * l2 * s2 * d1 ** 2 + m2 * G * l2 * np.sin(t1 + t2)
        want = np.array([M11 * a1 + M12 * a2 + h1, M12 * a1 + M22 * a2 + h2])
        np.testing.assert_allclose(tau, want, rtol=1e-11, atol=1e-11)


def _mass_matrix(tree, q):
    n = len(q)
    z = np.zeros(n)
    return np.stack([rnea(*tree, q, z, np.eye(n)[j], gravity=0.0) for j in range(n)], axis=1)


def test_mass_matrix_symmetric_positive_definite():
    tree = _tree(1)
    q, _, _ = _state(3)
    M = _mass_matrix(tree, q)
    np.testing.assert_allclose(M, M.T, atol=1e-12)
    assert np.linalg.eigvalsh(M).min() > 0


def test_power_identity():
    # with h_v = RNEA(q, qdot, 0) without gravity = C(q, qdot) qdot:
    # qdot^T h_v = 1/2 qdot^T (dM/dt) qdot, dM/dt along qdot by central differences
    tree = _tree(2)
    q, qd, _ = _state(4)
    hv = rnea(*tree, q, qd, np.zeros(18), gravity=0.0)
    eps = 1e-6
    Md = (_mass_matrix(tree, q + eps * qd) - _mass_matrix(tree, q - eps * qd)) / (2 * eps)
    assert qd @ hv == pytest.approx(0.5 * qd @ Md @ qd, rel=1e-6)


def test_gravity_equals_upward_base_acceleration():
    tree = _tree(0)
    q, qd, qdd = _state(5)
    a = rnea(*tree, q, qd, qdd)
    b = rnea(*tree, q, qd, qdd, base_a=(0.0, 0.0, G), gravity=0.0)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-10)


def test_base_linear_velocity_does_not_matter():
    # joint torques depend on the base's rotation, angular velocity and the
    # accelerations, not on its linear velocity (Galilean invariance)
    tree = _tree(3)
    q, qd, qdd = _state(6)
    kw = dict(base_R=mdl.rotation([0.1, -0.2, 0.7]), base_w=(0.3, -0.5, 0.8), base_dw=(1.0, 0.4, -2.0),
              base_a=(0.5, -1.5, 2.0))
    a = rnea(*tree, q, qd, qdd, base_v=(0.0, 0.0, 0.0), **kw)
    b = rnea(*tree, q, qd, qdd, base_v=(3.0, -2.0, 1.0), **kw)
    np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-9)


def test_rotation_about_the_vertical():
    # the same motion turned about the world's z axis (gravity unchanged)
    tree = _tree(4)
    q, qd, qdd = _state(7)
    R0 = mdl.rotation([0.15, 0.05, -0.3])
    w, dw, ab, vb = (np.array(v) for v in ((0.2, 0.1, -0.4), (0.5, -1.0, 0.3), (0.4, 0.2, -1.0), (0.3, 0.0, 0.1)))
    Z = rot_axis((0.0, 0.0, 1.0), 0.9)
    a = rnea(*tree, q, qd, qdd, base_R=R0, base_w=w, base_v=vb, base_dw=dw, base_a=ab)
    b = rnea(*tree, q, qd, qdd, base_R=Z @ R0, base_w=Z @ w, base_v=Z @ vb, base_dw=Z @ dw, base_a=Z @ ab)
    np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-9)


def test_tree_torque_map_uses_rnea():
    # with a tree, the oracle's torque map is RNEA - J^T W (+ PD); without,
    # the diagonal joint model
    from oracle.solve import agent_params, solve_agent
    from workload import make_agents
    model, inp = make_agents("small", np.arange(2))
    tm = dict(model)
    tm.update(make_trees("small", np.arange(2)))
    m0, m1 = agent_params(model, 0), agent_params(tm, 0)
    a = solve_agent(m0, inp["x0"][0], inp["cmd"][0], float(inp["phase"][0]), inp["qd_meas"][0])
    b = solve_agent(m1, inp["x0"][0], inp["cmd"][0], float(inp["phase"][0]), inp["qd_meas"][0])
    np.testing.assert_allclose(a["u"], b["u"])           # the QP does not see the tree
    assert np.abs(a["tau"] - b["tau"]).max() > 1e-3
    x0, x1, u0, u1 = b["x"][0], b["x"][1], b["u"][0], b["u"][1]
    dt = float(m1["dt"])
    inv = rnea(chain_parents(TREE_CHAINS, 18), m1["tree_axis"], m1["tree_offset"], m1["tree_mass"],
               m1["tree_com"], m1["tree_inertia"], x0[12:30], u0[12:30], (u1[12:30] - u0[12:30]) / dt,
               base_R=mdl.rotation(x0[3:6]), base_w=x0[9:12], base_v=x0[6:9],
               base_dw=(x1[9:12] - x0[9:12]) / dt, base_a=(x1[6:9] - x0[6:9]) / dt)
    diff = b["tau"] - a["tau"]
    np.testing.assert_allclose(diff, inv - (np.asarray(m0["M_j"]) * (u1[12:30] - u0[12:30]) / dt
                                            + np.asarray(m0["h_j"])), rtol=1e-9, atol=1e-9)
