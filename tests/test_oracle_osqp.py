"""Pins for the oracle's literal OSQP iteration (oracle/osqp.py; paper
Sec. III-B, Eq. kkt_system, Alg. 1; OSQP's update steps).

(i)   a one-variable problem iterated twice by hand (every step of the update:
      the KKT solve, z~, the relaxation, the projection and the dual update);
(ii)  the iteration's fixed point is the optimum: on horizon QPs of the
      generated workloads it converges to the interior-point solution;
(iii) the dual update keeps every multiplier in the normal cone of its
      bound: y >= 0 at an upper bound, <= 0 at a lower bound, 0 inside;
(iv)  the exact KKT solve gives z~ = A x~ (the second block row of
      Eq. kkt_system), which pins the sign of its -rho^-1 block.
"""
import numpy as np
import pytest

from oracle import ipm, osqp, qp as qpmod
from oracle.solve import agent_params
from workload import make_agents


def test_one_variable_iterations_by_hand():
    # minimise x^2 - 4x subject to 0 <= x <= 1 (P = 2, q = -4, A = 1), with
    # sigma = rho = 1 and alpha = 1.6, from x = z = y = 0.
    # iteration 1: [[3, 1], [1, -1]] [x~, nu] = [4, 0]  ->  x~ = nu = 1;
    #   z~ = 0 + (1 - 0) = 1; x = 1.6; zr = 1.6; z = clip(1.6) = 1; y = 0.6
    # iteration 2: rhs = [1.6 + 4, 1 - 0.6] = [5.6, 0.4]  ->  x~ = 1.5,
    #   nu = 1.1; z~ = 1 + 0.5 = 1.5; x = 2.4 - 0.96 = 1.44;
    #   zr = 2.4 - 0.6 = 1.8; z = clip(2.4) = 1; y = 0.6 + 0.8 = 1.4
    lq = osqp.LiteralQP(P=np.array([[2.0]]), q=np.array([-4.0]), A=np.array([[1.0]]), l=np.array([0.0]),
                        u=np.array([1.0]), rho=np.array([1.0]), n_dyn=0)
    tr = []
    osqp.iterate(lq, np.zeros(1), np.zeros(1), np.zeros(1), 2, sigma=1.0, alpha=1.6, trace=tr)
    want = [(1.0, 1.0, 1.6, 1.0, 0.6), (1.5, 1.5, 1.44, 1.0, 1.4)]
    for got, w in zip(tr, want):
        assert np.allclose([g[0] for g in got], w, rtol=0, atol=1e-14)
    # and it converges to the optimum x = 1 with the multiplier y = 2
    # (stationarity 2 x - 4 + y = 0)
    x, z, y = osqp.iterate(lq, np.zeros(1), np.zeros(1), np.zeros(1), 200, sigma=1.0, alpha=1.6)
    assert abs(x[0] - 1.0) < 1e-12 and abs(y[0] - 2.0) < 1e-12


def _agent_qp(i, N):
    mm, inp = make_agents("uneven", [i])
    m = agent_params(mm, 0)
    m["N"] = N
    x0 = inp["x0"][0]
    qp, _ = qpmod.agent_qp(m, x0, inp["cmd"][0], inp["phase"][0])
    return m, x0, qp


@pytest.mark.parametrize("i,N", [(0, 3), (5, 4), (11, 3)])
def test_fixed_point_is_the_interior_point_optimum(i, N):
    m, x0, qp = _agent_qp(i, N)
    lq = osqp.literal_form(qp, rho=0.1)
    x, z, y = osqp.start_point(lq, qp, x0, m["q_nom"])
    x, z, y, it = osqp.solve_until(lq, x, z, y, eps_abs=1e-11, eps_rel=1e-11, max_iter=60000,
                                   check_every=50)
    ref = ipm.solve_qp(qp.P, qp.q, qp.E, qp.e, qp.C, qp.lo, qp.hi)
    assert ref.converged
    scale = 1.0 + np.abs(ref.z).max()
    assert np.abs(x - ref.z).max() <= 1e-7 * scale, (it, np.abs(x - ref.z).max())


def test_multipliers_stay_in_the_normal_cone():
    m, x0, qp = _agent_qp(7, 5)
    lq = osqp.literal_form(qp, rho=0.1)
    x, z, y = osqp.start_point(lq, qp, x0, m["q_nom"])
    tr = []
    osqp.iterate(lq, x, z, y, 30, trace=tr)
    ineq = lq.l != lq.u
    for (_, _, _, zk, yk) in tr:
        at_up = ineq & np.isclose(zk, lq.u, rtol=0, atol=1e-12)
        at_lo = ineq & np.isclose(zk, lq.l, rtol=0, atol=1e-12)
        inside = ineq & ~at_up & ~at_lo
        assert np.all(yk[at_up] >= -1e-12)
        assert np.all(yk[at_lo] <= 1e-12)
        assert np.all(np.abs(yk[inside]) <= 1e-9)


def test_kkt_solve_gives_z_tilde_equal_A_x_tilde():
    m, x0, qp = _agent_qp(3, 4)
    lq = osqp.literal_form(qp, rho=0.1)
    x, z, y = osqp.start_point(lq, qp, x0, m["q_nom"])
    tr = []
    osqp.iterate(lq, x, z, y, 5, trace=tr)
    for (xt, zt, _, _, _) in tr:
        assert np.abs(lq.A @ xt - zt).max() <= 1e-7 * (1.0 + np.abs(zt).max())


def test_ruiz_one_iteration_by_hand():
    # P = diag(4, 1), q = (2, 0), A = [[2, 0]]: KKT column norms (4, 1) of
    # the variables and 2 of the row, so D = (1/2, 1), E = 1/sqrt(2); then
    # P = diag(1, 1), q = (1, 0), A = [[1/sqrt(2), 0]]; the cost scale is
    # 1 / max(mean(1, 1), 1) = 1; bounds scale by E
    lq = osqp.LiteralQP(P=np.diag([4.0, 1.0]), q=np.array([2.0, 0.0]), A=np.array([[2.0, 0.0]]),
                        l=np.array([-1.0]), u=np.array([3.0]), rho=np.array([0.1]), n_dyn=0)
    sq, D, E, c = osqp.ruiz(lq, 1)
    r = 1.0 / np.sqrt(2.0)
    assert np.allclose(D, [0.5, 1.0], atol=1e-15) and np.allclose(E, [r], atol=1e-15) and c == 1.0
    assert np.allclose(sq.P, np.eye(2), atol=1e-15) and np.allclose(sq.q, [1.0, 0.0], atol=1e-15)
    assert np.allclose(sq.A, [[r, 0.0]], atol=1e-15)
    assert np.allclose([sq.l[0], sq.u[0]], [-r, 3 * r], atol=1e-15)


def test_ruiz_equilibrates_and_keeps_the_optimum():
    m, x0, qp = _agent_qp(5, 4)
    lq = osqp.literal_form(qp, rho=0.1)
    sq, D, E, c = osqp.ruiz(lq, 10)
    # the scaled KKT matrix's columns have inf-norms near 1 (the unscaled ones
    # spread over orders of magnitude)
    def spread(l):
        col = np.maximum(np.abs(l.P).max(axis=0), np.abs(l.A).max(axis=0))
        row = np.abs(l.A).max(axis=1)
        v = np.concatenate([col, row])
        return v.max() / v.min()
    assert spread(lq) > 100.0 and spread(sq) < 1.1
    # the scaled problem has the same optimum, mapped back by D
    x, z, y = osqp.start_point(lq, qp, x0, m["q_nom"])
    xs, zs, ys, it = osqp.solve_until(sq, x / D, E * z, np.zeros_like(y), eps_abs=1e-12, eps_rel=1e-12,
                                      max_iter=60000, check_every=50)
    ref = ipm.solve_qp(qp.P, qp.q, qp.E, qp.e, qp.C, qp.lo, qp.hi)
    scale = 1.0 + np.abs(ref.z).max()
    assert np.abs(D * xs - ref.z).max() <= 1e-7 * scale, (it, np.abs(D * xs - ref.z).max())
