"""Pins for the oracle's ADMM with exact dynamics in the x-update
(oracle/admm.py: the iteration of the Riccati forms and of the paper's
fixed-N_QP mode; Alg. 1, Sec. III-B, OSQP's update steps).

(i)   two iterations of a two-variable problem worked by hand, and its limit;
(ii)  every x-update meets the dynamics exactly (E z~ = e);
(iii) the multipliers stay in the normal cone of their bounds;
(iv)  the fixed point is the interior-point optimum on horizon QPs of the
      workload.
"""
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import admm, ipm, qp as qpmod
from oracle.solve import agent_params
from workload import make_agents


def _toy():
    # minimise u^2 + x^2 subject to x = u + 1 (E = [-1, 1], e = 1) and
    # 0 <= u <= 0.25 (C = [1, 0]); z = (u, x)
    return SimpleNamespace(P=np.diag([2.0, 2.0]), q=np.zeros(2), E=np.array([[-1.0, 1.0]]), e=np.array([1.0]),
                           C=np.array([[1.0, 0.0]]), lo=np.array([0.0]), hi=np.array([0.25]), N=1)


def test_two_iterations_by_hand():
    # rho = sigma = alpha = 1.  Iteration 1 from z = w = y = 0:
    #   4u - nu = 0, 3x + nu = 0, x - u = 1  ->  u~ = -3/7, x~ = 4/7;
    #   w~ = -3/7; w = clip(-3/7, 0, 0.25) = 0; y = -3/7.
    # Iteration 2: rhs (sigma u + (rho w - y), sigma x) = (0, 4/7):
    #   4u - nu = 0, 3x + nu = 4/7, x - u = 1  ->  u~ = -17/49, x~ = 32/49;
    #   w = clip(-17/49 - 3/7) = 0; y = -3/7 - 17/49 = -38/49.
    t = _toy()
    tr = []
    admm.iterate(t, np.zeros(2), np.zeros(1), np.zeros(1), 2, rho=1.0, sigma=1.0, alpha=1.0, trace=tr)
    (zt1, wt1, z1, w1, y1), (zt2, wt2, z2, w2, y2) = tr
    assert np.allclose(zt1, [-3 / 7, 4 / 7], rtol=0, atol=1e-15) and np.allclose(wt1, [-3 / 7], atol=1e-15)
    assert np.allclose(w1, [0.0], atol=0) and np.allclose(y1, [-3 / 7], atol=1e-15)
    assert np.allclose(zt2, [-17 / 49, 32 / 49], rtol=0, atol=1e-15)
    assert np.allclose(w2, [0.0], atol=0) and np.allclose(y2, [-38 / 49], atol=1e-15)
    # the limit: u = 0 on its lower bound, x = 1, and stationarity
    # 2u + 2x + y = 0 gives y = -2
    z, w, y = admm.iterate(t, np.zeros(2), np.zeros(1), np.zeros(1), 400, rho=1.0, sigma=1.0, alpha=1.6)
    assert np.allclose(z, [0.0, 1.0], atol=1e-12) and abs(y[0] + 2.0) < 1e-12


def test_rho_eq_on_equality_rows_and_free_rows_dropped():
    t = _toy()
    t.C = np.array([[1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    t.lo = np.array([0.0, 0.5, -np.inf])
    t.hi = np.array([0.25, 0.5, np.inf])
    keep, rr = admm.row_steps(t, 0.1)
    assert keep.tolist() == [True, True, False]
    assert np.allclose(rr, [0.1, 100.0], rtol=1e-15)


def _agent_qp(i, N):
    mm, inp = make_agents("uneven", [i])
    m = agent_params(mm, 0)
    m["N"] = N
    x0 = inp["x0"][0]
    qp, _ = qpmod.agent_qp(m, x0, inp["cmd"][0], inp["phase"][0])
    return m, x0, qp


def test_dynamics_exact_and_normal_cone():
    m, x0, qp = _agent_qp(7, 5)
    z, w, y = admm.start_point(qp, x0, m["q_nom"])
    tr = []
    admm.iterate(qp, z, w, y, 30, trace=tr)
    keep, _ = admm.row_steps(qp, 0.1)
    lo, hi = qp.lo[keep], qp.hi[keep]
    ineq = lo != hi
    for (zt, _, _, wk, yk) in tr:
        assert np.abs(qp.E @ zt - qp.e).max() <= 1e-9 * (1.0 + np.abs(qp.e).max())
        at_up = ineq & np.isclose(wk, hi, rtol=0, atol=1e-12)
        at_lo = ineq & np.isclose(wk, lo, rtol=0, atol=1e-12)
        inside = ineq & ~at_up & ~at_lo
        assert np.all(yk[at_up] >= -1e-12) and np.all(yk[at_lo] <= 1e-12)
        assert np.all(np.abs(yk[inside]) <= 1e-9)


@pytest.mark.parametrize("i,N", [(0, 3), (5, 4), (11, 3)])
def test_fixed_point_is_the_interior_point_optimum(i, N):
    m, x0, qp = _agent_qp(i, N)
    z, w, y = admm.start_point(qp, x0, m["q_nom"])
    z, w, y = admm.iterate(qp, z, w, y, 40000)
    ref = ipm.solve_qp(qp.P, qp.q, qp.E, qp.e, qp.C, qp.lo, qp.hi)
    assert ref.converged
    assert np.abs(z - ref.z).max() <= 1e-7 * (1.0 + np.abs(ref.z).max()), np.abs(z - ref.z).max()
