"""Pins for the oracle's kinematic rows (oracle/refs.py kin_rows: the no-slip
and swing-height rows of Eq. mpc_formulation, the swing curve of Eqs.
bezier_1..5).

(i)   the quintic's control points by hand, and its five conditions plus the
      reading's sixth evaluated from the Bernstein form and by finite
      differences (not through the control-point formulas);
(ii)  a node's contact state and swing progress by hand;
(iii) the rows' values equal the foot's velocity and height computed from the
      model's lever r_i(q) by finite differences (pins the Jacobian's row and
      orientation, the velocity lanes and the ground reference);
(iv)  stage k's rows follow node k+1's contact state;
(v)   the interior-point optimum meets them (foot velocities and heights
      recomputed from r_i(q)), and the literal iteration converges to it.
"""
import math

import numpy as np
import pytest

from oracle import ipm, model as mdl, osqp, qp as qpmod, refs
from oracle.solve import agent_params
from workload import make_agents

KIN = dict(z_swing=0.075, v_to=0.1, v_td=-0.1)


def _b(t, b):
    return sum(math.comb(5, j) * t ** j * (1 - t) ** (5 - j) * b[j] for j in range(6))


def _db(t, b, h=1e-6):
    return (_b(t + h, b) - _b(t - h, b)) / (2 * h)


def test_bezier_points_by_hand():
    # symmetric: b1 = v_to / 5 = 0.1, b4 = -v_td / 5 = 0.1,
    # b2 + b3 = (3.2 - 0.5 - 0.5) / 10 = 0.22, b3 - b2 = 1.5 (b1 - b4) = 0
    assert np.allclose(refs.bezier_points(0.1, 0.5, -0.5), [0, 0.1, 0.11, 0.11, 0.1, 0], rtol=0, atol=1e-15)
    # B(0.25) = (405 b1 + 270 b2 + 90 b3 + 15 b4) / 1024 = 81.6 / 1024
    assert abs(refs.bezier(0.25, [0, 0.1, 0.11, 0.11, 0.1, 0]) - 81.6 / 1024) < 1e-15
    # asymmetric: b4 = 0.04, b2 + b3 = (3.2 - 0.5 - 0.2) / 10 = 0.25,
    # b3 - b2 = (3 b1 - 3 b4) / 2 = 0.09
    assert np.allclose(refs.bezier_points(0.1, 0.5, -0.2), [0, 0.1, 0.08, 0.17, 0.04, 0], rtol=0, atol=1e-15)


@pytest.mark.parametrize("z,vto,vtd", [(0.075, 0.1, -0.1), (0.15, 0.4, -0.05), (0.1, 0.0, 0.3)])
def test_bezier_conditions(z, vto, vtd):
    b = refs.bezier_points(z, vto, vtd)
    assert abs(_b(0.0, b)) < 1e-15 and abs(_b(1.0, b)) < 1e-15          # Eqs. bezier_1, 2
    assert abs(_b(0.5, b) - z) < 1e-15                                   # Eq. bezier_3
    assert abs((_b(1e-7, b) - _b(0.0, b)) / 1e-7 - vto) < 1e-5          # Eq. bezier_4
    assert abs((_b(1.0, b) - _b(1.0 - 1e-7, b)) / 1e-7 - vtd) < 1e-5    # Eq. bezier_5
    assert abs(_db(0.5, b)) < 1e-8                                       # the sixth condition
    for t in (0.1, 0.37, 0.8):
        assert abs(refs.bezier(t, b) - _b(t, b)) < 1e-15


def test_node_contact_by_hand():
    m = dict(dt=0.02, period=0.8, duty=[0.5, 0.5], offset=[0.0, 0.5])
    # node 5 from phase 0.3: phi = 0.3 + 5 * 0.025 = 0.425; foot 0 s = 0.425
    # (stance), foot 1 s = 0.925 (swing, t_sw = 0.425 / 0.5)
    st, tsw = refs.node_contact(m, 0.3, 5)
    assert st.tolist() == [True, False]
    assert tsw[0] == 0.0 and abs(tsw[1] - 0.85) < 1e-12
    # the schedule's own nodes agree
    m["N"] = 30
    sched = refs.contact_schedule(m, 0.3)
    for n in range(30):
        assert refs.node_contact(m, 0.3, n)[0].tolist() == sched[n].tolist()


def _agent(wl, i):
    mm, inp = make_agents(wl, [i])
    return agent_params(mm, 0), inp["x0"][0], inp["cmd"][0], inp["phase"][0]


def test_rows_are_foot_velocity_and_height():
    m, x0, cmd, ph = _agent("uneven", 3)
    g = np.random.default_rng(7)
    x = g.normal(size=30)
    u = g.normal(size=30)
    for k in range(int(m["N"])):
        Cu, Cx, lo, hi = refs.kin_rows(m, cmd, ph, k, KIN)
        st, tsw = refs.node_contact(m, ph, k + 1)
        val = Cu @ u + Cx @ x
        for i in range(2):
            # foot position p + r_i(q) moved along (v, joint rates u[12:30])
            h = 1e-6
            pos = lambda t: x[0:3] + t * x[6:9] + mdl.foot_lever(m, x[12:30] + t * u[12:30], i)
            vel = (pos(h) - pos(-h)) / (2 * h)
            assert np.allclose(val[3 * i:3 * i + 3], vel, rtol=0, atol=1e-8)
            height = x[2] + mdl.foot_lever(m, x[12:30], i)[2] - m["lever"][i][2]
            jz_qnom = np.asarray(m["J_leg"][i][2]) @ np.asarray(m["q_nom"][5 * i:5 * i + 5])
            assert abs(val[6 + i] - jz_qnom - height) < 1e-12
            if st[i]:
                assert (lo[3 * i:3 * i + 3] == 0).all() and (hi[3 * i:3 * i + 3] == 0).all()
                assert lo[6 + i] == -np.inf and hi[6 + i] == np.inf
            else:
                assert (lo[3 * i:3 * i + 3] == -np.inf).all() and (hi[3 * i:3 * i + 3] == np.inf).all()
                b = refs.bezier_points(KIN["z_swing"], KIN["v_to"], KIN["v_td"])
                assert lo[6 + i] == hi[6 + i]
                assert abs(hi[6 + i] - jz_qnom - (cmd[0] + _b(tsw[i], b))) < 1e-12


def test_stage_rows_follow_the_next_node():
    # find a stage whose foot changes contact between nodes k and k+1
    for i in range(12):
        m, x0, cmd, ph = _agent("uneven", i)
        N = int(m["N"])
        for k in range(N - 1):
            a = refs.node_contact(m, ph, k)[0]
            b = refs.node_contact(m, ph, k + 1)[0]
            if (a != b).any():
                _, _, lo, hi = refs.kin_rows(m, cmd, ph, k, KIN)
                for f in range(2):
                    assert (lo[3 * f] == 0.0) == bool(b[f])
                    assert np.isfinite(lo[6 + f]) == (not b[f])
                return
    pytest.fail("no contact change in the sample")


@pytest.mark.parametrize("i", [3, 7])
def test_optimum_meets_the_rows_and_is_the_literal_fixed_point(i):
    m, x0, cmd, ph = _agent("uneven", i)
    m["N"] = 5
    qp, ex = qpmod.agent_qp(m, x0, cmd, ph, kin=KIN)
    r = ipm.solve_qp(qp.P, qp.q, qp.E, qp.e, qp.C, qp.lo, qp.hi)
    assert r.converged
    b = refs.bezier_points(KIN["z_swing"], KIN["v_to"], KIN["v_td"])
    n_st = n_sw = 0
    for k in range(qp.N):
        u, x = qp.u(r.z, k), qp.x(r.z, k + 1)
        st, tsw = refs.node_contact(m, ph, k + 1)
        for f in range(2):
            if st[f]:
                h = 1e-6
                pos = lambda t: x[0:3] + t * x[6:9] + mdl.foot_lever(m, x[12:30] + t * u[12:30], f)
                assert np.abs((pos(h) - pos(-h)) / (2 * h)).max() < 1e-7
                n_st += 1
            else:
                height = x[2] + mdl.foot_lever(m, x[12:30], f)[2] - m["lever"][f][2]
                assert abs(height - cmd[0] - _b(tsw[f], b)) < 1e-8
                n_sw += 1
    assert n_st > 0 and n_sw > 0
    lq = osqp.literal_form(qp, rho=0.1)
    xx, z, y = osqp.start_point(lq, qp, x0, m["q_nom"])
    xx, z, y, it = osqp.solve_until(lq, xx, z, y, eps_abs=1e-11, eps_rel=1e-11, max_iter=60000, check_every=50)
    assert np.abs(xx - r.z).max() <= 1e-7 * (1.0 + np.abs(r.z).max()), it
