"""Pins for the oracle's QP assembly and interior-point solve.

(i)  closed-form affine LQR when no inequality is active;
(ii) brute-force active-set enumeration on toy 2-stage QPs;
(iii) KKT invariants on solves of the generated workloads;
(iv) a standing agent whose optimum is the reference, with its torque
     worked by hand (paper Eqs. rnea, mpc_torque).
"""
import numpy as np
import pytest

from oracle import activeset, ipm, kkt, lqr, qp as qpmod, refs
from oracle.solve import agent_params, solve_agent
from workload import make_agents, gen


def _loose(m):
    m = dict(m)
    m["mu"], m["fz_max"], m["qd_max"], m["q_lim"] = 1e3, 1e6, 1e6, 1e6
    return m


@pytest.mark.parametrize("i,gait", [(0, gen.GAIT_STAND), (3, gen.GAIT_STAND),
                                    (5, gen.GAIT_WALK), (7, gen.GAIT_HOP)])
def test_ipm_matches_closed_form_lqr(i, gait):
    mm, inp = make_agents("small", [i])
    m = _loose(agent_params(mm, 0))
    period, duty, off = gen._GAIT_TABLE[gait]
    m["period"], m["duty"], m["offset"] = period, np.array(duty), np.array(off)
    x0 = inp["x0"][0]
    x0[6:12] *= 0.1          # small motion: f_z stays well inside its bounds
    cmd = inp["cmd"][0] * np.array([1, 0.1, 0.1, 0.1])
    out = solve_agent(m, x0, cmd, inp["phase"][0], inp["qd_meas"][0])
    ex = out["extras"]
    st = ex["stance"]
    # nothing but the swing-foot equalities may be active
    y = out["y"]
    for k in range(m["N"]):
        for f in range(2):
            if st[k, f]:
                assert np.all(np.abs(y[k, 6 * f:6 * f + 6]) < 1e-9)
    assert np.all(np.abs(y[:, 12:]) < 1e-9)
    fixed = np.zeros((m["N"], 30), dtype=bool)
    for k in range(m["N"]):
        for f in range(2):
            if not st[k, f]:
                fixed[k, 6 * f:6 * f + 6] = True
    dt = m["dt"]
    x, u = lqr.affine_lqr(ex["A"], ex["B"], ex["c"], 2 * dt * m["Q"], 2 * dt * m["R"],
                          x0, ex["x_ref"], ex["u_ref"], fixed)
    scale = 1.0 + np.abs(u).max()
    assert np.abs(out["u"] - u).max() <= 1e-9 * scale
    assert np.abs(out["x"] - x).max() <= 1e-9 * (1.0 + np.abs(x).max())


def _toy_qp(rng, N=2, nx=3, nu=2):
    """Random 2-stage toy MPC QP in the oracle's standard form."""
    n = N * (nx + nu)
    P = np.diag(rng.uniform(0.1, 2.0, n))
    q = rng.normal(size=n) * 3          # pulls the optimum onto some bounds
    E = np.zeros((N * nx, n))
    for k in range(N):
        bu, bx = k * (nx + nu), k * (nx + nu) + nu
        E[k * nx:(k + 1) * nx, bx:bx + nx] = np.eye(nx)
        E[k * nx:(k + 1) * nx, bu:bu + nu] = -rng.normal(size=(nx, nu))
        if k > 0:
            px = (k - 1) * (nx + nu) + nu
            E[k * nx:(k + 1) * nx, px:px + nx] = -rng.normal(size=(nx, nx)) * 0.5
    # feasible by construction: bounds bracket C z0 for a point z0 with E z0 = e
    z0 = rng.normal(size=n) * 0.3
    e = E @ z0
    m = 8
    C = rng.normal(size=(m, n))
    Cz0 = C @ z0
    lo = Cz0 - rng.uniform(0.05, 0.5, m)
    hi = Cz0 + rng.uniform(0.05, 0.5, m)
    lo[0] = -np.inf                       # one-sided rows
    hi[1] = np.inf
    lo[2] = hi[2] = Cz0[2]                # an equality row
    lo[3], hi[3] = -np.inf, np.inf        # a free row
    return P, q, E, e, C, lo, hi


@pytest.mark.parametrize("seed", range(12))
def test_ipm_matches_brute_force_active_set(seed):
    rng = np.random.default_rng(100 + seed)
    P, q, E, e, C, lo, hi = _toy_qp(rng)
    bf = activeset.brute_force_qp(P, q, E, e, C, lo, hi)
    assert bf is not None
    r = ipm.solve_qp(P, q, E, e, C, lo, hi)
    assert r.converged
    assert np.abs(r.z - bf[0]).max() <= 1e-8 * (1 + np.abs(bf[0]).max())
    # the toy problems do exercise active inequality rows
    if seed == 0:
        n_act = sum(1 for i in range(C.shape[0]) if bf[2][i] != 0)
        assert n_act >= 2


@pytest.mark.parametrize("name,i", [("small", 0), ("small", 4), ("small", 12),
                                    ("uneven", 3), ("uneven", 11), ("uneven", 40)])
def test_kkt_invariants_on_workload_solves(name, i):
    mm, inp = make_agents(name, [i])
    m = agent_params(mm, 0)
    out = solve_agent(m, inp["x0"][0], inp["cmd"][0], inp["phase"][0], inp["qd_meas"][0])
    qp = out["qp"]
    r = out["ipm"]
    assert r.converged
    km = kkt.kkt_measures(qp.P, qp.q, qp.E, qp.e, qp.C, qp.lo, qp.hi, r.z, r.nu, r.y)
    scale = 1.0 + np.abs(qp.q).max()
    assert km["stationarity"] <= 1e-8 * scale
    assert km["equality"] <= 1e-9
    assert km["violation"] <= 1e-9
    assert km["dual_sign"] <= 1e-9
    assert km["complementarity"] <= 1e-8


def test_standing_equilibrium_torque_by_hand():
    mm, inp = make_agents("small", [2])
    m = agent_params(mm, 0)
    period, duty, off = gen._GAIT_TABLE[gen.GAIT_STAND]
    m["period"], m["duty"], m["offset"] = period, np.array(duty), np.array(off)
    # symmetric levers: (r_L + r_R) is vertical, so (r_L + r_R) x (0,0,mg/2) = 0
    m["lever"] = np.array([[0.1, 0.07, -0.05], [-0.1, -0.07, 0.02]])
    x0 = np.zeros(30)
    x0[2] = 0.6
    x0[12:30] = m["q_nom"]
    cmd = (0.6, 0.0, 0.0, 0.0)
    out = solve_agent(m, x0, cmd, 0.25, np.zeros(18))
    W = 0.5 * m["mass"] * 9.81
    tau = m["h_j"].copy()
    for foot in range(2):
        for jj in range(5):
            tau[5 * foot + jj] -= m["J_leg"][foot][2][jj] * W
    assert np.allclose(out["u"][0, [2, 8]], W, atol=1e-8)
    assert np.allclose(out["tau"], tau, atol=1e-8)
    assert abs(out["V"]) < 1e-8


def test_feasibility_lp_on_a_textbook_pair():
    # x <= 0 and x >= 1 (no point), against 0 <= x <= 1 (a segment)
    from types import SimpleNamespace
    from oracle.feasibility import is_feasible
    bad = SimpleNamespace(C=np.array([[1.0], [1.0]]), lo=np.array([-np.inf, 1.0]), hi=np.array([0.0, np.inf]),
                          E=np.zeros((0, 1)), e=np.zeros(0))
    ok = SimpleNamespace(C=np.array([[1.0]]), lo=np.array([0.0]), hi=np.array([1.0]),
                         E=np.zeros((0, 1)), e=np.zeros(0))
    assert not is_feasible(bad)
    assert is_feasible(ok)


@pytest.mark.parametrize("i,joint,side", [(0, 0, 1.0), (2, 7, -1.0), (5, 17, 1.0)])
def test_feasibility_lp_matches_the_joint_reachability_bound(i, joint, side):
    # |q0_j| <= q_lim + dt qd_max is the exact first-stage reachability
    # condition; the LP over the whole horizon QP must flip at the same place
    from oracle.feasibility import is_feasible, joint_limits_reachable
    model, inp = make_agents("uneven", np.arange(8))
    m = agent_params(model, i)
    lim = float(m["q_lim"]) + float(m["dt"]) * float(m["qd_max"])
    for scale, want in ((0.999, True), (1.001, False)):
        x0 = np.array(inp["x0"][i], float)
        x0[12 + joint] = side * scale * lim
        qp, _ = qpmod.agent_qp(m, x0, inp["cmd"][i], float(inp["phase"][i]))
        assert joint_limits_reachable(m, x0) == want
        assert is_feasible(qp) == want, (scale, want)


@pytest.mark.parametrize("name", ["uneven", "mixed16k"])
def test_workload_agents_are_feasible(name):
    from oracle.feasibility import is_feasible
    model, inp = make_agents(name, np.arange(6))
    for i in range(6):
        m = agent_params(model, i)
        qp, _ = qpmod.agent_qp(m, np.asarray(inp["x0"][i], float), inp["cmd"][i], float(inp["phase"][i]))
        assert is_feasible(qp)
