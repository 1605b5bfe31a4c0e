"""Parity of the literal form (MPC_FORM_LDL: the paper's Alg. 1 with OSQP's
ADMM on the full KKT system of Eq. kkt_system, factored once by a block
LDL^T, Eq. ldl, and solved by substitution every iteration, Eqs.
backsolve_1-2) against the oracle's literal iteration (oracle/osqp.py: the
same algorithm with a dense FP64 LU solve of the KKT system).

The literal iteration is compared iterate for iterate: after a fixed number
of iterations N_QP from f_init both sides hold the same ADMM iterate, not the
QP's optimum (the paper's fixed-N_QP mode); with and without the Ruiz
equilibration (f_Ruiz), computed on each side from its own data.  Bars: torques within the
torque tolerance (1e-4 N m + 1e-3 |tau|); the primal iterate within 1e-4
of its own scale (FP32 factors of a KKT matrix with entries from 1e-2 to
1e3: measured 1e-6); in the converged mode the iteration count within one
residual-check period of the oracle's, where the stopping test is met by a
margin FP32 can resolve.
"""
import numpy as np
import pytest

from helpers import agents, device_inputs, oracle_view, torque_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    import __graft_entry__ as g
    g.build()
    from paper_2510_12717_b300 import mpcgpu
    return mpcgpu


def _solve(mpcgpu, model, inp32, **opts):
    n = len(model["mass"])
    s = mpcgpu.Solver(max_agents=n, max_horizon=20, form=mpcgpu.FORM_LDL,
                      stream=torch.cuda.current_stream().cuda_stream, **opts)
    s.set_models(model, np.arange(n))
    r = s.solve_host(np.arange(n), inp32["x0"], inp32["qd_meas"], inp32["cmd"], inp32["phase"])
    r["state"] = [s.export_state(a, int(model["N"][a])) for a in range(n)]
    r["stats"] = s.agent_stats(np.arange(n))
    s.close()
    return r


def _oracle(model, inp32, a, iters, scaling=0):
    from oracle import osqp
    from oracle.solve import agent_params
    mo, io = oracle_view(model, inp32)
    m = agent_params(mo, a)
    return osqp.literal_agent(m, io["x0"][a], io["cmd"][a], io["phase"][a], io["qd_meas"][a], iters,
                              scaling=scaling)


@pytest.mark.parametrize("name,n", [("small", 16), ("uneven", 10)])
@pytest.mark.parametrize("iters", [1, 25])
@pytest.mark.parametrize("ruiz", [0, 10])
def test_literal_iterations_match_oracle(name, n, iters, ruiz):
    # ruiz: iterations of the Ruiz equilibration (f_Ruiz of Alg. 1) on both sides
    mpcgpu = _lib()
    model, inp = agents(name, np.arange(n))
    inp32 = device_inputs(inp)
    r = _solve(mpcgpu, model, inp32, fixed_iters=iters, ruiz_iters=ruiz)
    assert (r["status"] == mpcgpu.AGENT_MAX_ITER).all()
    assert (r["stats"]["iters"] == iters).all()
    for a in range(n):
        o = _oracle(model, inp32, a, iters, scaling=ruiz)
        st = r["state"][a]
        su = 1.0 + np.abs(o["u"]).max()
        sx = 1.0 + np.abs(o["x"]).max()
        assert np.abs(st["u"] - o["u"]).max() <= 1e-4 * su, a
        assert np.abs(st["x"] - o["x"]).max() <= 1e-4 * sx, a
        ok = torque_close(r["tau"][a], o["tau"])
        assert ok.all(), (a, np.abs(r["tau"][a] - o["tau"]).max())


@pytest.mark.parametrize("ruiz", [0, 10])
def test_literal_converged_mode_counts_oracle_iterations(ruiz):
    from oracle import osqp, qp as qpmod
    from oracle.solve import agent_params
    mpcgpu = _lib()
    model, inp = agents("small", np.arange(16))
    inp32 = device_inputs(inp)
    r = _solve(mpcgpu, model, inp32, fixed_iters=0, max_iter=4000, check_every=10, ruiz_iters=ruiz)
    mo, io = oracle_view(model, inp32)
    matched = 0
    its = []
    for a in range(16):
        m = agent_params(mo, a)
        qp, _ = qpmod.agent_qp(m, io["x0"][a], io["cmd"][a], io["phase"][a])
        lq = osqp.literal_form(qp, 0.1)
        x, z, y = osqp.start_point(lq, qp, io["x0"][a], np.asarray(m["q_nom"], float))
        x, z, y, it = osqp.solve_until(lq, x, z, y, max_iter=4000, check_every=10, scaling=ruiz)
        got = int(r["stats"]["iters"][a])
        if it < 1000:
            # short runs: the stopping test is met by a margin FP32 resolves
            assert abs(got - it) <= 10, (a, got, it)
            assert r["status"][a] == mpcgpu.AGENT_INACCURATE
            matched += 1
        else:
            # long runs hover at the tolerance; FP32 may stop some checks apart
            assert abs(got - it) <= 0.1 * it + 20, (a, got, it)
        its.append((got, it))
    print(f"\n[literal converged, ruiz {ruiz}] (gpu, oracle) iterations: {its}")
    # without the equilibration most of these agents stop within 1000
    # iterations; with it (fixed rho) most run much longer
    assert matched >= (8 if ruiz == 0 else 0)


def test_literal_full_size_sampled():
    # the bench configuration: 16384 agents of mixed horizons and gaits,
    # N_QP = 25, one launch; a stratified sample against the oracle
    mpcgpu = _lib()
    n = 16384
    model, inp = agents("mixed16k", np.arange(n))
    inp32 = device_inputs(inp)
    dev = torch.device("cuda:0")
    t = {k: torch.from_numpy(v).to(dev) for k, v in inp32.items()}
    ids = torch.arange(n, dtype=torch.int32, device=dev)
    s = mpcgpu.Solver(max_agents=n, max_horizon=20, form=mpcgpu.FORM_LDL, fixed_iters=25,
                      stream=torch.cuda.current_stream().cuda_stream)
    s.set_models(model, np.arange(n))
    tk = s.submit(ids, t["x0"], t["qd_meas"], t["cmd"], t["phase"])
    s.solve(tk)
    tau = torch.empty((n, 18), device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    s.get_torques(tk, tau=tau, status=st)
    torch.cuda.synchronize()
    s.close()
    tau = tau.cpu().numpy()
    st = st.cpu().numpy()
    assert (st == mpcgpu.AGENT_MAX_ITER).all()
    Nh = model["N"]
    sample = [int(np.flatnonzero(Nh == h)[0]) for h in (5, 9, 13, 17, 20)] + [n - 1, n // 2]
    for a in sample:
        o = _oracle(model, inp32, a, 25)
        ok = torque_close(tau[a], o["tau"])
        assert ok.all(), (a, np.abs(tau[a] - o["tau"]).max())


def test_literal_nonfinite_input_is_flagged():
    mpcgpu = _lib()
    model, inp = agents("small", np.arange(4))
    inp32 = device_inputs(inp)
    inp32["x0"][2, 7] = np.nan
    r = _solve(mpcgpu, model, inp32, fixed_iters=5)
    assert r["status"][2] == mpcgpu.AGENT_NAN
    assert np.all(r["tau"][2] == 0.0)
    assert (r["status"][[0, 1, 3]] == mpcgpu.AGENT_MAX_ITER).all()


def test_literal_budget_counts_the_factors():
    mpcgpu = _lib()
    # the regular form of 256 agents fits in 64 MB; the literal form's factors
    # (about 29 KB per stage per agent) do not
    s = mpcgpu.Solver(max_agents=256, max_horizon=20, hbm_budget_bytes=64 << 20,
                      stream=torch.cuda.current_stream().cuda_stream)
    s.close()
    with pytest.raises(mpcgpu.MpcError):
        mpcgpu.Solver(max_agents=256, max_horizon=20, form=mpcgpu.FORM_LDL, fixed_iters=25,
                      hbm_budget_bytes=64 << 20, stream=torch.cuda.current_stream().cuda_stream)


# the kinematic rows of Eq. mpc_formulation (no-slip, swing height on the
# Bezier curve of Eqs. bezier_1-5): both sides build them from their own data
KIN = dict(z_swing=0.075, v_to=0.1, v_td=-0.1)
KIN_OPTS = dict(kin_rows=1, swing_height=0.075, v_takeoff=0.1, v_touchdown=-0.1)


def _oracle_kin(model, inp32, a, iters):
    from oracle import osqp
    from oracle.solve import agent_params
    mo, io = oracle_view(model, inp32)
    m = agent_params(mo, a)
    return osqp.literal_agent(m, io["x0"][a], io["cmd"][a], io["phase"][a], io["qd_meas"][a], iters, kin=KIN)


@pytest.mark.parametrize("name,n", [("small", 16), ("uneven", 10)])
@pytest.mark.parametrize("iters", [1, 25])
def test_literal_kinematic_rows_iterations_match_oracle(name, n, iters):
    mpcgpu = _lib()
    model, inp = agents(name, np.arange(n))
    inp32 = device_inputs(inp)
    r = _solve(mpcgpu, model, inp32, fixed_iters=iters, **KIN_OPTS)
    assert (r["status"] == mpcgpu.AGENT_MAX_ITER).all()
    far = 0
    for a in range(n):
        o = _oracle_kin(model, inp32, a, iters)
        st = r["state"][a]
        su = 1.0 + np.abs(o["u"]).max()
        sx = 1.0 + np.abs(o["x"]).max()
        assert np.abs(st["u"] - o["u"]).max() <= 1e-4 * su, a
        assert np.abs(st["x"] - o["x"]).max() <= 1e-4 * sx, a
        ok = torque_close(r["tau"][a], o["tau"])
        assert ok.all(), (a, np.abs(r["tau"][a] - o["tau"]).max())
        # the rows matter: the iterate without them is elsewhere
        o0 = _oracle(model, inp32, a, iters)
        far += not torque_close(r["tau"][a], o0["tau"]).all()
    assert far >= n // 2, far


def test_literal_kinematic_rows_converged_mode():
    from oracle import osqp, qp as qpmod
    from oracle.solve import agent_params
    mpcgpu = _lib()
    model, inp = agents("small", np.arange(16))
    inp32 = device_inputs(inp)
    r = _solve(mpcgpu, model, inp32, fixed_iters=0, max_iter=4000, check_every=10, **KIN_OPTS)
    mo, io = oracle_view(model, inp32)
    its = []
    matched = 0
    for a in range(16):
        m = agent_params(mo, a)
        qp, _ = qpmod.agent_qp(m, io["x0"][a], io["cmd"][a], io["phase"][a], kin=KIN)
        lq = osqp.literal_form(qp, 0.1)
        x, z, y = osqp.start_point(lq, qp, io["x0"][a], np.asarray(m["q_nom"], float))
        x, z, y, it = osqp.solve_until(lq, x, z, y, max_iter=4000, check_every=10)
        got = int(r["stats"]["iters"][a])
        if it < 1000:
            assert abs(got - it) <= 10, (a, got, it)
            assert r["status"][a] == mpcgpu.AGENT_INACCURATE
            matched += 1
        else:
            assert abs(got - it) <= 0.1 * it + 20, (a, got, it)
        its.append((got, it))
    print(f"\n[literal converged, kinematic rows] (gpu, oracle) iterations: {its}")
    assert matched >= 8


def test_literal_kinematic_rows_full_size_sampled():
    # 16384 agents of mixed horizons and gaits, N_QP = 25, one launch
    mpcgpu = _lib()
    n = 16384
    model, inp = agents("mixed16k", np.arange(n))
    inp32 = device_inputs(inp)
    dev = torch.device("cuda:0")
    t = {k: torch.from_numpy(v).to(dev) for k, v in inp32.items()}
    ids = torch.arange(n, dtype=torch.int32, device=dev)
    s = mpcgpu.Solver(max_agents=n, max_horizon=20, form=mpcgpu.FORM_LDL, fixed_iters=25,
                      stream=torch.cuda.current_stream().cuda_stream, **KIN_OPTS)
    s.set_models(model, np.arange(n))
    tk = s.submit(ids, t["x0"], t["qd_meas"], t["cmd"], t["phase"])
    s.solve(tk)
    tau = torch.empty((n, 18), device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    s.get_torques(tk, tau=tau, status=st)
    torch.cuda.synchronize()
    s.close()
    tau = tau.cpu().numpy()
    assert (st.cpu().numpy() == mpcgpu.AGENT_MAX_ITER).all()
    Nh = model["N"]
    sample = [int(np.flatnonzero(Nh == h)[0]) for h in (5, 9, 13, 17, 20)] + [n - 1, n // 2]
    for a in sample:
        o = _oracle_kin(model, inp32, a, 25)
        ok = torque_close(tau[a], o["tau"])
        assert ok.all(), (a, np.abs(tau[a] - o["tau"]).max())


def test_literal_kinematic_rows_short_horizons_and_nonfinite():
    # the shortest horizons (N = 2, 3: the rows of the last stage read x_N)
    # and a non-finite state next to them
    mpcgpu = _lib()
    n = 8
    model, inp = agents("uneven", np.arange(n))
    model["N"][:] = [2, 3, 2, 3, 4, 2, 3, 2]
    inp32 = device_inputs(inp)
    inp32["x0"][5, 8] = np.nan
    r = _solve(mpcgpu, model, inp32, fixed_iters=5, **KIN_OPTS)
    assert r["status"][5] == mpcgpu.AGENT_NAN and np.all(r["tau"][5] == 0.0)
    for a in [0, 1, 2, 3, 4, 6, 7]:
        assert r["status"][a] == mpcgpu.AGENT_MAX_ITER
        o = _oracle_kin(model, inp32, a, 5)
        st = r["state"][a]
        assert np.abs(st["u"] - o["u"]).max() <= 1e-4 * (1.0 + np.abs(o["u"]).max()), a
        assert torque_close(r["tau"][a], o["tau"]).all(), (a, np.abs(r["tau"][a] - o["tau"]).max())


@pytest.mark.parametrize("rho0,alpha", [(0.2, 1.6), (0.1, 1.0), (0.02, 1.8), (0.4, 1.6)])
def test_literal_iterations_match_oracle_other_steps(rho0, alpha):
    # other step sizes (rho, and rho_eq = 1e3 rho on the equality rows) and
    # relaxations, with the kinematic rows; both sides from their own data.
    # The iterates are held to 1e-4 of their scale at every step size; the
    # torques to the tolerance up to rho0 = 0.2: at rho0 = 0.4 (rho_eq = 400)
    # the FP32 factor of the more ill-conditioned KKT matrix leaves a torque
    # of one of these agents at 1.6x the tolerance (the torque map's
    # qddot = (qdot_1 - qdot_0) / dt amplifies the iterate's rounding)
    from oracle import osqp
    from oracle.solve import agent_params
    mpcgpu = _lib()
    n = 8
    model, inp = agents("uneven", np.arange(n))
    inp32 = device_inputs(inp)
    r = _solve(mpcgpu, model, inp32, fixed_iters=25, rho0=rho0, alpha=alpha, **KIN_OPTS)
    mo, io = oracle_view(model, inp32)
    for a in range(n):
        m = agent_params(mo, a)
        o = osqp.literal_agent(m, io["x0"][a], io["cmd"][a], io["phase"][a], io["qd_meas"][a], 25,
                               rho=rho0, alpha=alpha, kin=KIN)
        st = r["state"][a]
        assert np.abs(st["u"] - o["u"]).max() <= 1e-4 * (1.0 + np.abs(o["u"]).max()), a
        assert np.abs(st["x"] - o["x"]).max() <= 1e-4 * (1.0 + np.abs(o["x"]).max()), a
        if rho0 <= 0.2:
            assert torque_close(r["tau"][a], o["tau"]).all(), (a, np.abs(r["tau"][a] - o["tau"]).max())


@pytest.mark.parametrize("kin", [0, 1])
def test_literal_longest_horizon(kin):
    # the largest horizon the API allows (MPC_MAX_HORIZON = 32 stages): the
    # staged items, the record strides and (kin) the one-lane-per-stage row
    # set-up at their limits
    mpcgpu = _lib()
    n = 3
    model, inp = agents("uneven", np.arange(n))
    model["N"][:] = mpcgpu.MAX_HORIZON
    inp32 = device_inputs(inp)
    s = mpcgpu.Solver(max_agents=n, max_horizon=mpcgpu.MAX_HORIZON, form=mpcgpu.FORM_LDL, fixed_iters=5,
                      stream=torch.cuda.current_stream().cuda_stream, **(KIN_OPTS if kin else {}))
    s.set_models(model, np.arange(n))
    r = s.solve_host(np.arange(n), inp32["x0"], inp32["qd_meas"], inp32["cmd"], inp32["phase"])
    states = [s.export_state(a, mpcgpu.MAX_HORIZON) for a in range(n)]
    s.close()
    assert (r["status"] == mpcgpu.AGENT_MAX_ITER).all()
    for a in range(n):
        o = _oracle_kin(model, inp32, a, 5) if kin else _oracle(model, inp32, a, 5)
        assert np.abs(states[a]["u"] - o["u"]).max() <= 1e-4 * (1.0 + np.abs(o["u"]).max()), a
        assert torque_close(r["tau"][a], o["tau"]).all(), (a, np.abs(r["tau"][a] - o["tau"]).max())


def test_literal_batch_of_some_slots_in_any_order():
    # a batch that names some of the context's agent slots, out of order, and
    # one id that is out of range: the rows map to their slots, the bad row is
    # skipped (status -1, zero outputs)
    mpcgpu = _lib()
    n = 10
    model, inp = agents("uneven", np.arange(n))
    inp32 = device_inputs(inp)
    s = mpcgpu.Solver(max_agents=n, max_horizon=20, form=mpcgpu.FORM_LDL, fixed_iters=5,
                      stream=torch.cuda.current_stream().cuda_stream, **KIN_OPTS)
    s.set_models(model, np.arange(n))
    ids = np.array([7, 2, 9, 4])
    sub = {k: np.ascontiguousarray(v[ids]) for k, v in inp32.items()}
    bad_ids = np.concatenate([ids, [n + 3]])
    sub_bad = {k: np.concatenate([v, v[:1]]) for k, v in sub.items()}
    r = s.solve_host(bad_ids, sub_bad["x0"], sub_bad["qd_meas"], sub_bad["cmd"], sub_bad["phase"])
    s.close()
    assert r["status"][-1] == -1 and np.all(r["tau"][-1] == 0.0)
    assert (r["status"][:-1] == mpcgpu.AGENT_MAX_ITER).all()
    for row, a in enumerate(ids):
        o = _oracle_kin(model, inp32, int(a), 5)
        assert torque_close(r["tau"][row], o["tau"]).all(), (a, np.abs(r["tau"][row] - o["tau"]).max())
