"""System behaviour of the batching form on the GPU: CUDA-graph replay,
concurrent batches on two streams, the autotuner."""
import numpy as np
import pytest

from helpers import agents, device_inputs, torque_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpcgpu():
    import __graft_entry__ as g
    g.build()
    from paper_2510_12717_b300 import mpcgpu as m
    m.load()
    return m


def _dev(inp32):
    return {k: torch.from_numpy(v).to("cuda:0") for k, v in inp32.items()}


def _solve(s, ids_d, t, n, stream=None):
    tk = s.submit(ids_d, t["x0"], t["qd_meas"], t["cmd"], t["phase"])
    s.solve(tk, stream=stream)
    tau = torch.empty((n, 18), device="cuda:0")
    st = torch.empty(n, dtype=torch.int32, device="cuda:0")
    s.get_torques(tk, tau=tau, status=st)
    return tau, st


def test_graph_replay_is_bitwise_equal(mpcgpu):
    ids = np.arange(64)
    model, inp = agents("uneven", ids)
    t = _dev(device_inputs(inp))
    ids_d = torch.from_numpy(ids.astype(np.int32)).cuda()
    side = torch.cuda.Stream()          # graphs are captured on a non-default stream
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        cs = side.cuda_stream
        ref = mpcgpu.Solver(max_agents=64, max_horizon=20, stream=cs, warm_start=0)
        ref.set_models(model, ids)
        r0 = ref.stats()["kernel_launches"]
        tau0, st0 = _solve(ref, ids_d, t, 64)
        per_solve = ref.stats()["kernel_launches"] - r0
        g = mpcgpu.Solver(max_agents=64, max_horizon=20, stream=cs, warm_start=0, graph=1)
        g.set_models(model, ids)
        outs = [_solve(g, ids_d, t, 64) for _ in range(2)]    # capture, then a replay
        l0 = g.stats()["kernel_launches"]
        outs.append(_solve(g, ids_d, t, 64))                  # a second replay
        replay_launches = g.stats()["kernel_launches"] - l0
    torch.cuda.synchronize()
    assert g.stats()["graph_replays"] == 2
    assert replay_launches == per_solve >= 4   # the replay counts every kernel the graph holds
    for tau, st in outs:
        assert torch.equal(tau, tau0) and torch.equal(st, st0)
    ref.close(); g.close()


def test_two_streams_match_sequential(mpcgpu):
    ids = np.arange(96)
    model, inp = agents("uneven", ids)
    inp32 = device_inputs(inp)
    cs = torch.cuda.current_stream().cuda_stream
    seq = mpcgpu.Solver(max_agents=96, max_horizon=20, stream=cs, warm_start=0)
    seq.set_models(model, ids)
    ids_d = torch.from_numpy(ids.astype(np.int32)).cuda()
    tau_seq, _ = _solve(seq, ids_d, _dev(inp32), 96)
    torch.cuda.synchronize()
    par = mpcgpu.Solver(max_agents=96, max_horizon=20, stream=cs, warm_start=0)
    par.set_models(model, ids)
    halves = [np.arange(0, 48), np.arange(48, 96)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    res = []
    torch.cuda.synchronize()
    for h, sm in zip(halves, streams):
        part = {k: v[h] for k, v in inp32.items()}
        with torch.cuda.stream(sm):
            t = _dev(part)
            hid = torch.from_numpy(h.astype(np.int32)).cuda()
            sm.synchronize()
            res.append(_solve(par, hid, t, len(h), stream=sm.cuda_stream))
    torch.cuda.synchronize()
    got = torch.cat([r[0] for r in res]).cpu().numpy()
    assert np.array_equal(got, tau_seq.cpu().numpy())
    seq.close(); par.close()


def test_autotune_picks_a_solving_configuration(mpcgpu):
    ids = np.arange(256)
    model, inp = agents("uneven", ids)
    inp32 = device_inputs(inp)
    t = _dev(inp32)
    ids_d = torch.from_numpy(ids.astype(np.int32)).cuda()
    s = mpcgpu.Solver(max_agents=256, max_horizon=20, stream=torch.cuda.current_stream().cuda_stream)
    s.set_models(model, ids)
    tk = s.submit(ids_d, t["x0"], t["qd_meas"], t["cmd"], t["phase"])
    rep = s.autotune(tk, repeats=1)
    # shape stage (variant x resident blocks per SM: 2 + 3) then schedule stage (2 x 3)
    assert len(rep["candidates"]) == 11
    ch = rep["chosen"]
    assert rep["key"]["size_bin"] == 8 and len(rep["table"]) == 1      # 256 agents: floor(log2) = 8
    assert abs(rep["key"]["mean_horizon"] - model["N"].mean()) <= 0.005      # reported to 2 decimals
    assert rep["table"][0]["grid_per_sm"] == ch["grid_per_sm"]
    assert s.stats()["variant"] == ch["variant"] and s.stats()["check_every"] == ch["check_every"]
    s.solve(tk)
    tau = torch.empty((256, 18), device="cuda:0")
    st = torch.empty(256, dtype=torch.int32, device="cuda:0")
    s.get_torques(tk, tau=tau, status=st)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    # the tuned configuration reaches the same optimum as the default one
    ref = mpcgpu.Solver(max_agents=256, max_horizon=20, stream=torch.cuda.current_stream().cuda_stream)
    ref.set_models(model, ids)
    r = ref.solve_host(ids, inp32["x0"], inp32["qd_meas"], inp32["cmd"], inp32["phase"])
    assert torque_close(tau.cpu().numpy(), r["tau"]).all()
    s.close(); ref.close()


def test_polish_attempt_histogram(mpcgpu):
    # the context's histogram of accepted-polish solve counts covers every
    # live agent, agrees with the per-agent outcome, and most warm agents
    # need one solve
    ids = np.arange(64)
    model, _ = agents("uneven", ids)
    s = mpcgpu.Solver(max_agents=64, max_horizon=20, stream=torch.cuda.current_stream().cuda_stream)
    s.set_models(model, ids)
    for replan in (0, 1):
        _, inp = agents("uneven", ids, replan=replan)
        inp32 = device_inputs(inp)
        s.solve_host(ids.astype(np.int32), inp32["x0"], inp32["qd_meas"], inp32["cmd"], inp32["phase"])
        hist = s.stats()["polish_attempts"]
        st = s.agent_stats(ids.astype(np.int32))
        assert len(hist) == 9 and sum(hist) == 64
        assert hist[0] == int((st["polished"] == 0).sum())
    assert hist[1] >= 0.75 * 64
    s.close()


def test_async_model_upload_equals_sync(mpcgpu):
    # mpc_set_models_async on a stream of its own, ordered before the solve
    # by waiting on that stream: the same models as mpc_set_models, so the
    # same torques, bit for bit; a swap replaces an agent's model either way
    from workload import make_agents
    n = 24
    ids = np.arange(n)
    model, inp = make_agents("uneven", ids)
    other, _ = make_agents("uneven", np.arange(100, 100 + n))
    f32 = {k: np.ascontiguousarray(v, np.float32) for k, v in inp.items()}
    cur = torch.cuda.current_stream().cuda_stream
    side = torch.cuda.Stream()
    a = mpcgpu.Solver(max_agents=n, max_horizon=20, stream=cur)
    b = mpcgpu.Solver(max_agents=n, max_horizon=20, stream=cur)
    a.set_models(other, ids)
    a.set_models(model, ids)
    b.set_models(other, ids)
    b.set_models_async(model, ids, side.cuda_stream)
    side.synchronize()
    ra = a.solve_host(ids, f32["x0"], f32["qd_meas"], f32["cmd"], f32["phase"])
    rb = b.solve_host(ids, f32["x0"], f32["qd_meas"], f32["cmd"], f32["phase"])
    a.close()
    b.close()
    assert (ra["status"] == 0).all()
    assert np.array_equal(ra["tau"], rb["tau"]) and np.array_equal(ra["status"], rb["status"])
