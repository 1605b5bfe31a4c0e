"""Failure detection on the GPU without a fault: a bounded device wait that
runs out.

The test hook `wait_test_agent` arms the first stage-block wait of one agent
with no copy behind it, so that wait gives up after `spin_limit` polls with
nothing in flight.  That agent must come back MPC_AGENT_TIMEOUT with zeroed
outputs, the event must be counted, every other agent of the batch must be
solved exactly as without the hook, and the context must stay usable.
"""
import numpy as np
import pytest

from helpers import agents, device_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpcgpu():
    import __graft_entry__ as g
    g.build()
    from paper_2510_12717_b300 import mpcgpu as m
    m.load()
    return m


@pytest.mark.parametrize("form", [1, 0], ids=["fused", "plain"])
def test_wait_that_runs_out_times_out_one_agent(mpcgpu, form):
    n, bad = 24, 7
    ids = np.arange(n)
    model, inp = agents("uneven", ids)
    inp32 = device_inputs(inp)
    stream = torch.cuda.current_stream().cuda_stream

    def solve(**opts):
        s = mpcgpu.Solver(max_agents=n, max_horizon=20, form=form, stream=stream, **opts)
        s.set_models(model, ids)
        outs = [s.solve_host(ids, inp32["x0"], inp32["qd_meas"], inp32["cmd"], inp32["phase"]) for _ in range(2)]
        stats = s.stats()
        s.close()
        return outs, stats

    ref, ref_stats = solve()
    got, stats = solve(spin_limit=1 << 12, wait_test_agent=bad)
    assert ref_stats["wait_timeouts"] == 0
    # one event per solve: the agent's first wait runs out in both replans
    assert stats["wait_timeouts"] == 2
    others = np.setdiff1d(ids, [bad])
    for r, g in zip(ref, got):
        assert (r["status"] == 0).all()
        assert g["status"][bad] == mpcgpu.AGENT_TIMEOUT
        assert (g["tau"][bad] == 0).all() and g["value"][bad] == 0
        assert (g["status"][others] == 0).all()
        assert np.array_equal(g["tau"][others], r["tau"][others])
    # the device and a fresh context are unaffected
    again, again_stats = solve()
    assert again_stats["wait_timeouts"] == 0
    assert np.array_equal(again[0]["tau"], ref[0]["tau"])


def test_spin_limit_and_test_agent_are_validated(mpcgpu):
    with pytest.raises(mpcgpu.MpcError):
        mpcgpu.Solver(max_agents=4, max_horizon=10, spin_limit=0)
    with pytest.raises(mpcgpu.MpcError):
        mpcgpu.Solver(max_agents=4, max_horizon=10, wait_test_agent=4)


def test_literal_form_wait_that_runs_out_times_out_one_agent(mpcgpu):
    # the literal form's bulk copies of the stage factors (one warp per agent):
    # the first staged item of one agent is armed with no copy behind it
    n, bad = 12, 5
    ids = np.arange(n)
    model, inp = agents("uneven", ids)
    inp32 = device_inputs(inp)
    stream = torch.cuda.current_stream().cuda_stream

    def solve(**opts):
        s = mpcgpu.Solver(max_agents=n, max_horizon=20, form=mpcgpu.FORM_LDL, fixed_iters=5, stream=stream,
                          **opts)
        s.set_models(model, ids)
        out = s.solve_host(ids, inp32["x0"], inp32["qd_meas"], inp32["cmd"], inp32["phase"])
        stats = s.stats()
        s.close()
        return out, stats

    ref, ref_stats = solve()
    got, stats = solve(spin_limit=1 << 12, wait_test_agent=bad)
    assert ref_stats["wait_timeouts"] == 0 and stats["wait_timeouts"] == 1
    others = np.setdiff1d(ids, [bad])
    assert (ref["status"] == mpcgpu.AGENT_MAX_ITER).all()
    assert got["status"][bad] == mpcgpu.AGENT_TIMEOUT
    assert (got["tau"][bad] == 0).all()
    assert (got["status"][others] == mpcgpu.AGENT_MAX_ITER).all()
    assert np.array_equal(got["tau"][others], ref["tau"][others])
    again, again_stats = solve()
    assert again_stats["wait_timeouts"] == 0 and np.array_equal(again["tau"], ref["tau"])
