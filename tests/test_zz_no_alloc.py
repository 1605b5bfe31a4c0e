"""The allocation-free entry point, mpc_solve_static.

It exists for callers that cannot allocate device memory when they need a
solve (simulator plugins that may only use the buffers handed to them,
real-time loops that must not enter the device allocator once running, or
processes where another framework owns the allocator).
Its workspace is a static device array inside the library, so this test
checks that two calls in a row through it give the same torques, within the
parity tolerance, as the regular context-based entry point on the same
inputs.  The file sorts last so that a run stopping at its first failure has
already run every other test.
"""
import numpy as np
import pytest

from helpers import agents, device_inputs, torque_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _regular(mpcgpu, model, inp32, dev):
    n = len(model["mass"])
    s = mpcgpu.Solver(max_agents=n, max_horizon=20, warm_start=0,
                      stream=torch.cuda.current_stream().cuda_stream)
    s.set_models(model, np.arange(n))
    r = s.solve_host(np.arange(n), inp32["x0"], inp32["qd_meas"], inp32["cmd"], inp32["phase"])
    s.close()
    return r


def _static(mpcgpu, model, inp32, dev):
    n = len(model["mass"])
    t = {k: torch.from_numpy(v).to(dev) for k, v in inp32.items()}
    tau = torch.full((n, 18), float("nan"), device=dev)
    status = torch.full((n,), -7, dtype=torch.int32, device=dev)
    rc = mpcgpu.solve_static(model, t["x0"], t["qd_meas"], t["cmd"], t["phase"], tau=tau, status=status,
                             stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == mpcgpu.MPC_OK
    return dict(tau=tau.cpu().numpy(), status=status.cpu().numpy())


def test_static_entry_matches_regular_entry_twice():
    import __graft_entry__ as g
    g.build()
    from paper_2510_12717_b300 import mpcgpu
    dev = torch.device("cuda:0")
    # call 1: 12 mixed-horizon agents; call 2: 9 other agents, next replan
    cases = [("uneven", np.arange(12), 0), ("uneven", np.arange(40, 49), 1)]
    for name, ids, replan in cases:
        model, inp = agents(name, ids, replan=replan)
        inp32 = device_inputs(inp)
        ref = _regular(mpcgpu, model, inp32, dev)
        got = _static(mpcgpu, model, inp32, dev)
        assert np.array_equal(got["status"], ref["status"])
        assert torque_close(got["tau"], ref["tau"]).all()


def test_static_entry_full_layout_matches_regular_entry():
    # exactly the static maximum: 64 agents, all at horizon 20, so every
    # per-agent region of the static array is used to its end
    import __graft_entry__ as g
    g.build()
    from paper_2510_12717_b300 import mpcgpu
    dev = torch.device("cuda:0")
    model, inp = agents("uneven", np.arange(mpcgpu.STATIC_MAX_AGENTS), replan=2)
    model["N"][:] = mpcgpu.STATIC_MAX_HORIZON
    inp32 = device_inputs(inp)
    ref = _regular(mpcgpu, model, inp32, dev)
    got = _static(mpcgpu, model, inp32, dev)
    assert (ref["status"] == 0).all()
    assert np.array_equal(got["status"], ref["status"])
    ok = torque_close(got["tau"], ref["tau"])
    assert ok.all(), np.argwhere(~ok)


def test_static_entry_rejects_horizon_beyond_limit():
    import __graft_entry__ as g
    g.build()
    from paper_2510_12717_b300 import mpcgpu
    model, inp = agents("uneven", np.arange(1))
    model["N"][:] = mpcgpu.STATIC_MAX_HORIZON + 1
    dev = torch.device("cuda:0")
    t = {k: torch.from_numpy(v).to(dev) for k, v in device_inputs(inp).items()}
    rc = mpcgpu.solve_static(model, t["x0"], t["qd_meas"], t["cmd"], t["phase"])
    assert rc == mpcgpu.MPC_ERR_INVALID


def test_static_entry_rejects_oversize_batch():
    import __graft_entry__ as g
    g.build()
    from paper_2510_12717_b300 import mpcgpu
    model, inp = agents("uneven", np.arange(mpcgpu.STATIC_MAX_AGENTS + 1))
    dev = torch.device("cuda:0")
    t = {k: torch.from_numpy(v).to(dev) for k, v in device_inputs(inp).items()}
    rc = mpcgpu.solve_static(model, t["x0"], t["qd_meas"], t["cmd"], t["phase"])
    assert rc == mpcgpu.MPC_ERR_INVALID
