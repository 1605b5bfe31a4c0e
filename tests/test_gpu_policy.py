"""Residual policy + joint-torque blending (paper Sec. IV, Eq. joint-torque)
on the tensor cores, against the FP64 oracle pipeline (IPM -> policy)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import ATOL, RTOL, agents, device_inputs, oracle_view  # noqa: E402

LAMBDA = 0.1
# Tolerances on the actions: both sides round every layer input to bfloat16;
# they differ by FP32 vs FP64 accumulation (~1e-6 relative), which flips a
# rounding decision now and then: one flip moves an activation by one bfloat16
# step (2^-8 relative) and the next layer's outputs by about
# |w| |h| 2^-8 ~ 0.06 * 1 * 0.004 = 2.4e-4; a few flips per agent stay below
# the bound below.  The blended torque adds lambda K_p times that.
A_ATOL, A_RTOL = 2e-3, 1e-2


@pytest.fixture(scope="module")
def mpcgpu():
    import __graft_entry__ as g
    g.build()
    from paper_2510_12717_b300 import mpcgpu as m
    m.load()
    return m


def _solve_with_policy(mpcgpu, model, inp32, weights):
    dev = torch.device("cuda:0")
    n = len(model["mass"])
    s = mpcgpu.Solver(max_agents=n, max_horizon=int(model["N"].max()), stream=torch.cuda.current_stream().cuda_stream)
    s.set_models(model, np.arange(n, dtype=np.int32))
    s.set_policy(weights, LAMBDA)
    t = {k: torch.from_numpy(v).to(dev) for k, v in inp32.items()}
    ids = torch.arange(n, dtype=torch.int32, device=dev)
    tk = s.submit(ids, t["x0"], t["qd_meas"], t["cmd"], t["phase"])
    s.solve(tk)
    tau_b = torch.empty((n, 18), device=dev)
    act = torch.empty((n, 10), device=dev)
    s.policy_torques(tk, tau=tau_b, action=act)
    out = dict(tau=torch.empty((n, 18), device=dev), q_set=torch.empty((n, 18), device=dev),
               qd_set=torch.empty((n, 18), device=dev), value=torch.empty(n, device=dev),
               status=torch.empty(n, dtype=torch.int32, device=dev))
    s.get_torques(tk, **out)
    torch.cuda.synchronize()
    s.close()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["tau_blend"] = tau_b.cpu().numpy()
    res["action"] = act.cpu().numpy()
    return res


def test_policy_and_blend_match_oracle(mpcgpu):
    from oracle.policy import policy_batch
    from oracle.solve import solve_batch
    from workload import make_policy
    ids = np.arange(40)        # 40 agents: three partial 16-agent tiles
    model, inp = agents("uneven", ids)
    inp32 = device_inputs(inp)
    w = make_policy()
    r = _solve_with_policy(mpcgpu, model, inp32, w)
    assert (r["status"] == 0).all()
    m, i = oracle_view(model, inp32)
    ref = solve_batch(m, i)
    acts, taus = policy_batch(m, i, ref["tau"], ref["V"], w, LAMBDA)
    da = np.abs(r["action"] - acts)
    print(f"\n[policy] actions max |da| {da.max():.2e}, |a| max {np.abs(acts).max():.2f}")
    assert (da <= A_ATOL + A_RTOL * np.abs(acts)).all(), np.argwhere(da > A_ATOL + A_RTOL * np.abs(acts))
    kp = np.asarray(m["Kp"])[:, :10]
    tol = ATOL + RTOL * np.abs(taus)
    tol[:, :10] += LAMBDA * kp * (A_ATOL + A_RTOL * np.abs(acts))
    dt = np.abs(r["tau_blend"] - taus)
    assert (dt <= tol).all(), np.argwhere(dt > tol)


def test_zero_policy_blend_is_pd_about_nominal(mpcgpu):
    # zero weights and biases: a = 0 exactly, so the blended torque is the
    # MPC torque plus lambda (K_p (q_nom - q) - K_d qdot) on the legs
    ids = np.arange(20)
    model, inp = agents("uneven", ids)
    inp32 = device_inputs(inp)
    w = {f"W{l}": np.zeros(s, np.float32) for l, s in ((1, (54, 256)), (2, (256, 256)), (3, (256, 256)), (4, (256, 10)))}
    w.update({f"b{l}": np.zeros(d, np.float32) for l, d in ((1, 256), (2, 256), (3, 256), (4, 10))})
    r = _solve_with_policy(mpcgpu, model, inp32, w)
    assert np.array_equal(r["action"], np.zeros_like(r["action"]))
    q = inp32["x0"][:, 12:22].astype(np.float64)
    want = r["tau"].astype(np.float64)
    want[:, :10] += LAMBDA * (model["Kp"][:, :10] * (model["q_nom"][:, :10] - q) -
                              model["Kd"][:, :10] * inp32["qd_meas"][:, :10])
    np.testing.assert_allclose(r["tau_blend"], want, rtol=1e-6, atol=1e-5)
