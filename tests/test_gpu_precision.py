"""Precision modes of the Riccati factor (FP32, TF32 / BF16 tensor-core stage
products, FP64 stage Schur complement) against the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import agents, device_inputs, oracle_view, torque_close  # noqa: E402

_REF = {}


@pytest.fixture(scope="module")
def mpcgpu():
    import __graft_entry__ as g
    g.build()
    from paper_2510_12717_b300 import mpcgpu as m
    m.load()
    return m


def _solve(mpcgpu, model, inps, precision, refine):
    n = len(model["mass"])
    s = mpcgpu.Solver(max_agents=n, max_horizon=int(model["N"].max()),
                      stream=torch.cuda.current_stream().cuda_stream, precision=precision, refine_steps=refine)
    s.set_models(model, np.arange(n))
    out = []
    for inp32 in inps:
        r = s.solve_host(np.arange(n, dtype=np.int32), inp32["x0"], inp32["qd_meas"], inp32["cmd"], inp32["phase"])
        out.append((r, s.agent_stats(np.arange(n, dtype=np.int32))))
    s.close()
    return out


def _case(name, n):
    from oracle.solve import solve_batch
    key = (name, n)
    if key not in _REF:
        ids = np.arange(n)
        model, _ = agents(name, ids)
        inps, refs = [], []
        for replan in (0, 1):
            _, inp = agents(name, ids, replan=replan)
            inp32 = device_inputs(inp)
            m, i = oracle_view(model, inp32)
            inps.append(inp32)
            refs.append(solve_batch(m, i))
        _REF[key] = (model, inps, refs)
    return _REF[key]


@pytest.mark.parametrize("precision,refine", [(0, 1), (3, 1)], ids=["fp32+refine", "fp64schur+refine"])
def test_fp32_and_fp64_factor_match_oracle(mpcgpu, precision, refine):
    model, inps, refs = _case("uneven", 32)
    for (r, st), ref in zip(_solve(mpcgpu, model, inps, precision, refine), refs):
        assert (r["status"] == 0).all()
        ok = torque_close(r["tau"], ref["tau"])
        assert ok.all(), np.argwhere(~ok)


@pytest.mark.parametrize("precision", [1, 2], ids=["tf32", "bf16"])
def test_tensor_core_factor_with_refinement_matches_oracle(mpcgpu, precision):
    # TF32 / BF16 stage products, their rounding won back by the automatic
    # refinement steps (2 for TF32, 3 for BF16): every agent solved and within
    # the FP64 torque tolerance; the norm-wise error is printed per replan
    model, inps, refs = _case("uneven", 32)
    for replan, ((r, st), ref) in enumerate(zip(_solve(mpcgpu, model, inps, precision, -1), refs)):
        assert (r["status"] == 0).all(), np.argwhere(r["status"] != 0)
        rel = np.linalg.norm(r["tau"] - ref["tau"], axis=1) / np.maximum(np.linalg.norm(ref["tau"], axis=1), 1e-9)
        print(f"\n[precision {precision} replan {replan}] median rel err {np.median(rel):.2e}, max {rel.max():.2e}")
        ok = torque_close(r["tau"], ref["tau"])
        assert ok.all(), np.argwhere(~ok)


def test_tensor_core_products_track_fp32(mpcgpu):
    # the tensor-core products only change the factor's rounding: solved
    # agents of the three modes agree to the products' precision
    model, inps, refs = _case("uneven", 32)
    base = _solve(mpcgpu, model, inps[:1], 0, 1)[0][0]["tau"]
    for precision, tol in ((1, 2e-2), (2, 2e-1)):
        tau = _solve(mpcgpu, model, inps[:1], precision, 1)[0][0]["tau"]
        rel = np.linalg.norm(tau - base, axis=1) / np.maximum(np.linalg.norm(base, axis=1), 1e-9)
        assert np.median(rel) < tol, (precision, np.median(rel))


def test_ill_conditioned_accuracy_reported(mpcgpu):
    # Q, R spread over [1e-4, 1e4]: FP32 loses digits in the factor; one
    # refinement step keeps most agents within the torque tolerance; the
    # TF32 / BF16 factors are reported only
    model, inps, refs = _case("mixed16k_ill", 32)
    for precision, refine, need in ((0, 1, 0.8), (3, 1, 0.8), (1, -1, None), (2, -1, None)):
        for replan, ((r, st), ref) in enumerate(zip(_solve(mpcgpu, model, inps, precision, refine), refs)):
            fin = np.isfinite(r["tau"]).all(axis=1)
            ok = torque_close(r["tau"], ref["tau"]).all(axis=1) & fin
            print(f"\n[ill-conditioned precision {precision} refine {refine} replan {replan}] "
                  f"within tolerance {ok.mean():.3f}, solved {(r['status'] == 0).mean():.3f}, "
                  f"polished {(st['polished'] > 0).mean():.3f}")
            if need is not None:
                assert fin.all()
                assert ok.mean() >= need
