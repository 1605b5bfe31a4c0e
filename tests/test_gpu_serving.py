"""Serving form: continuous batching over two streams with churn."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_serving_loop_runs_and_solves_everything():
    import __graft_entry__ as g
    g.build()
    from paper_2510_12717_b300.serve import ServingEngine
    from workload import make_agents, perturb_inputs
    total, pool = 640, 512
    ids = np.arange(total)
    model, inp = make_agents("serving", ids)
    reps = [inp]
    for r in range(1, 3):
        reps.append(perturb_inputs("serving", reps[-1], ids, r))
    reps = [{k: np.ascontiguousarray(v, np.float32) for k, v in x.items()} for x in reps]
    eng = ServingEngine(model, reps, pool=pool, streams=2, max_batch=256)
    st = eng.run(rate=40000.0, duration=0.25, churn_period=0.05, churn_frac=0.05)
    eng.close()
    print("\n[serving]", st, "statuses", eng.status_counts)
    assert st["not_solved"] == 0
    assert st["solves"] > 0 and st["batches"] >= 4
    assert eng.churned >= 3 * round(0.05 * pool)
    assert st["p50_ms"] is not None and st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]


def test_budget_admission():
    import __graft_entry__ as g
    g.build()
    from paper_2510_12717_b300 import mpcgpu
    with pytest.raises(mpcgpu.MpcError) as e:
        mpcgpu.Solver(max_agents=16384, max_horizon=20, hbm_budget_bytes=1 << 30)
    assert e.value.status == mpcgpu.MPC_ERR_BUDGET
    s = mpcgpu.Solver(max_agents=1024, max_horizon=20, hbm_budget_bytes=1 << 30)
    assert s.stats()["arena_bytes"] <= 1 << 30
    s.close()
