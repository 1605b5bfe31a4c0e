"""Serving form: the native continuous-batching server (mpc_server_*) with
churn, and its answers against direct solves of the same states."""
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


def test_server_answers_equal_direct_solves():
    # every agent's answer from the server equals a direct solve of the same
    # state on a context with the same history (each agent's solve depends
    # only on its own state and warm start); two rounds: all agents, then a
    # subset whose requests coalesce (the newest state wins)
    import __graft_entry__ as g
    g.build()
    from paper_2510_12717_b300 import mpcgpu
    from workload import make_agents, perturb_inputs
    n = 96
    ids = np.arange(n)
    model, inp = make_agents("serving", ids)
    r1 = perturb_inputs("serving", inp, ids, 1)
    r2 = perturb_inputs("serving", r1, ids, 2)
    f32 = lambda x: {k: np.ascontiguousarray(v, np.float32) for k, v in x.items()}
    inp, r1, r2 = f32(inp), f32(r1), f32(r2)
    stream = torch.cuda.current_stream().cuda_stream
    direct = mpcgpu.Solver(max_agents=n, max_horizon=20, stream=stream)
    served = mpcgpu.Solver(max_agents=n, max_horizon=20, stream=stream)
    direct.set_models(model, ids)
    served.set_models(model, ids)
    slots = ids.astype(np.int32)
    d1 = direct.solve_host(slots, inp["x0"], inp["qd_meas"], inp["cmd"], inp["phase"])
    sub = slots[::3]
    d2 = direct.solve_host(sub, r2["x0"][sub], r2["qd_meas"][sub], r2["cmd"][sub], r2["phase"][sub])
    srv = mpcgpu.Server(served, n, max_batch=40, max_inflight=2)
    srv.start()
    srv.push(slots, inp["x0"], inp["qd_meas"], inp["cmd"], inp["phase"], np.zeros(n))
    srv.drain(30.0)
    a1 = srv.results()
    # round 2: the subset's replan-1 state, then its replan-2 state in the same push (coalesced)
    both = np.concatenate([sub, sub])
    cat = lambda k: np.concatenate([r1[k][sub], r2[k][sub]])
    t = srv.clock()
    srv.push(both, cat("x0"), cat("qd_meas"), cat("cmd"), cat("phase"), np.full(len(both), t))
    srv.drain(30.0)
    a2 = srv.results()
    srv.stop()
    srv.close()
    served.close()
    direct.close()
    assert a1["answered"] == n and a1["batches"] >= 3          # max_batch 40 splits the first round
    assert np.array_equal(a1["tau"], d1["tau"]) and (a1["status"] == 0).all()
    assert a2["answered"] == n + len(both) and a2["solves"] == n + len(sub)   # the pairs coalesced
    assert np.array_equal(a2["tau"][sub], d2["tau"])
    assert len(a2["latency"]) == n + len(both) and (a2["latency"] >= 0).all()


@pytest.mark.parametrize("mode", [1, 2])
def test_server_with_deferral_answers_equal_direct_solves(mode):
    # joints moved next to their limits: the polish from the previous active
    # set fails for several agents; with deferral on, the server answers the
    # rest from the batch and finishes those in batches of their own; every
    # answer is the optimum a direct solve finds (a deferred agent's
    # active-set method may take another path to it: the bar is the torque
    # tolerance)
    import __graft_entry__ as g
    g.build()
    from paper_2510_12717_b300 import mpcgpu
    from workload import make_inputs, make_agents
    n = 40
    ids = np.arange(n)
    model, _ = make_agents("uneven", ids)
    f32 = lambda x: {k: np.ascontiguousarray(v, np.float32) for k, v in x.items()}
    reps = [f32(make_inputs("uneven", ids, r)[1]) for r in range(3)]
    sign = np.sign(np.random.default_rng(11).standard_normal((n, 18)))
    reps[2]["x0"][:, 12:30] = np.float32(1.45) * sign
    stream = torch.cuda.current_stream().cuda_stream
    direct = mpcgpu.Solver(max_agents=n, max_horizon=20, stream=stream)
    served = mpcgpu.Solver(max_agents=n, max_horizon=20, stream=stream)
    direct.set_models(model, ids)
    served.set_models(model, ids)
    slots = ids.astype(np.int32)
    for r in (0, 1):
        direct.solve_host(slots, reps[r]["x0"], reps[r]["qd_meas"], reps[r]["cmd"], reps[r]["phase"])
        served.solve_host(slots, reps[r]["x0"], reps[r]["qd_meas"], reps[r]["cmd"], reps[r]["phase"])
    d = direct.solve_host(slots, reps[2]["x0"], reps[2]["qd_meas"], reps[2]["cmd"], reps[2]["phase"])
    dst = direct.agent_stats(slots)
    fell_back = dst["polished"] != 2
    srv = mpcgpu.Server(served, n, max_batch=n, max_inflight=2)
    srv.set_defer(mode)
    srv.start()
    srv.push(slots, reps[2]["x0"], reps[2]["qd_meas"], reps[2]["cmd"], reps[2]["phase"], np.zeros(n))
    srv.drain(30.0)
    a = srv.results()
    deferred = srv.deferred()
    srv.stop()
    srv.close()
    served.close()
    direct.close()
    assert fell_back.sum() >= 2 and deferred >= fell_back.sum()
    assert a["answered"] == n and a["solves"] == n and a["batches"] >= 2
    assert (a["status"] == 0).all() and (d["status"] == 0).all()
    tol = 1e-4 + 1e-3 * np.abs(d["tau"])
    assert (np.abs(a["tau"] - d["tau"]) <= tol).all()
