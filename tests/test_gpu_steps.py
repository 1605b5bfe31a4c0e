"""Step-level parity of the CUDA path (Alg. 1's f_init / f_param and the
linearisation, rows A1 and A2): the horizon QP that the set-up kernel forms,
read back through mpc_export_qp, against the oracle's own construction of the
same QP (oracle/refs.py for the contact schedule, references and row bounds;
oracle/model.py's complex-step linearisation for A_k, B_k, c_k).

A wrong block of the analytic Jacobians is caught here directly, not only
through the torques of a whole solve.  The two sides share no code: the
oracle differentiates the model numerically in FP64, the device writes the
Jacobians by hand in FP32, so the bar is FP32 rounding of the device's
arithmetic on FP32 inputs.
"""
import numpy as np
import pytest

from helpers import agents, device_inputs, oracle_view

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpcgpu():
    import __graft_entry__ as g
    g.build()
    from paper_2510_12717_b300 import mpcgpu as m
    m.load()
    return m


def _pick():
    # every gait, both horizon extremes, and a warm replan of each
    from workload import make_agents
    pool, _ = make_agents("uneven", np.arange(300))
    pick = []
    for g in range(5):
        pick += list(np.nonzero(pool["gait"] == g)[0][:2])
    pick += list(np.nonzero(pool["N"] == 5)[0][:1]) + list(np.nonzero(pool["N"] == 20)[0][:1])
    return np.array(sorted(set(int(p) for p in pick)))


@pytest.mark.parametrize("replan", [0, 1])
def test_setup_forms_the_oracle_qp(mpcgpu, replan):
    from oracle import model as mdl, refs
    from oracle.solve import agent_params
    ids = _pick()
    model, inp0 = agents("uneven", ids)
    s = mpcgpu.Solver(max_agents=len(ids), max_horizon=20, stream=torch.cuda.current_stream().cuda_stream)
    slots = np.arange(len(ids))
    s.set_models(model, slots)
    inps = [device_inputs(inp0)]
    if replan:
        inps.append(device_inputs(agents("uneven", ids, replan=1)[1]))
    for inp32 in inps:
        s.solve_host(slots, inp32["x0"], inp32["qd_meas"], inp32["cmd"], inp32["phase"])
    inp32 = inps[-1]
    m64, i64 = oracle_view(model, inp32)
    worst = {}
    for a in slots:
        m = agent_params(m64, a)
        N = int(m["N"])
        got = s.export_qp(int(a), N)
        x0 = i64["x0"][a]
        stance = refs.contact_schedule(m, float(i64["phase"][a]))
        x_ref, u_ref = refs.references(m, x0, i64["cmd"][a], stance)
        A, B, c = mdl.linearise(m, x0, u_ref)
        rows = [refs.stage_rows(m, stance[k]) for k in range(N)]
        lo = np.stack([r[2] for r in rows]).astype(np.float32)
        hi = np.stack([r[3] for r in rows]).astype(np.float32)
        # row bounds (and with them the contact schedule): exact
        assert np.array_equal(got["lo"], lo), a
        assert np.array_equal(got["hi"], hi), a

        def close(name, g, r, atol, rtol):
            err = np.abs(g - r) / (atol + rtol * np.abs(r))
            worst[name] = max(worst.get(name, 0.0), float(err.max()))
            assert err.max() <= 1.0, (name, a, np.unravel_index(err.argmax(), err.shape), float(err.max()))

        close("x_ref", got["x_ref"], x_ref, 1e-6, 1e-5)
        close("u_ref", got["u_ref"], u_ref, 1e-6, 1e-5)
        close("A", got["A"], np.stack(A), 1e-6, 1e-5)
        close("B", got["B"], np.stack(B), 1e-7, 1e-5)
        close("c", got["c"], np.stack(c), 2e-6, 1e-5)
    s.close()
    print(f"\n[step A1/A2 replan {replan}] worst error / tolerance: "
          + ", ".join(f"{k} {v:.3f}" for k, v in worst.items()))
