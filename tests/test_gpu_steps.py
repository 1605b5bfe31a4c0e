"""Step-level parity of the CUDA path.  Alg. 1's f_init / f_param and the
linearisation (rows A1 and A2): the horizon QP that the set-up kernel forms,
read back through mpc_export_qp, against the oracle's own construction of the
same QP (oracle/refs.py for the contact schedule, references and row bounds;
oracle/model.py's complex-step linearisation for A_k, B_k, c_k).

A wrong block of the analytic Jacobians is caught here directly, not only
through the torques of a whole solve.  The two sides share no code: the
oracle differentiates the model numerically in FP64, the device writes the
Jacobians by hand in FP32, so the bar is FP32 rounding of the device's
arithmetic on FP32 inputs.  One ADMM iteration (rows A3-A5: the Riccati
factor and sweeps of the x-update, relaxation, projection, dual update)
against the same iteration written out densely in FP64.
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


def test_admm_iteration_equals_dense_kkt_solve(mpcgpu):
    # rows A3-A5: one ADMM iteration (the Riccati factor of P + sigma I +
    # C^T diag(rho_r) C with the dynamics exact, its backward and forward
    # sweeps, then relaxation, projection and the dual update) against the same
    # iteration written out densely in FP64: the equality-constrained QP of the
    # x-update solved through its full KKT matrix, then OSQP's updates row by
    # row with np.clip.  Iterate: the state after 5 iterations of a first solve
    # (generic w, y, not at a fixed point), imported into a fresh context.
    from oracle import refs
    from oracle.solve import agent_params
    ids = np.arange(6)
    model, inp = agents("uneven", ids)
    inp32 = device_inputs(inp)
    slots = np.arange(len(ids))
    opts = dict(stream=torch.cuda.current_stream().cuda_stream, polish=0, warm_polish=0, adaptive_rho=0)
    s = mpcgpu.Solver(max_agents=len(ids), max_horizon=20, fixed_iters=5, **opts)
    s.set_models(model, slots)
    s.solve_host(slots, inp32["x0"], inp32["qd_meas"], inp32["cmd"], inp32["phase"])
    Ns = [int(model["N"][a]) for a in slots]
    st0 = [s.export_state(int(a), Ns[a]) for a in slots]
    qps = [s.export_qp(int(a), Ns[a]) for a in slots]
    s.close()
    s = mpcgpu.Solver(max_agents=len(ids), max_horizon=20, fixed_iters=1, **opts)
    s.set_models(model, slots)
    for a in slots:
        s.import_state(int(a), st0[a])
    s.solve_host(slots, inp32["x0"], inp32["qd_meas"], inp32["cmd"], inp32["phase"])
    st1 = [s.export_state(int(a), Ns[a]) for a in slots]
    s.close()
    cfg = mpcgpu.MpcConfig()
    mpcgpu.load().mpc_default_config(mpcgpu.C.byref(cfg))
    sigma, alpha = float(cfg.sigma), float(cfg.alpha)
    m64, i64 = oracle_view(model, inp32)
    worst = 0.0
    for a in slots:
        N, q0, q1 = Ns[a], qps[a], st0[a]
        m = agent_params(m64, a)
        dt = float(m["dt"])
        Q, R = np.asarray(m["Q"], float), np.asarray(m["R"], float)
        rho = float(q1["rho"])
        stance = refs.contact_schedule(m, float(i64["phase"][a]))
        n = 60 * N
        P = np.zeros((n, n)); qv = np.zeros(n)
        E = np.zeros((30 * N, n)); e = np.zeros(30 * N)
        C = np.zeros((56 * N, n)); lo = np.zeros(56 * N); hi = np.zeros(56 * N)
        for k in range(N):
            Cu, Cx, l_k, h_k = refs.stage_rows(m, stance[k])
            iu, ix, ir = slice(60 * k, 60 * k + 30), slice(60 * k + 30, 60 * k + 60), slice(56 * k, 56 * k + 56)
            C[ir, iu], C[ir, ix] = Cu, Cx
            lo[ir], hi[ir] = l_k, h_k
            P[iu, iu] += np.diag(2 * dt * R + sigma)
            P[ix, ix] += np.diag(2 * dt * Q + sigma)
            qv[iu] = -2 * dt * R * q0["u_ref"][k] - sigma * q1["u"][k]
            qv[ix] = -2 * dt * Q * q0["x_ref"][k + 1] - sigma * q1["x"][k + 1]
            er = slice(30 * k, 30 * k + 30)
            E[er, ix] = np.eye(30)
            E[er, iu] = -q0["B"][k]
            if k == 0:
                e[er] = q0["c"][0] + q0["A"][0] @ i64["x0"][a]
            else:
                E[er, 60 * (k - 1) + 30:60 * (k - 1) + 60] = -q0["A"][k]
                e[er] = q0["c"][k]
        # the row classes of the ADMM penalty: equality rows 1e3 rho, bounded rows rho, free rows 0
        cls = np.where(lo == hi, 1e3, np.where(np.isfinite(lo) | np.isfinite(hi), 1.0, 0.0))
        rr = rho * cls
        w_old = np.concatenate([q1["w"][k] for k in range(N)]).astype(float)
        y_old = np.concatenate([q1["y"][k] for k in range(N)]).astype(float)
        P += C.T @ (rr[:, None] * C)
        qv -= C.T @ (rr * w_old - y_old)
        K = np.block([[P, E.T], [E, np.zeros((30 * N, 30 * N))]])
        zt = np.linalg.solve(K, np.concatenate([-qv, e]))[:n]
        z_old = np.concatenate([np.concatenate([q1["u"][k], q1["x"][k + 1]]) for k in range(N)]).astype(float)
        z_new = alpha * zt + (1 - alpha) * z_old
        wh = alpha * (C @ zt) + (1 - alpha) * w_old
        with np.errstate(divide="ignore", invalid="ignore"):
            w_new = np.where(rr > 0, np.clip(wh + y_old / np.where(rr > 0, rr, 1.0), lo, hi), wh)
        y_new = np.where(rr > 0, y_old + rr * (wh - w_new), 0.0)
        got_z = np.concatenate([np.concatenate([st1[a]["u"][k], st1[a]["x"][k + 1]]) for k in range(N)])
        got_w = np.concatenate([st1[a]["w"][k] for k in range(N)])
        got_y = np.concatenate([st1[a]["y"][k] for k in range(N)])
        # FP32 factor and sweeps against FP64: norm-wise relative error of
        # the iterate within 1e-5 (about 170 FP32 units; measured 1e-7 to 3e-6)
        ez = np.linalg.norm(got_z - z_new) / np.linalg.norm(z_new)
        ew = np.linalg.norm(got_w - w_new) / max(np.linalg.norm(w_new), 1e-12)
        ey = np.linalg.norm(got_y - y_new) / max(np.linalg.norm(y_new), 1e-12)
        worst = max(worst, ez, ew, ey)
        print(f"\n[ADMM step, agent {a}, N {N}] rel err z {ez:.2e} w {ew:.2e} y {ey:.2e}")
        assert ez <= 1e-5 and ew <= 1e-5 and ey <= 1e-5, (a, ez, ew, ey)
