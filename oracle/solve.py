"""The oracle's whole per-agent pipeline (paper Alg. 1, solved exactly).

f_param (schedule, references, bounds) -> linearisation -> dense QP ->
interior-point solve -> torque map.  A process pool (spawn start method, one
BLAS thread per worker) runs agents in parallel.

Oracle code: test infrastructure only.
"""
from __future__ import annotations

import os

import numpy as np

from . import ipm, qp as qpmod, torque


def agent_params(model: dict, a: int) -> dict:
    return {k: v[a] for k, v in model.items()}


def solve_agent(m: dict, x0, cmd, phase, qd_meas, *, tol_mu=1e-13, tol_res=1e-11):
    x0 = np.asarray(x0, float)
    qp, ex = qpmod.agent_qp(m, x0, cmd, phase)
    r = ipm.solve_qp(qp.P, qp.q, qp.E, qp.e, qp.C, qp.lo, qp.hi,
                     tol_mu=tol_mu, tol_res=tol_res)
    N = qp.N
    u = np.stack([qp.u(r.z, k) for k in range(N)])
    x = np.vstack([x0[None, :]] + [qp.x(r.z, k)[None, :] for k in range(1, N + 1)])
    tau, q_set, qd_set = torque.torque_map(m, x0, qd_meas, u[0], u[1], x1=x[1])
    return dict(tau=tau, q_set=q_set, qd_set=qd_set, V=qp.objective(r.z),
                x=x, u=u, y=r.y.reshape(N, 56), ipm=r, qp=qp, extras=ex)


def _worker(args):
    m, x0, cmd, phase, qd = args
    out = solve_agent(m, x0, cmd, phase, qd)
    r = out["ipm"]
    return (out["tau"], out["q_set"], out["qd_set"], out["V"], out["x"], out["u"],
            out["y"], r.converged, r.iters, out["extras"]["stance"])


_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _init_worker():
    for var in _THREAD_VARS:
        os.environ[var] = "1"
    try:
        from threadpoolctl import threadpool_limits
        threadpool_limits(1)
    except Exception:
        pass


def solve_batch(model: dict, inputs: dict, idx=None, processes: int | None = None):
    """Solve agents `idx` (default all).  Returns a dict of per-agent results.

    processes=0 runs serially in this process.
    """
    B = len(model["mass"])
    idx = list(range(B)) if idx is None else list(idx)
    jobs = [(agent_params(model, a), inputs["x0"][a], inputs["cmd"][a],
             inputs["phase"][a], inputs["qd_meas"][a]) for a in idx]
    if processes == 0 or len(jobs) == 1:
        res = [_worker(j) for j in jobs]
    else:
        import multiprocessing as mp
        n = processes or len(os.sched_getaffinity(0))
        ctx = mp.get_context("spawn")
        # workers start with one BLAS thread each (set before they import numpy)
        saved = {v: os.environ.get(v) for v in _THREAD_VARS}
        os.environ.update({v: "1" for v in _THREAD_VARS})
        try:
            with ctx.Pool(n, initializer=_init_worker) as pool:
                res = pool.map(_worker, jobs, chunksize=1)
        finally:
            for v, old in saved.items():
                if old is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = old
    return dict(
        tau=np.stack([r[0] for r in res]), q_set=np.stack([r[1] for r in res]),
        qd_set=np.stack([r[2] for r in res]), V=np.array([r[3] for r in res]),
        x=[r[4] for r in res], u=[r[5] for r in res], y=[r[6] for r in res],
        converged=np.array([r[7] for r in res]), iters=np.array([r[8] for r in res]),
        stance=[r[9] for r in res], idx=np.array(idx),
    )
