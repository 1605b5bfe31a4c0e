"""Continuous-batching serving over the C ABI (one GPU): a request driver
for the library's native server (mpc_server_*, csrc/server.cu).

Requests for agent replans arrive as a Poisson stream.  Agents are slots of
one solver context (admitted under an HBM budget at creation); each keeps its
warm start and factor caches resident on the device.  The native server
holds a per-slot pending table (later requests of an agent coalesce into its
pending one: the newest state wins) and a worker thread that, whenever fewer
than `streams` batches are on the GPU, forms the next batch from every agent
with pending requests and no batch in flight, copies it to the device,
solves it on its own stream and answers its requests when it completes.
With `defer` = 1 (the default) an agent whose polish first fails does not
hold its batch for the length of an ADMM solve: it comes back deferred and
the server finishes it (ADMM from the saved start) in a batch of its own, so
one slow agent delays only its own requests (2: also agents that two reduced
KKT solves of the polish do not settle; 0: off).
This driver replays the arrival process in real time: every few hundred
microseconds it pushes the requests that have arrived, with their states and
arrival times.  Every `churn_period` seconds (1 s = 100 replans of an agent
at 100 Hz) a fraction of the agents leaves and as many new agents join (the
server swaps their models in once no batch of theirs is in flight).

Request states: each agent walks forward in time from its initial inputs;
a request is one 10 ms environment step: gait phase += phase_step, and the
state takes one step of a mean-reverting walk around the agent's initial
state, x <- x_init + a (x - x_init) + step_sigma N(0, I), as a robot under
feedback control stays near its reference (a plain random walk drifts past
the joint limits within a few seconds and makes the QPs infeasible).  The
requests of an agent that arrive together carry the state after all of
their steps (they coalesce in the server anyway).

Latency of a request = completion time of the batch that answered it minus
its arrival time, on the server's clock.
"""
from __future__ import annotations

import time

import numpy as np

from . import mpcgpu


class ServingEngine:
    def __init__(self, model: dict, inputs, *, pool: int, streams: int = 2, max_batch: int = 0,
                 hbm_budget_bytes: int = 8 << 30, device: int = 0, step_sigma: float = 0.02,
                 phase_step: float = 0.02, revert: float = 0.95, seed: int = 0, defer: int = 1,
                 **solver_opts):
        """model: SoA agent models (workload.make_agents layout) of every agent
        that may ever join (live + reserve); inputs: their initial per-agent
        input dict (x0, qd_meas, cmd, phase), or a list whose first entry is.
        pool: number of slots (live agents at a time); streams: batches on the
        GPU at a time."""
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        torch.cuda.set_device(self.dev)
        self.model = model
        if isinstance(inputs, (list, tuple)):
            inputs = inputs[0]
        self.walk = StateWalk(inputs, step_sigma=step_sigma, phase_step=phase_step, revert=revert, seed=seed)
        self.total = len(model["mass"])
        self.pool = pool
        self.streams = streams
        self.defer = defer
        self.max_batch = max_batch or pool
        self.solver = mpcgpu.Solver(max_agents=pool, max_horizon=int(np.max(model["N"])), device=device,
                                    stream=torch.cuda.current_stream(self.dev).cuda_stream,
                                    hbm_budget_bytes=hbm_budget_bytes, **solver_opts)
        # slot s holds agent slot_agent[s]
        self.slot_agent = np.arange(pool)
        self.reserve = list(range(pool, self.total))
        self.churned = 0
        self.solver.set_models(model, np.arange(pool, dtype=np.int32), idx=self.slot_agent)
        self.status_counts = {}

    def close(self):
        self.solver.close()

    def _pick_churn(self, frac: float, rng):
        """Slots whose agents leave and the reserve agents that join them."""
        k = int(round(frac * self.pool))
        if k == 0 or len(self.reserve) < k:
            return None, None
        slots = np.sort(rng.choice(self.pool, k, replace=False))
        self.reserve.extend(int(a) for a in self.slot_agent[slots])
        new = np.asarray([self.reserve.pop(0) for _ in range(k)])
        self.churned += k
        self.slot_agent[slots] = new
        return slots.astype(np.int32), new

    def run(self, rate: float, duration: float, *, seed: int = 0, churn_period: float = 1.0,
            churn_frac: float = 0.05, warmup_batches: int = 2):
        """Serve a Poisson stream of `rate` requests/s for `duration` seconds
        of arrivals.  Returns latency and throughput statistics."""
        rng = np.random.default_rng(seed)
        n_req = rng.poisson(rate * duration)
        t_arr = np.sort(rng.uniform(0.0, duration, n_req))
        slot_req = rng.integers(0, self.pool, n_req).astype(np.int32)
        # warm the solver (models resident, first factorisations) before the clock starts
        slots_all = np.arange(self.pool, dtype=np.int32)
        for _ in range(warmup_batches):
            x0, qd, cmd, ph = self.walk.advance(self.slot_agent, np.ones(self.pool, dtype=np.int64))
            self.solver.solve_host(slots_all, x0, qd, cmd, ph)
        W = self.walk
        srv = mpcgpu.Server(self.solver, self.pool, self.max_batch, self.streams)
        srv.set_defer(self.defer)
        load = None
        next_churn = churn_period if churn_period and churn_period > 0 else float("inf")
        try:
            srv.start()
            # the requests come from a native thread (a Python loop falls behind
            # the arrival process by milliseconds); this thread only swaps agents
            a = self.slot_agent
            load = mpcgpu.Load(srv, t_arr, slot_req, W.XI[a], W.CMD[a], W.PH[a], revert=W.revert,
                               sigma=W.step_sigma, phase_step=float(W.phase_step), seed=seed + 1)
            t_start = srv.clock()
            while srv.clock() - t_start < duration:
                if srv.clock() - t_start >= next_churn:
                    slots, new = self._pick_churn(churn_frac, rng)
                    if slots is not None:
                        srv.set_models(self.model, slots, idx=new)
                        load.reset(slots, W.XI[new], W.CMD[new], W.PH[new])
                    next_churn += churn_period
                time.sleep(1e-3)
            lag = load.wait(timeout_s=max(60.0, 20 * duration))
            srv.drain(timeout_s=max(60.0, 20 * duration))
            wall = srv.clock()
            res = srv.results()
            blog = srv.batches()
            n_deferred = srv.deferred()
            srv.stop()
        finally:
            if load is not None:
                load.close()
            srv.close()
        st = res["status"]
        for v in np.unique(st[st >= 0]):
            self.status_counts[int(v)] = int(np.count_nonzero(st == v))
        lat = res["latency"]
        dur = 1e3 * (blog[:, 1] - blog[:, 0])      # launch to completion of each batch
        return dict(requests=int(n_req), rate=rate, duration=duration, wall_s=wall, solves=int(res["solves"]),
                    not_solved=int(res["not_solved"]), solves_per_s=res["solves"] / wall, batches=int(res["batches"]),
                    mean_batch=res["solves"] / max(res["batches"], 1),
                    p50_ms=float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
                    p99_ms=float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
                    coalesced_frac=1.0 - res["solves"] / max(n_req, 1), swapped=int(res["swapped"]),
                    batch_ms_p50=float(np.percentile(dur, 50)) if len(dur) else None,
                    batch_ms_p99=float(np.percentile(dur, 99)) if len(dur) else None,
                    batch_ms_max=float(dur.max()) if len(dur) else None,
                    push_lag_ms_p99=lag[1] * 1e3, push_lag_ms_max=lag[2] * 1e3, deferred=n_deferred)


class StateWalk:
    """Synthetic per-agent request states.  One environment step: phase +=
    phase_step, x <- x_init + a (x - x_init) + sigma xi (xi ~ N(0, I)),
    qd_meas ~ 0.1 N(0, I), commanded height = current height (the other
    command entries stay).  s coalesced steps take the s-step transition:
    decay a^s, noise scale sigma sqrt((1 - a^2s) / (1 - a^2)).  The noise is
    drawn once into a pool and read as windows at random offsets (synthetic
    states; fresh normals per batch dominated the host loop).  Arrays are kept
    per field and contiguous, so a batch is a few gathers and one scatter."""

    def __init__(self, inputs, *, step_sigma=0.02, phase_step=0.02, revert=0.95, seed=0, pool_size=1 << 22):
        self.X = np.array(inputs["x0"], dtype=np.float32, copy=True)
        self.XI = self.X.copy()
        self.CMD = np.array(inputs["cmd"], dtype=np.float32, copy=True)
        self.PH = np.array(inputs["phase"], dtype=np.float32, copy=True)
        self.phase_step = np.float32(phase_step)
        self.revert = float(revert)
        self.step_sigma = float(step_sigma)
        steps = np.arange(_MAX_STEPS + 1, dtype=np.float64)
        a = float(revert)
        var = steps if a == 1.0 else (1.0 - a ** (2.0 * steps)) / (1.0 - a * a)
        self.decay_tab = (a ** steps).astype(np.float32)
        self.sdev_tab = (step_sigma * np.sqrt(var)).astype(np.float32)
        self.rng = np.random.default_rng(seed)
        self.noise = self.rng.standard_normal(pool_size, dtype=np.float32)

    def draw(self, shape):
        """A window of the pool at a random offset (a fixed cyclic order would
        repeat each agent's noise with a fixed period and correlate the walk)."""
        size = int(np.prod(shape))
        at = int(self.rng.integers(0, len(self.noise) - size + 1))
        return self.noise[at:at + size].reshape(shape)

    def advance(self, agents, steps):
        """Walk the agents' states `steps` environment steps forward; returns
        (x0, qd_meas, cmd, phase) of the batch, fresh arrays in batch order."""
        n = len(agents)
        s = np.minimum(np.asarray(steps, dtype=np.int64), _MAX_STEPS)
        x = self.X[agents]
        xi = self.XI[agents]
        x -= xi
        x *= self.decay_tab[s][:, None]
        x += xi
        x += self.sdev_tab[s][:, None] * self.draw((n, 30))
        self.X[agents] = x
        ph = self.PH[agents] + self.phase_step * s.astype(np.float32)
        ph -= np.floor(ph)
        self.PH[agents] = ph
        cmd = self.CMD[agents]
        cmd[:, 0] = x[:, 2]
        return x, 0.1 * self.draw((n, 18)), cmd, ph


_MAX_STEPS = 1024        # coalesced steps beyond this take this many
