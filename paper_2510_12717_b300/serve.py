"""Continuous-batching serving loop over the C ABI (one GPU).

Requests for agent replans arrive as a Poisson stream.  Agents are slots of
one solver context (admitted under an HBM budget at creation); each keeps its
warm start and factor caches resident on the device.  A request waits in a
per-agent pending set: later requests of the same agent coalesce into it (the
newest state wins).  Whenever one of the streams is free, all pending agents
that are not already in flight (up to max_batch) form the next batch, which
is copied from pinned memory, solved on that stream (mpc_solve_on) and read
back, overlapping with the batch on the other stream.  Every `churn_period`
seconds (1 s = 100 replans of an agent at 100 Hz) a fraction of the live
agents leaves and as many new agents join: agents between requests (none of
their batches in flight), so the swap needs no wait for the device.

Request states: each agent walks forward in time from its initial inputs;
a request is one 10 ms environment step: gait phase += phase_step, and the
state takes one step of a mean-reverting walk around the agent's initial
state, x <- x_init + a (x - x_init) + step_sigma N(0, I), as a robot under
feedback control stays near its reference (a plain random walk drifts past
the joint limits within a few seconds and makes the QPs infeasible).  A
batch answering s coalesced requests of an agent solves its state s steps
on from its previous solve (the s-step transition of the same walk).

Latency of a request = completion time of the batch that answered it minus
its arrival time (time since the run started, on the host clock).
"""
from __future__ import annotations

import time

import numpy as np

from . import mpcgpu


class ServingEngine:
    def __init__(self, model: dict, inputs, *, pool: int, streams: int = 2, max_batch: int = 0,
                 hbm_budget_bytes: int = 8 << 30, device: int = 0, step_sigma: float = 0.02,
                 phase_step: float = 0.02, revert: float = 0.95, seed: int = 0, **solver_opts):
        """model: SoA agent models (workload.make_agents layout) of every agent
        that may ever join (live + reserve); inputs: their initial per-agent
        input dict (x0, qd_meas, cmd, phase), or a list whose first entry is.
        pool: number of slots (live agents at a time)."""
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.model = model
        if isinstance(inputs, (list, tuple)):
            inputs = inputs[0]
        self.walk = StateWalk(inputs, step_sigma=step_sigma, phase_step=phase_step, revert=revert, seed=seed)
        self.total = len(model["mass"])
        self.pool = pool
        self.max_batch = max_batch or pool
        self.solver = mpcgpu.Solver(max_agents=pool, max_horizon=int(np.max(model["N"])), device=device,
                                    stream=torch.cuda.current_stream(self.dev).cuda_stream,
                                    hbm_budget_bytes=hbm_budget_bytes, **solver_opts)
        # slot s holds agent slot_agent[s]
        self.slot_agent = np.arange(pool)
        self.reserve = list(range(pool, self.total))
        self.churned = 0
        self.solver.set_models(model, np.arange(pool, dtype=np.int32), idx=self.slot_agent)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(streams)]
        mb = self.max_batch
        pin = dict(pin_memory=True)
        self.h_in = [dict(ids=torch.empty(mb, dtype=torch.int32, **pin), x0=torch.empty((mb, 30), **pin),
                          qd=torch.empty((mb, 18), **pin), cmd=torch.empty((mb, 4), **pin),
                          ph=torch.empty(mb, **pin)) for _ in streams_range(streams)]
        self.d_in = [dict(ids=torch.empty(mb, dtype=torch.int32, device=self.dev),
                          x0=torch.empty((mb, 30), device=self.dev), qd=torch.empty((mb, 18), device=self.dev),
                          cmd=torch.empty((mb, 4), device=self.dev), ph=torch.empty(mb, device=self.dev))
                     for _ in streams_range(streams)]
        self.d_out = [dict(tau=torch.empty((mb, 18), device=self.dev),
                           st=torch.empty(mb, dtype=torch.int32, device=self.dev)) for _ in streams_range(streams)]
        self.h_out = [dict(tau=torch.empty((mb, 18), **pin), st=torch.empty(mb, dtype=torch.int32, **pin))
                      for _ in streams_range(streams)]

    def close(self):
        self.solver.close()

    # ---------------------------------------------------------------- churn
    def churn(self, frac: float, rng, idle=None):
        """A fraction of the live agents leaves; as many reserve agents join.
        idle: mask of the slots that may leave (no batch of theirs in flight)."""
        k = int(round(frac * self.pool))
        cand = np.arange(self.pool) if idle is None else np.nonzero(idle)[0]
        k = min(k, len(cand))
        if k == 0 or len(self.reserve) < k:
            return 0
        slots = np.sort(rng.choice(cand, k, replace=False))
        # the joining agent's model replaces the leaving one's in its slot:
        # mpc_set_models resets the slot's warm start (no per-slot release)
        self.reserve.extend(int(a) for a in self.slot_agent[slots])
        new = [self.reserve.pop(0) for _ in range(k)]
        self.churned += k
        self.slot_agent[slots] = new
        self.solver.set_models(self.model, slots.astype(np.int32), idx=np.asarray(new))
        return k

    # ---------------------------------------------------------------- run
    def run(self, rate: float, duration: float, *, seed: int = 0, churn_period: float = 1.0,
            churn_frac: float = 0.05, warmup_batches: int = 2):
        """Serve a Poisson stream of `rate` requests/s for `duration` seconds
        of arrivals.  Returns latency and throughput statistics."""
        rng = np.random.default_rng(seed)
        n_req = rng.poisson(rate * duration)
        t_arr = np.sort(rng.uniform(0.0, duration, n_req))
        slot_req = rng.integers(0, self.pool, n_req)
        # per-slot request lists (arrival order) for latency bookkeeping
        order = np.argsort(slot_req, kind="stable")
        starts = np.searchsorted(slot_req[order], np.arange(self.pool + 1))
        times_by_slot = t_arr[order]
        arrived = np.zeros(self.pool, dtype=np.int64)     # requests arrived so far, per slot
        served = np.zeros(self.pool, dtype=np.int64)      # requests answered, per slot
        in_flight = np.zeros(self.pool, dtype=bool)
        lat = []
        batches = 0
        solves = 0
        sizes = []
        busy = [None] * len(self.streams)
        next_req = 0
        # warm the solver (models resident, first factorisations) before the clock starts
        self.bad_status = 0
        self.status_counts = {}
        self.batch_log = []
        for _ in range(warmup_batches):
            for lo in range(0, self.pool, self.max_batch):
                sl = np.arange(lo, min(lo + self.max_batch, self.pool))
                self._solve_sync(sl, np.ones(len(sl), dtype=np.int64))
        next_churn = churn_period if churn_period and churn_period > 0 else float("inf")
        t0 = time.perf_counter()
        while True:
            now = time.perf_counter() - t0
            # arrivals
            hi = np.searchsorted(t_arr, now, side="right")
            if hi > next_req:
                np.add.at(arrived, slot_req[next_req:hi], 1)
                next_req = hi
            # completions
            for si, b in enumerate(busy):
                if b is not None and b["event"].query():
                    t_done = time.perf_counter() - t0
                    sl, cover = b["slots"], b["cover"]
                    stv = self.h_out[si]["st"].numpy()[:len(sl)]
                    self.bad_status += int(np.count_nonzero(stv != 0))
                    for v in np.unique(stv):
                        self.status_counts[int(v)] = self.status_counts.get(int(v), 0) + int(np.count_nonzero(stv == v))
                    self.batch_log.append((len(sl), t_done - b["t_start"], b["t_start"]))
                    lat.append(self._latencies(times_by_slot, starts, served, sl, cover, t_done))
                    served[sl] = cover
                    in_flight[sl] = False
                    solves += len(sl)
                    busy[si] = None
            # new batches on free streams
            for si in range(len(self.streams)):
                if busy[si] is not None:
                    continue
                ready = np.nonzero((arrived > served) & ~in_flight)[0]
                if len(ready) == 0:
                    continue
                sl = ready[:self.max_batch]
                busy[si] = self._launch(si, sl, arrived[sl] - served[sl])
                busy[si]["cover"] = arrived[sl].copy()
                busy[si]["t_start"] = time.perf_counter() - t0
                in_flight[sl] = True
                batches += 1
                sizes.append(len(sl))
            if now >= next_churn:
                # leave/join: slots with no batch in flight are swapped (the
                # model upload is ordered before any later batch of theirs)
                self.churn(churn_frac, rng, idle=~in_flight)
                next_churn += churn_period
            if next_req >= n_req and all(b is None for b in busy) and not np.any(arrived > served):
                break
            if now > duration * 20 + 60:
                break
        wall = time.perf_counter() - t0
        lat = np.concatenate(lat) if lat else np.zeros(0)
        return dict(requests=int(n_req), rate=rate, duration=duration, wall_s=wall, solves=int(solves),
                    not_solved=int(self.bad_status),
                    solves_per_s=solves / wall, batches=batches, mean_batch=float(np.mean(sizes)) if sizes else 0.0,
                    p50_ms=float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
                    p99_ms=float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
                    coalesced_frac=1.0 - solves / max(n_req, 1))

    @staticmethod
    def _latencies(times_by_slot, starts, served, sl, cover, t_done):
        # requests [served, cover) of each slot in the batch are answered now
        cnt = cover - served[sl]
        if cnt.sum() == 0:
            return np.zeros(0)
        first = starts[sl] + served[sl]
        idx = np.repeat(first - np.cumsum(cnt) + cnt, cnt) + np.arange(cnt.sum())
        return t_done - times_by_slot[idx]

    def _fill(self, si, sl, steps):
        h = self.h_in[si]
        n = len(sl)
        x0, qd, cmd, ph = self.walk.advance(self.slot_agent[sl], steps)
        h["ids"].numpy()[:n] = sl
        h["x0"].numpy()[:n] = x0
        h["qd"].numpy()[:n] = qd
        h["cmd"].numpy()[:n] = cmd
        h["ph"].numpy()[:n] = ph
        return n

    def _launch(self, si, sl, steps):
        torch = self.torch
        n = self._fill(si, sl, steps)
        st = self.streams[si]
        d, h, do, ho = self.d_in[si], self.h_in[si], self.d_out[si], self.h_out[si]
        with torch.cuda.stream(st):
            for k in ("ids", "x0", "qd", "cmd", "ph"):
                d[k][:n].copy_(h[k][:n], non_blocking=True)
            tk = self.solver.submit(d["ids"][:n], d["x0"][:n], d["qd"][:n], d["cmd"][:n], d["ph"][:n])
            self.solver.solve(tk, stream=st.cuda_stream)
            self.solver.get_torques(tk, tau=do["tau"][:n], status=do["st"][:n])
            ho["tau"][:n].copy_(do["tau"][:n], non_blocking=True)
            ho["st"][:n].copy_(do["st"][:n], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return dict(slots=sl, event=ev)

    def _solve_sync(self, sl, steps):
        b = self._launch(0, sl, steps)
        b["event"].synchronize()


def streams_range(n):
    return range(n)


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
