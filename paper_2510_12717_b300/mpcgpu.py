"""ctypes binding of libmpcgpu.so (C ABI in include/mpcgpu.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Device buffers are torch CUDA tensors (passed by data_ptr());
streams are torch streams.  There is no CPU fallback: load() raises when the
library is missing or cannot be loaded.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpcgpu.so")

MPC_OK, MPC_ERR_INVALID, MPC_ERR_BUDGET, MPC_ERR_CUDA = 0, 1, 2, 3
MPC_ERR_NOT_READY, MPC_ERR_TIMEOUT, MPC_ERR_STATE = 4, 5, 6
AGENT_SOLVED, AGENT_MAX_ITER, AGENT_PRIMAL_INFEAS, AGENT_DUAL_INFEAS, AGENT_NAN, AGENT_TIMEOUT = 0, 1, 2, 3, 4, 5
AGENT_INACCURATE, AGENT_DEFERRED = 6, 7
SOLVE_DEFER_ADMM, SOLVE_ADMM_ONLY, SOLVE_DEFER_SLOW, SOLVE_DEFER_COLD = 1, 2, 4, 8
FORM_PLAIN, FORM_FUSED, FORM_LDL = 0, 1, 2
FP32, TF32, BF16, FP64, TF32X3 = 0, 1, 2, 3, 4
PEAK_FP32_FMA, PEAK_FP64_FMA, PEAK_TF32_MMA_SYNC, PEAK_BF16_MMA_SYNC = 0, 1, 2, 3

STATUS_NAMES = {0: "MPC_OK", 1: "MPC_ERR_INVALID", 2: "MPC_ERR_BUDGET", 3: "MPC_ERR_CUDA",
                4: "MPC_ERR_NOT_READY", 5: "MPC_ERR_TIMEOUT", 6: "MPC_ERR_STATE"}


class MpcConfig(C.Structure):
    _fields_ = [
        ("device", C.c_int), ("stream", C.c_void_p), ("max_agents", C.c_int),
        ("max_horizon", C.c_int), ("hbm_budget_bytes", C.c_size_t), ("precision", C.c_int),
        ("form", C.c_int), ("rho0", C.c_float), ("sigma", C.c_float), ("alpha", C.c_float),
        ("eps_abs", C.c_float), ("eps_rel", C.c_float), ("max_iter", C.c_int),
        ("fixed_iters", C.c_int), ("check_every", C.c_int), ("adaptive_rho", C.c_int),
        ("polish", C.c_int), ("warm_start", C.c_int), ("variant", C.c_int),
        ("early_polish", C.c_float), ("graph", C.c_int), ("warm_polish", C.c_int),
        ("refine_steps", C.c_int), ("spin_limit", C.c_int), ("wait_test_agent", C.c_int),
        ("ruiz_iters", C.c_int), ("kin_rows", C.c_int), ("swing_height", C.c_float),
        ("v_takeoff", C.c_float), ("v_touchdown", C.c_float),
    ]


class MpcAgentModel(C.Structure):
    _fields_ = [
        ("mass", C.c_double), ("inertia", C.c_double * 3), ("lever", (C.c_double * 3) * 2),
        ("J_leg", ((C.c_double * 5) * 6) * 2), ("M_j", C.c_double * 18), ("h_j", C.c_double * 18),
        ("Kp", C.c_double * 18), ("Kd", C.c_double * 18), ("Q", C.c_double * 30),
        ("R", C.c_double * 30), ("mu", C.c_double), ("fz_max", C.c_double),
        ("qd_max", C.c_double), ("q_lim", C.c_double), ("N", C.c_int), ("dt", C.c_double),
        ("gait", C.c_int), ("period", C.c_double), ("duty", C.c_double * 2),
        ("offset", C.c_double * 2), ("q_nom", C.c_double * 18),
    ]


# numpy mirror of mpc_agent_model (C alignment), for vectorised packing
MODEL_DTYPE = np.dtype([
    ("mass", "f8"), ("inertia", "f8", 3), ("lever", "f8", (2, 3)), ("J_leg", "f8", (2, 6, 5)),
    ("M_j", "f8", 18), ("h_j", "f8", 18), ("Kp", "f8", 18), ("Kd", "f8", 18), ("Q", "f8", 30),
    ("R", "f8", 30), ("mu", "f8"), ("fz_max", "f8"), ("qd_max", "f8"), ("q_lim", "f8"),
    ("N", "i4"), ("dt", "f8"), ("gait", "i4"), ("period", "f8"), ("duty", "f8", 2),
    ("offset", "f8", 2), ("q_nom", "f8", 18),
], align=True)

class MpcTreeModel(C.Structure):
    _fields_ = [
        ("axis", (C.c_double * 3) * 18), ("offset", (C.c_double * 3) * 18), ("mass", C.c_double * 18),
        ("com", (C.c_double * 3) * 18), ("inertia", (C.c_double * 3) * 18),
    ]


# numpy mirror of mpc_tree_model; field name -> key of the model dict (workload.make_trees)
TREE_DTYPE = np.dtype([("axis", "f8", (18, 3)), ("offset", "f8", (18, 3)), ("mass", "f8", 18),
                       ("com", "f8", (18, 3)), ("inertia", "f8", (18, 3))], align=True)
TREE_KEYS = {"axis": "tree_axis", "offset": "tree_offset", "mass": "tree_mass", "com": "tree_com",
             "inertia": "tree_inertia"}


def pack_trees(trees: dict, idx=None) -> np.ndarray:
    """Tree arrays (tree_axis, tree_offset, tree_mass, tree_com, tree_inertia)
    -> mpc_tree_model array."""
    B = len(trees["tree_mass"])
    idx = np.arange(B) if idx is None else np.asarray(idx)
    out = np.zeros(len(idx), dtype=TREE_DTYPE)
    for name, key in TREE_KEYS.items():
        out[name] = np.asarray(trees[key])[idx]
    return out


# every function the header declares: name -> (restype, argtypes)
_P, _I32P, _U64P = C.c_void_p, C.c_void_p, C.POINTER(C.c_uint64)
SIGNATURES = {
    "mpc_default_config": (C.c_int, [C.POINTER(MpcConfig)]),
    "mpc_create": (C.c_int, [C.POINTER(MpcConfig), C.POINTER(C.c_void_p)]),
    "mpc_destroy": (C.c_int, [_P]),
    "mpc_set_models": (C.c_int, [_P, C.c_int32, _P, _P]),
    "mpc_set_model": (C.c_int, [_P, C.c_int32, _P]),
    "mpc_release_agent": (C.c_int, [_P, C.c_int32]),
    "mpc_submit": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, _P, _U64P]),
    "mpc_solve": (C.c_int, [_P, C.c_uint64]),
    "mpc_solve_on": (C.c_int, [_P, C.c_uint64, _P]),
    "mpc_solve_ex": (C.c_int, [_P, C.c_uint64, _P, C.c_int32]),
    "mpc_set_models_async": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "mpc_autotune": (C.c_int, [_P, C.c_uint64, C.c_int32, C.c_char_p, C.c_size_t]),
    "mpc_get_torques": (C.c_int, [_P, C.c_uint64, _P, _P, _P, _P, _P]),
    "mpc_solve_host": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "mpc_get_agent_stats": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, _P, _P, _P, _P]),
    "mpc_export_state": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, _P]),
    "mpc_import_state": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, C.c_float]),
    "mpc_export_qp": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, _P, _P, _P]),
    "mpc_solve_static": (C.c_int, [C.c_int32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "mpc_get_stats": (C.c_int, [_P, C.c_char_p, C.c_size_t]),
    "mpc_last_error": (C.c_char_p, [_P]),
    "mpc_set_policy": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, C.c_float]),
    "mpc_policy_torques": (C.c_int, [_P, C.c_uint64, _P, _P]),
    "mpc_set_trees": (C.c_int, [_P, C.c_int32, _P, _P]),
    "mpc_measure_peak": (C.c_int, [C.c_int32, _P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mpc_server_create": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_void_p)]),
    "mpc_server_start": (C.c_int, [_P]),
    "mpc_server_set_defer": (C.c_int, [_P, C.c_int32]),
    "mpc_server_deferred": (C.c_int64, [_P]),
    "mpc_server_push": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, _P, _P]),
    "mpc_server_set_models": (C.c_int, [_P, C.c_int32, _P, _P]),
    "mpc_server_drain": (C.c_int, [_P, C.c_double]),
    "mpc_server_clock": (C.c_double, [_P]),
    "mpc_server_results": (C.c_int, [_P, _P, C.c_int64, C.POINTER(C.c_int64), _P, _P, _P]),
    "mpc_server_batches": (C.c_int, [_P, _P, C.c_int64, C.POINTER(C.c_int64)]),
    "mpc_server_stop": (C.c_int, [_P]),
    "mpc_server_last_error": (C.c_char_p, [_P]),
    "mpc_server_destroy": (C.c_int, [_P]),
    "mpc_load_start": (C.c_int, [_P, C.c_int64, _P, _P, C.c_int32, _P, _P, _P, C.c_float, C.c_float, C.c_float,
                                 C.c_uint64, C.POINTER(C.c_void_p)]),
    "mpc_load_reset": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P]),
    "mpc_load_wait": (C.c_int, [_P, C.c_double, _P]),
    "mpc_load_destroy": (C.c_int, [_P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libmpcgpu.so and declare its signatures.  Raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libmpcgpu.so not built ({path}); run __graft_entry__.build() "
                           "or python -m paper_2510_12717_b300.build")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MpcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def pack_models(model: dict, idx=None) -> np.ndarray:
    """SoA model dict (workload.make_agents layout) -> mpc_agent_model array."""
    B = len(model["mass"])
    idx = np.arange(B) if idx is None else np.asarray(idx)
    out = np.zeros(len(idx), dtype=MODEL_DTYPE)
    for name in MODEL_DTYPE.names:
        out[name] = np.asarray(model[name])[idx]
    return out


STATIC_MAX_AGENTS = 64
STATIC_MAX_HORIZON = 20
MAX_HORIZON = 32          # MPC_MAX_HORIZON: the largest horizon a context may take


def solve_static(model: dict, x0, qd_meas, cmd, phase, *, tau=None, q_set=None, qd_set=None,
                 value=None, status=None, stream=None, idx=None) -> int:
    """mpc_solve_static: allocation-free cold solve of up to 64 agents.

    For callers that cannot allocate device memory at solve time.  Inputs and
    outputs are caller-owned device tensors; returns the mpc_status code.
    """
    lib = load()
    recs = pack_models(model, idx)
    return lib.mpc_solve_static(len(recs), recs.ctypes.data, _ptr(x0), _ptr(qd_meas), _ptr(cmd),
                                _ptr(phase), _ptr(tau), _ptr(q_set), _ptr(qd_set), _ptr(value),
                                _ptr(status), stream)


def measure_peak(kind: int, stream=None) -> tuple[float, float]:
    """mpc_measure_peak: (TFLOP/s, ms per launch) of one arithmetic unit."""
    lib = load()
    tf, ms = C.c_double(0.0), C.c_double(0.0)
    st = lib.mpc_measure_peak(kind, stream, C.byref(tf), C.byref(ms))
    if st != MPC_OK:
        raise MpcError(st, f"mpc_measure_peak({kind}) failed")
    return tf.value, ms.value


class Solver:
    """One library context (mpc_create ... mpc_destroy)."""

    def __init__(self, max_agents: int = 16384, max_horizon: int = 20, *, form: int = FORM_FUSED,
                 device: int = 0, stream=None, hbm_budget_bytes: int = 0, **opts):
        self.lib = load()
        cfg = MpcConfig()
        self._check(self.lib.mpc_default_config(C.byref(cfg)), None)
        cfg.device = device
        cfg.stream = stream
        cfg.max_agents = max_agents
        cfg.max_horizon = max_horizon
        cfg.form = form
        cfg.hbm_budget_bytes = hbm_budget_bytes
        for k, v in opts.items():
            if not hasattr(cfg, k):
                raise TypeError(f"unknown solver option {k}")
            setattr(cfg, k, v)
        self.cfg = cfg
        h = C.c_void_p()
        st = self.lib.mpc_create(C.byref(cfg), C.byref(h))
        if st != MPC_OK:
            raise MpcError(st, "mpc_create failed")
        self.ctx = h

    def _check(self, st, ctx=True):
        if st != MPC_OK:
            msg = self.lib.mpc_last_error(self.ctx).decode() if ctx else ""
            raise MpcError(st, msg)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.mpc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- models
    def set_models(self, model: dict, agent_ids, idx=None):
        """mpc_set_models; when the model dict also holds kinematic trees
        (tree_* keys, workload.make_trees), mpc_set_trees for the same agents."""
        recs = pack_models(model, idx)
        ids = np.ascontiguousarray(agent_ids, dtype=np.int32)
        assert len(ids) == len(recs)
        self._check(self.lib.mpc_set_models(self.ctx, len(ids), _ptr(ids), recs.ctypes.data))
        if "tree_axis" in model:
            self.set_trees(model, ids, idx)

    def set_models_async(self, model: dict, agent_ids, stream, idx=None):
        """mpc_set_models_async: the upload is enqueued on `stream` (a
        cudaStream_t handle) and the call returns at once (no trees)."""
        recs = pack_models(model, idx)
        ids = np.ascontiguousarray(agent_ids, dtype=np.int32)
        assert len(ids) == len(recs)
        self._check(self.lib.mpc_set_models_async(self.ctx, len(ids), _ptr(ids), recs.ctypes.data, stream))

    def set_trees(self, trees: dict, agent_ids, idx=None):
        """mpc_set_trees: kinematic trees for the agents' torque maps."""
        recs = pack_trees(trees, idx)
        ids = np.ascontiguousarray(agent_ids, dtype=np.int32)
        assert len(ids) == len(recs)
        self._check(self.lib.mpc_set_trees(self.ctx, len(ids), _ptr(ids), recs.ctypes.data))

    def release(self, agent_id: int):
        self._check(self.lib.mpc_release_agent(self.ctx, int(agent_id)))

    # -- device-buffer path
    def submit(self, ids, x0, qd_meas, cmd, phase) -> int:
        t = C.c_uint64()
        self._check(self.lib.mpc_submit(self.ctx, int(ids.shape[0]), _ptr(ids), _ptr(x0), _ptr(qd_meas),
                                        _ptr(cmd), _ptr(phase), C.byref(t)))
        return t.value

    def solve(self, ticket: int, stream=None, flags: int = 0):
        """mpc_solve (context stream) or mpc_solve_on (stream: a cudaStream_t
        handle); with flags (SOLVE_DEFER_ADMM, SOLVE_ADMM_ONLY) mpc_solve_ex."""
        if flags:
            self._check(self.lib.mpc_solve_ex(self.ctx, C.c_uint64(ticket), stream, int(flags)))
        elif stream is None:
            self._check(self.lib.mpc_solve(self.ctx, C.c_uint64(ticket)))
        else:
            self._check(self.lib.mpc_solve_on(self.ctx, C.c_uint64(ticket), stream))

    def autotune(self, ticket: int, repeats: int = 2) -> dict:
        """mpc_autotune: time the tunables on the ticket's batch, keep the fastest."""
        import json
        buf = C.create_string_buffer(8192)
        self._check(self.lib.mpc_autotune(self.ctx, C.c_uint64(ticket), repeats, buf, 8192))
        return json.loads(buf.value.decode())

    def get_torques(self, ticket: int, tau=None, q_set=None, qd_set=None, value=None, status=None):
        self._check(self.lib.mpc_get_torques(self.ctx, C.c_uint64(ticket), _ptr(tau), _ptr(q_set),
                                             _ptr(qd_set), _ptr(value), _ptr(status)))

    # -- residual policy (paper Sec. IV) blended into the MPC torques
    def set_policy(self, weights: dict, blend_lambda: float = 0.1):
        """weights: W1..W4 ([in][out]) and b1..b4 as FP32 arrays
        (workload.make_policy layout)."""
        arrs = []
        for l in (1, 2, 3, 4):
            arrs.append(np.ascontiguousarray(weights[f"W{l}"], np.float32))
            arrs.append(np.ascontiguousarray(weights[f"b{l}"], np.float32))
        self._keep_policy = arrs
        self._check(self.lib.mpc_set_policy(self.ctx, *[_ptr(a) for a in arrs], C.c_float(blend_lambda)))

    def policy_torques(self, ticket: int, tau=None, action=None):
        """Enqueue the policy for a solved ticket (before get_torques)."""
        self._check(self.lib.mpc_policy_torques(self.ctx, C.c_uint64(ticket), _ptr(tau), _ptr(action)))

    # -- host-buffer path (numpy in, numpy out)
    def solve_host(self, ids, x0, qd_meas, cmd, phase, *, tau=None, q_set=None, qd_set=None,
                   value=None, status=None):
        n = len(ids)
        ids = np.ascontiguousarray(ids, np.int32)
        x0 = np.ascontiguousarray(x0, np.float32)
        qd_meas = np.ascontiguousarray(qd_meas, np.float32)
        cmd = np.ascontiguousarray(cmd, np.float32)
        phase = np.ascontiguousarray(phase, np.float32)
        tau = np.empty((n, 18), np.float32) if tau is None else tau
        q_set = np.empty((n, 18), np.float32) if q_set is None else q_set
        qd_set = np.empty((n, 18), np.float32) if qd_set is None else qd_set
        value = np.empty(n, np.float32) if value is None else value
        status = np.empty(n, np.int32) if status is None else status
        self._check(self.lib.mpc_solve_host(self.ctx, n, _ptr(ids), _ptr(x0), _ptr(qd_meas), _ptr(cmd),
                                            _ptr(phase), _ptr(tau), _ptr(q_set), _ptr(qd_set),
                                            _ptr(value), _ptr(status)))
        return dict(tau=tau, q_set=q_set, qd_set=qd_set, value=value, status=status)

    # -- inspection
    def agent_stats(self, ids):
        ids = np.ascontiguousarray(ids, np.int32)
        n = len(ids)
        it = np.empty(n, np.int32)
        rf = np.empty(n, np.int32)
        po = np.empty(n, np.int32)
        rp = np.empty(n, np.float32)
        rd = np.empty(n, np.float32)
        pn = np.empty(n, np.float32)
        dn = np.empty(n, np.float32)
        self._check(self.lib.mpc_get_agent_stats(self.ctx, n, _ptr(ids), _ptr(it), _ptr(rf), _ptr(po),
                                                 _ptr(rp), _ptr(rd), _ptr(pn), _ptr(dn)))
        return dict(iters=it, refactors=rf, polished=po, prim_res=rp, dual_res=rd, prim_scaled=pn,
                    dual_scaled=dn)

    def export_state(self, agent_id: int, N: int):
        x = np.empty((N + 1, 30), np.float32)
        u = np.empty((N, 30), np.float32)
        w = np.empty((N, 56), np.float32)
        y = np.empty((N, 56), np.float32)
        rho = np.empty(1, np.float32)
        self._check(self.lib.mpc_export_state(self.ctx, int(agent_id), _ptr(x), _ptr(u), _ptr(w),
                                              _ptr(y), _ptr(rho)))
        return dict(x=x, u=u, w=w, y=y, rho=float(rho[0]))

    def export_qp(self, agent_id: int, N: int) -> dict:
        """mpc_export_qp: references, row bounds and linearised dynamics of the
        agent's last solve."""
        out = dict(x_ref=np.empty((N + 1, 30), np.float32), u_ref=np.empty((N, 30), np.float32),
                   lo=np.empty((N, 56), np.float32), hi=np.empty((N, 56), np.float32),
                   A=np.empty((N, 30, 30), np.float32), B=np.empty((N, 30, 30), np.float32),
                   c=np.empty((N, 30), np.float32))
        self._check(self.lib.mpc_export_qp(self.ctx, int(agent_id), *[_ptr(out[k]) for k in
                                                                     ("x_ref", "u_ref", "lo", "hi", "A", "B", "c")]))
        return out

    def import_state(self, agent_id: int, st: dict):
        arrs = [np.ascontiguousarray(st[k], np.float32) for k in ("x", "u", "w", "y")]
        self._check(self.lib.mpc_import_state(self.ctx, int(agent_id), *[_ptr(a) for a in arrs],
                                              C.c_float(st["rho"])))

    def stats(self) -> dict:
        import json
        buf = C.create_string_buffer(4096)
        self._check(self.lib.mpc_get_stats(self.ctx, buf, 4096))
        return json.loads(buf.value.decode())


class Server:
    """Continuous-batching server over a Solver's context (mpc_server_*).

    While it runs the context is the server's: make no other Solver call
    until stop().  Inputs are copied on push; results() copies the answered
    requests' latencies, each slot's last torques and status, and counters."""

    def __init__(self, solver: Solver, pool: int, max_batch: int = 0, max_inflight: int = 2):
        self.lib = load()
        self.solver = solver
        self.pool = pool
        h = C.c_void_p()
        st = self.lib.mpc_server_create(solver.ctx, pool, max_batch or pool, max_inflight, C.byref(h))
        if st != MPC_OK:
            raise MpcError(st, "mpc_server_create failed")
        self.srv = h

    def _check(self, st):
        if st != MPC_OK:
            raise MpcError(st, self.lib.mpc_server_last_error(self.srv).decode())

    def set_defer(self, mode: int = 1):
        """mpc_server_set_defer (before start()): 1 = agents whose polish
        first fails, 2 = also those two reduced KKT solves do not settle,
        3 = as 2 for cold agents and as 1 for warm ones, finish in batches
        of their own; 0 = off."""
        self._check(self.lib.mpc_server_set_defer(self.srv, int(mode)))

    def deferred(self) -> int:
        return int(self.lib.mpc_server_deferred(self.srv))

    def start(self):
        self._check(self.lib.mpc_server_start(self.srv))

    def clock(self) -> float:
        return self.lib.mpc_server_clock(self.srv)

    def push(self, slots, x0, qd_meas, cmd, phase, t_arrive):
        slots = np.ascontiguousarray(slots, np.int32)
        x0 = np.ascontiguousarray(x0, np.float32)
        qd_meas = np.ascontiguousarray(qd_meas, np.float32)
        cmd = np.ascontiguousarray(cmd, np.float32)
        phase = np.ascontiguousarray(phase, np.float32)
        t_arrive = np.ascontiguousarray(t_arrive, np.float64)
        self._check(self.lib.mpc_server_push(self.srv, len(slots), _ptr(slots), _ptr(x0), _ptr(qd_meas),
                                             _ptr(cmd), _ptr(phase), _ptr(t_arrive)))

    def set_models(self, model: dict, slots, idx=None):
        recs = pack_models(model, idx)
        slots = np.ascontiguousarray(slots, np.int32)
        self._keep = recs
        self._check(self.lib.mpc_server_set_models(self.srv, len(slots), _ptr(slots), recs.ctypes.data))

    def drain(self, timeout_s: float = 60.0):
        self._check(self.lib.mpc_server_drain(self.srv, C.c_double(timeout_s)))

    def results(self):
        n = C.c_int64(0)
        self._check(self.lib.mpc_server_results(self.srv, None, 0, C.byref(n), None, None, None))
        lat = np.empty(max(n.value, 1), np.float64)
        tau = np.empty((self.pool, 18), np.float32)
        status = np.empty(self.pool, np.int32)
        cnt = np.zeros(6, np.int64)
        self._check(self.lib.mpc_server_results(self.srv, _ptr(lat), len(lat), C.byref(n), _ptr(tau),
                                                _ptr(status), _ptr(cnt)))
        keys = ("pushed", "answered", "batches", "solves", "not_solved", "swapped")
        return dict(latency=lat[:min(n.value, len(lat))], tau=tau, status=status, **dict(zip(keys, cnt.tolist())))

    def batches(self):
        """Completed batches: array [n][3] of launch time, completion time (s), agents."""
        n = C.c_int64(0)
        self._check(self.lib.mpc_server_batches(self.srv, None, 0, C.byref(n)))
        log = np.zeros((max(n.value, 1), 3), np.float64)
        self._check(self.lib.mpc_server_batches(self.srv, _ptr(log), len(log), C.byref(n)))
        return log[:n.value]

    def stop(self):
        self._check(self.lib.mpc_server_stop(self.srv))

    def close(self):
        if getattr(self, "srv", None):
            self.lib.mpc_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Load:
    """Synthetic request source replaying an arrival trace in real time into
    a Server (mpc_load_*): one mean-reverting walk step of the agent's state
    per request, from a native thread."""

    def __init__(self, server: Server, t_arrive, slots, x_init, cmd, phase, *, revert=0.95, sigma=0.02,
                 phase_step=0.02, seed=0):
        self.lib = load()
        t = np.ascontiguousarray(t_arrive, np.float64)
        sl = np.ascontiguousarray(slots, np.int32)
        x = np.ascontiguousarray(x_init, np.float32)
        c = np.ascontiguousarray(cmd, np.float32)
        p = np.ascontiguousarray(phase, np.float32)
        h = C.c_void_p()
        st = self.lib.mpc_load_start(server.srv, len(t), _ptr(t), _ptr(sl), server.pool, _ptr(x), _ptr(c), _ptr(p),
                                     C.c_float(revert), C.c_float(sigma), C.c_float(phase_step), C.c_uint64(seed),
                                     C.byref(h))
        if st != MPC_OK:
            raise MpcError(st, "mpc_load_start failed")
        self.h = h

    def reset(self, slots, x_init, cmd, phase):
        sl = np.ascontiguousarray(slots, np.int32)
        st = self.lib.mpc_load_reset(self.h, len(sl), _ptr(sl), _ptr(np.ascontiguousarray(x_init, np.float32)),
                                     _ptr(np.ascontiguousarray(cmd, np.float32)),
                                     _ptr(np.ascontiguousarray(phase, np.float32)))
        if st != MPC_OK:
            raise MpcError(st, "mpc_load_reset failed")

    def wait(self, timeout_s: float = 60.0):
        """Blocks until every request was pushed; returns (median, p99, max) push lag in seconds."""
        lag = np.zeros(3, np.float64)
        st = self.lib.mpc_load_wait(self.h, C.c_double(timeout_s), _ptr(lag))
        if st != MPC_OK:
            raise MpcError(st, "mpc_load_wait failed")
        return tuple(lag.tolist())

    def close(self):
        if getattr(self, "h", None):
            self.lib.mpc_load_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
