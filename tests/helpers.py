"""Shared helpers of the GPU tests: inputs as the device sees them, the
oracle on the same inputs, and the tolerance of the parity bar."""
import numpy as np

from workload import make_agents, make_inputs

# torque tolerance (elementwise allclose) and residual bar
RTOL, ATOL = 1e-3, 1e-4
RES_TOL = 1e-4
# model fields kept in double precision on the device (schedule decisions)
_DOUBLE_FIELDS = {"dt", "period", "duty", "offset", "N", "gait"}


def device_inputs(inp):
    """Inputs rounded to float32, as the C ABI takes them."""
    return {k: np.ascontiguousarray(v, dtype=np.float32) for k, v in inp.items()}


def oracle_view(model, inp32):
    """Model and inputs for the oracle: float32-representable values (what the
    device stores) promoted to float64; schedule fields kept as given."""
    m = {}
    for k, v in model.items():
        m[k] = v if k in _DOUBLE_FIELDS else np.asarray(v, np.float32).astype(np.float64)
    i = {k: v.astype(np.float64) for k, v in inp32.items()}
    return m, i


def torque_close(got, ref):
    return np.abs(got - ref) <= ATOL + RTOL * np.abs(ref)


def agents(name, ids=None, replan=0):
    if replan:
        return make_inputs(name, ids, replan)
    return make_agents(name, ids)
