"""The arithmetic-throughput microbenchmarks that give the solver's roofline
its measured ceilings: each runs, and none reports more than its unit can do
at the maximum SM clock (a rate above that would mean a miscounted kernel)."""
import math

import pytest

pytestmark = pytest.mark.gpu

N_SM, FP32_LANES, FP64_LANES, MAX_MHZ = 148, 128, 64, 2032.0


@pytest.fixture(scope="module")
def mpcgpu():
    import __graft_entry__ as g
    g.build()
    from paper_2510_12717_b300 import mpcgpu
    return mpcgpu


def test_fp32_fma_rate_is_bounded_by_the_derived_peak(mpcgpu):
    tf, ms = mpcgpu.measure_peak(mpcgpu.PEAK_FP32_FMA)
    derived = N_SM * FP32_LANES * 2 * MAX_MHZ * 1e6 / 1e12
    assert ms > 0
    assert 0.25 * derived < tf <= 1.02 * derived, (tf, derived)


def test_fp64_and_mma_sync_rates_are_finite(mpcgpu):
    fp32, _ = mpcgpu.measure_peak(mpcgpu.PEAK_FP32_FMA)
    fp64, _ = mpcgpu.measure_peak(mpcgpu.PEAK_FP64_FMA)
    tf32, _ = mpcgpu.measure_peak(mpcgpu.PEAK_TF32_MMA_SYNC)
    bf16, _ = mpcgpu.measure_peak(mpcgpu.PEAK_BF16_MMA_SYNC)
    for v in (fp64, tf32, bf16):
        assert math.isfinite(v) and v > 0
    # one FP64 FMA lane per two FP32 lanes at most on any part of this family
    assert fp64 <= N_SM * FP64_LANES * 2 * MAX_MHZ * 1e6 / 1e12 * 1.02
