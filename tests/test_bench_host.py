"""Host logic of bench.py (CPU): the clock-sample window and throttle reasons,
weak-scaling shards, whole-job throughput, and the algorithmic FLOP count."""
import datetime
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _row(t, mhz, reasons=()):
    stamp = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ", ".join("Active" if n in reasons else "Not Active" for n in names)
    return f"{stamp}, 0, {mhz}, 2032, 500.0, 0x0, {flags}\n"


def test_clock_summary_keeps_the_timed_window(tmp_path):
    b = _bench()
    c = b.ClockSampler(0)
    c.path = str(tmp_path / "clocks.csv")
    t0 = 1_800_000_000.0
    with open(c.path, "w") as f:
        f.write(_row(t0 - 1.0, 1100, ("hw_slowdown",)))       # before the window: ignored
        f.write(_row(t0 + 0.02, 2032))
        f.write(_row(t0 + 0.04, 2000, ("sw_power_cap",)))
        f.write(_row(t0 + 0.06, 2032))
        f.write(_row(t0 + 2.0, 900, ("hw_thermal_slowdown",)))  # after: ignored
    c.t_begin, c.t_end = t0, t0 + 0.07
    s = c.summary()
    assert s["samples"] == 3 and s["window"] == "timed region"
    assert s["sm_mhz"] == 2032.0 and s["sm_max_mhz"] == 2032.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_nearest_sample_and_unsampled(tmp_path):
    b = _bench()
    c = b.ClockSampler(0)
    c.path = str(tmp_path / "clocks.csv")
    t0 = 1_800_000_000.0
    with open(c.path, "w") as f:
        f.write(_row(t0 - 3.0, 1500))
        f.write(_row(t0 + 0.5, 1900))
    c.t_begin, c.t_end = t0, t0 + 0.1          # no sample inside: the nearest one
    s = c.summary()
    assert s["samples"] == 1 and s["sm_mhz"] == 1900.0 and s["window"].startswith("nearest")
    c.path = str(tmp_path / "missing.csv")
    assert c.summary()["reasons"] == ["unsampled"]


def test_shards_and_throughput():
    b = _bench()
    world, n = 4, 1000
    ids = np.concatenate([b.shard_ids(n, r, world) for r in range(world)])
    np.testing.assert_array_equal(ids, np.arange(world * n))      # a partition, no overlap
    v, ms = b.job_throughput(n, 10, 250.0, 1)
    assert ms == 250.0 and abs(v - n * 10 / 0.25) < 1e-6


def test_flop_model():
    b = _bench()
    N = np.array([10, 20])
    zero = np.zeros(2, int)
    polished = b.flops_per_agent(N, zero, zero, np.array([2, 2]))
    with_admm = b.flops_per_agent(N, np.array([50, 50]), zero, np.array([1, 1]))
    assert polished[1] == 2 * polished[0]                 # linear in the horizon
    assert (with_admm > polished).all()                   # ADMM adds its factor and iterations
    # the factor's count: two dense 22^3 products, a symmetric inverse, the
    # sparse A/B products by their nonzeros, one mat-vec
    n = 22
    assert b.FACTOR_STAGE == 2 * 2 * n ** 3 + n ** 3 + 2 * n * (3 * 64 + 2 * 74) + 2 * n * n
    assert polished[0] == 10 * (b.POLISH_STAGE + b.REFINE_STAGE)
    two = b.flops_per_agent(N, zero, zero, np.array([2, 2]), attempts=2.0)
    assert np.allclose(two - polished, polished)          # a second reduced solve costs the same
    assert b.attempts_mean([0, 3, 1]) == 1.25


def test_literal_bytes_per_iteration():
    b = _bench()
    # per stage: L by columns and by rows (3105 each), 1/D (90), the state and
    # row data; G_k in both passes for the stages that couple to a neighbour
    one = 4 * (2 * 3105 + 90 + b.LDL_STATE)
    assert b.ldl_bytes_per_iteration(np.array([1]))[0] == one
    assert b.ldl_bytes_per_iteration(np.array([3]))[0] == 3 * one + 4 * 2 * 2 * 900
    # the kinematic rows: the L31 rows staged in both passes, the eight rows' data
    kin = b.ldl_bytes_per_iteration(np.array([3]), kin=1)[0] - b.ldl_bytes_per_iteration(np.array([3]))[0]
    assert kin == 3 * 4 * (2 * 96 + 2 * 2 * 8 + 3 * 8)
