"""Pins for the oracle's schedule and references (paper Sec. III-A)."""
import math
import os

import numpy as np
import pytest

from oracle import refs
from workload import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "contact_schedule.txt")
GAITS = {"walk": gen.GAIT_WALK, "stand": gen.GAIT_STAND, "hop": gen.GAIT_HOP,
         "single_l": gen.GAIT_SINGLE_L, "single_r": gen.GAIT_SINGLE_R}


def _model(gait, N):
    period, duty, off = gen._GAIT_TABLE[gait]
    return dict(N=N, dt=0.02, period=period, duty=np.array(duty),
                offset=np.array(off), mass=25.0, q_nom=np.zeros(18))


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        g, ph, n, left, right = line.split()
        rows.append((g, float(ph), int(n), left, right))
    return rows


@pytest.mark.parametrize("row", _golden(), ids=lambda r: f"{r[0]}-{r[1]}")
def test_contact_schedule_golden(row):
    g, ph, n, left, right = row
    st = refs.contact_schedule(_model(GAITS[g], n), ph)
    assert "".join(str(int(b)) for b in st[:, 0]) == left
    assert "".join(str(int(b)) for b in st[:, 1]) == right


def test_force_reference_weight_split():
    # desired f_z = weight / number of feet in stance (paper Sec. III-A)
    m = _model(gen.GAIT_WALK, 10)
    st = np.array([[1, 1], [1, 0], [0, 1], [0, 0]] + [[1, 1]] * 6, dtype=bool)
    x0 = np.zeros(30)
    _, u_ref = refs.references(m, x0, (0.6, 0.0, 0.0, 0.0), st)
    w = 25.0 * 9.81
    assert u_ref[0, 2] == pytest.approx(w / 2) and u_ref[0, 8] == pytest.approx(w / 2)
    assert u_ref[1, 2] == pytest.approx(w) and u_ref[1, 8] == 0.0
    assert u_ref[2, 2] == 0.0 and u_ref[2, 8] == pytest.approx(w)
    assert np.all(u_ref[3] == 0.0)
    assert np.all(u_ref[:, [0, 1, 3, 4, 5, 6, 7, 9, 10, 11]] == 0.0)
    assert np.all(u_ref[:, 12:] == 0.0)


def test_state_reference_heuristic():
    # Eqs. des_traj_1..5: height, integrated yaw, velocity in the yaw frame
    m = _model(gen.GAIT_WALK, 4)
    m["q_nom"] = np.arange(18) * 0.01
    x0 = np.zeros(30)
    x0[5] = 0.3
    cmd = (0.62, 0.8, -0.2, 0.5)
    st = np.ones((4, 2), dtype=bool)
    x_ref, _ = refs.references(m, x0, cmd, st)
    for k in range(5):
        yaw = 0.3 + k * 0.02 * 0.5
        assert x_ref[k, 2] == 0.62 and x_ref[k, 5] == pytest.approx(yaw)
        # rotating (0.8, -0.2) by yaw keeps its norm and its angle offset
        vx, vy = x_ref[k, 6], x_ref[k, 7]
        assert math.hypot(vx, vy) == pytest.approx(math.hypot(0.8, -0.2))
        assert math.atan2(vy, vx) == pytest.approx(yaw + math.atan2(-0.2, 0.8))
        assert x_ref[k, 11] == 0.5
        assert np.all(x_ref[k, [0, 1, 3, 4, 8, 9, 10]] == 0.0)
        assert np.all(x_ref[k, 12:] == m["q_nom"])


def test_stage_rows_layout():
    m = dict(mu=0.5, fz_max=600.0, qd_max=10.0, q_lim=1.5)
    Cu, Cx, lo, hi = refs.stage_rows(m, np.array([True, False]))
    u = np.zeros(30)
    u[0:3] = (10.0, -4.0, 100.0)
    r = Cu @ u
    # pyramid rows of the stance foot: +-f_x - mu f_z, +-f_y - mu f_z
    assert r[12:16] == pytest.approx([10 - 50, -10 - 50, -4 - 50, 4 - 50])
    assert np.all(hi[12:16] == 0.0) and np.all(np.isinf(lo[12:16]))
    # swing foot: its wrench is fixed to zero, its pyramid rows are free
    assert np.all(lo[6:12] == 0.0) and np.all(hi[6:12] == 0.0)
    assert np.all(np.isinf(lo[16:20])) and np.all(np.isinf(hi[16:20]))
    assert (lo[2], hi[2]) == (0.0, 600.0)
    assert np.all(Cx[38:56, 12:30] == np.eye(18)) and np.all(hi[38:] == 1.5)
