"""Host logic of the serving loop (CPU): the synthetic request-state walk."""
import numpy as np

from paper_2510_12717_b300.serve import StateWalk


def _inputs(n=4096, seed=0):
    g = np.random.default_rng(seed)
    return dict(x0=g.standard_normal((n, 30)).astype(np.float32),
                qd_meas=np.zeros((n, 18), np.float32),
                cmd=np.zeros((n, 4), np.float32),
                phase=g.uniform(0, 1, n).astype(np.float32))


def test_s_steps_at_once_equal_s_single_steps_without_noise():
    a, s = 0.9, 3
    w1 = StateWalk(_inputs(), revert=a, pool_size=1 << 16)
    w3 = StateWalk(_inputs(), revert=a, pool_size=1 << 16)
    w1.noise[:] = 0.0
    w3.noise[:] = 0.0
    ids = np.arange(64)
    w1.X[ids] += 1.0                              # start off x_init
    w3.X[ids] += 1.0
    for _ in range(s):
        w1.advance(ids, np.ones(64, np.int64))
    x3 = w3.advance(ids, np.full(64, s))[0]
    np.testing.assert_allclose(x3, w1.X[ids], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(x3 - w3.XI[ids], a ** s, rtol=1e-5)
    # the s-step noise scale is the geometric sum of the single-step variances
    sig = 0.02
    want = sig * np.sqrt(sum(a ** (2 * i) for i in range(s)))
    assert abs(float(w3.sdev_tab[s]) - want) < 1e-7


def test_walk_is_stationary_around_the_initial_state():
    a, sig = 0.95, 0.02
    w = StateWalk(_inputs(), revert=a, step_sigma=sig, seed=3)
    ids = np.arange(4096)
    for _ in range(200):
        w.advance(ids, np.ones(4096, np.int64))
    d = w.X - w.XI
    assert abs(float(d.mean())) < 2e-3
    assert abs(float(d.std()) - sig / np.sqrt(1 - a * a)) < 0.1 * sig / np.sqrt(1 - a * a)


def test_phase_height_command_and_joint_rates():
    w = StateWalk(_inputs(), phase_step=0.02)
    ids = np.array([5, 9, 11])
    ph0 = w.PH[ids].copy()
    x, qd, cmd, ph = w.advance(ids, np.array([1, 2, 60]))
    np.testing.assert_allclose(ph, (ph0 + 0.02 * np.array([1, 2, 60])) % 1.0, atol=1e-5)
    assert ((ph >= 0) & (ph < 1)).all()
    np.testing.assert_array_equal(cmd[:, 0], x[:, 2])
    assert qd.shape == (3, 18) and np.abs(qd).max() > 0
    np.testing.assert_array_equal(w.X[ids], x)
    np.testing.assert_array_equal(w.PH[ids], ph)
