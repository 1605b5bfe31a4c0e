"""Pins of the residual-policy oracle (paper Sec. IV: observation, MLP,
Eq. joint-torque blending) against independent values."""
import numpy as np
import pytest

from oracle import policy


def test_bf16_rounding_matches_torch_cast():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.uniform(-6, 6, 4000),
                        # exact ties: halfway between neighbours, both parities
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.0 - 2.0 ** -8, 3.0 + 2.0 ** -7,
                                  0.0, -0.0, 65504.0])]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(policy.bf16_round(x), ref)


def test_bf16_ties_go_to_even():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: even mantissa is 1.0
    assert policy.bf16_round(1.0 + 2.0 ** -8) == 1.0
    # 1 + 3 * 2^-8 lies halfway between 1 + 2^-7 and 1 + 2^-6: even is 1 + 2^-6
    assert policy.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6


def test_elu_values():
    assert policy.elu(2.5) == 2.5
    assert abs(policy.elu(-1.0) - (np.exp(-1.0) - 1.0)) < 1e-15
    assert policy.elu(0.0) == 0.0


def test_observation_layout():
    # x0 = [p, theta, v, omega, q]: fill each block with distinct markers
    x0 = np.concatenate([[1, 2, 3], [4, 5, 6], [7, 8, 9], [10, 11, 12], 100 + np.arange(18)]).astype(float)
    qd = 200 + np.arange(18.0)
    o = policy.observation(x0, qd, 0.25, (0.0, 0.5), -7.0)
    assert o.shape == (54,)
    assert list(o[0:3]) == [1, 2, 3] and list(o[3:6]) == [4, 5, 6]        # p, theta
    assert list(o[6:24]) == list(100 + np.arange(18.0))                   # q_j
    assert list(o[24:27]) == [10, 11, 12] and list(o[27:30]) == [7, 8, 9]  # omega, v
    assert list(o[30:48]) == list(qd)                                     # qdot_j
    # phase 0.25: left foot (offset 0) at a quarter period, right at 3/4
    np.testing.assert_allclose(o[48:53], [0.25, 1.0, 0.0, -1.0, 0.0], atol=1e-15)
    assert o[53] == -7.0


def test_mlp_with_selection_weights():
    # W1 copies obs 0..9 into hidden 0..9 (rest 0), W2, W3 identity, W4 picks
    # hidden 0..9: for positive inputs the network is the identity on them
    w = {f"b{l}": np.zeros(d) for l, d in ((1, 256), (2, 256), (3, 256), (4, 10))}
    w["W1"] = np.zeros((54, 256)); w["W1"][np.arange(10), np.arange(10)] = 1.0
    w["W2"] = np.eye(256); w["W3"] = np.eye(256)
    w["W4"] = np.zeros((256, 10)); w["W4"][np.arange(10), np.arange(10)] = 1.0
    o = np.zeros(54); o[:10] = [0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 3.5, 4.0, 4.5, 5.0]   # exact in bf16
    np.testing.assert_array_equal(policy.mlp(o, w), o[:10])
    # a negative input goes through ELU three times
    o[0] = -1.0
    e = np.expm1(-1.0)
    want = policy.bf16_round(np.expm1(policy.bf16_round(np.expm1(policy.bf16_round(e)))))
    assert abs(policy.mlp(o, w)[0] - want) < 1e-15


def test_blend_hand_values():
    tau = np.arange(18.0)
    a = np.full(10, 0.1)
    q = np.full(18, 0.2); q_hat = np.full(18, 0.3); qd = np.full(18, 2.0)
    kp = np.full(18, 30.0); kd = np.full(18, 1.0)
    out = policy.blend(tau, a, q, qd, q_hat, kp, kd, 0.1)
    # legs: 30 (0.1 + 0.3 - 0.2) - 1 * 2 = 4, times 0.1 = 0.4; arms unchanged
    np.testing.assert_allclose(out[:10], np.arange(10.0) + 0.4, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(out[10:], np.arange(10.0, 18.0))
