"""Residual policy and joint-torque blending (paper Sec. IV "Residual
Architecture": observation o in R^54, MLP of three 256-wide ELU layers, leg
actions a in R^10; "Blending Strategy", Eq. (joint-torque), lambda = 0.1).

TEST INFRASTRUCTURE ONLY (see the package header).  Plain NumPy, FP64
arithmetic; the layer inputs and the weights are rounded to bfloat16 where
the GPU's tensor-core kernel rounds them, so that the two compare closely.

Readings (the paper lists 3+3+18+3+3+18+1 = 49 entries plus the contact-phase
variables phi and states 54): phi has 5 entries, the gait phase and
(sin, cos) of 2 pi (phase + offset_i) for each foot; qdot_j is the measured
joint velocity; q_hat (default joint positions) is the agent's nominal pose.
"""
from __future__ import annotations

import numpy as np

OBS, HID, ACT = 54, 256, 10
LAMBDA = 0.1


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64.
    The value is first rounded to float32, as the kernel holds it."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    bias = np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))
    r = ((u + bias) & np.uint64(0xFFFF0000)).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def elu(x):
    x = np.asarray(x, dtype=np.float64)
    return np.where(x > 0.0, x, np.expm1(np.minimum(x, 0.0)))


def observation(x0, qd_meas, phase, offsets, value):
    """o = [p, theta, q_j, omega, v, qdot_j, phi(5), V_MPC] for one agent;
    x0 = [p, theta, v, omega, q] as the MPC state."""
    x0 = np.asarray(x0, dtype=np.float64)
    ph = float(phase)
    phi = [ph]
    for off in offsets:
        ang = 2.0 * np.pi * (ph + float(off))
        phi += [np.sin(ang), np.cos(ang)]
    return np.concatenate([x0[0:3], x0[3:6], x0[12:30], x0[9:12], x0[6:9],
                           np.asarray(qd_meas, dtype=np.float64), phi, [float(value)]])


def mlp(o, w):
    """a = W4^T h3 + b4, h_l = elu(W_l^T h_{l-1} + b_l), h0 = o; every layer's
    input and weights rounded to bfloat16, sums and biases in FP64."""
    h = np.asarray(o, dtype=np.float64)
    for layer in (1, 2, 3, 4):
        W = bf16_round(w[f"W{layer}"])
        z = bf16_round(h) @ W + np.asarray(w[f"b{layer}"], dtype=np.float64)
        h = elu(z) if layer < 4 else z
    return h


def blend(tau_mpc, a, q, qd, q_hat, kp, kd, lam=LAMBDA):
    """Eq. (joint-torque): tau_res = K_p (a + q_hat - q) - K_d qdot on the 10
    leg joints; tau = tau_MPC + lambda tau_res (arms keep tau_MPC)."""
    tau = np.array(tau_mpc, dtype=np.float64, copy=True)
    legs = slice(0, ACT)
    tau_res = np.asarray(kp)[legs] * (np.asarray(a) + np.asarray(q_hat)[legs] - np.asarray(q)[legs]) \
        - np.asarray(kd)[legs] * np.asarray(qd)[legs]
    tau[legs] += lam * tau_res
    return tau


def policy_batch(model, inputs, tau_mpc, value, w, lam=LAMBDA):
    """(actions [B,10], blended torques [B,18]) for a batch of agents."""
    B = len(model["mass"])
    acts = np.zeros((B, ACT))
    taus = np.zeros((B, 18))
    for a in range(B):
        o = observation(inputs["x0"][a], inputs["qd_meas"][a], inputs["phase"][a],
                        model["offset"][a], value[a])
        act = mlp(o, w)
        acts[a] = act
        taus[a] = blend(tau_mpc[a], act, np.asarray(inputs["x0"][a])[12:30], inputs["qd_meas"][a],
                        model["q_nom"][a], model["Kp"][a], model["Kd"][a], lam)
    return acts, taus
