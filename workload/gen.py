"""Seeded generator of synthetic humanoid MPC agents and replan inputs.

Every agent has its own counter-based random stream (Philox keyed by
splitmix64 of the workload seed and the agent id), so an agent's parameters
and inputs do not depend on which batch it is drawn in.

Distributions (a stand-in for the paper's simulator rollouts, Sec. IV):
  mass U[20,30] kg; body inertia diagonal U[0.5,2] kg m^2; foot lever arms
  U[-0.15,0.15]^3 m; Q, R diagonal log-uniform in [1e-2,1e2] ([1e-4,1e4] for
  the ill-conditioned variant); friction mu U[0.4,1] (U[0.3,1] for the mixed
  workloads); base position (0,0,U[0.55,0.65]); attitude U[-0.1,0.1]^3;
  base linear/angular velocity N(0,0.1); joints U[-0.5,0.5]; nominal joints
  equal to the first replan's joints; command (height = base height,
  vx U[-1,1], vy U[-0.5,0.5], wz U[-1,1]); phase U[0,1); dt = 0.02 s;
  K_p = 30, K_d = 1, joint inertia M_j U[0.02,0.3], bias torque h_j U[-5,5],
  leg Jacobian entries U[-0.5,0.5]; measured joint velocity N(0,0.1).

This module holds no arithmetic of the method itself.
"""
from __future__ import annotations

import numpy as np

NX = 30      # state: p(3) theta(3) v(3) omega(3) q(18)
NU = 30      # input: f_L(3) m_L(3) f_R(3) m_R(3) qdot(18)
NJ = 18      # joints: 0-4 left leg, 5-9 right leg, 10-17 arms
NCON = 56    # inequality rows per stage

GAIT_WALK, GAIT_STAND, GAIT_HOP, GAIT_SINGLE_L, GAIT_SINGLE_R = 0, 1, 2, 3, 4
GAIT_NAMES = {0: "walk", 1: "stand", 2: "hop", 3: "single_l", 4: "single_r"}

# gait -> (period s, duty per foot, phase offset per foot)
_GAIT_TABLE = {
    GAIT_WALK: (0.5, (0.5, 0.5), (0.0, 0.5)),
    GAIT_STAND: (0.5, (1.0, 1.0), (0.0, 0.0)),
    GAIT_HOP: (0.5, (0.5, 0.5), (0.0, 0.0)),
    GAIT_SINGLE_L: (0.5, (1.0, 0.0), (0.0, 0.0)),   # left foot stance, right swing
    GAIT_SINGLE_R: (0.5, (0.0, 1.0), (0.0, 0.0)),   # right foot stance, left swing
}

SEED_BASE = 2510_12717

# name -> spec; idx is the workload's index in the seed
WORKLOADS = {
    "small": dict(idx=0, n_agents=16, horizon=(10, 10), gaits="walk",
                  mu=(0.4, 1.0), qr=(1e-2, 1e2)),
    "uniform": dict(idx=1, n_agents=4096, horizon=(10, 10), gaits="walk",
                    mu=(0.4, 1.0), qr=(1e-2, 1e2)),
    "uneven": dict(idx=2, n_agents=8192, horizon=(5, 20), gaits="mixed",
                   mu=(0.3, 1.0), qr=(1e-2, 1e2)),
    "mixed16k": dict(idx=3, n_agents=16384, horizon=(5, 20), gaits="mixed",
                     mu=(0.3, 1.0), qr=(1e-2, 1e2)),
    "mixed16k_ill": dict(idx=3, n_agents=16384, horizon=(5, 20), gaits="mixed",
                         mu=(0.3, 1.0), qr=(1e-4, 1e4)),
    "serving": dict(idx=4, n_agents=16384, horizon=(5, 20), gaits="mixed",
                    mu=(0.3, 1.0), qr=(1e-2, 1e2)),
}

_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One step of the splitmix64 mixer (Steele, Lea, Flood 2014)."""
    z = (x + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def agent_rng(seed: int, agent_id: int, stream: int = 0) -> np.random.Generator:
    """Counter-based generator for one agent (and one stream of that agent)."""
    k0 = splitmix64(splitmix64(seed & _M64) ^ (agent_id & _M64))
    k1 = splitmix64(k0 ^ ((stream + 1) * 0xD1B54A32D192ED03 & _M64))
    return np.random.Generator(np.random.Philox(key=[k0, k1]))


def workload_spec(name: str) -> dict:
    spec = dict(WORKLOADS[name])
    spec["name"] = name
    spec["seed"] = SEED_BASE + spec["idx"]
    return spec


def _pick_gait(u: float, mixed: bool) -> int:
    if not mixed:
        return GAIT_WALK
    if u < 0.3:
        return GAIT_WALK
    if u < 0.6:
        return GAIT_STAND
    if u < 0.9:
        return GAIT_HOP
    return GAIT_SINGLE_L if u < 0.95 else GAIT_SINGLE_R


def make_agents(name: str, agent_ids=None, *, zero_xy_weight: bool = False):
    """Draw agent models and first-replan inputs for workload `name`.

    Returns (model, inputs): dicts of numpy arrays, leading axis = agent.
    model : mass, inertia[3], lever[2,3], J_leg[2,6,5], M_j[18], h_j[18],
            Kp[18], Kd[18], Q[30], R[30], mu, fz_max, qd_max, q_lim, N (int32),
            dt, gait (int32), period, duty[2], offset[2], q_nom[18]
    inputs: x0[30], qd_meas[18], cmd[4] = (c_h, c_vx, c_vy, c_wz), phase
    """
    spec = workload_spec(name)
    if agent_ids is None:
        agent_ids = np.arange(spec["n_agents"])
    agent_ids = np.asarray(agent_ids, dtype=np.int64)
    B = len(agent_ids)
    mixed = spec["gaits"] == "mixed"
    nlo, nhi = spec["horizon"]
    mulo, muhi = spec["mu"]
    qrlo, qrhi = np.log(spec["qr"][0]), np.log(spec["qr"][1])

    m = dict(
        mass=np.empty(B), inertia=np.empty((B, 3)), lever=np.empty((B, 2, 3)),
        J_leg=np.empty((B, 2, 6, 5)), M_j=np.empty((B, NJ)), h_j=np.empty((B, NJ)),
        Kp=np.full((B, NJ), 30.0), Kd=np.full((B, NJ), 1.0),
        Q=np.empty((B, NX)), R=np.empty((B, NU)), mu=np.empty(B),
        fz_max=np.full(B, 600.0), qd_max=np.full(B, 10.0), q_lim=np.full(B, 1.5),
        N=np.empty(B, dtype=np.int32), dt=np.full(B, 0.02),
        gait=np.empty(B, dtype=np.int32), period=np.empty(B),
        duty=np.empty((B, 2)), offset=np.empty((B, 2)), q_nom=np.empty((B, NJ)),
    )
    inp = dict(x0=np.empty((B, NX)), qd_meas=np.empty((B, NJ)),
               cmd=np.empty((B, 4)), phase=np.empty(B))

    for a, aid in enumerate(agent_ids):
        g = agent_rng(spec["seed"], int(aid))
        U = g.random(216)
        Z = g.standard_normal(24)
        m["mass"][a] = 20.0 + 10.0 * U[0]
        m["inertia"][a] = 0.5 + 1.5 * U[1:4]
        m["lever"][a] = (-0.15 + 0.3 * U[4:10]).reshape(2, 3)
        m["J_leg"][a] = (-0.5 + U[10:70]).reshape(2, 6, 5)
        m["M_j"][a] = 0.02 + 0.28 * U[70:88]
        m["h_j"][a] = -5.0 + 10.0 * U[88:106]
        m["Q"][a] = np.exp(qrlo + (qrhi - qrlo) * U[106:136])
        m["R"][a] = np.exp(qrlo + (qrhi - qrlo) * U[136:166])
        m["mu"][a] = mulo + (muhi - mulo) * U[166]
        m["N"][a] = nlo + min(int(U[167] * (nhi - nlo + 1)), nhi - nlo)
        gait = _pick_gait(U[168], mixed)
        m["gait"][a] = gait
        period, duty, off = _GAIT_TABLE[gait]
        m["period"][a] = period
        m["duty"][a] = duty
        m["offset"][a] = off
        x0 = np.zeros(NX)
        x0[2] = 0.55 + 0.1 * U[169]
        x0[3:6] = -0.1 + 0.2 * U[170:173]
        x0[6:12] = 0.1 * Z[0:6]
        x0[12:30] = -0.5 + U[173:191]
        inp["x0"][a] = x0
        m["q_nom"][a] = x0[12:30]
        inp["cmd"][a] = (x0[2], -1.0 + 2.0 * U[191], -0.5 + U[192], -1.0 + 2.0 * U[193])
        inp["phase"][a] = U[194]
        inp["qd_meas"][a] = 0.1 * Z[6:24]
    if zero_xy_weight:
        m["Q"][:, 0:2] = 0.0
    return m, inp


def perturb_inputs(name: str, inputs: dict, agent_ids, replan: int, *,
                   sigma: float = 0.02, phase_step: float = 0.02) -> dict:
    """Inputs of replan `replan` (>= 1): x0 += N(0, sigma), phase += phase_step.

    The perturbation of an agent is drawn from its own stream `replan`, so it
    does not depend on batching either.  phase_step = 0.01 s / 0.5 s period.
    """
    spec = workload_spec(name)
    agent_ids = np.asarray(agent_ids, dtype=np.int64)
    out = {k: v.copy() for k, v in inputs.items()}
    for a, aid in enumerate(agent_ids):
        g = agent_rng(spec["seed"], int(aid), stream=replan)
        out["x0"][a] += sigma * g.standard_normal(NX)
        out["qd_meas"][a] = 0.1 * g.standard_normal(NJ)
    out["cmd"][:, 0] = out["x0"][:, 2]
    ph = out["phase"] + phase_step
    out["phase"] = ph - np.floor(ph)
    return out


def make_inputs(name: str, agent_ids=None, replan: int = 0):
    """(model, inputs) of replan `replan` for the given agents."""
    spec = workload_spec(name)
    if agent_ids is None:
        agent_ids = np.arange(spec["n_agents"])
    model, inp = make_agents(name, agent_ids)
    for r in range(1, replan + 1):
        inp = perturb_inputs(name, inp, agent_ids, r)
    return model, inp


def take_agents(d: dict, idx) -> dict:
    """Select a subset of agents (rows) from a model or inputs dict."""
    idx = np.asarray(idx)
    return {k: np.ascontiguousarray(v[idx]) for k, v in d.items()}


# ---------------------------------------------------------------- residual policy
POLICY_OBS, POLICY_HIDDEN, POLICY_ACT = 54, 256, 10


def make_policy(seed: int = 2510_12717 + 100) -> dict:
    """Random weights of the residual MLP 54 -> 256 -> 256 -> 256 -> 10 (the
    trained weights are not available): W_l ~ N(0, 1/fan_in) stored [in][out],
    b_l ~ N(0, 0.01), FP32.  Random draws only."""
    g = np.random.Generator(np.random.Philox(key=splitmix64(seed)))
    dims = [POLICY_OBS, POLICY_HIDDEN, POLICY_HIDDEN, POLICY_HIDDEN, POLICY_ACT]
    out = {}
    for layer in range(4):
        fan_in, fan_out = dims[layer], dims[layer + 1]
        out[f"W{layer + 1}"] = (g.standard_normal((fan_in, fan_out)) / np.sqrt(fan_in)).astype(np.float32)
        out[f"b{layer + 1}"] = (0.01 * g.standard_normal(fan_out)).astype(np.float32)
    return out


# ---------------------------------------------------------------- kinematic trees
# 18 revolute joints in four chains hanging off the floating base: (first
# joint, length) of the left leg, right leg, left arm, right arm.  A chain's
# first joint has the base as parent, every other joint the previous one.
TREE_CHAINS = ((0, 5), (5, 5), (10, 4), (14, 4))
_TREE_STREAM = 1 << 20
_LEG_AXES = ((0.0, 0.0, 1.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 1.0, 0.0), (0.0, 1.0, 0.0))
_ARM_AXES = ((0.0, 1.0, 0.0), (1.0, 0.0, 0.0), (0.0, 0.0, 1.0), (0.0, 1.0, 0.0))


def make_trees(name: str, agent_ids=None) -> dict:
    """Seeded synthetic kinematic trees, one per agent (the robot's model
    files are not available).  Per joint j: axis (unit vector in its parent
    link's frame, a hip/knee/ankle or shoulder/elbow pattern tilted by up to
    0.1 per component), offset of the joint from the parent frame's origin
    (legs: hip at (0, +-0.1, -0.1), thigh and shank 0.3-0.4 m; arms: shoulder
    at (0, +-0.2, 0.3), upper arm 0.2-0.3 m), link mass (legs 0.5-5 kg, arms
    0.5-1.5 kg), centre of mass in the link frame, and the diagonal of the
    link's rotational inertia about its centre of mass.  Random draws only."""
    spec = workload_spec(name)
    if agent_ids is None:
        agent_ids = np.arange(spec["n_agents"])
    agent_ids = np.asarray(agent_ids, dtype=np.int64)
    B = len(agent_ids)
    axis = np.zeros((B, NJ, 3))
    offset = np.zeros((B, NJ, 3))
    mass = np.zeros((B, NJ))
    com = np.zeros((B, NJ, 3))
    inertia = np.zeros((B, NJ, 3))
    seed = SEED_BASE + spec["idx"]
    leg_mass = ((1.0, 2.0), (1.0, 2.0), (3.0, 5.0), (2.0, 4.0), (0.5, 1.0))
    for a, aid in enumerate(agent_ids):
        g = agent_rng(seed, int(aid), stream=_TREE_STREAM)
        for c, (j0, length) in enumerate(TREE_CHAINS):
            side = 1.0 if c % 2 == 0 else -1.0
            leg = c < 2
            for t in range(length):
                j = j0 + t
                ax = np.array(_LEG_AXES[t] if leg else _ARM_AXES[t]) + g.uniform(-0.1, 0.1, 3)
                axis[a, j] = ax / np.linalg.norm(ax)
                if leg:
                    if t == 0:
                        offset[a, j] = (g.uniform(-0.02, 0.02), side * g.uniform(0.08, 0.12), g.uniform(-0.12, -0.08))
                    elif t < 3:
                        offset[a, j] = (0.0, 0.0, -g.uniform(0.03, 0.06))
                    else:
                        offset[a, j] = (0.0, 0.0, -g.uniform(0.3, 0.4))
                    mass[a, j] = g.uniform(*leg_mass[t])
                    com[a, j] = (g.uniform(-0.02, 0.02), g.uniform(-0.02, 0.02), -g.uniform(0.02, 0.2))
                    inertia[a, j] = g.uniform(0.002, 0.05, 3)
                else:
                    if t == 0:
                        offset[a, j] = (g.uniform(-0.02, 0.02), side * g.uniform(0.18, 0.22), g.uniform(0.25, 0.35))
                    elif t < 3:
                        offset[a, j] = (0.0, side * g.uniform(0.0, 0.03), -g.uniform(0.02, 0.05))
                    else:
                        offset[a, j] = (0.0, 0.0, -g.uniform(0.2, 0.3))
                    mass[a, j] = g.uniform(0.5, 1.5)
                    com[a, j] = (g.uniform(-0.02, 0.02), g.uniform(-0.02, 0.02), -g.uniform(0.02, 0.15))
                    inertia[a, j] = g.uniform(0.001, 0.02, 3)
    return dict(tree_axis=axis, tree_offset=offset, tree_mass=mass, tree_com=com, tree_inertia=inertia)
