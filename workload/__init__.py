"""Seeded synthetic inputs for the batched kinodynamic-MPC hot path.

This package draws random numbers and nothing else: it holds none of the
method's arithmetic (no schedule, reference, dynamics, QP or torque math).
Both the CPU oracle and the CUDA path take their inputs from here.
"""
from .gen import (  # noqa: F401
    GAIT_WALK, GAIT_STAND, GAIT_HOP, GAIT_SINGLE_L, GAIT_SINGLE_R, GAIT_NAMES,
    NX, NU, NJ, NCON, WORKLOADS, splitmix64, agent_rng, make_agents,
    make_inputs, perturb_inputs, take_agents, workload_spec, make_policy,
    POLICY_OBS, POLICY_HIDDEN, POLICY_ACT, TREE_CHAINS, make_trees,
)
