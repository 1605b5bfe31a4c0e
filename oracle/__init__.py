"""Plain, slow, FP64 CPU oracle of the batched kinodynamic-MPC hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
anything in this package; only the tests, the smoke check and the CPU-baseline
leg of the benchmark use it.  It shares no code with the CUDA path: the two
meet only in the seeded input generator (package `workload`), which holds none
of the method's arithmetic.

What it computes (paper: Sec. III-A "Formulation", Eq. (mpc_formulation);
Sec. III-B Eq. (kkt_system); Sec. III-C Alg. 1, Eqs. (rnea), (mpc_torque)):

  refs.py    contact schedule, desired trajectory (Eqs. des_traj_1..5),
             references and constraint bounds for every stage
  model.py   floating-base model (Eq. base_dynamics in its centroidal form,
             footnote of Sec. III-A) and its linearisation by complex step
  qp.py      the dense horizon QP of Eq. (mpc_formulation), linearised
  ipm.py     dense primal-dual Mehrotra predictor-corrector interior point
             solve of that QP (the exact optimum the GPU's ADMM converges to)
  torque.py  first-stage solution -> joint torques (Eqs. rnea, mpc_torque)
  solve.py   the whole per-agent pipeline, and a process pool over agents
  policy.py  residual policy (Sec. IV: observation, 3 x 256 ELU MLP, leg
             actions) and joint-torque blending (Eq. joint-torque)
  lqr.py     closed-form affine finite-horizon LQR (a pin for the IPM)
  activeset.py brute-force active-set enumeration on toy QPs (a pin)
  kkt.py     KKT stationarity / feasibility / complementarity checks (a pin)
  feasibility.py  primal feasibility of the QP's constraint set (an LP by
             HiGHS), the reference for the solver's infeasibility status
  osqp.py    the literal iteration: OSQP's ADMM on the full KKT system
             (Eq. kkt_system), with the optional Ruiz equilibration
  admm.py    the Riccati forms' iteration: the same ADMM with the dynamics
             exact in every x-update (the paper's fixed-N_QP mode)

Pins (tests/test_oracle_*.py, all CPU): closed-form LQR when no constraint is
active, brute-force active sets on toy QPs, KKT invariants on every solve,
complex-step vs central-difference Jacobians, rigid-body invariants, a
rotation-derivative check of the Euler-rate map, hand-worked contact
schedules (tests/golden/), a hand-computed standing torque, and the
closed-form joint-reachability bound for the feasibility LP.
"""
