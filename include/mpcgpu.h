/*
 * mpcgpu.h - C ABI of the batched kinodynamic-MPC solver (B300, sm_103a).
 *
 * One call of the library replans many independent humanoid agents at once:
 * for each agent it forms the horizon QP of the paper's kinodynamic MPC
 * (Sec. III-A, Eq. (mpc_formulation); desired trajectory Eqs. (des_traj_1)-
 * (des_traj_5); contact schedule of Sec. III-A), linearised about the
 * agent's current state (real-time iteration, Sec. III-B), solves it with
 * OSQP-style ADMM (Sec. III-B, Eq. (kkt_system); the KKT solve is done by a
 * per-stage Riccati recursion instead of a sparse LDL, Eqs. (ldl),
 * (backsolve_1)-(backsolve_2)), and maps the first-stage solution to joint
 * torques (Sec. III-C, Eqs. (rnea), (mpc_torque)); Alg. 1 is the whole path.
 *
 * Conventions used by every entry point:
 *   - Pointers are DEVICE pointers unless the argument name ends in _host.
 *   - The caller owns every buffer it passes; the library never frees one.
 *     The library owns its device arenas (models, warm starts, factor
 *     caches, scratch), allocated in mpc_create and freed in mpc_destroy.
 *   - Work is enqueued on the context's stream (mpc_config.stream); results
 *     are valid once that stream has reached the point after the call.
 *   - Errors are return codes; nothing throws or aborts across the ABI.
 *     mpc_last_error() gives a one-line description of the last failure.
 *   - One host thread per context.
 *
 * Per-agent layouts (float32, row-major, agent-major):
 *   x0[n][30]      state: p(3), Theta = (roll, pitch, yaw)(3), v(3) world,
 *                  w(3) world, q(18): joints 0-4 left leg, 5-9 right leg,
 *                  10-17 arms
 *   qd_meas[n][18] measured joint velocities (the K_d term of Eq. mpc_torque)
 *   cmd[n][4]      command (c_h, c_vx, c_vy, c_wz) of Eqs. (des_traj_*)
 *   phase[n]       gait phase in [0, 1)
 *   tau[n][18], q_set[n][18], qd_set[n][18], value[n], agent_status[n]
 */
#ifndef MPCGPU_H
#define MPCGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPC_NX 30    /* state size */
#define MPC_NU 30    /* input size: f_L(3) m_L(3) f_R(3) m_R(3) qdot(18) */
#define MPC_NJ 18    /* joints */
#define MPC_NROW 56  /* inequality rows per stage */
#define MPC_MAX_HORIZON 32

typedef enum {
  MPC_OK = 0,
  MPC_ERR_INVALID = 1,   /* bad argument, unknown agent, unsupported option */
  MPC_ERR_BUDGET = 2,    /* arenas would exceed hbm_budget_bytes */
  MPC_ERR_CUDA = 3,      /* a CUDA runtime call failed */
  MPC_ERR_NOT_READY = 4, /* ticket not solved yet / unknown ticket */
  MPC_ERR_TIMEOUT = 5,   /* a bounded device wait gave up */
  MPC_ERR_STATE = 6      /* call out of order (e.g. solve before submit) */
} mpc_status;

typedef enum {
  MPC_AGENT_SOLVED = 0,        /* a polished point passed the KKT check of its active set
                                  (the optimum up to rounding) */
  MPC_AGENT_MAX_ITER = 1,      /* iteration cap reached (or fixed-N_QP mode) */
  MPC_AGENT_PRIMAL_INFEAS = 2, /* no point satisfies the constraints: OSQP's certificate
                                  (the multiplier change of the last ADMM iteration,
                                  with the dynamics multipliers from the costate
                                  recursion) held at a residual check, tolerance
                                  1e-4 relative; outputs are those of the last
                                  iterate, and the next replan cold-starts */
  MPC_AGENT_DUAL_INFEAS = 3,   /* never produced: every row of the cost is bounded
                                  below on the dynamics (Q, R >= 0, x0 fixed) */
  MPC_AGENT_NAN = 4,           /* non-finite input or iterate; outputs zeroed */
  MPC_AGENT_TIMEOUT = 5,       /* a bounded device wait gave up; outputs zeroed */
  MPC_AGENT_INACCURATE = 6,    /* ADMM met its stopping test but no polish passed the KKT
                                  check (or polish is off): the outputs are ADMM's iterate,
                                  as accurate as that test, not certified to be the
                                  optimum; the warm start is kept */
  MPC_AGENT_DEFERRED = 7       /* only with a DEFER flag of mpc_solve_ex, outputs zeroed.
                                  DEFER_ADMM: the polish first failed its KKT check and the
                                  agent's ADMM start (the last polished point, its row values
                                  and multipliers) was written to its warm start instead of
                                  running ADMM: solve it again with MPC_SOLVE_ADMM_ONLY and
                                  the same inputs.  DEFER_SLOW: the polish first had not
                                  passed after two reduced KKT solves; its corrected active
                                  set is kept: solve it again with no flag and the same
                                  inputs, which continues from it (likewise DEFER_COLD) */
} mpc_agent_status;

/* Precision of the Riccati factor's two dense 22 x 22 stage products per
 * stage (K = -H_uu^-1 H_ux and H_ux^T K) and of its Schur inverse: FP32 on the
 * CUDA cores; TF32 / BF16 on the tensor cores (mma.sync, FP32 accumulation);
 * FP64 Schur inverse; TF32X3 = error-compensated split TF32 on the tensor
 * cores (three mma per tile, FP32-level accuracy; Ootomo and Yokota 2022). */
typedef enum { MPC_FP32 = 0, MPC_TF32 = 1, MPC_BF16 = 2, MPC_FP64 = 3, MPC_TF32X3 = 4 } mpc_precision;

/* Launch form of a context's solves.  PLAIN and FUSED solve with the
 * per-stage Riccati recursion (polish first, ADMM fallback).  LDL is the
 * paper's literal solve (Alg. 1, Sec. III-B): OSQP's ADMM on the full KKT
 * system of Eq. (kkt_system), factored once per solve by a batched block
 * LDL^T (Eq. ldl; the inequality rows' pivots first, then per stage the
 * block of u_k, the stage's dynamics multipliers and x_{k+1}) and solved by
 * forward / backward substitution in every iteration (Eqs. backsolve_1-2);
 * every solve starts from f_init (cold), rho stays at rho0, no polish.  With
 * fixed_iters > 0 it runs exactly that many iterations (the paper's N_QP;
 * agent_status MPC_AGENT_MAX_ITER), otherwise until OSQP's stopping test at
 * a residual check every check_every iterations (MPC_AGENT_INACCURATE: not
 * certified by a polish) or max_iter.  Its factors take about 29 KB per
 * stage per agent of device memory (max_agents x max_horizon stages). */
typedef enum { MPC_FORM_PLAIN = 0, MPC_FORM_FUSED = 1, MPC_FORM_LDL = 2 } mpc_form;

/* Unit measured by mpc_measure_peak. */
typedef enum {
  MPC_PEAK_FP32_FMA = 0,      /* FP32 fused multiply-add on the CUDA cores */
  MPC_PEAK_FP64_FMA = 1,      /* FP64 fused multiply-add */
  MPC_PEAK_TF32_MMA_SYNC = 2, /* mma.sync m16n8k8 TF32, FP32 accumulation */
  MPC_PEAK_BF16_MMA_SYNC = 3  /* mma.sync m16n8k16 BF16, FP32 accumulation */
} mpc_peak_kind;

typedef enum {
  MPC_GAIT_WALK = 0, MPC_GAIT_STAND = 1, MPC_GAIT_HOP = 2,
  MPC_GAIT_SINGLE_L = 3, MPC_GAIT_SINGLE_R = 4
} mpc_gait;

/* Solver and context options.  mpc_default_config() fills the defaults:
 * rho0 0.1, sigma 1e-6, alpha 1.6, eps_abs = eps_rel = 1e-5, max_iter 4000,
 * fixed_iters 0, check_every 10, adaptive_rho 1, polish 1, warm_start 1,
 * form FUSED, precision FP32, max_horizon 20, variant 1, early_polish 100,
 * graph 0, warm_polish 1, refine_steps -1, spin_limit 4194304, wait_test_agent -1,
 * ruiz_iters 0, kin_rows 0, swing_height 0.075, v_takeoff 0.1, v_touchdown -0.1.
 * OSQP's parameters (Stellato et al. 2020,
 * Sec. 3.2, to which the paper defers after Eq. (backsolve_2)). */
typedef struct mpc_config {
  int device;                 /* CUDA device ordinal */
  void* stream;               /* cudaStream_t; NULL = the legacy default stream */
  int max_agents;             /* agent ids are 0 .. max_agents-1 */
  int max_horizon;            /* largest N any agent may use (<= MPC_MAX_HORIZON) */
  size_t hbm_budget_bytes;    /* cap on all device arenas; 0 = no cap */
  int precision;              /* mpc_precision of the Riccati factor (the rest is FP32):
                                 FP32; TF32 / BF16 = the two dense stage-block
                                 products (K = -H_uu^-1 H_ux and H_ux^T K) on the
                                 tensor cores (mma.sync), FP32 accumulation; FP64 =
                                 the stage Schur complement H_uu inverted in FP64;
                                 TF32X3 = the two products in split TF32 on the
                                 tensor cores (FP32-level accuracy).
                                 With polish first on (polish, warm_polish,
                                 fixed_iters 0), a TF32 / BF16 agent whose polish
                                 first fails falls back to FP32 factors for its
                                 ADMM solve and later polishes; otherwise every
                                 factor uses the requested precision */
  int form;                   /* mpc_form: PLAIN = one kernel per step (set-up, factor,
                                 ADMM, polish, torque map; static grids); FUSED = a
                                 set-up kernel, one persistent kernel that solves
                                 every agent (polish first, ADMM fallback, polish) over
                                 a longest-first work queue, and a torque-map kernel;
                                 LDL = the paper's literal KKT solve (see mpc_form) */
  float rho0, sigma, alpha;   /* ADMM step size, proximal weight, relaxation */
  float eps_abs, eps_rel;     /* OSQP-style stopping tolerances */
  int max_iter;               /* iteration cap */
  int fixed_iters;            /* >0: run exactly this many iterations (paper's N_QP) */
  int check_every;            /* residual / rho check period */
  int adaptive_rho;           /* OSQP rho update (refactor when off by 5x) */
  int polish;                 /* OSQP-style active-set polish after ADMM */
  int warm_start;             /* start from the agent's previous solution */
  int variant;                /* kernel build: 1 = 2 resident blocks/SM (no register
                                 spills), 2 = 3 blocks/SM (more warps, some spills) */
  float early_polish;         /* try the polish once both residuals are within this
                                 factor of the tolerance (0 = only after ADMM) */
  int graph;                  /* 1: the fused solve is captured as a CUDA graph the
                                 first time a batch (buffers, ticket slot, stream)
                                 is solved and replayed afterwards (only on a
                                 non-default stream; direct launches otherwise) */
  int warm_polish;            /* 1: polish first, from the previous replan's final
                                 active set (warm start) or from the equality rows
                                 alone (cold agent); ADMM runs only if that fails
                                 its KKT check */
  int refine_steps;           /* iterative-refinement steps on each polish solve
                                 (0..4); -1 = automatic: 2 for TF32 and 3 for BF16
                                 stage products, 1 for FP32 / FP64 */
  int spin_limit;             /* polls of a bounded device wait (a stage block's bulk
                                 copy into shared memory) before it gives up; the
                                 agent then gets MPC_AGENT_TIMEOUT with zeroed
                                 outputs, the kernel waits (bounded again) for that
                                 warp's copies still in flight and the warp takes no
                                 further agent (the rest of the batch is solved by
                                 the other warps); mpc_get_stats counts the events
                                 ("wait_timeouts").  > 0 */
  int wait_test_agent;        /* failure-detection test only: the first stage-block
                                 wait of this agent id is armed with no copy behind
                                 it, so it runs out after spin_limit polls with
                                 nothing in flight.  -1 = off (the default) */
  int ruiz_iters;             /* literal form (MPC_FORM_LDL) only: iterations of OSQP's
                                 modified Ruiz equilibration of the KKT system before
                                 its factorisation (f_Ruiz of Alg. 1; 0..50, default 0
                                 = unscaled: with the fixed step size of this form the
                                 equilibrated problem converges more slowly on these
                                 QPs; OSQP pairs its scaling with an adaptive rho) */
  int kin_rows;               /* literal form (MPC_FORM_LDL) only, and without Ruiz
                                 scaling: 1 adds the kinematic rows of Eq.
                                 (mpc_formulation) to every stage k, read at node k+1
                                 on (u_k, x_{k+1}): per foot in stance the no-slip rows
                                 v_{k+1} + J_leg[0:3] qdot_leg,k = 0 (J(q) qdot = 0,
                                 with the node's joint rates those of u_k), per foot in
                                 swing the height row p_z + J_leg[2] (q_leg - q_nom) =
                                 c_h + B(t_sw), B the quintic of Eqs. (bezier_1-5) with
                                 dB/dt(0.5) = 0 as its sixth condition.  Rows 56-63 of
                                 the stage (56 + 3i + r: no-slip of foot i, component r;
                                 62 + i: swing height of foot i).  Default 0 */
  float swing_height;         /* z_swing of Eq. (bezier_3), m (default 0.075) */
  float v_takeoff;            /* v_to of Eq. (bezier_4), m/s (default 0.1) */
  float v_touchdown;          /* v_td of Eq. (bezier_5), m/s (default -0.1) */
} mpc_config;

/* One agent's model (host memory, float64; stored as float32 on the device,
 * except the schedule fields dt, period, duty, offset, which stay float64 so
 * that stance/swing decisions are taken in double precision). */
typedef struct mpc_agent_model {
  double mass;              /* kg */
  double inertia[3];        /* body-frame principal inertia, kg m^2 */
  double lever[2][3];       /* nominal foot lever arms from the CoM, m */
  double J_leg[2][6][5];    /* per foot: wrench rows (f 0-2, m 3-5) x 5 leg joints */
  double M_j[18];           /* joint inertia (diagonal joint-space model) */
  double h_j[18];           /* joint bias torque */
  double Kp[18], Kd[18];    /* PD gains of Eq. (mpc_torque) */
  double Q[30], R[30];      /* diagonal cost weights of Eq. (mpc_formulation) */
  double mu, fz_max, qd_max, q_lim;
  int N;                    /* horizon (2 .. max_horizon) */
  double dt;                /* node spacing, s */
  int gait;                 /* mpc_gait (informational; duty/offset define it) */
  double period;            /* gait period, s */
  double duty[2];           /* stance fraction per foot (1 = always stance) */
  double offset[2];         /* phase offset per foot */
  double q_nom[18];         /* nominal joint angles */
} mpc_agent_model;

/* One agent's kinematic tree for the torque map's inverse dynamics (paper
 * Sec. III-C, Eq. (rnea): M(q) qddot + h(q, qdot) by the recursive
 * Newton-Euler algorithm).  Host memory, float64; stored as float32.  18
 * revolute joints in four chains hanging off the floating base, in the
 * joint order of the state: 0-4 left leg, 5-9 right leg, 10-13 left arm,
 * 14-17 right arm; a chain's first joint has the base as parent, every other
 * joint the previous one.  Joint j turns about axis[j] (a unit vector in its
 * parent link's frame) at offset[j] from the parent frame's origin (the base
 * frame's origin is the base position p of the state); link j's frame is the
 * parent's translated to the joint and rotated by q_j about the axis. */
typedef struct mpc_tree_model {
  double axis[18][3];
  double offset[18][3];     /* m */
  double mass[18];          /* link mass, kg */
  double com[18][3];        /* link centre of mass in the link frame, m */
  double inertia[18][3];    /* diagonal of the link's inertia about its centre of mass
                               in the link frame, kg m^2 */
} mpc_tree_model;

typedef struct mpc_ctx mpc_ctx;

/* Fill *cfg with the defaults above (device 0, NULL stream, max_agents 16384). */
mpc_status mpc_default_config(mpc_config* cfg);

/* Create a context: allocates every device arena for cfg->max_agents agents
 * of horizon up to cfg->max_horizon.  MPC_ERR_BUDGET if that exceeds
 * cfg->hbm_budget_bytes (non-zero).  *out is NULL on failure. */
mpc_status mpc_create(const mpc_config* cfg, mpc_ctx** out);

/* Free everything the context owns (synchronises its stream first). */
mpc_status mpc_destroy(mpc_ctx* ctx);

/* Admit or update agents: copies n host models (models_host[n]) into the
 * device model arena at agent_ids_host[n] and clears their warm starts.
 * Synchronous with respect to the host buffers. */
mpc_status mpc_set_models(mpc_ctx* ctx, int32_t n, const int32_t* agent_ids_host,
                          const mpc_agent_model* models_host);

/* Single-agent form of mpc_set_models. */
mpc_status mpc_set_model(mpc_ctx* ctx, int32_t agent_id, const mpc_agent_model* model_host);

/* Give agents a kinematic tree (trees_host[n], at agent_ids_host[n]): from
 * the next solve their torque map computes M(q) qddot + h(q, qdot) of Eq.
 * (rnea) by the recursive Newton-Euler algorithm over the tree, the floating
 * base moving as the MPC predicts (orientation and angular velocity of x0,
 * accelerations (x_1 - x_0)/dt of its twist, gravity 9.81 m/s^2 along -z),
 * in place of the diagonal joint model M_j qddot_j + h_j; the contact term
 * -J_leg^T W keeps the model's leg Jacobian.  An agent without a tree, or
 * whose model was uploaded again since (mpc_set_models clears the tree),
 * uses the diagonal model.  The QP does not depend on the tree.  Synchronous
 * with respect to the host buffers.  Errors: MPC_ERR_INVALID for a bad count,
 * an id out of range, a NULL buffer, a non-finite value, an axis that is not
 * a unit vector (|norm - 1| > 1e-6), a negative mass or inertia. */
mpc_status mpc_set_trees(mpc_ctx* ctx, int32_t n, const int32_t* agent_ids_host,
                         const mpc_tree_model* trees_host);

/* mpc_set_models without waiting: the models are packed into the context's
 * pinned host staging (allocated by the first call) and uploaded on `stream`
 * (a cudaStream_t), and the call returns at once.  The upload is complete when
 * that stream has reached the point after the call; until then no batch may
 * solve these agents, and no further model upload (of either kind) may
 * start, since both reuse the context's staging buffers.  For a caller that
 * swaps agents while other batches run (the server's churn).  A call with
 * n = 0 only allocates the staging (page-locking it takes milliseconds; the
 * server does it when it is created).  Errors as mpc_set_models. */
mpc_status mpc_set_models_async(mpc_ctx* ctx, int32_t n, const int32_t* agent_ids_host,
                                const mpc_agent_model* models_host, void* stream);

/* Remove an agent: its slot no longer accepts submissions. */
mpc_status mpc_release_agent(mpc_ctx* ctx, int32_t agent_id);

/* Register one replan batch of n agents (device buffers, layouts above).
 * Nothing runs yet; the buffers must stay valid until mpc_solve has been
 * enqueued.  *ticket identifies the batch.  At most 64 tickets are pending
 * (a ticket's slot is reused only after its solve and gather have completed
 * on the device); MPC_ERR_STATE when none is free. */
mpc_status mpc_submit(mpc_ctx* ctx, int32_t n, const int32_t* agent_ids,
                      const float* x0, const float* qd_meas, const float* cmd,
                      const float* phase, uint64_t* ticket);

/* Enqueue the whole hot path (Alg. 1) for the ticket's agents on the
 * context's stream:
 * schedule/references/bounds, linearisation, assembly, Riccati factor, ADMM
 * iterations with residual checks and rho updates, polish, torque map, and
 * the write-back of each agent's warm start. */
mpc_status mpc_solve(mpc_ctx* ctx, uint64_t ticket);

/* mpc_solve on a caller-chosen stream (a cudaStream_t; NULL = legacy default
 * stream).  Batches solved concurrently on different streams must not share
 * an agent: their per-agent state would race.  Each ticket has its own work
 * queue, so concurrent tickets are otherwise independent.  The ticket's
 * results are gathered on the same stream by mpc_get_torques. */
mpc_status mpc_solve_on(mpc_ctx* ctx, uint64_t ticket, void* stream);

/* Flags of mpc_solve_ex (fused form only), for latency-bound callers that
 * answer most of a batch at once and finish its slow agents in a batch of
 * their own.  DEFER_ADMM: an agent whose polish first fails is not taken
 * through ADMM in this solve; it ends MPC_AGENT_DEFERRED.  ADMM_ONLY: no
 * polish first; every agent runs ADMM from its warm start (with the polish
 * attempts along the way and the final polish), the second half of a
 * DEFER_ADMM solve.  DEFER_SLOW (alone): the polish first stops after two
 * reduced KKT solves (the active-set method's first guess and one
 * correction); an agent it has not solved by then ends MPC_AGENT_DEFERRED and
 * a solve without flags continues it (more corrections, then ADMM if needed),
 * with the same result as an uninterrupted solve. */
typedef enum {
  MPC_SOLVE_DEFER_ADMM = 1, MPC_SOLVE_ADMM_ONLY = 2, MPC_SOLVE_DEFER_SLOW = 4,
  MPC_SOLVE_DEFER_COLD = 8   /* alone: DEFER_SLOW for cold agents (no warm start: a first
                                solve, or one after a model swap); a warm agent is deferred
                                only when its polish first fails; continue with no flag */
} mpc_solve_flags;

/* mpc_solve_on with flags (0 = mpc_solve_on).  MPC_ERR_INVALID for an
 * unknown flag or flags on a form other than FUSED. */
mpc_status mpc_solve_ex(mpc_ctx* ctx, uint64_t ticket, void* stream, int32_t flags);

/* Tune the batching form's launch configuration on the ticket's batch by
 * timing candidates (`repeats` timed solves each, after one untimed solve) on
 * the context's stream, in two stages: the kernel shape (variant = register
 * cap and so resident warps, x the persistent kernel's resident blocks per
 * SM: all that fit, or fewer agents in flight), then the ADMM schedule
 * (residual-check period x early-polish threshold) on the best shape.  Among
 * the candidates that solve the most agents the fastest wins.  The choice is
 * stored in the context's configuration and in its table of tuned entries,
 * keyed by (precision, floor(log2 batch size)): every later solve of a batch
 * with that key uses the entry (with the tuned batch's mean horizon recorded
 * beside it).  The batch's agents are solved repeatedly (their warm starts
 * advance); the ticket stays submitted.  report (may be NULL) receives a JSON
 * summary: the choice, its key, every candidate, the table.  Synchronous. */
mpc_status mpc_autotune(mpc_ctx* ctx, uint64_t ticket, int32_t repeats, char* report, size_t cap);

/* Enqueue a gather of the ticket's results into caller buffers (any may be
 * NULL): tau, q_set, qd_set [n][18], value[n] = QP objective at the
 * solution, agent_status[n] (mpc_agent_status; -1 and zero outputs for a
 * batch row whose id is out of range or not admitted, which the solve
 * skipped).  Releases the ticket. */
mpc_status mpc_get_torques(mpc_ctx* ctx, uint64_t ticket, float* tau, float* q_set,
                           float* qd_set, float* value, int32_t* agent_status);

/* Host-buffer convenience (the end-to-end path): copies the inputs from host
 * memory, submits, solves, gathers and copies the results back, then
 * synchronises the stream.  Output pointers may be NULL. */
mpc_status mpc_solve_host(mpc_ctx* ctx, int32_t n, const int32_t* agent_ids_host,
                          const float* x0_host, const float* qd_meas_host,
                          const float* cmd_host, const float* phase_host,
                          float* tau_host, float* q_set_host, float* qd_set_host,
                          float* value_host, int32_t* agent_status_host);

/* Per-agent solver statistics of the last solve of each agent, copied to
 * host arrays (any may be NULL): ADMM iterations, refactorisations, polish
 * accepted (0 no, 1 after ADMM, 2 by the polish first, without ADMM),
 * final unscaled primal and dual residuals (inf-norms), and the scaled
 * residuals: the largest primal row violation / stationarity component over
 * its own tolerance eps_abs + eps_rel * (magnitude of that row's or
 * component's terms), the convergence measure (<= 1 converged).
 * Synchronises the stream. */
mpc_status mpc_get_agent_stats(mpc_ctx* ctx, int32_t n, const int32_t* agent_ids_host,
                               int32_t* iters_host, int32_t* refactors_host,
                               int32_t* polished_host, float* prim_res_host,
                               float* dual_res_host, float* prim_scaled_host,
                               float* dual_scaled_host);

/* Checkpoint / inspection of one agent's solver state (host buffers):
 * x[(N+1)][30], u[N][30] = last primal solution (after polish, if accepted),
 * w[N][56] = projected constraint values, y[N][56] = row multipliers,
 * rho.  Synchronises the stream. */
mpc_status mpc_export_state(mpc_ctx* ctx, int32_t agent_id, float* x_host, float* u_host,
                            float* w_host, float* y_host, float* rho_host);

/* Inspection of one agent's horizon QP as its last solve formed it (host
 * buffers, each may be NULL): steps f_init / f_param and the linearisation of
 * Alg. 1, i.e. the desired trajectory (Eqs. des_traj_1-5) xref[(N+1)][30] and
 * uref[N][30], the row bounds of Eq. (mpc_formulation)'s constraints
 * lo[N][56], hi[N][56] (rows: 0-11 foot wrenches, 12-19 friction pyramid,
 * 20-37 joint rates, 38-55 joints at stage k+1; +-inf = free), and the
 * dynamics linearised about x0 and u_ref,k (Sec. III-B),
 * x_{k+1} = A_k x_k + B_k u_k + c_k: A[N][30][30], B[N][30][30], c[N][30],
 * row-major.  Synchronises the stream.  Errors: MPC_ERR_INVALID for an
 * unknown agent. */
mpc_status mpc_export_qp(mpc_ctx* ctx, int32_t agent_id, float* xref_host, float* uref_host,
                         float* lo_host, float* hi_host, float* A_host, float* B_host, float* c_host);

/* Restore a state written by mpc_export_state (sets the warm start). */
mpc_status mpc_import_state(mpc_ctx* ctx, int32_t agent_id, const float* x_host,
                            const float* u_host, const float* w_host, const float* y_host,
                            float rho);

/* Allocation-free solve, for callers that cannot allocate device memory
 * when they need a solve: simulator plugins that may only use the buffers
 * handed to them, real-time control loops that must not enter the device
 * allocator once running, or processes whose device allocator belongs to
 * another framework.  The paper has no counterpart; it is a deployment
 * convenience.
 *
 * Solves n <= 64 agents of horizon N <= 20 (models_host[n], host memory) in
 * one cold-started fused pass with the default options of
 * mpc_default_config(), on `stream` (a cudaStream_t; NULL = default stream).
 * Inputs x0, qd_meas, cmd, phase and outputs tau, q_set, qd_set, value,
 * agent_status are device buffers with the layouts above (outputs may be
 * NULL).  All workspace lives in one static device array of about 11 MB that
 * every GPU loading this library holds until the process exits; no call
 * allocates or frees device memory.
 *   - The first call on a device resolves the array's device address (with
 *     that device current).
 *   - A call cannot be captured into a CUDA graph: it copies the packed
 *     models from pageable host staging, and a replay would read whatever a
 *     later call packed there.
 *   - Every call shares the one device array, which keeps the previous
 *     call's contents (warm-start markers and the horizons of unused slots
 *     are cleared each call), and the packed models pass through host
 *     staging arrays shared by the whole process: any two calls that overlap
 *     in time race, on the host and on the GPU, whatever their threads,
 *     devices or streams.  Calls made one after another from one thread are
 *     safe.
 * Returns MPC_ERR_INVALID for n > 64, a horizon > 20, an invalid model or a
 * NULL input; MPC_ERR_CUDA when a runtime call fails. */
mpc_status mpc_solve_static(int32_t n, const mpc_agent_model* models_host, const float* x0,
                            const float* qd_meas, const float* cmd, const float* phase,
                            float* tau, float* q_set, float* qd_set, float* value,
                            int32_t* agent_status, void* stream);

/* JSON summary of the context (sizes, arenas, counters) into buf, and
 * "polish_attempts": a histogram over the live agents of their last solve's
 * accepted polish, entry a = agents whose polish took a reduced KKT solves
 * (the first guess and its corrections), entry 0 = no polish accepted (the
 * iteration count of the active-set method).  Synchronises the stream. */
mpc_status mpc_get_stats(mpc_ctx* ctx, char* buf, size_t cap);

/* Residual policy and joint-torque blending after the MPC (paper Sec. IV,
 * "Residual Architecture" and "Blending Strategy", Eq. (joint-torque)).
 * mpc_set_policy uploads the MLP 54 -> 256 -> 256 -> 256 -> 10 (ELU hidden
 * layers): host FP32 weights W_l stored [in][out] row-major (W1 54 x 256,
 * W2 and W3 256 x 256, W4 256 x 10) and biases b_l; the device keeps the
 * weights in bfloat16 (round to nearest even) and the biases in FP32.
 * blend_lambda is the blending factor lambda (0.1 in the paper).  May be
 * called again to replace the weights.  Errors: MPC_ERR_INVALID for a NULL
 * pointer or a non-finite lambda. */
mpc_status mpc_set_policy(mpc_ctx* ctx, const float* W1, const float* b1, const float* W2,
                          const float* b2, const float* W3, const float* b3, const float* W4,
                          const float* b4, float blend_lambda);

/* Evaluate the policy for a solved ticket and blend its actions into the MPC
 * torques; call between mpc_solve and mpc_get_torques (which releases the
 * ticket).  Per agent (batch row order): the observation
 * o = [p, theta, q_j, omega, v, qdot_j, phi, V_MPC] in R^54, with qdot_j the
 * measured joint velocity and phi = (phase, sin and cos of 2 pi (phase +
 * offset_i) for both feet); the actions a in R^10 (leg joints 0-9); the
 * torques tau = tau_MPC + lambda (K_p (a + q_nom - q) - K_d qdot) on the legs
 * and tau_MPC on the arms.  Each layer runs on the tensor cores with
 * bfloat16 inputs and FP32 accumulation.  Outputs (device, either may be
 * NULL): tau [n][18], action [n][10].  Enqueued on the ticket's stream.
 * Errors: MPC_ERR_STATE if no policy is set, MPC_ERR_NOT_READY for an
 * unknown or unsolved ticket. */
mpc_status mpc_policy_torques(mpc_ctx* ctx, uint64_t ticket, float* tau_dev, float* action_dev);

/* Measured arithmetic ceiling of one unit, the denominator of the solver's
 * roofline: a throughput kernel (64 warps per SM, independent dependency
 * chains on that unit only) run once to warm up and five times timed with
 * CUDA events on `stream` (a cudaStream_t, NULL = the legacy default stream)
 * on the current device.  Outputs (host): tflops = FLOP per launch / mean
 * launch time (an FMA counts 2 FLOP, an m16n8kK mma 2 x 16 x 8 x K); ms (may
 * be NULL) = mean launch time in milliseconds.  Synchronises the stream.
 * Errors: MPC_ERR_INVALID for an unknown kind or a NULL tflops,
 * MPC_ERR_CUDA for a failed allocation or launch. */
mpc_status mpc_measure_peak(int32_t kind, void* stream, double* tflops, double* ms);

/* One-line description of the last error on this context (never NULL). */
const char* mpc_last_error(mpc_ctx* ctx);

/* ---------------------------------------------------------------- serving
 * Continuous batching (the serving form of the replan loop): agents are the
 * context's slots; their warm starts and factor caches stay on the device.
 * Requests (slot, state, arrival time) are pushed from any host thread; a
 * later request of a slot that is not yet in a batch replaces the earlier
 * one's state (coalescing: the newest state wins) and is answered by the
 * same solve.  A worker thread, started by mpc_server_start, owns the
 * context until mpc_server_stop: whenever fewer than max_inflight batches
 * are on the GPU it forms the next one from every slot with pending requests
 * and no batch in flight (oldest request first, at most max_batch slots),
 * copies their states to the device and enqueues set-up, solve, gather and
 * the copy of the torques back on one of its own streams.  When that batch
 * completes, each request it covered is answered; its latency is the
 * completion time minus its arrival time on the server's clock
 * (mpc_server_clock: seconds since mpc_server_start).  While the server runs
 * the caller makes no other call on the context; the context outlives the
 * server.  Ownership: the server copies every input on push; results are
 * copied out by mpc_server_results.  Errors: MPC_ERR_INVALID for bad
 * arguments (a slot outside [0, pool), a NULL buffer); a CUDA or solver
 * error stops the worker and is returned by mpc_server_drain and
 * mpc_server_stop (text: mpc_server_last_error). */
typedef struct mpc_server mpc_server;

/* pool: slots served (<= the context's max_agents, ids 0..pool-1, each given
 * a model by mpc_set_models before); max_batch: largest batch; max_inflight:
 * regular batches on the GPU at a time (1..4; each has its own stream and
 * pinned and device buffers, allocated here, and one more lane of its own
 * carries the batches of deferred agents, see mpc_server_set_defer). */
mpc_status mpc_server_create(mpc_ctx* ctx, int32_t pool, int32_t max_batch, int32_t max_inflight,
                             mpc_server** out);
/* Deferral of slow agents (mode 0 = off, the default; set before
 * mpc_server_start).  Mode 1: batches are solved with MPC_SOLVE_DEFER_ADMM,
 * so an agent whose polish first fails does not hold its batch's answers
 * for the length of an ADMM solve; mode 2: with MPC_SOLVE_DEFER_SLOW, neither
 * does an agent that two reduced KKT solves of its polish do not settle;
 * mode 3: with MPC_SOLVE_DEFER_COLD, as mode 2 for cold agents (the first
 * requests after a model swap) and as mode 1 for the others.  The worker keeps
 * such agents (with their requests and states) and finishes them
 * (MPC_SOLVE_ADMM_ONLY in mode 1, no flag otherwise) in batches of their own
 * on an extra lane, answering their requests when those complete.
 * mpc_server_deferred gives the number of agents deferred so far.
 * MPC_ERR_INVALID for another mode. */
mpc_status mpc_server_set_defer(mpc_server* srv, int32_t mode);
int64_t mpc_server_deferred(mpc_server* srv);
/* Starts the worker and the server's clock.  MPC_ERR_STATE if started. */
mpc_status mpc_server_start(mpc_server* srv);
/* n requests (host arrays): slots [n], x0 [n][30], qd_meas [n][18], cmd [n][4],
 * phase [n], t_arrive [n] (seconds on the server's clock). */
mpc_status mpc_server_push(mpc_server* srv, int32_t n, const int32_t* slots, const float* x0,
                           const float* qd_meas, const float* cmd, const float* phase, const double* t_arrive);
/* Agents leaving and joining: each slot's model is replaced (its warm start
 * reset, as by mpc_set_models) by the worker once the slot has no batch in
 * flight; requests already pending for the slot are answered by the new
 * agent's solve. */
mpc_status mpc_server_set_models(mpc_server* srv, int32_t n, const int32_t* slots, const mpc_agent_model* models);
/* Waits until every pushed request is answered and every swap applied, at
 * most timeout_s seconds (MPC_ERR_TIMEOUT after that). */
mpc_status mpc_server_drain(mpc_server* srv, double timeout_s);
/* Seconds since mpc_server_start. */
double mpc_server_clock(mpc_server* srv);
/* Results so far (host buffers, each may be NULL except n_latency):
 * latency [cap] the answered requests' latencies in answer order (s),
 * *n_latency their count; tau [pool][18] and status [pool] each slot's last
 * answer (status -1: never answered); counters [6] = requests pushed,
 * answered, batches, agent-solves, solves not SOLVED, model swaps applied. */
mpc_status mpc_server_results(mpc_server* srv, double* latency, int64_t cap, int64_t* n_latency, float* tau,
                              int32_t* status, int64_t* counters);
/* The completed batches so far (host buffer, may be NULL): log [cap][3] =
 * launch time, completion time (s, server clock), agents; *n_batches their
 * count. */
mpc_status mpc_server_batches(mpc_server* srv, double* log, int64_t cap, int64_t* n_batches);
/* Stops the worker after its batches in flight have completed. */
mpc_status mpc_server_stop(mpc_server* srv);
const char* mpc_server_last_error(mpc_server* srv);
/* Stops the server if running and frees its streams and buffers. */
mpc_status mpc_server_destroy(mpc_server* srv);

/* Synthetic request source for measuring the server (the paper has no
 * counterpart; it stands in for the simulator's per-step requests): replays
 * n requests, arrival times t_arrive [n] (seconds from the end of this
 * call's set-up, non-decreasing; pushed with that moment added, on the
 * server's clock) for slots [n] (< pool), in real time from threads of its
 * own (the slots split between them) through mpc_server_push.  A request is one 10 ms environment step of
 * its agent: phase += phase_step, and one step of a mean-reverting walk of the
 * state about the agent's initial state x_init [pool][30] (host),
 * x <- x_init + revert (x - x_init) + sigma xi with xi ~ N(0, I); qd_meas =
 * 0.1 xi'; cmd [pool][4] with the commanded height set to the current one;
 * phase [pool] the initial phases.  Normal draws from a seeded counter-based
 * generator.  The trace is copied. */
typedef struct mpc_load mpc_load;
mpc_status mpc_load_start(mpc_server* srv, int64_t n, const double* t_arrive, const int32_t* slots, int32_t pool,
                          const float* x_init, const float* cmd, const float* phase, float revert, float sigma,
                          float phase_step, uint64_t seed, mpc_load** out);
/* New walk origins for slots whose agents changed (host arrays). */
mpc_status mpc_load_reset(mpc_load* load, int32_t n, const int32_t* slots, const float* x_init, const float* cmd,
                          const float* phase);
/* Waits (at most timeout_s) until every request has been pushed; lag_stats
 * [3] (may be NULL) = median, 99th percentile and largest delay between a
 * pushed chunk's oldest arrival time and its push (s). */
mpc_status mpc_load_wait(mpc_load* load, double timeout_s, double* lag_stats);
mpc_status mpc_load_destroy(mpc_load* load);

#ifdef __cplusplus
}
#endif

#endif /* MPCGPU_H */
