// Device-side data layout of the batched MPC solver.
//
// Every per-agent array lives in an arena indexed by the agent's slot
// (agent id).  Strides are fixed by the context's max_horizon (maxN).
//
// Index conventions (paper Sec. III-A, state and input of Eq. mpc_formulation
// in the centroidal reading):
//   x = [p 0-2, Theta 3-5, v 6-8, w 9-11, q 12-29]
//   u = [f_L 0-2, m_L 3-5, f_R 6-8, m_R 9-11, qdot 12-29]
// Indices 0-21 of x and u form the coupled block (base + leg joints): its
// stage matrices are dense 22x22.  Indices 22-29 are the eight arm joints,
// which decouple into scalar problems q+ = q + dt qdot.  Lane i of the warp
// that owns an agent handles index i of both x and u.
#pragma once
#include <stdint.h>

namespace mpc {

constexpr int NX = 30;
constexpr int NC = 22;      // coupled block size
constexpr int LD = 23;      // column stride of a 22x22 block (odd: no bank conflicts)
constexpr int LDD_HOST = 23;  // the same stride, for host code reading the lin record
constexpr int MB = 512;     // floats reserved per 22x22 block (22*23 = 506 used)
constexpr int NA = 8;       // arm joints
constexpr int NR = 56;      // inequality rows per stage
constexpr int RS = 64;      // stride of per-stage row arrays
constexpr int VS = 32;      // stride of per-stage lane vectors
constexpr int MAXN = 32;
constexpr int R24 = 24;     // row stride of the dense R24 blocks
constexpr int BLK = 528;    // floats of one R24 block (22 rows x 24)

// float model record (MODEL_F floats per agent).  M_TREE_ON != 0 marks an
// agent whose torque map runs the recursive Newton-Euler algorithm over its
// kinematic tree, stored from M_TREE on: per joint j (TREE_J floats at
// M_TREE + TREE_J j) the axis (3, parent frame), the joint's offset from the
// parent frame's origin (3), the link mass, its centre of mass (3, link
// frame) and the diagonal of its inertia about the centre of mass (3).
// Uploading a model clears both (mpc_set_models writes the whole record).
enum : int {
  M_MASS = 0, M_INVM = 1, M_INERTIA = 2, M_LEVER = 5, M_JLEG = 11,   // J_leg[f][r][j] at 11 + 30f + 5r + j
  M_MJ = 71, M_HJ = 89, M_KP = 107, M_KD = 125, M_Q = 143, M_R = 173,
  M_MU = 203, M_FZMAX = 204, M_QDMAX = 205, M_QLIM = 206, M_DT = 207,
  M_QNOM = 208, M_TREE_ON = 226, M_TREE = 256, MODEL_F = 512
};
enum : int { TREE_J = 13, TREE_F = 18 * TREE_J, TA_AXIS = 0, TA_OFF = 3, TA_MASS = 6, TA_COM = 7, TA_INER = 10 };
static_assert(M_TREE + TREE_F <= MODEL_F, "tree record exceeds the model record");
// double schedule record (SCHED_D doubles per agent)
enum : int { S_DT = 0, S_PERIOD = 1, S_DUTY = 2, S_OFF = 4, SCHED_D = 8 };
// per-agent input record (IN_F floats): x0, qd_meas, cmd, phase
enum : int { I_X0 = 0, I_QD = 32, I_CMD = 50, I_PHASE = 54, IN_F = 64 };
// per-agent output record (OUT_F floats)
// O_PRIM/O_DUAL: residual inf-norms; O_PRIM_N/O_DUAL_N: largest component over
// its own tolerance (<= 1 converged)
enum : int { O_TAU = 0, O_QSET = 18, O_QDSET = 36, O_V = 54, O_PRIM = 55, O_DUAL = 56, O_PRIM_N = 57,
             O_DUAL_N = 58, OUT_F = 64 };
// per-agent integer record (ST_I ints)
// T_ATTEMPTS: solves of the accepted polish (first + corrections; 0 = none accepted)
enum : int { T_STATUS = 0, T_ITERS = 1, T_REFAC = 2, T_POLISHED = 3, T_N = 4, T_WARM = 5, T_FIRST = 6,
             T_ATTEMPTS = 7, ST_I = 8 };

struct Arena {
  int max_agents;
  int maxN;
  // model
  const float* model;     // [A][MODEL_F]
  const double* sched;    // [A][SCHED_D]
  const int* horizon;     // [A]
  // warm-start / solution state
  float* xs;              // [A][(maxN+1)*VS]   x_k, lane-indexed
  float* us;              // [A][maxN*VS]
  float* ws;              // [A][maxN*RS]
  float* ys;              // [A][maxN*RS]
  float* rho;             // [A]
  int* warm_valid;        // [A] horizon the warm start was written with (0 = none)
  // outputs
  float* out;             // [A][OUT_F]
  int* stat;              // [A][ST_I]
  // scratch (solver workspace; contents meaningful only during a solve)
  float* inp;             // [A][IN_F]
  float* xref;            // [A][(maxN+1)*VS]
  float* uref;            // [A][maxN*VS]
  float* rlo;             // [A][maxN*RS] row lower bounds
  float* rhi;             // [A][maxN*RS]
  float* rcls;            // [A][maxN*RS] rho multiplier per row: 0 free, 1 ineq, 1e3 eq
  float* lin;             // [A][LIN_F]  A_base, B, per-stage dA (3x10) and c
  float* cK;              // [A][maxN*BLK] Riccati gains K_k (R24)
  float* cH;              // [A][maxN*BLK] inverse Schur blocks H_uu^-1 (R24)
  float* cEl;             // [A][maxN*128] polish: per-stage elimination of each input (float4 per lane)
  float* cD;              // [A][maxN*VS]  polish refinement: feed-forward terms of the correction
  float* cE;              // [A][maxN*64] e_k = P_{k+1} c_k (lanes 0-21), arm gain (22-29),
                          //   arm e (32-39), arm H_uu^-1 (54-61)
  float* xt;              // [A][(maxN+1)*VS] KKT-solve primal (x tilde)
  float* ut;              // [A][maxN*VS]
  float* dv;              // [A][maxN*VS]    feed-forward terms d_k
  int* act;               // [A][maxN*RS]    polish: active-set code per row
  int* order;             // [A] work queue of the persistent kernel: batch rows, longest first
  int* counter;           // [1] next queue position
  int* fault;             // [F_COUNT] device event counters (F_WAIT_TIMEOUTS: agents whose bounded
                          //   wait gave up; each retired its warp after draining its copies)
  // literal form only (MPC_FORM_LDL; NULL otherwise): the block LDL^T factors of
  // the full KKT system, per stage LDL_REC floats (strictly lower L by columns
  // and by rows, 1/D, the coupling block of the stage's dynamics rows to the
  // previous stage's x), the forward-substitution vectors, the dynamics
  // multipliers
  float* lL;              // [A][maxN*LDL_REC]
  float* lw;              // [A][maxN*LDL_W]
  float* ly;              // [A][maxN*VS]
  float* lS;              // [A][maxN*LDL_S] Ruiz scaling per stage (D of u_k and x_{k+1}, E of the
                          //   dynamics and inequality rows) and its per-iteration factors
  float* lc;              // [A] Ruiz cost scale c
};
// Ruiz scaling record of one stage (floats): D of u_k at LS_DU, of x_{k+1} at
// LS_DX, E of the stage's dynamics rows at LS_ED and of its 56 inequality rows
// at LS_EI; LS_T + the same offsets: one iteration's factors
enum : int { LS_DU = 0, LS_DX = 32, LS_ED = 64, LS_EI = 96, LS_T = 160, LDL_S = 320 };
// literal-form record of one stage: 90 block variables (u_k, the stage's 30
// dynamics multipliers, x_{k+1}); the strictly lower L without its
// structurally zero block (the x_{k+1} rows against the u_k columns), packed
// by columns at LDL_COL and by rows at LDL_ROW (3105 entries each), 1/D at
// LDL_IND, the 30 x 30 coupling block G_k (row-major) at LDL_G, and with
// the kinematic rows the three rows of L31 that they fill (the x_{k+1} rows of
// v, on u_k; row-major 3 x 30) at LDL_L31
enum : int { LDL_NB = 90, LDL_NL = 3105, LDL_COL = 0, LDL_ROW = 3108, LDL_IND = 6216, LDL_G = 6312,
             LDL_L31 = 7232, LDL_REC = 7328, LDL_W = 96 };
// kinematic rows of a stage (literal form): 56 + 3i + r no-slip of foot i,
// component r; 62 + i swing height of foot i
enum : int { KIN_ROW = 56, KIN_NR = 8 };
enum : int { F_WAIT_TIMEOUTS = 0, F_COUNT = 4 };

// lin record layout: dense A_base and B (column-major, stride 23), their
// compact columns (22 x 6 values, padded to 136), then per stage k the leg
// coupling block dA_k (3x10 at +0) and the affine term c_k (at +32)
enum : int { L_ABASE = 0, L_B = MB, L_AV = 2 * MB, L_BV = 2 * MB + 136, L_STAGE = 2 * MB + 272 };
__host__ __device__ constexpr int lin_floats(int maxN) { return L_STAGE + maxN * 64; }

struct Batch {
  int n;
  const int* ids;         // [n] agent slot per batch row
  const float* x0;        // [n][30]
  const float* qd;        // [n][18]
  const float* cmd;       // [n][4]
  const float* phase;     // [n]
  const int* order;       // [n] processing order of the rows (NULL: row order)
  int* counter;           // work-queue counter, zero at launch (NULL: static assignment)
};

// default poll count of a bounded mbarrier wait (mpc_config.spin_limit)
constexpr int kSpinLimit = 1 << 22;

struct SolverParams {
  float rho0, sigma, alpha, eps_abs, eps_rel, early_polish;
  int max_iter, fixed_iters, check_every, adaptive_rho, polish, warm_start, warm_polish;
  int precision;   // factor precision: PREC_FP32 / PREC_TF32 / PREC_BF16 / PREC_FP64
  int refine;      // iterative-refinement steps on a polish from the previous active set
  int refine_admm; // ... and on a polish that follows ADMM iterations
  int trees;       // 1: some agent has a kinematic tree; mpc_k_rnea runs after the solve
  int split;       // fused form: 1 = set-up and torque map as kernels of their own
  int spin_limit;  // polls of a bounded mbarrier wait before it gives up (MPC_AGENT_TIMEOUT)
  int wait_test_slot;  // failure-detection test: the first stage-block wait of this agent slot is
                       //   armed with no copy behind it, so it runs out (-1: off)
  int ruiz;            // literal form: Ruiz equilibration iterations (0: none)
  int defer;           // fused form: 1 = an agent whose polish first fails ends DEFERRED once its
                       //   ADMM warm start is written (no ADMM in this launch); 2 = an agent whose
                       //   polish first has not passed after 2 reduced solves ends DEFERRED with
                       //   its corrected active set kept (a later solve continues from it); 3 = as
                       //   2 for a cold agent, and a warm one when its polish first fails
  int kin;             // literal form: 1 = the kinematic rows 56-63 of every stage
  float kin_b[6];      // their swing curve's Bezier control points b_0 .. b_5
};

}  // namespace mpc
