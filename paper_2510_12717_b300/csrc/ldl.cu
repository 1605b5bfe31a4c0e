// Literal form of the paper's QP solve (MPC_FORM_LDL): OSQP's ADMM on the
// full KKT system of Eq. (kkt_system), factored once per solve into
// L_K D_K L_K^T (Eq. ldl) and solved by forward substitution, diagonal
// scaling and backward substitution in every iteration (Eqs. backsolve_1,
// backsolve_2); Alg. 1 with cuDSS_fac / cuDSS_solve replaced by the kernels
// below.  The ADMM update (f_ADMM) is OSQP's (Stellato et al. 2020, Sec. 3),
// to which the paper defers after Eq. (backsolve_2):
//
//   [[P + sigma I, A^T], [A, -rho^-1]] [x~; nu] = [sigma x - q; z - rho^-1 y]
//   z~ = z + rho^-1 (nu - y),  x <- alpha x~ + (1 - alpha) x,
//   zr = alpha z~ + (1 - alpha) z,  z <- clip(zr + rho^-1 y, l, u),
//   y <- y + rho (zr - z).
//
// The rows of A are the dynamics x_{k+1} - A_k x_k - B u_k = c_k (l = u, step
// size rho_eq = 1e3 rho) and the stage inequality rows (wrench boxes,
// friction pyramids, joint-rate boxes on u_k, joint boxes on x_{k+1}; rows
// with l = u take rho_eq, free rows are left out).
//
// Elimination order (a symmetric permutation of A_K; A_K is quasi-definite,
// so every order has an LDL^T factorisation with diagonal D): first the
// inequality rows, one 1 x 1 pivot -1/rho_r each (their Schur complement adds
// C^T diag(rho) C to the stage's u_k and x_{k+1} blocks and never leaves the
// stage), then per stage k the 90 block variables (u_k, the stage's dynamics
// multipliers, x_{k+1}).  In that order A_K is block tridiagonal in the
// stages: the only coupling between blocks k-1 and k is the entry -A_k of the
// dynamics rows of stage k on x_k.  The block factorisation: S_0 = M_0,
// S_k = M_k - A_k X_{k-1} A_k^T on the multiplier block, where X_{k-1} is the
// x_k block of S_{k-1}^-1 = L_xx^-T D_xx^-1 L_xx^-1 (x last in the block);
// with Y_k = A_k L_xx^-T, the off-diagonal factor is L_{k,k-1} = -Y_k D_xx^-1
// =: -G_k and the update is G_k Y_k^T.  The dense 90 x 90 blocks are factored
// without pivoting.
//
// Kernels (one warp per agent):
//   mpc_k_ldl_factor : assembles and factors the blocks stage by stage, the
//                      rows of its 30-wide sub-blocks in registers; writes L (packed by columns for the
//                      forward substitution and by rows for the backward one,
//                      so that both read coalesced), 1/D and G_k
//   mpc_k_ldl_admm   : one warp runs the iterations; per iteration a forward pass over the
//                      stages (right-hand side, coupling, unit lower solve)
//                      and a backward pass (1/D, coupling, unit upper solve,
//                      then the stage's relaxation, projection and dual
//                      updates); fixed N_QP (the paper's mode) or until OSQP's
//                      stopping test with a residual check every check_every
// The set-up kernel before them (schedule, references, bounds, linearisation,
// the cold start of f_init) and the torque map after them are the solver's
// own.  Every iteration reads each stage's factors from global memory.
#include "solver_dev.cuh"
#include "solver.h"

namespace mpc {
namespace {

constexpr int NB = LDL_NB;
constexpr int F_FLOATS = 30 * 32;                        // factor kernel: shared floats per warp

// Packed strictly lower L without the zero block (rows 60-89 x columns
// 0-29): column j holds rows j+1 .. 59 (j < 30) or j+1 .. 89; row i holds
// columns 0 .. i-1 (i < 60) or 30 .. i-1.  L(i, j) is at col_off(j) + i - j - 1
// by columns and at row_off(i) + j - row_skip(i) by rows.
__host__ __device__ constexpr int col_off(int j) {
  return j <= 30 ? 59 * j - j * (j - 1) / 2 : 1335 + 59 * (j - 30) - (j - 30) * (j - 31) / 2;
}
__host__ __device__ constexpr int row_off(int i) { return i <= 60 ? i * (i - 1) / 2 : 1770 + (i - 1) * (i - 60) / 2; }
__host__ __device__ constexpr int row_skip(int i) { return i >= 60 ? 30 : 0; }
static_assert(col_off(89) == LDL_NL && row_off(90) == LDL_NL, "packed layout size");
// Stored positions: one float of padding before the second and two before the
// third 30-wide group of columns (of rows), so that each group starts on a
// 16-byte boundary and the iterations can stage it by a bulk copy of its own
// (3107 of the 3108 floats of each layout in use).
__host__ __device__ constexpr int col_pos(int j) { return col_off(j) + (j >= 30) + (j >= 60); }
__host__ __device__ constexpr int row_pos(int i) { return row_off(i) + (i >= 30) + (i >= 60); }
// the three staged parts of a pass: forward part p = columns 30p .. 30p + 29
// (88 for p = 2), backward part p = rows 89 .. 60, 59 .. 30, 29 .. 1; their
// start in the layout and the floats copied (rounded up to 16 bytes)
__host__ __device__ constexpr int fwd_start(int p) { return col_pos(30 * p); }
__host__ __device__ constexpr int bwd_start(int p) { return p == 0 ? row_pos(60) : p == 1 ? row_pos(30) : 0; }
__host__ __device__ constexpr int part_floats(int p) { return p == 2 ? 436 : 1336; }
static_assert(fwd_start(1) % 4 == 0 && fwd_start(2) % 4 == 0 && bwd_start(0) % 4 == 0 && bwd_start(1) % 4 == 0,
              "staged parts start on 16-byte boundaries");
static_assert(fwd_start(2) + part_floats(2) <= LDL_ROW - LDL_COL && bwd_start(0) + part_floats(0) <= LDL_ROW - LDL_COL &&
              col_pos(88) + 1 <= fwd_start(2) + part_floats(2) && row_pos(89) + 59 <= bwd_start(0) + part_floats(0) &&
              col_pos(59) + 30 <= fwd_start(1) + part_floats(1) && row_pos(59) + 59 <= bwd_start(1) + part_floats(1) &&
              col_pos(29) + 30 <= fwd_start(0) + part_floats(0) && row_pos(29) + 29 <= bwd_start(2) + part_floats(2),
              "each part holds its columns (rows) within its layout");

__device__ __forceinline__ bool live_row(const Arena& a, const Batch& b, int row) {
  if (row >= b.n) return false;
  const int s = b.ids[row];
  return s >= 0 && s < a.max_agents && a.horizon[s] >= 2 && a.horizon[s] <= a.maxN;
}

// entry (r, c) of the dynamics matrix A_k of the coupled block and the arms
// (A_base plus the contact-dependent leg-joint block dA_k of rows 9-11)
__device__ __forceinline__ float a_entry(const float* lin, int k, int r, int c) {
  if (r < NC) {
    if (c >= NC) return 0.f;
    float v = lin[L_ABASE + c * LDD + r];
    if (r >= 9 && r < 12 && c >= 12) v += lin[L_STAGE + k * 64 + (r - 9) * 10 + (c - 12)];
    return v;
  }
  return c == r ? 1.f : 0.f;
}
__device__ __forceinline__ float b_entry(const float* lin, float dt, int r, int c) {
  if (r < NC) return c < NC ? lin[L_B + c * LDD + r] : 0.f;
  return c == r ? dt : 0.f;
}
// coefficient of input c (0 f_x, 1 f_y, 2 f_z of one foot) in the foot's
// friction-pyramid row t (f_x - mu f_z, -f_x - mu f_z, f_y - mu f_z, -f_y - mu f_z)
__device__ __forceinline__ float pyr_coef(int c, int t, float mu) {
  if (c == 2) return -mu;
  if (c == 0) return t == 0 ? 1.f : (t == 1 ? -1.f : 0.f);
  return t == 2 ? 1.f : (t == 3 ? -1.f : 0.f);
}
// value of inequality row r (0..55) of a stage at (u_k, x_{k+1})
__device__ __forceinline__ float row_value(int r, const float* U, const float* X, float mu) {
  if (r < 12) return U[r];
  if (r < 20) {
    const int f = (r - 12) >> 2, t = (r - 12) & 3, b = 6 * f;
    const float s = (t < 2 ? U[b] : U[b + 1]) * ((t & 1) ? -1.f : 1.f);
    return s - mu * U[b + 2];
  }
  if (r < 38) return U[r - 8];
  return X[r - 26];
}

// ------------------------------------------------------------------ kinematic rows
// The no-slip and swing-height rows of Eq. (mpc_formulation), read at node
// k+1 on (u_k, x_{k+1}) (rows KIN_ROW + q):
//   q = 3i + r (r = 0, 1, 2): v_{k+1,r} + J_leg,i[r] . qdot_leg,i = 0 (foot i in stance)
//   q = 6 + i:               p_z + J_leg,i[2] . q_leg,i = c_h + B(t_sw) + J_leg,i[2] . q_nom,i (swing)
// Their coefficients in shared memory, by lane: KU row q (q < 6) holds the u
// coefficients of no-slip row q (its x coefficient is 1 at lane 6 + r); KC
// row i the x coefficients of foot i's height row.
constexpr int KIN_SM = 8 * 32;
__device__ __forceinline__ void kin_fill(float* ks, const float* md, int lane) {
  for (int q = 0; q < 8; ++q) {
    const int f = q < 6 ? q / 3 : q - 6, r = q < 6 ? q % 3 : 2;
    const int j = lane - 12 - 5 * f;
    float v = (j >= 0 && j < 5) ? md[M_JLEG + 30 * f + 5 * r + j] : 0.f;
    if (q >= 6 && lane == 2) v = 1.f;
    ks[q * 32 + lane] = v;
  }
  __syncwarp();
}
// value of kinematic row q at (u_k, x_{k+1})
__device__ __forceinline__ float kin_value(int q, const float* U, const float* X, const float* ks) {
  const int f = q < 6 ? q / 3 : q - 6;
  const int b = 12 + 5 * f;
  const float* c = ks + q * 32 + b;
  float v;
  if (q < 6) {
    v = X[6 + q % 3];
#pragma unroll
    for (int j = 0; j < 5; ++j) v = fmaf(c[j], U[b + j], v);
  } else {
    v = X[2];
#pragma unroll
    for (int j = 0; j < 5; ++j) v = fmaf(c[j], X[b + j], v);
  }
  return v;
}

// Bounds, classes and the cold start of the kinematic rows of every stage:
// node k+1's contact state from the schedule in double precision (the
// operation order of the set-up kernel's), its swing progress
// t_sw = (s - d_i) / (1 - d_i) and the height B(t_sw) of the Bezier curve
// (control points in SolverParams), in double precision.  Lane k: stage k.
__global__ void __launch_bounds__(32) mpc_k_ldl_kin(Arena a, Batch b, SolverParams prm) {
  const int lane = threadIdx.x;
  const int row = blockIdx.x;
  if (!live_row(a, b, row)) return;
  const int slot = b.ids[row];
  const AgentPtrs ap = agent_ptrs(a, slot);
  if (ap.st[T_STATUS] == MPC_AGENT_NAN_) return;
  const int N = ap.N;
  const float* md = ap.mdl;
  const int k = lane;
  if (k >= N) return;
  const double step = __ddiv_rn(ap.sch[S_DT], ap.sch[S_PERIOD]);
  double ph = __dadd_rn((double)ap.inp[I_PHASE], __dmul_rn((double)(k + 1), step));
  ph = __dsub_rn(ph, floor(ph));
  float* lo = ap.rlo + k * RS + KIN_ROW;
  float* hi = ap.rhi + k * RS + KIN_ROW;
  float* cl = ap.rcls + k * RS + KIN_ROW;
  float* w = ap.w + k * RS + KIN_ROW;
  float* y = ap.y + k * RS + KIN_ROW;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    double s = __dadd_rn(ph, ap.sch[S_OFF + i]);
    s = __dsub_rn(s, floor(s));
    const double d = ap.sch[S_DUTY + i];
    const bool stance = s < d;
    for (int r = 0; r < 3; ++r) {
      lo[3 * i + r] = stance ? 0.f : -INFINITY;
      hi[3 * i + r] = stance ? 0.f : INFINITY;
      cl[3 * i + r] = stance ? 1000.f : 0.f;
      w[3 * i + r] = 0.f;
      y[3 * i + r] = 0.f;
    }
    if (stance) {
      lo[6 + i] = -INFINITY; hi[6 + i] = INFINITY; cl[6 + i] = 0.f; w[6 + i] = 0.f;
    } else {
      const double t = (s - d) / (1.0 - d), t1 = 1.0 - t;
      // Bernstein weights C(5, j) t^j (1 - t)^(5 - j)
      const double t2 = t * t, u2 = t1 * t1;
      const double wj[6] = {u2 * u2 * t1, 5.0 * t * u2 * u2, 10.0 * t2 * u2 * t1, 10.0 * t2 * t * u2,
                            5.0 * t2 * t2 * t1, t2 * t2 * t};
      double bz = 0.0;
      for (int j = 0; j < 6; ++j) bz += wj[j] * (double)prm.kin_b[j];
      double h = (double)ap.inp[I_CMD] + bz;
      for (int j = 0; j < 5; ++j) h += (double)md[M_JLEG + 30 * i + 10 + j] * (double)md[M_QNOM + 5 * i + j];
      lo[6 + i] = hi[6 + i] = (float)h;
      cl[6 + i] = 1000.f;
      w[6 + i] = (float)h;   // the cold start's z: its row value projected onto [h, h]
    }
    y[6 + i] = 0.f;
  }
}

// ------------------------------------------------------------------ factor
// One warp per agent; lane l (< 30) holds row l of each 30 x 30 block in
// registers.  The stage's 90 x 90 block M_k = [[A11, ., .], [A21, A22, .],
// [0, I, A33]] (u_k, multipliers, x_{k+1}; A11 = R_t with the pyramid
// couplings, A21 = -B, A22 = -rho_eq^-1 I - A_k X_{k-1} A_k^T, A33 = Q_t) is
// factored as a supernodal LDL^T over its three 30-wide groups:
//   A11 = L11 D1 L11^T;  L21 = A21 L11^-T D1^-1;  L22 D2 L22^T = A22 - L21 D1 L21^T;
//   L31 = 0 (the x_{k+1} rows have no entry on u_k);  L32 = L22^-T D2^-1;
//   L33 D3 L33^T = A33 - L32 D2 L32^T,
// the same factors as the dense right-looking LDL^T of M_k in this order.
// A 30 x 30 LDL^T of rows held in registers: at pivot j the unscaled column
// entry t_c = S(c, j) of row c is broadcast from lane c by a shuffle.
__device__ __forceinline__ void ldl30(float (&a)[30], float& d, int lane) {
#pragma unroll
  for (int j = 0; j < 30; ++j) {
    const float t = a[j];
    const float ij = 1.f / __shfl_sync(FULL, t, j);
    const float l = t * ij;
#pragma unroll
    for (int c = j + 1; c < 30; ++c) {
      const float tc = __shfl_sync(FULL, t, c);
      if (lane >= c) a[c] = fmaf(-l, tc, a[c]);
    }
    if (lane == j) d = t;
    if (lane > j) a[j] = l;
  }
}
// y L^T = a for row vectors (L unit lower, row c of L in register array Lr of
// lane c): y_c = a_c - sum_{c' < c} L(c, c') y_c'
__device__ __forceinline__ void trsv_rows(float (&y)[30], const float (&Lr)[30]) {
#pragma unroll
  for (int c = 1; c < 30; ++c) {
#pragma unroll
    for (int q = 0; q < c; ++q) y[c] = fmaf(-__shfl_sync(FULL, Lr[q], c), y[q], y[c]);
  }
}

// row i of L, columns j0 .. j0 + 29 (only j < i when diag), into both layouts
template <bool DIAG>
__device__ __forceinline__ void put_row(float* rec, int i, int j0, const float (&v)[30], int lane) {
  if (lane >= 30) return;
  float* Lr = rec + LDL_ROW;
  float* Lc = rec + LDL_COL;
#pragma unroll
  for (int c = 0; c < 30; ++c) {
    const int j = j0 + c;
    if (!DIAG || j < i) {
      Lr[row_pos(i) + j - row_skip(i)] = v[c];
      Lc[col_pos(j) + i - j - 1] = v[c];
    }
  }
}

// KIN: with the kinematic rows.  Their pivots, eliminated first like the
// other rows', add C^T diag(rho) C to the blocks: to A11 (u_k) the no-slip
// rows' J^T J on a foot's leg rates, to A33 (x_{k+1}) their unit entries on v
// and the height rows' c c^T, and to A31 the no-slip rows' cross terms between
// v_{k+1} and the leg rates.  So three rows of L31 (x_{k+1} rows 6-8) are no
// longer zero: L31 = A31 L11^-T D1^-1; L32 = (A32 - L31 D1 L21^T) L22^-T D2^-1;
// A33 loses L31 D1 L31^T as well.
constexpr int F_KIN = KIN_SM + 3 * 32 + 2 * 3 * 33 + 2;     // KU/KC, L31 rows, Y31 and M32 (stride 33)
template <bool KIN>
__global__ void __launch_bounds__(32) mpc_k_ldl_factor(Arena a, Batch b, SolverParams prm) {
  const int lane = threadIdx.x;
  const int row = blockIdx.x;
  if (!live_row(a, b, row)) return;
  const int slot = b.ids[row];
  const AgentPtrs ap = agent_ptrs(a, slot);
  if (ap.st[T_STATUS] == MPC_AGENT_NAN_) return;
  extern __shared__ __align__(16) float fsm[];
  float* T = fsm;                   // 30 rows of stride 32: the scaled rows of the last solve
  float* ks = fsm + F_FLOATS;       // KIN: coefficients of the kinematic rows
  float* T31 = ks + KIN_SM;         // KIN: the three scaled rows of L31 (stride 32)
  float* Y31 = T31 + 3 * 32;        // KIN: ... unscaled (stride 33)
  float* M32 = Y31 + 3 * 33;        // KIN: rows 6-8 of L31 D1 L21^T (stride 33)
  const float* md = ap.mdl;
  const float* lin = ap.lin;
  const int N = ap.N;
  const float dt = md[M_DT], mu = md[M_MU], sigma = prm.sigma;
  const float rho = *ap.rho, rho_eq = 1e3f * rho;
  const int l = lane < 30 ? lane : 29;   // lanes 30, 31 shadow row 29 (their results are unused)
  float* rec0 = a.lL + (size_t)slot * a.maxN * LDL_REC;
  // Ruiz scaling (all ones without equilibration): the factor is that of the
  // scaled system, P -> c D P D, A -> E A D
  const float* S0 = a.lS + (size_t)slot * a.maxN * LDL_S;
  const float cs = a.lc[slot];
  float mrow[30];                        // row l of A_k X_{k-1} A_k^T (0 at k = 0)
#pragma unroll
  for (int c = 0; c < 30; ++c) mrow[c] = 0.f;
  if (KIN) kin_fill(ks, md, lane);
  const bool is3 = KIN && lane >= 6 && lane < 9;   // KIN: lanes 6-8 hold the x_{k+1} rows of v
  const int r3c = is3 ? lane - 6 : 0;
  for (int k = 0; k < N; ++k) {
    float* rec = rec0 + (size_t)k * LDL_REC;
    const float* cls = ap.rcls + k * RS;
    const float* Sk = S0 + (size_t)k * LDL_S;
    const float du = Sk[LS_DU + l], dx = Sk[LS_DX + l], ed = Sk[LS_ED + l];
    const float* ei = Sk + LS_EI;
    // ---- A11 = R_t: diagonal, and the pyramid couplings of row f_z of a foot
    float av[30];
#pragma unroll
    for (int c = 0; c < 30; ++c) av[c] = 0.f;
    {
      const int ru = l < 12 ? l : l + 8;
      float dg = cs * du * du * 2.f * dt * md[M_R + l] + sigma + rho * cls[ru] * (ei[ru] * du) * (ei[ru] * du);
      if (l < 12 && (l % 6) < 3) {
        const int f = l / 6, cc = l - 6 * f, p = 12 + 4 * f, b0 = 6 * f;
        float w[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) w[t] = rho * cls[p + t] * ei[p + t] * ei[p + t];
        dg += du * du * (cc == 0 ? w[0] + w[1] : (cc == 1 ? w[2] + w[3] : mu * mu * (w[0] + w[1] + w[2] + w[3])));
        if (cc == 2) {
          const float db0 = Sk[LS_DU + b0], db1 = Sk[LS_DU + b0 + 1];
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            if (c == l - 2) av[c] = mu * (w[1] - w[0]) * db0 * du;
            if (c == l - 1) av[c] = mu * (w[3] - w[2]) * db1 * du;
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 30; ++c)
        if (c == l) av[c] = dg;
    }
    // KIN: the step sizes of the stage's kinematic rows (0 on a free row),
    // the no-slip rows' J^T diag(rho) J on A11
    float rk[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) rk[q] = KIN ? rho * cls[KIN_ROW + q] : 0.f;
    if (KIN) {
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const float aq = rk[q] * ks[q * 32 + l];
#pragma unroll
        for (int c = 0; c < 30; ++c) av[c] = fmaf(aq, ks[q * 32 + c], av[c]);
      }
    }
    const float q33 = cs * dx * dx * 2.f * dt * md[M_Q + l] + sigma +
                      (l >= 12 ? rho * cls[l + 26] * (ei[l + 26] * dx) * (ei[l + 26] * dx) : 0.f);
    const float a32 = ed * dx;           // the x_{k+1} entry of dynamics row l, scaled
    const float ed1 = k + 1 < N ? Sk[LDL_S + LS_ED + l] : 1.f;   // E of the next stage's dynamics row l
    float dd0 = 1.f, dd1 = 1.f, dd2 = 1.f;
    // KIN: this lane's share of the height rows' c c^T and of the no-slip
    // rows' unit entries on A33; rows 6-8 of L31 D1 L31^T
    const float h6 = KIN ? rk[6] * ks[6 * 32 + l] : 0.f, h7 = KIN ? rk[7] * ks[7 * 32 + l] : 0.f;
    const float nd = is3 ? rk[r3c] + rk[3 + r3c] : 0.f;
    float m33[3] = {0.f, 0.f, 0.f};
    // ---- the three groups in turn: factor the (updated) diagonal block,
    // store its rows, solve the next off-diagonal block's rows against it
    // (A21 = -B, A32 = I, and for the coupling A_{k+1}), scale them by 1/D,
    // and form the next diagonal block's update from the scaled rows
#pragma unroll 1
    for (int g = 0; g < 3; ++g) {
      float d = 1.f;
      ldl30(av, d, lane);
      if (g == 0) dd0 = d;
      else if (g == 1) dd1 = d;
      else dd2 = d;
      put_row<true>(rec, 30 * g + l, 30 * g, av, lane);
      if (g == 2 && k + 1 == N) break;
      if (KIN && g == 0) {
        // rows 6-8 of L31: the rows of A31 solved against L11, then scaled
        float y3[30];
#pragma unroll
        for (int c = 0; c < 30; ++c) y3[c] = is3 ? fmaf(rk[r3c], ks[r3c * 32 + c], rk[3 + r3c] * ks[(3 + r3c) * 32 + c]) : 0.f;
        trsv_rows(y3, av);
#pragma unroll
        for (int c = 0; c < 30; ++c) {
          const float v = y3[c] / __shfl_sync(FULL, d, c);
          if (is3) {
            rec[LDL_L31 + r3c * 30 + c] = v;
            T31[r3c * 32 + c] = v;
            Y31[r3c * 33 + c] = y3[c];
          }
        }
        __syncwarp();
      }
      float y[30];
#pragma unroll
      for (int c = 0; c < 30; ++c)
        y[c] = g == 0 ? -b_entry(lin, dt, l, c) * ed * __shfl_sync(FULL, du, c)
                      : (g == 1 ? (c == l ? a32 : 0.f) - (is3 ? M32[r3c * 33 + c] : 0.f)
                                : a_entry(lin, k + 1, l, c) * ed1 * __shfl_sync(FULL, dx, c));
      trsv_rows(y, av);
      float ys[30];
#pragma unroll
      for (int c = 0; c < 30; ++c) ys[c] = y[c] / __shfl_sync(FULL, d, c);
      if (KIN && g == 0) {
        // column l of rows 6-8 of L31 D1 L21^T, from this lane's row of L21
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          float acc = 0.f;
#pragma unroll
          for (int m = 0; m < 30; ++m) acc = fmaf(Y31[q * 33 + m], ys[m], acc);
          if (lane < 30) M32[q * 33 + l] = acc;
        }
      }
      if (g < 2) {
        put_row<false>(rec, 30 * (g + 1) + l, 30 * g, ys, lane);
      } else if (lane < 30) {
        float* G = rec0 + (size_t)(k + 1) * LDL_REC + LDL_G;
#pragma unroll
        for (int c = 0; c < 30; ++c) G[lane * 30 + c] = ys[c];
      }
      __syncwarp();
      if (lane < 30)
#pragma unroll
        for (int c = 0; c < 30; ++c) T[lane * 32 + c] = ys[c];
      __syncwarp();
      // row l of (unscaled rows) x (scaled rows)^T
#pragma unroll
      for (int s2 = 0; s2 < 30; ++s2) {
        float acc = 0.f;
        const float4* r4 = reinterpret_cast<const float4*>(T + s2 * 32);
#pragma unroll
        for (int q = 0; q < 7; ++q) {
          const float4 v = r4[q];
          acc = fmaf(y[4 * q], v.x, acc);
          acc = fmaf(y[4 * q + 1], v.y, acc);
          acc = fmaf(y[4 * q + 2], v.z, acc);
          acc = fmaf(y[4 * q + 3], v.w, acc);
        }
        acc = fmaf(y[28], T[s2 * 32 + 28], acc);
        acc = fmaf(y[29], T[s2 * 32 + 29], acc);
        if (g == 0) av[s2] = (s2 == l ? -1.f / rho_eq : 0.f) - mrow[s2] - acc;
        else if (g == 1) {
          float v = (s2 == l ? q33 : 0.f) - acc;
          if (KIN) {
            // the kinematic rows on A33, less L31 D1 L31^T
            v = fmaf(h6, ks[6 * 32 + s2], fmaf(h7, ks[7 * 32 + s2], v));
            if (s2 == l) v += nd;
            if (s2 >= 6 && s2 < 9 && is3) v -= m33[s2 - 6];
          }
          av[s2] = v;
        } else mrow[s2] = acc;
      }
      if (KIN && g == 0 && is3) {
        // rows 6-8 of L31 D1 L31^T
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          float acc = 0.f;
          for (int m = 0; m < 30; ++m) acc = fmaf(Y31[r3c * 33 + m], T31[q * 32 + m], acc);
          m33[q] = acc;
        }
      }
      __syncwarp();
    }
    if (lane < 30) {
      // (the x_{k+1} rows have no entry on u_k: L31 = 0, not stored)
      rec[LDL_IND + l] = 1.f / dd0;
      rec[LDL_IND + 30 + l] = 1.f / dd1;
      rec[LDL_IND + 60 + l] = 1.f / dd2;
    }
  }
}

// ------------------------------------------------------------------ Ruiz (f_Ruiz)
// OSQP's modified Ruiz equilibration of the KKT matrix [[P, A^T], [A, 0]]
// (Stellato et al. 2020, Sec. 5.1), stage by stage: each iteration divides
// every variable's and row's column by the square root of its inf-norm in the
// currently scaled matrix (below 1e-4 counted as 1, above 1e4 as 1e4), then
// scales the cost by 1 / max(mean column inf-norm of P, |q|_inf).  A column
// of u_k meets P, the stage's dynamics rows (through B) and its box and
// pyramid rows; one of x_{k+1} meets P, the stage's dynamics rows (identity),
// the next stage's (through A_{k+1}) and its joint box; a dynamics row meets
// x_{k+1}, u_k and (k >= 1) x_k.  One warp per agent; A_base and B (signed,
// 30 x 30 with the arms) in shared memory.
__device__ __forceinline__ float ruiz_lim(float v) { return v < 1e-4f ? 1.f : fminf(v, 1e4f); }

__global__ void __launch_bounds__(32) mpc_k_ldl_ruiz(Arena a, Batch b, SolverParams prm) {
  const int lane = threadIdx.x;
  const int row = blockIdx.x;
  if (!live_row(a, b, row)) return;
  const int slot = b.ids[row];
  const AgentPtrs ap = agent_ptrs(a, slot);
  if (ap.st[T_STATUS] == MPC_AGENT_NAN_) return;
  extern __shared__ __align__(16) float rsm[];
  float* sA = rsm;                  // A_base (rows of stride 31)
  float* sB = rsm + 30 * 31;        // B
  const float* md = ap.mdl;
  const float* lin = ap.lin;
  const int N = ap.N;
  const float dt = md[M_DT], mu = md[M_MU];
  float* S0 = a.lS + (size_t)slot * a.maxN * LDL_S;
  for (int k = 0; k < N; ++k)
    for (int t = lane; t < LS_T; t += 32) S0[(size_t)k * LDL_S + t] = 1.f;
  if (prm.ruiz <= 0) {        // no equilibration: every factor 1
    if (lane == 0) a.lc[slot] = 1.f;
    return;
  }
  for (int t = lane; t < 900; t += 32) {
    const int r = t / 30, c = t - 30 * r;
    sA[r * 31 + c] = r < NC ? (c < NC ? lin[L_ABASE + c * LDD + r] : 0.f) : (c == r ? 1.f : 0.f);
    sB[r * 31 + c] = b_entry(lin, dt, r, c);
  }
  __syncwarp();
  // entry (r, c) of A_k: A_base plus the stage's leg-joint block dA_k
  auto ak = [&](int k, int r, int c) {
    float v = sA[r * 31 + c];
    if (r >= 9 && r < 12 && c >= 12 && c < NC) v += lin[L_STAGE + k * 64 + (r - 9) * 10 + (c - 12)];
    return v;
  };
  float cs = 1.f;
  const int j = lane < 30 ? lane : 29;
  const float Ru = 2.f * dt * md[M_R + j], Qx = 2.f * dt * md[M_Q + j];
  for (int it = 0; it < prm.ruiz; ++it) {
    // ---- pass 1: the inf-norms of the current scaled matrix -> the factors
    for (int k = 0; k < N; ++k) {
      float* Sk = S0 + (size_t)k * LDL_S;
      const float* Sn = k + 1 < N ? Sk + LDL_S : nullptr;
      const float* Sp = k ? Sk - LDL_S : nullptr;
      const float* cls = ap.rcls + k * RS;
      if (lane < 30) {
        // column u_k,j
        const float du = Sk[LS_DU + j];
        float m = 0.f;
        for (int i = 0; i < 30; ++i) m = fmaxf(m, Sk[LS_ED + i] * fabsf(sB[i * 31 + j]));
        const int ru = j < 12 ? j : j + 8;
        if (cls[ru] > 0.f) m = fmaxf(m, Sk[LS_EI + ru]);
        if (j < 12 && (j % 6) < 3) {
          const int f = j / 6, cc = j - 6 * f, p = 12 + 4 * f;
          for (int t = 0; t < 4; ++t)
            if (cls[p + t] > 0.f) m = fmaxf(m, Sk[LS_EI + p + t] * fabsf(pyr_coef(cc, t, mu)));
        }
        const float colu = fmaxf(cs * du * du * Ru, du * m);
        // column x_{k+1},j
        const float dx = Sk[LS_DX + j];
        m = Sk[LS_ED + j];
        if (Sn)
          for (int i = 0; i < 30; ++i) m = fmaxf(m, Sn[LS_ED + i] * fabsf(ak(k + 1, i, j)));
        if (j >= 12 && cls[j + 26] > 0.f) m = fmaxf(m, Sk[LS_EI + j + 26]);
        const float colx = fmaxf(cs * dx * dx * Qx, dx * m);
        // dynamics row k, j: x_{k+1} - A_k x_k - B u_k
        m = Sk[LS_DX + j];
        for (int c = 0; c < 30; ++c) m = fmaxf(m, Sk[LS_DU + c] * fabsf(sB[j * 31 + c]));
        if (Sp)
          for (int c = 0; c < 30; ++c) m = fmaxf(m, Sp[LS_DX + c] * fabsf(ak(k, j, c)));
        const float rowd = Sk[LS_ED + j] * m;
        Sk[LS_T + LS_DU + j] = rsqrtf(ruiz_lim(colu));
        Sk[LS_T + LS_DX + j] = rsqrtf(ruiz_lim(colx));
        Sk[LS_T + LS_ED + j] = rsqrtf(ruiz_lim(rowd));
      }
      // inequality rows of the stage
      for (int h = 0; h < 2; ++h) {
        const int r = lane + 32 * h;
        if (r >= NR) break;
        float e = 1.f;
        if (cls[r] > 0.f) {
          float m;
          if (r < 12) m = Sk[LS_DU + r];
          else if (r < 20) {
            const int f = (r - 12) >> 2, t = (r - 12) & 3, b0 = 6 * f;
            m = fmaxf(Sk[LS_DU + b0 + (t < 2 ? 0 : 1)], mu * Sk[LS_DU + b0 + 2]);
          } else if (r < 38) m = Sk[LS_DU + r - 8];
          else m = Sk[LS_DX + r - 26];
          e = rsqrtf(ruiz_lim(Sk[LS_EI + r] * m));
        }
        Sk[LS_T + LS_EI + r] = e;
      }
    }
    __syncwarp();
    // ---- pass 2: apply them; then the cost scale
    float sum_p = 0.f, q_max = 0.f;
    for (int k = 0; k < N; ++k) {
      float* Sk = S0 + (size_t)k * LDL_S;
      if (lane < 30) {
        Sk[LS_DU + j] *= Sk[LS_T + LS_DU + j];
        Sk[LS_DX + j] *= Sk[LS_T + LS_DX + j];
        Sk[LS_ED + j] *= Sk[LS_T + LS_ED + j];
        const float du = Sk[LS_DU + j], dx = Sk[LS_DX + j];
        sum_p += cs * (du * du * Ru + dx * dx * Qx);
        q_max = fmaxf(q_max, cs * fmaxf(fabsf(du * Ru * ap.uref[k * VS + j]), fabsf(dx * Qx * ap.xref[(k + 1) * VS + j])));
      }
      for (int h = 0; h < 2; ++h) {
        const int r = lane + 32 * h;
        if (r < NR) Sk[LS_EI + r] *= Sk[LS_T + LS_EI + r];
      }
    }
    const float mean_p = warp_sum(sum_p) / (60.f * N);
    const float g = 1.f / ruiz_lim(fmaxf(mean_p, warp_max(q_max)));
    cs *= g;
    __syncwarp();
  }
  if (lane == 0) a.lc[slot] = cs;
}

// ------------------------------------------------------------------ solves
// Unit lower solve L w = b of one block, part p of L by columns (shared
// memory, the part's first column at Lc); the lane holds entries lane,
// lane + 32, lane + 64 (< 90) in e0, e1, e2.  Part 0 is columns 0-29, 1 is
// 30-59, 2 is 60-88.  KIN: rows 66-68 (the v rows of x_{k+1}) also have
// entries in columns 0-29, the three rows of L31 (L3, row-major 3 x 30).
template <int P, bool KIN>
__device__ __forceinline__ void fwd_part(const float* Lc, const float* L3, float& e0, float& e1, float& e2, int lane) {
#pragma unroll
  for (int j = 30 * P; j < (P == 2 ? NB - 1 : 30 * P + 30); ++j) {
    const int o = col_pos(j) - fwd_start(P) - j - 1;   // L(i, j) at o + i, i > j
    const float wj = j < 32 ? __shfl_sync(FULL, e0, j) : (j < 64 ? __shfl_sync(FULL, e1, j - 32)
                                                                 : __shfl_sync(FULL, e2, j - 64));
    // columns j < 30 have no rows 60-89 (the zero block)
    if (lane > j) e0 = fmaf(-Lc[o + lane], wj, e0);
    if (lane + 32 > j && (j >= 30 || lane + 32 < 60)) e1 = fmaf(-Lc[o + lane + 32], wj, e1);
    if (lane + 64 > j && lane < NB - 64 && j >= 30) e2 = fmaf(-Lc[o + lane + 64], wj, e2);
    if (KIN && j < 30 && lane >= 2 && lane < 5) e2 = fmaf(-L3[(lane - 2) * 30 + j], wj, e2);
  }
}
// Unit upper solve L^T v = w of one block, part p of L by rows (the part's
// first row at Lr): part 0 is rows 89-60, 1 is 59-30, 2 is 29-1.
template <int P, bool KIN>
__device__ __forceinline__ void bwd_part(const float* Lr, const float* L3, float& e0, float& e1, float& e2, int lane) {
#pragma unroll
  for (int j = (P == 0 ? NB - 1 : P == 1 ? 59 : 29); j >= (P == 0 ? 60 : P == 1 ? 30 : 1); --j) {
    const int o = row_pos(j) - bwd_start(P) - row_skip(j);   // L(j, i) at o + i, i < j (i >= 30 for j >= 60)
    const float vj = j < 32 ? __shfl_sync(FULL, e0, j) : (j < 64 ? __shfl_sync(FULL, e1, j - 32)
                                                                 : __shfl_sync(FULL, e2, j - 64));
    if (lane < j && (j < 60 || lane >= 30)) e0 = fmaf(-Lr[o + lane], vj, e0);
    if (lane + 32 < j) e1 = fmaf(-Lr[o + lane + 32], vj, e1);
    if (lane + 64 < j) e2 = fmaf(-Lr[o + lane + 64], vj, e2);
    if (KIN && j >= 66 && j < 69 && lane < 30) e0 = fmaf(-L3[(j - 66) * 30 + lane], vj, e0);
  }
}

// Staging of the factors: the iterations walk the stages forward (items
// t = 3k + p: part p of L_k by columns, with G_k in part 0) and backward
// (items t = 3N + 3(N-1-k) + p: part p of L_k by rows, with 1/D_k and G_{k+1}
// in part 0); each item is copied into one of two shared-memory buffers by
// bulk copies (completion on the buffer's mbarrier) while the previous item
// computes.  Parts of about 5.3 KB instead of whole 12.4 KB stage blocks keep
// the buffers small, so that more warps fit on an SM.  A wait gives up after
// `limit` polls: the warp then issues nothing more, waits (bounded) for the
// copies in flight and ends the agent's solve with MPC_AGENT_TIMEOUT.  `dry`
// (failure-detection test only) arms the first item's barrier with no copy
// behind it, so that its wait runs out with nothing in flight into that
// buffer.
constexpr int BUF_L = 0, BUF_G = 1336, BUF_D = 2236, BUF_L31 = 2332, BUF_FLOATS = 2432;
struct Stager {
  float* buf[2];
  uint64_t* bar;      // two mbarriers
  uint32_t phase;     // bit b: parity of buffer b's next completion
  uint32_t pending;   // bit b: a copy into buffer b not yet waited for
  bool dead;
  bool dry;
  int limit;
};
// KIN: the items carry the three rows of L31 too
// KIN: part 0 carries the three rows of L31 too
template <bool KIN>
__device__ __forceinline__ void stage_issue(Stager& sg, int b, const float* rec0, int N, int t, int lane) {
  if (sg.dead) return;
  __syncwarp();   // every lane is done with the buffer's previous contents
  if (sg.dry) {
    // armed for a copy that is never issued (nothing in flight: not pending)
    if (lane == 0) mbar_expect_tx(sg.bar + b, part_floats(0) * 4);
    sg.dry = false;
    return;
  }
  if (lane == 0) {
    const bool fwd = t < 3 * N;
    const int u = fwd ? t : t - 3 * N;
    const int k = fwd ? u / 3 : N - 1 - u / 3;
    const int p = u - 3 * (u / 3);
    const float* rec = rec0 + (size_t)k * LDL_REC;
    const uint32_t bl = part_floats(p) * 4, bg = 900 * 4, bd = 96 * 4;
    const bool g = p == 0 && (fwd ? k >= 1 : k + 1 < N);
    const bool d = p == 0 && !fwd;
    const uint32_t b3 = KIN && p == 0 ? 96 * 4 : 0;
    mbar_expect_tx(sg.bar + b, bl + (g ? bg : 0) + (d ? bd : 0) + b3);
    tma_load_1d(sg.buf[b] + BUF_L, rec + (fwd ? LDL_COL + fwd_start(p) : LDL_ROW + bwd_start(p)), bl, sg.bar + b);
    if (g) tma_load_1d(sg.buf[b] + BUF_G, fwd ? rec + LDL_G : rec + LDL_REC + LDL_G, bg, sg.bar + b);   // G_k or G_{k+1}
    if (d) tma_load_1d(sg.buf[b] + BUF_D, rec + LDL_IND, bd, sg.bar + b);
    if (b3) tma_load_1d(sg.buf[b] + BUF_L31, rec + LDL_L31, b3, sg.bar + b);
  }
  sg.pending |= 1u << b;
}
__device__ __forceinline__ void stage_wait(Stager& sg, int b) {
  if (sg.dead) return;
  if (!__all_sync(FULL, mbar_wait(sg.bar + b, (sg.phase >> b) & 1u, sg.limit))) {
    sg.dead = true;
    return;
  }
  sg.phase ^= 1u << b;
  sg.pending &= ~(1u << b);
}
__device__ __forceinline__ void stage_drain(Stager& sg) {
  for (int b = 0; b < 2; ++b)
    if (sg.pending & (1u << b)) mbar_wait(sg.bar + b, (sg.phase >> b) & 1u, sg.limit);
  sg.pending = 0;
  __syncwarp();
}

struct LdlRes { float rp, rd, sp, sd; };

// OSQP's residuals of the unscaled iterate (x = D x_s, z = z_s / E,
// y = E y_s / c): primal |A x - z|, dual |P x + q + A^T y| (inf-norms) and
// their scales max(|A x|, |z|), max(|P x|, |A^T y|, |q|).  xv: 160 floats of
// shared scratch (u_k, x_{k+1}, x_k, the dynamics multipliers of stages k, k+1).
// ks: the kinematic rows' coefficients (shared memory), or null without them.
__device__ __noinline__ LdlRes ldl_residuals(const AgentPtrs& ap, const float* ly, const float* S0, float cs, float* xv,
                                const float* ks, int lane) {
  const int N = ap.N;
  const float* md = ap.mdl;
  const float* lin = ap.lin;
  const float dt = md[M_DT], mu = md[M_MU];
  const float ic = 1.f / cs;
  LdlRes r{0.f, 0.f, 0.f, 0.f};
  float* U = xv;          // u_k
  float* X = xv + 32;     // x_{k+1}
  float* XP = xv + 64;    // x_k
  float* Y0 = xv + 96;    // dynamics multipliers of stage k
  float* Y1 = xv + 128;   // ... of stage k + 1
  for (int k = 0; k < N; ++k) {
    const float* Sk = S0 + (size_t)k * LDL_S;
    const int c30 = lane < 30 ? lane : 29;
    U[lane] = Sk[LS_DU + c30] * ap.u[k * VS + lane];
    X[lane] = Sk[LS_DX + c30] * ap.x[(k + 1) * VS + lane];
    XP[lane] = k ? Sk[LS_DX - LDL_S + c30] * ap.x[k * VS + lane] : ap.x[lane];
    Y0[lane] = Sk[LS_ED + c30] * ly[k * VS + lane] * ic;
    Y1[lane] = k + 1 < N ? Sk[LDL_S + LS_ED + c30] * ly[(k + 1) * VS + lane] * ic : 0.f;
    __syncwarp();
    const float* ei = Sk + LS_EI;
    if (lane < 30) {
      const int i = lane;
      // dynamics row i: x_{k+1} - A_k x_k - B u_k - c_k
      float ax = 0.f, bu = 0.f;
      for (int c = 0; c < 30; ++c) {
        ax = fmaf(a_entry(lin, k, i, c), XP[c], ax);
        bu = fmaf(b_entry(lin, dt, i, c), U[c], bu);
      }
      // the row's A x and z in OSQP's terms (x_0 is data: at k = 0 its term
      // belongs to z)
      const float ck = i < NC ? lin[L_STAGE + k * 64 + 32 + i] : 0.f;
      const float axr = k ? X[i] - ax - bu : X[i] - bu;
      const float zr = k ? ck : ck + ax;
      r.rp = fmaxf(r.rp, fabsf(axr - zr));
      r.sp = fmaxf(r.sp, fmaxf(fabsf(axr), fabsf(zr)));
      // stationarity of u_k and x_{k+1}
      float gu = 2.f * dt * md[M_R + i] * U[i], qu = -2.f * dt * md[M_R + i] * ap.uref[k * VS + i];
      float gx = 2.f * dt * md[M_Q + i] * X[i], qx = -2.f * dt * md[M_Q + i] * ap.xref[(k + 1) * VS + i];
      float atu = 0.f, atx = Y0[i];
      for (int c = 0; c < 30; ++c) atu = fmaf(-b_entry(lin, dt, c, i), Y0[c], atu);
      if (k + 1 < N)
        for (int c = 0; c < 30; ++c) atx = fmaf(-a_entry(lin, k + 1, c, i), Y1[c], atx);
      const float* cls = ap.rcls + k * RS;
      const float* yy = ap.y + k * RS;
      const int ru = i < 12 ? i : i + 8;
      if (cls[ru] > 0.f) atu += ei[ru] * yy[ru] * ic;
      if (i < 12 && (i % 6) < 3) {
        const int f = i / 6, c = i - 6 * f, p = 12 + 4 * f;
        for (int t = 0; t < 4; ++t)
          if (cls[p + t] > 0.f) atu = fmaf(pyr_coef(c, t, mu), ei[p + t] * yy[p + t] * ic, atu);
      }
      if (i >= 12 && cls[i + 26] > 0.f) atx += ei[i + 26] * yy[i + 26] * ic;
      if (ks) {
        // the kinematic rows (a free row's multiplier stays 0)
        const float* yk = yy + KIN_ROW;
        for (int q = 0; q < 6; ++q) atu = fmaf(ks[q * 32 + i], yk[q], atu);
        if (i >= 6 && i < 9) atx += yk[i - 6] + yk[i - 3];
        atx = fmaf(ks[6 * 32 + i], yk[6], fmaf(ks[7 * 32 + i], yk[7], atx));
      }
      r.rd = fmaxf(r.rd, fmaxf(fabsf(gu + qu + atu), fabsf(gx + qx + atx)));
      r.sd = fmaxf(r.sd, fmaxf(fmaxf(fabsf(gu), fabsf(gx)), fmaxf(fmaxf(fabsf(atu), fabsf(atx)),
                                                                   fmaxf(fabsf(qu), fabsf(qx)))));
    }
    // inequality rows
    for (int h = 0; h < 2; ++h) {
      const int rr = lane + 32 * h;
      if (rr < (ks ? KIN_ROW + KIN_NR : NR) && ap.rcls[k * RS + rr] > 0.f) {
        const float cz = rr >= KIN_ROW ? kin_value(rr - KIN_ROW, U, X, ks) : row_value(rr, U, X, mu);
        const float z = ap.w[k * RS + rr] / ei[rr];
        r.rp = fmaxf(r.rp, fabsf(cz - z));
        r.sp = fmaxf(r.sp, fmaxf(fabsf(cz), fabsf(z)));
      }
    }
    __syncwarp();
  }
  r.rp = warp_max(r.rp); r.rd = warp_max(r.rd); r.sp = warp_max(r.sp); r.sd = warp_max(r.sd);
  return r;
}

// ------------------------------------------------------------------ iterations
// Per-lane global inputs of one stage (lane i < 30: u_i, dynamics row i,
// x_i), loaded one stage ahead of their use.  Forward pass: the iterate, the
// references, the affine term, the dynamics multiplier, and the slack,
// multiplier and class of every inequality row on u_i (its box row, and for a
// force input the foot's four pyramid rows with their coefficients) and on
// x_i (the joint box).
struct FIn {
  float u, ur, x, xr, yl, ck;
  float du, dx, ed;             // scaling of u_i, x_i and dynamics row i
  float cr, zr, yr, er;         // box row of u_i (class, slack, multiplier, scaling)
  float cq, zq, yq, eq;         // joint box of x_i
  float cp[4], zp[4], yp[4], kp[4], ep[4];
  float kc, kz, ky;             // lanes 0-7: kinematic row KIN_ROW + lane (class, slack, multiplier)
};
// SC: the problem is Ruiz-scaled (otherwise every scaling factor is 1 and none is loaded)
template <bool SC, bool KIN>
__device__ __forceinline__ FIn load_fin(const AgentPtrs& ap, const float* ly, const float* S0, int k, int lane) {
  FIn f;
  f.kc = f.kz = f.ky = 0.f;
  if (KIN && lane < KIN_NR) {
    f.kc = ap.rcls[k * RS + KIN_ROW + lane];
    f.kz = ap.w[k * RS + KIN_ROW + lane];
    f.ky = ap.y[k * RS + KIN_ROW + lane];
  }
  f.u = f.ur = f.x = f.xr = f.yl = f.ck = 0.f;
  f.du = f.dx = f.ed = 1.f;
  f.cr = f.zr = f.yr = f.cq = f.zq = f.yq = 0.f;
  f.er = f.eq = 1.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) { f.cp[q] = f.zp[q] = f.yp[q] = f.kp[q] = 0.f; f.ep[q] = 1.f; }
  if (lane < 30) {
    const int i = lane;
    const float* cls = ap.rcls + k * RS;
    const float* zz = ap.w + k * RS;
    const float* yy = ap.y + k * RS;
    const float* Sk = S0 + (size_t)k * LDL_S;
    const float* ei = Sk + LS_EI;
    if (SC) {
      f.du = Sk[LS_DU + i];
      f.dx = Sk[LS_DX + i];
      f.ed = Sk[LS_ED + i];
    }
    f.u = ap.u[k * VS + i];
    f.ur = ap.uref[k * VS + i];
    f.x = ap.x[(k + 1) * VS + i];
    f.xr = ap.xref[(k + 1) * VS + i];
    f.yl = ly[k * VS + i];
    f.ck = i < NC ? ap.lin[L_STAGE + k * 64 + 32 + i] : 0.f;
    const int ru = i < 12 ? i : i + 8;
    f.cr = cls[ru]; f.zr = zz[ru]; f.yr = yy[ru];
    if (SC) f.er = ei[ru];
    if (i >= 12) { f.cq = cls[i + 26]; f.zq = zz[i + 26]; f.yq = yy[i + 26]; if (SC) f.eq = ei[i + 26]; }
    if (i < 12 && (i % 6) < 3) {
      const int ff = i / 6, c = i - 6 * ff, p = 12 + 4 * ff;
      const float mu = ap.mdl[M_MU];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        f.cp[q] = cls[p + q]; f.zp[q] = zz[p + q]; f.yp[q] = yy[p + q]; f.kp[q] = pyr_coef(c, q, mu);
        if (SC) f.ep[q] = ei[p + q];
      }
    }
  }
  return f;
}
// Backward pass: the forward vector w_k, the iterate, the dynamics
// multiplier, and slack, multiplier, class and bounds of rows lane and lane + 32.
struct BIn {
  float w0, w1, w2, u, x, yl, du, dx;
  float c0, z0, y0, lo0, hi0, e0, c1, z1, y1, lo1, hi1, e1;
};
template <bool SC, bool KIN>
__device__ __forceinline__ BIn load_bin(const AgentPtrs& ap, const float* ly, const float* lw, const float* S0,
                                        int k, int lane) {
  BIn b;
  b.du = b.dx = b.e0 = b.e1 = 1.f;
  if (SC) {
    const float* Sk = S0 + (size_t)k * LDL_S;
    const int c30 = lane < 30 ? lane : 29;
    b.du = Sk[LS_DU + c30];
    b.dx = Sk[LS_DX + c30];
    b.e0 = Sk[LS_EI + lane];
    b.e1 = lane + 32 < NR ? Sk[LS_EI + lane + 32] : 1.f;
  }
  b.w0 = lw[k * LDL_W + lane];
  b.w1 = lw[k * LDL_W + lane + 32];
  b.w2 = lane < NB - 64 ? lw[k * LDL_W + lane + 64] : 0.f;
  b.u = ap.u[k * VS + lane];
  b.x = ap.x[(k + 1) * VS + lane];
  b.yl = ly[k * VS + lane];
  const int r0 = lane, r1 = lane + 32;
  b.c0 = ap.rcls[k * RS + r0]; b.z0 = ap.w[k * RS + r0]; b.y0 = ap.y[k * RS + r0];
  b.lo0 = ap.rlo[k * RS + r0]; b.hi0 = ap.rhi[k * RS + r0];
  if (r1 < (KIN ? KIN_ROW + KIN_NR : NR)) {
    b.c1 = ap.rcls[k * RS + r1]; b.z1 = ap.w[k * RS + r1]; b.y1 = ap.y[k * RS + r1];
    b.lo1 = ap.rlo[k * RS + r1]; b.hi1 = ap.rhi[k * RS + r1];
  } else {
    b.c1 = b.z1 = b.y1 = b.lo1 = b.hi1 = 0.f;
  }
  return b;
}

constexpr int W_ADMM = 2 * BUF_FLOATS + 96 + 160 + 32 + 4;   // shared floats of the one warp of a block
constexpr int W_ADMM_KIN = W_ADMM + KIN_SM + 32;               // ... with the kinematic rows
// KIN: with the kinematic rows (never with SC: the two are not combined)
// (ten resident blocks per SM: the register allocation for them spills least)
template <bool SC, bool KIN>
__global__ void __launch_bounds__(32, 10) mpc_k_ldl_admm(Arena a, Batch b, SolverParams prm) {
  static_assert(!(SC && KIN), "the kinematic rows run unscaled");
  const int lane = threadIdx.x;
  const int row = blockIdx.x;
  if (!live_row(a, b, row)) return;
  const int slot = b.ids[row];
  const AgentPtrs ap = agent_ptrs(a, slot);
  if (ap.st[T_STATUS] == MPC_AGENT_NAN_) return;
  extern __shared__ __align__(16) float asm_[];
  float* rb = asm_ + 2 * BUF_FLOATS;    // the stage's 90-vector, by block index
  float* xv = rb + 96;                  // scratch: the unscaled stage vectors (updates, residuals)
  float* cv = xv + 160;                 // coupling vector: x part of w_{k-1} / multiplier part of v_{k+1}
  Stager sg;
  sg.buf[0] = asm_;
  sg.buf[1] = asm_ + BUF_FLOATS;
  sg.bar = reinterpret_cast<uint64_t*>(cv + 32);
  sg.phase = 0u; sg.pending = 0u; sg.dead = false;
  sg.dry = slot == prm.wait_test_slot;
  float* ks = asm_ + W_ADMM;            // KIN: the kinematic rows' coefficients
  float* kt = ks + KIN_SM;              // KIN: rho_r z_r - y_r of the stage's kinematic rows
  sg.limit = prm.spin_limit > 0 ? prm.spin_limit : kSpinLimit;
  if (lane == 0) {
    mbar_init(sg.bar, 1);
    mbar_init(sg.bar + 1, 1);
    fence_mbar_init();
  }
  __syncwarp();
  const float* md = ap.mdl;
  const float* lin = ap.lin;
  const int N = ap.N;
  const float dt = md[M_DT], mu = md[M_MU];
  const float sigma = prm.sigma, alpha = prm.alpha;
  if (KIN) kin_fill(ks, md, lane);
  const float rho = *ap.rho, rho_eq = 1e3f * rho;
  const float* rec0 = a.lL + (size_t)slot * a.maxN * LDL_REC;
  float* lw = a.lw + (size_t)slot * a.maxN * LDL_W;
  float* ly = a.ly + (size_t)slot * a.maxN * VS;
  const int i = lane;   // lanes 0-29: u_i, dynamics row i, x_i of each stage
  const float Ru = lane < 30 ? 2.f * dt * md[M_R + i] : 0.f;
  const float Qx = lane < 30 ? 2.f * dt * md[M_Q + i] : 0.f;
  // dynamics rows of stage 0: x_1 - B u_0 = c_0 + A_0 x0
  float a0x0 = 0.f;
  if (lane < 30)
    for (int c = 0; c < 30; ++c) a0x0 = fmaf(a_entry(lin, 0, i, c), ap.inp[I_X0 + c], a0x0);
  for (int k = 0; k < N; ++k) ly[k * VS + lane] = 0.f;
  // the iterations run on the Ruiz-scaled problem (all ones without it): the
  // f_init start scaled in, x_s = D^-1 x, z_s = E z (y = 0)
  const float* S0 = a.lS + (size_t)slot * a.maxN * LDL_S;
  const float cs = SC ? a.lc[slot] : 1.f;
  for (int k = 0; SC && k < N; ++k) {
    const float* Sk = S0 + (size_t)k * LDL_S;
    if (lane < 30) {
      ap.u[k * VS + lane] /= Sk[LS_DU + lane];
      ap.x[(k + 1) * VS + lane] /= Sk[LS_DX + lane];
    }
    for (int h = 0; h < 2; ++h) {
      const int r = lane + 32 * h;
      if (r < NR && ap.rcls[k * RS + r] > 0.f) ap.w[k * RS + r] *= Sk[LS_EI + r];
    }
  }
  __syncwarp();
  const bool fixed = prm.fixed_iters > 0;
  const int max_it = fixed ? prm.fixed_iters : prm.max_iter;
  const int every = prm.check_every > 0 ? prm.check_every : 10;
  int status = MPC_AGENT_MAX_ITER_, it = 0;
  LdlRes res{0.f, 0.f, 0.f, 0.f};
  const int T = 6 * N;                 // staged items per iteration (three parts per stage and pass)
  stage_issue<KIN>(sg, 0, rec0, N, 0, lane);
  for (it = 1; it <= max_it && !sg.dead; ++it) {
    const bool last = it == max_it;
    // ---- forward pass: b_k (+ G_k w_{k-1,x}), w_k = L_k^-1 b_k; the
    // stage's global inputs are loaded one stage ahead
    FIn fin = load_fin<SC, KIN>(ap, ly, S0, 0, lane);
    for (int k = 0; k < N; ++k) {
      const int t = 3 * k, bcur = t & 1;
      stage_issue<KIN>(sg, bcur ^ 1, rec0, N, t + 1, lane);
      const FIn f = fin;
      if (k + 1 < N) fin = load_fin<SC, KIN>(ap, ly, S0, k + 1, lane);
      float bu = 0.f, bl = 0.f, bx = 0.f;
      if (lane < 30) {
        // sigma x_s - q_s + C_s^T (rho z_s - y_s), q_s = c D q, C_s = E C D
        bu = sigma * f.u + cs * f.du * Ru * f.ur;
        if (f.cr > 0.f) bu += f.du * f.er * (rho * f.cr * f.zr - f.yr);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (f.cp[q] > 0.f) bu = fmaf(f.kp[q] * f.du * f.ep[q], rho * f.cp[q] * f.zp[q] - f.yp[q], bu);
        bl = f.ed * (f.ck + (k ? 0.f : a0x0)) - f.yl / rho_eq;
        bx = sigma * f.x + cs * f.dx * Qx * f.xr;
        if (f.cq > 0.f) bx += f.dx * f.eq * (rho * f.cq * f.zq - f.yq);
      }
      if (KIN) {
        // C^T (rho z - y) of the kinematic rows
        if (lane < KIN_NR) kt[lane] = rho * f.kc * f.kz - f.ky;
        __syncwarp();
        if (lane < 30) {
#pragma unroll
          for (int q = 0; q < 6; ++q) bu = fmaf(ks[q * 32 + i], kt[q], bu);
          if (i >= 6 && i < 9) bx += kt[i - 6] + kt[i - 3];
          bx = fmaf(ks[6 * 32 + i], kt[6], fmaf(ks[7 * 32 + i], kt[7], bx));
        }
      }
      stage_wait(sg, bcur);
      if (sg.dead) break;
      const float* buf = sg.buf[bcur];
      if (lane < 30) {
        if (k) {
          const float* g = buf + BUF_G + i * 30;
          for (int c = 0; c < 30; ++c) bl = fmaf(g[c], cv[c], bl);
        }
        rb[i] = bu;
        rb[30 + i] = bl;
        rb[60 + i] = bx;
      }
      __syncwarp();
      float e0 = rb[lane], e1 = rb[lane + 32], e2 = lane < NB - 64 ? rb[lane + 64] : 0.f;
      fwd_part<0, KIN>(buf + BUF_L, buf + BUF_L31, e0, e1, e2, lane);
      // parts 1 and 2 (the last stage's part 2 issues the backward pass's first item)
      stage_issue<KIN>(sg, bcur, rec0, N, t + 2, lane);
      stage_wait(sg, bcur ^ 1);
      if (sg.dead) break;
      fwd_part<1, KIN>(sg.buf[bcur ^ 1] + BUF_L, nullptr, e0, e1, e2, lane);
      stage_issue<KIN>(sg, bcur ^ 1, rec0, N, t + 3, lane);
      stage_wait(sg, bcur);
      if (sg.dead) break;
      fwd_part<2, KIN>(sg.buf[bcur] + BUF_L, nullptr, e0, e1, e2, lane);
      lw[k * LDL_W + lane] = e0;
      lw[k * LDL_W + lane + 32] = e1;
      if (lane < NB - 64) lw[k * LDL_W + lane + 64] = e2;
      __syncwarp();
      // x part of w_k for the next stage's coupling (entries 60-89)
      if (lane >= 28) cv[lane - 28] = e1;
      if (lane < NB - 64) cv[lane + 4] = e2;
      __syncwarp();
    }
    if (sg.dead) break;
    // ---- backward pass: v_k = L_k^-T (D_k^-1 w_k + G_{k+1}^T v_{k+1,mult}),
    // then the stage's update; inputs one stage ahead
    BIn bin = load_bin<SC, KIN>(ap, ly, lw, S0, N - 1, lane);
    for (int k = N - 1; k >= 0; --k) {
      const int t = 3 * N + 3 * (N - 1 - k), bcur = t & 1;
      stage_issue<KIN>(sg, bcur ^ 1, rec0, N, t + 1, lane);
      const BIn q = bin;
      if (k >= 1) bin = load_bin<SC, KIN>(ap, ly, lw, S0, k - 1, lane);
      stage_wait(sg, bcur);
      if (sg.dead) break;
      const float* buf = sg.buf[bcur];
      const float* iD = buf + BUF_D;
      rb[lane] = q.w0 * iD[lane];
      rb[lane + 32] = q.w1 * iD[lane + 32];
      if (lane < NB - 64) rb[lane + 64] = q.w2 * iD[lane + 64];
      __syncwarp();
      if (k + 1 < N && lane < 30) {
        const float* g = buf + BUF_G;
        float s = 0.f;
        for (int r = 0; r < 30; ++r) s = fmaf(g[r * 30 + i], cv[r], s);
        rb[60 + i] += s;
      }
      __syncwarp();
      float e0 = rb[lane], e1 = rb[lane + 32], e2 = lane < NB - 64 ? rb[lane + 64] : 0.f;
      bwd_part<0, KIN>(buf + BUF_L, buf + BUF_L31, e0, e1, e2, lane);
      // parts 1 and 2; the next item: this iteration's next stage, or the
      // next iteration's first
      stage_issue<KIN>(sg, bcur, rec0, N, t + 2, lane);
      stage_wait(sg, bcur ^ 1);
      if (sg.dead) break;
      bwd_part<1, KIN>(sg.buf[bcur ^ 1] + BUF_L, nullptr, e0, e1, e2, lane);
      if (t + 3 < T) stage_issue<KIN>(sg, bcur ^ 1, rec0, N, t + 3, lane);
      else if (!last) stage_issue<KIN>(sg, bcur ^ 1, rec0, N, 0, lane);
      stage_wait(sg, bcur);
      if (sg.dead) break;
      bwd_part<2, KIN>(sg.buf[bcur] + BUF_L, nullptr, e0, e1, e2, lane);
      __syncwarp();
      rb[lane] = e0;
      rb[lane + 32] = e1;
      if (lane < NB - 64) rb[lane + 64] = e2;
      __syncwarp();
      // rb = (x~ of u_k, nu of the dynamics rows, x~ of x_{k+1})
      if (lane < 30) {
        const float nu = rb[30 + i];
        cv[i] = nu;
        ap.u[k * VS + i] = alpha * rb[i] + (1.f - alpha) * q.u;
        ap.x[(k + 1) * VS + i] = alpha * rb[60 + i] + (1.f - alpha) * q.x;
        // dynamics rows (z = l = u always): zr - z = alpha (nu - y) / rho_eq
        ly[k * VS + i] = (1.f - alpha) * q.yl + alpha * nu;
      }
      // the rows' z~ = E C D x~: the stage's x~ times D
      xv[lane] = lane < 30 ? q.du * rb[lane] : 0.f;
      xv[32 + lane] = lane < 30 ? q.dx * rb[60 + lane] : 0.f;
      __syncwarp();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int rr = lane + 32 * h;
        const float cl = h ? q.c1 : q.c0;
        if (rr < (KIN ? KIN_ROW + KIN_NR : NR) && cl > 0.f) {
          const float rr_rho = rho * cl;
          const float er = h ? q.e1 : q.e0;
          const float zt = (KIN && rr >= KIN_ROW) ? kin_value(rr - KIN_ROW, xv, xv + 32, ks)
                                                  : er * row_value(rr, xv, xv + 32, mu);
          const float zo = h ? q.z1 : q.z0, yo = h ? q.y1 : q.y0;
          const float zh = alpha * zt + (1.f - alpha) * zo;
          const float zn = fminf(fmaxf(zh + yo / rr_rho, er * (h ? q.lo1 : q.lo0)), er * (h ? q.hi1 : q.hi0));
          ap.y[k * RS + rr] = yo + rr_rho * (zh - zn);
          ap.w[k * RS + rr] = zn;
        }
      }
      __syncwarp();
    }
    if (sg.dead) break;
    const bool check = !fixed && (it % every == 0 || last);
    if (check || (fixed && last)) {
      res = ldl_residuals(ap, ly, S0, cs, xv, KIN ? ks : nullptr, lane);
      if (!(isfinite(res.rp) && isfinite(res.rd))) { status = MPC_AGENT_NAN_; break; }
      if (check && res.rp <= prm.eps_abs + prm.eps_rel * res.sp && res.rd <= prm.eps_abs + prm.eps_rel * res.sd) {
        status = MPC_AGENT_INACCURATE_;   // ADMM's stopping test, no polish: not certified
        break;
      }
    }
  }
  if (it > max_it) it = max_it;
  if (sg.dead) {
    status = MPC_AGENT_TIMEOUT_;
    if (lane == 0) atomicAdd(a.fault + F_WAIT_TIMEOUTS, 1);
  }
  // copies issued for an iteration that did not run (a stop after a check)
  stage_drain(sg);
  // the iterate scaled back: x = D x_s, z = z_s / E, y = E y_s / c
  for (int k = 0; SC && k < N; ++k) {
    const float* Sk = S0 + (size_t)k * LDL_S;
    if (lane < 30) {
      ap.u[k * VS + lane] *= Sk[LS_DU + lane];
      ap.x[(k + 1) * VS + lane] *= Sk[LS_DX + lane];
      ly[k * VS + lane] *= Sk[LS_ED + lane] / cs;
    }
    for (int h = 0; h < 2; ++h) {
      const int r = lane + 32 * h;
      if (r < NR && ap.rcls[k * RS + r] > 0.f) {
        ap.w[k * RS + r] /= Sk[LS_EI + r];
        ap.y[k * RS + r] *= Sk[LS_EI + r] / cs;
      }
    }
  }
  __syncwarp();
  // a non-finite iterate leaves no torques
  bool bad = false;
  for (int k = 0; k <= N; ++k) bad |= lane < 30 && !isfinite(ap.x[k * VS + lane]);
  for (int k = 0; k < N; ++k) bad |= lane < 30 && !isfinite(ap.u[k * VS + lane]);
  if (warp_or(bad) && status != MPC_AGENT_TIMEOUT_) status = MPC_AGENT_NAN_;
  if (lane == 0) {
    ap.st[T_STATUS] = status;
    ap.st[T_ITERS] = it;
    ap.st[T_REFAC] = 0;
    ap.st[T_POLISHED] = 0;
    ap.st[T_ATTEMPTS] = 0;
    ap.out[O_PRIM] = res.rp;
    ap.out[O_DUAL] = res.rd;
    ap.out[O_PRIM_N] = 0.f;
    ap.out[O_DUAL_N] = 0.f;
    *ap.warm = 0;   // every solve of this form starts from f_init
  }
}

}  // namespace

template <typename K>
static cudaError_t set_smem(K kern, int floats, bool carveout) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(floats * sizeof(float)));
  if (e == cudaSuccess && carveout)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  return e;
}

cudaError_t launch_ldl(const Arena& a, const Batch& b, const SolverParams& prm, cudaStream_t st, int* launches) {
  static int configured = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured != dev) {
    // the iteration kernel's one-warp blocks hold about 21 KB of shared
    // memory: it asks for the largest shared-memory carveout, so that ten fit
    // on an SM
    cudaError_t e = set_smem(mpc_k_ldl_factor<false>, F_FLOATS, false);
    if (e == cudaSuccess) e = set_smem(mpc_k_ldl_factor<true>, F_FLOATS + F_KIN, false);
    if (e == cudaSuccess) e = set_smem(mpc_k_ldl_admm<false, false>, W_ADMM, true);
    if (e == cudaSuccess) e = set_smem(mpc_k_ldl_admm<true, false>, W_ADMM, true);
    if (e == cudaSuccess) e = set_smem(mpc_k_ldl_admm<false, true>, W_ADMM_KIN, true);
    if (e != cudaSuccess) return e;
    configured = dev;
  }
  if (b.n <= 0) return cudaSuccess;
  if (prm.kin && prm.ruiz > 0) return cudaErrorInvalidValue;
  mpc_k_ldl_ruiz<<<b.n, 32, 2 * 30 * 31 * sizeof(float), st>>>(a, b, prm);
  if (prm.kin) {
    mpc_k_ldl_kin<<<b.n, 32, 0, st>>>(a, b, prm);
    mpc_k_ldl_factor<true><<<b.n, 32, (F_FLOATS + F_KIN) * sizeof(float), st>>>(a, b, prm);
    mpc_k_ldl_admm<false, true><<<b.n, 32, W_ADMM_KIN * sizeof(float), st>>>(a, b, prm);
  } else {
    mpc_k_ldl_factor<false><<<b.n, 32, F_FLOATS * sizeof(float), st>>>(a, b, prm);
    if (prm.ruiz > 0) mpc_k_ldl_admm<true, false><<<b.n, 32, W_ADMM * sizeof(float), st>>>(a, b, prm);
    else mpc_k_ldl_admm<false, false><<<b.n, 32, W_ADMM * sizeof(float), st>>>(a, b, prm);
  }
  if (launches) *launches += prm.kin ? 4 : 3;
  return cudaGetLastError();
}

}  // namespace mpc
