// Kernels of the batched MPC solver (sm_103a).  One warp per agent.
// Included by one translation unit per kernel variant (solver_v*.cu).
//
// Two launch forms of the same device steps:
//   plain : mpc_k_setup -> mpc_k_factor -> mpc_k_admm -> mpc_k_polish -> mpc_k_torque,
//           one launch per step, all intermediates in the global arenas;
//   fused : mpc_k_fused runs every step of an agent in one warp, keeping the
//           constant stage matrices in shared memory between steps.
// Both run the same sequence: ADMM with residual checks, rho updates and an
// early polish attempt once the residuals are within early_polish x the tolerance;
// a final polish after ADMM if none was accepted; the torque map.
#pragma once
#include "solver_dev.cuh"
#include "solver.h"

namespace mpc {
namespace {   // everything but launch_variant is private to the variant's translation unit

// ============================================================ small helpers
// diagonal of the x_k block of the ADMM KKT matrix (k >= 1): 2 dt Q + sigma
// + rho on the joint-box row of stage k-1
__device__ __forceinline__ float qt_x(const AgentPtrs& ap, int k, int i, float rho, float sigma) {
  const float* md = ap.mdl;
  float v = 2.f * md[M_DT] * md[M_Q + i] + sigma;
  if (i >= 12 && i < 30) v += rho * ap.rcls[(k - 1) * RS + i + 26];
  return v;
}

// A_k x for the coupled block, lane row: dense A_base (column-major) plus
// the contact-dependent block dA_k (rows 9-11 x columns 12-21)
__device__ __forceinline__ float ak_mv(const float* Ab, const float* dA, const float* v, int lane) {
  float r = cm_mv_s(Ab, v, lane);
  if (lane >= 9 && lane < 12) {
    const float* row = dA + (lane - 9) * 10;
#pragma unroll
    for (int c = 0; c < 10; ++c) r = fmaf(row[c], v[12 + c], r);
  }
  return r;
}

// compact A values of stage k: the leg-joint columns take dA_k
__device__ __forceinline__ void set_stage_A(float* sm, const float* dA, int lane) {
  if (lane >= 12 && lane < NC) {
    float* av = sm + S_AV + lane * 6;
    av[0] = 1.f;   // identity entry (the polish may zero it for a stage)
#pragma unroll
    for (int t = 1; t < 4; ++t) av[t] = dA[(t - 1) * 10 + (lane - 12)];
  }
  __syncwarp();
}

__device__ __forceinline__ void copy_n(float* dst, const float* src, int n4, int lane) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
  float4* d4 = reinterpret_cast<float4*>(dst);
  for (int t = lane; t < n4; t += 32) d4[t] = s4[t];
}
__device__ __forceinline__ void copy_blk(float* dst, const float* src, int lane) { copy_n(dst, src, BLK / 4, lane); }
// ============================================================ setup (A1, A2)
// Contact schedule, references, bounds (f_param), analytic linearisation
// about x0 and u_ref (f_KKT Jacobians), warm or cold start (f_init).
// Returns false (agent marked NaN) when an input is not finite.
__device__ __noinline__ bool setup_agent(const AgentPtrs& ap, float* sm, int lane, const SolverParams& prm) {
  const int N = ap.N;
  const float* md = ap.mdl;
  float* vec = sm + S_VEC;
  float* xbar = vec + V_X * 64;
  int* flags = reinterpret_cast<int*>(vec + V_FLAGS * 64);

  const float xi = lane < 30 ? ap.inp[I_X0 + lane] : 0.f;
  bool bad = lane < 30 && !isfinite(xi);
  if (lane < 18) bad |= !isfinite(ap.inp[I_QD + lane]);
  if (lane < 5) bad |= !isfinite(ap.inp[I_CMD + lane]);
  if (warp_or(bad)) return false;
  xbar[lane] = xi;

  // contact schedule (double precision, no contraction): lane k -> stage k
  if (lane < N) {
    const double step = __ddiv_rn(ap.sch[S_DT], ap.sch[S_PERIOD]);
    double ph = __dadd_rn((double)ap.inp[I_PHASE], __dmul_rn((double)lane, step));
    ph = __dsub_rn(ph, floor(ph));
    int f = 0;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      double s = __dadd_rn(ph, ap.sch[S_OFF + i]);
      s = __dsub_rn(s, floor(s));
      if (s < ap.sch[S_DUTY + i]) f |= 1 << i;
    }
    flags[lane] = f;
  }
  __syncwarp();

  const float fzmax = md[M_FZMAX], qdmax = md[M_QDMAX], qlim = md[M_QLIM];
  // stage bounds: per stage, lane r writes rows r and r + 32 (coalesced)
  for (int k = 0; k < N; ++k) {
    const int f = flags[k];
    float* lo = ap.rlo + k * RS;
    float* hi = ap.rhi + k * RS;
    float* cl = ap.rcls + k * RS;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = lane + 32 * h;
      if (r >= NR) break;
      float l, u, c;
      if (r < 12) {                                 // foot wrench boxes
        const int i = r / 6, cc = r - 6 * i;
        if ((f >> i) & 1) {
          const bool z = (cc == 2);
          l = z ? 0.f : -INFINITY; u = z ? fzmax : INFINITY; c = z ? 1.f : 0.f;
        } else {
          l = 0.f; u = 0.f; c = 1000.f;
        }
      } else if (r < 20) {                          // friction pyramids
        const bool stance = (f >> ((r - 12) / 4)) & 1;
        l = -INFINITY; u = stance ? 0.f : INFINITY; c = stance ? 1.f : 0.f;
      } else if (r < 38) {                          // joint rates
        l = -qdmax; u = qdmax; c = 1.f;
      } else {                                      // joint positions (on x_{k+1})
        l = -qlim; u = qlim; c = 1.f;
      }
      lo[r] = l;
      hi[r] = u;
      cl[r] = c;
    }
  }

  // references: desired trajectory (Eqs. des_traj_1..5) and force split
  const float dt = md[M_DT];
  const float ch = ap.inp[I_CMD], cvx = ap.inp[I_CMD + 1], cvy = ap.inp[I_CMD + 2], cwz = ap.inp[I_CMD + 3];
  // yaw_k and its cosine and sine for every stage k = 0..N at once (lane k,
  // lane 0 also k = 32)
  float* vyaw = vec + V_T * 64;
  float* vcos = vec + V_G * 64;
  float* vsin = vec + V_D * 64;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int k = lane + 32 * h;
    if (k <= N) {
      const float yaw = xbar[5] + ((float)k * dt) * cwz;
      float sy, cy;
      sincosf(yaw, &sy, &cy);
      vyaw[k] = yaw;
      vcos[k] = cy;
      vsin[k] = sy;
    }
  }
  __syncwarp();
  const float qn = (lane >= 12 && lane < 30) ? md[M_QNOM + lane - 12] : 0.f;
  for (int k = 0; k <= N; ++k) {
    float v = 0.f;
    if (lane == 2) v = ch;
    else if (lane == 5) v = vyaw[k];
    else if (lane == 6) v = vcos[k] * cvx - vsin[k] * cvy;
    else if (lane == 7) v = vsin[k] * cvx + vcos[k] * cvy;
    else if (lane == 11) v = cwz;
    else if (lane >= 12 && lane < 30) v = qn;
    ap.xref[k * VS + lane] = v;
  }
  __syncwarp();
  const float weight = md[M_MASS] * GRAV;
  for (int k = 0; k < N; ++k) {
    const int f = flags[k];
    const float share = weight / (float)__popc(f);
    float v = 0.f;
    if (lane == 2 && (f & 1)) v = share;
    if (lane == 8 && (f & 2)) v = share;
    ap.uref[k * VS + lane] = v;
  }

  // ---- linearisation about (x0, u_ref_k): analytic Jacobians, forward Euler
  const float roll = xbar[3], pitch = xbar[4], yaw0 = xbar[5];
  const float cr = cosf(roll), sr = sinf(roll), cp = cosf(pitch), sp = sinf(pitch);
  const float cy = cosf(yaw0), sy = sinf(yaw0);
  const M3 R = {{cy * cp, cy * sp * sr - sy * cr, cy * sp * cr + sy * sr,
                 sy * cp, sy * sp * sr + cy * cr, sy * sp * cr - cy * sr,
                 -sp, cp * sr, cp * cr}};
  const float I0 = md[M_INERTIA], I1 = md[M_INERTIA + 1], I2 = md[M_INERTIA + 2];
  M3 Iw, Iwi;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Iw.m[3 * r + c] = m3(R, r, 0) * I0 * m3(R, c, 0) + m3(R, r, 1) * I1 * m3(R, c, 1) + m3(R, r, 2) * I2 * m3(R, c, 2);
      Iwi.m[3 * r + c] = m3(R, r, 0) / I0 * m3(R, c, 0) + m3(R, r, 1) / I1 * m3(R, c, 1) + m3(R, r, 2) / I2 * m3(R, c, 2);
    }
  const float w0 = xbar[9], w1 = xbar[10], w2 = xbar[11];
  const float ic = 1.f / cp, tp = sp * ic;
  const M3 Einv = {{cy * ic, sy * ic, 0.f, -sy, cy, 0.f, cy * tp, sy * tp, 1.f}};
  const float ea = cy * w0 + sy * w1, eb = -sy * w0 + cy * w1;
  // d(E^-1 w)/dTheta, columns (roll, pitch, yaw)
  const M3 dE = {{0.f, ea * sp * ic * ic, eb * ic, 0.f, 0.f, -ea, 0.f, ea * ic * ic, tp * eb}};
  const float Iww0 = Iw.m[0] * w0 + Iw.m[1] * w1 + Iw.m[2] * w2;
  const float Iww1 = Iw.m[3] * w0 + Iw.m[4] * w1 + Iw.m[5] * w2;
  const float Iww2 = Iw.m[6] * w0 + Iw.m[7] * w1 + Iw.m[8] * w2;
  // gyroscopic Jacobian: I_w^-1 (-[w]x I_w + [I_w w]x)
  M3 sw = skew3(w0, w1, w2), sIw = skew3(Iww0, Iww1, Iww2);
  M3 swI = mul3(sw, Iw);
  M3 gin;
#pragma unroll
  for (int t = 0; t < 9; ++t) gin.m[t] = sIw.m[t] - swI.m[t];
  const M3 gyro = mul3(Iwi, gin);
  // foot levers r_i(q) = lever_i + J_r,i (q_leg,i - q_nom,leg,i)
  float rl[2][3];
#pragma unroll
  for (int f = 0; f < 2; ++f)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float v = md[M_LEVER + 3 * f + c];
      for (int j = 0; j < 5; ++j)
        v += md[M_JLEG + 30 * f + 5 * c + j] * (xbar[12 + 5 * f + j] - md[M_QNOM + 5 * f + j]);
      rl[f][c] = v;
    }
  const float invm = md[M_INVM];

  // A_base = I + dt f_x (without the contact-dependent leg coupling) and
  // B = dt f_u, dense column-major: lane j fills column j
  float* Ab = sm + S_AB;
  float* Bm = sm + S_B;
  if (lane < NC) {
    const int j = lane;
    for (int i = 0; i < NC; ++i) {
      float a = (i == j) ? 1.f : 0.f;
      if (i < 3 && j == i + 6) a += dt;
      if (i >= 3 && i < 6 && j >= 3 && j < 6) a += dt * m3(dE, i - 3, j - 3);
      if (i >= 3 && i < 6 && j >= 9 && j < 12) a += dt * m3(Einv, i - 3, j - 9);
      if (i >= 9 && i < 12 && j >= 9 && j < 12) a += dt * m3(gyro, i - 9, j - 9);
      Ab[j * LDD + i] = a;
      float b = 0.f;
      if (i >= 6 && i < 9 && (j == i - 6 || j == i)) b = dt * invm;
      if (i >= 9 && i < 12 && j < 12) {
        const int f = j / 6, c = j - 6 * f, r = i - 9;
        if (c < 3) {
          // I_w^-1 [r_f]x, column c
          const M3 S = skew3(rl[f][0], rl[f][1], rl[f][2]);
          b = dt * (m3(Iwi, r, 0) * m3(S, 0, c) + m3(Iwi, r, 1) * m3(S, 1, c) + m3(Iwi, r, 2) * m3(S, 2, c));
        } else {
          b = dt * m3(Iwi, r, c - 3);
        }
      }
      if (i >= 12 && j == i) b = dt;
      Bm[j * LDD + i] = b;
    }
  }
  __syncwarp();
  // compact columns of A_base and B
  if (lane < NC) {
    const int j = lane;
    for (int t = 0; t < 6; ++t) {
      sm[S_AV + j * 6 + t] = t < acnt(j) ? Ab[j * LDD + arow(j, t)] : 0.f;
      sm[S_BV + j * 6 + t] = t < bcnt(j) ? Bm[j * LDD + brow(j, t)] : 0.f;
    }
  }
  __syncwarp();
  // stash for the separate-kernel form and the factor's reloads
  copy_n(ap.lin + L_ABASE, Ab, 2 * MB / 4, lane);
  copy_n(ap.lin + L_AV, sm + S_AV, 272 / 4, lane);

  // per stage: dA_k = dt dw/dq_leg (depends on the stance forces of u_ref_k)
  // and c_k = x0 + dt f(x0, u_ref_k) - A_k x0 - B u_ref_k
  // (the stance forces are those of u_ref_k, recomputed from the contact
  // flags; dA_k is staged in shared memory for the A_k x0 product, so neither
  // is read back from global memory right after it was written)
  // stage-independent parts, once: the dA_k entry of lane (r, col) per unit
  // stance force, A_base x0, and f(x0, u) = f0c + f0L F_L + f0R F_R
  float* vdA = vec + V_T * 64;
  float gdA = 0.f;
  int fsel = 0;
  if (lane < 30) {
    const int r = lane / 10, col = lane - 10 * r, f = col / 5, j = col - 5 * f;
    const float jr0 = md[M_JLEG + 30 * f + 0 * 5 + j], jr1 = md[M_JLEG + 30 * f + 1 * 5 + j];
    gdA = dt * (m3(Iwi, r, 0) * jr1 - m3(Iwi, r, 1) * jr0);
    fsel = f;
  }
  float Abx = 0.f, f0c = 0.f, f0L = 0.f, f0R = 0.f, BuL = 0.f, BuR = 0.f;
  if (lane < NC) {
    const int i = lane;
    Abx = cm_mv(Ab, xbar, lane);
    if (i < 3) f0c = xbar[6 + i];
    else if (i < 6) f0c = m3(Einv, i - 3, 0) * w0 + m3(Einv, i - 3, 1) * w1 + m3(Einv, i - 3, 2) * w2;
    else if (i == 8) { f0c = -GRAV; f0L = invm; f0R = invm; }
    else if (i >= 9 && i < 12) {
      // I_w^-1 (r_L x f_L + r_R x f_R - w x I_w w) with f = (0, 0, F)
      const int r = i - 9;
      const float g0 = w1 * Iww2 - w2 * Iww1, g1 = w2 * Iww0 - w0 * Iww2, g2 = w0 * Iww1 - w1 * Iww0;
      f0c = -(m3(Iwi, r, 0) * g0 + m3(Iwi, r, 1) * g1 + m3(Iwi, r, 2) * g2);
      f0L = m3(Iwi, r, 0) * rl[0][1] - m3(Iwi, r, 1) * rl[0][0];
      f0R = m3(Iwi, r, 0) * rl[1][1] - m3(Iwi, r, 1) * rl[1][0];
    }
    BuL = Bm[2 * LDD + i];
    BuR = Bm[8 * LDD + i];
  }
  for (int k = 0; k < N; ++k) {
    float* st = ap.lin + L_STAGE + k * 64;
    const int fk = flags[k];
    const float share = weight / (float)__popc(fk);
    const float FL = (fk & 1) ? share : 0.f, FR = (fk & 2) ? share : 0.f;
    if (lane < 30) {
      const float v = (fsel ? FR : FL) * gdA;
      st[lane] = v;
      vdA[lane] = v;
    }
    __syncwarp();
    if (lane < NC) {
      const int i = lane;
      float Ax = Abx;
      if (i >= 9 && i < 12) {
        const float* row = vdA + (i - 9) * 10;
#pragma unroll
        for (int c = 0; c < 10; ++c) Ax = fmaf(row[c], xbar[12 + c], Ax);
      }
      const float f0 = f0c + f0L * FL + f0R * FR;
      st[32 + i] = xbar[i] + dt * f0 - Ax - (BuL * FL + BuR * FR);
    }
    __syncwarp();
  }

  // warm or cold start (f_init: the current pose repeated over the horizon,
  // everything else zero; duals zero)
  const bool warm = prm.warm_start && (*ap.warm == N);
  if (lane == 0) ap.st[T_WARM] = warm ? 1 : 0;
  if (!warm) {
    for (int k = 0; k <= N; ++k) {
      float v = 0.f;
      if (lane < 6) v = xbar[lane];
      else if (lane >= 12 && lane < 30) v = md[M_QNOM + lane - 12];
      ap.x[k * VS + lane] = v;
    }
    for (int k = 0; k < N; ++k) ap.u[k * VS + lane] = 0.f;
    __syncwarp();
    for (int k = 0; k < N; ++k) {
      for (int r = lane; r < NR; r += 32) {
        const float v = (r >= 38) ? md[M_QNOM + r - 38] : 0.f;
        ap.w[k * RS + r] = fminf(fmaxf(v, ap.rlo[k * RS + r]), ap.rhi[k * RS + r]);
        ap.y[k * RS + r] = 0.f;
      }
    }
    if (lane == 0) *ap.rho = prm.rho0;
  }
  ap.x[lane] = xbar[lane];
  __syncwarp();
  return true;
}

// load the constant stage matrices (dense A_base, B and their compact
// columns) of the agent into smem
__device__ __forceinline__ void load_lin(const AgentPtrs& ap, float* sm, int lane) {
  copy_n(sm + S_AB, ap.lin + L_ABASE, 2 * MB / 4, lane);
  copy_n(sm + S_AV, ap.lin + L_AV, 272 / 4, lane);
  __syncwarp();
}

// ============================================================ factor (A3, A4)
// Backward Riccati recursion on the stage blocks of the KKT system of the
// ADMM x-update (P + sigma I + rho C^T C, dynamics as exact constraints).
// Per stage, lane j forms column j of P A_k and P B from the compact columns
// (at most 6 terms each), then column j of
//   H_uu = R_t + B^T (P B),  H_ux = B^T (P A),  T = A^T (P A)
// with compile-time sparsity; H_uu is inverted (2 x 2-block sweep), K = -H_uu^-1 H_ux
// and P <- T + H_ux^T K + diag(Q_t).  Caches per stage: K_k, H_uu,k^-1 (R24),
// e_k = P_{k+1} c_k, and the arm lanes' scalar gain, inverse and e.
// The polish step runs the same recursion on its reduced problem.
struct StageIn {
  const float* c;     // affine term c_k of the coupled lanes (smem vector)
  float rt_diag;      // this lane's diagonal of R_t
  float rt_off[3];    // force lanes: R_t(row b+r, j) of the foot block; arm lanes: [0] = B, [1] = c, [2] = A
  float qt;           // this lane's diagonal of Q_t for x_k (k >= 1)
  float rh;           // polish: this lane's linear cost of the reduced input
};
// per-lane results of one factor stage: e (coupled: (P_{k+1} c_k)_i; arm:
// P_{k+1} c), and for arm lanes the scalar gain and inverse
struct StageOut { float e, Ka, Hi; };

template <int PREC>
__device__ __forceinline__ StageOut factor_stage(const AgentPtrs& ap, float* sm, int lane, int k,
                                                 const StageIn& in, float* Pa, const LanePat& pat, int prec_rt,
                                                 bool store_h = true) {
  const int prec = PREC >= 0 ? PREC : prec_rt;
  StageOut so;
  so.e = so.Ka = so.Hi = 0.f;
  float* P = sm + S_P; float* H = sm + S_H; float* X = sm + S_X; float* K = sm + S_K;
  const float* av = sm + S_AV;
  const float* bv = sm + S_BV;
  const int j = lane < NC ? lane : NC - 1;
  // e = P c (before P is overwritten)
  const float e = r24_mtv(P, in.c, lane);
  // lane j: column j of P B, then H(:, j) = B^T (P B)(:, j) (H, X are not
  // read by other lanes before the next barrier, so they are written at once)
  {
    float pb[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) pb[i] = 0.f;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      const float b = bv[j * 6 + t];
      const int rb = pat.br[t];
#pragma unroll
      for (int i = 0; i < NC; ++i) pb[i] = fmaf(P[i * R24 + rb], b, pb[i]);
    }
    if (lane < NC) {
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        float h = 0.f;
#pragma unroll
        for (int t = 0; t < 6; ++t)
          if (t < bcnt(i)) h = fmaf(bv[i * 6 + t], pb[brow(i, t)], h);
        H[i * R24 + j] = h;
      }
    }
  }
  // column j of P A_k, then X(:, j) = B^T (P A)(:, j) and T(:, j) = A^T (P A)(:, j)
  float pa[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) pa[i] = 0.f;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const float a = av[j * 6 + t];
    const int ra = pat.ar[t];
#pragma unroll
    for (int i = 0; i < NC; ++i) pa[i] = fmaf(P[i * R24 + ra], a, pa[i]);
  }
  if (lane < NC) {
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      float x = 0.f;
#pragma unroll
      for (int t = 0; t < 6; ++t)
        if (t < bcnt(i)) x = fmaf(bv[i * 6 + t], pa[brow(i, t)], x);
      X[i * R24 + j] = x;
    }
  }
  __syncwarp();   // every lane has read P: T may overwrite it
  if (lane < NC) {
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      float tt = 0.f;
#pragma unroll
      for (int t = 0; t < 6; ++t)
        if (t < acnt(i)) tt = fmaf(av[i * 6 + t], pa[arow(i, t)], tt);
      P[i * R24 + j] = tt;
    }
    // + R_t column j: its diagonal and, for a force lane, its foot block
    H[j * R24 + j] += in.rt_diag;
    if (j < 12 && (j % 6) < 3) {
      const int b = (j / 6) * 6;
#pragma unroll
      for (int r = 0; r < 3; ++r)
        if (b + r != j) H[(b + r) * R24 + j] += in.rt_off[r];
    }
  }
  __syncwarp();
  // V_S (and V_H) are free during a factor stage
  if (prec == PREC_FP64) r24_inv_f64(H, reinterpret_cast<double*>(sm + S_VEC + V_S * 64), lane);
  else r24_inv(H, sm + S_VEC + V_S * 64, lane);
  // K = -H_uu^-1 H_ux (H_uu^-1 symmetric)
  if (prec == PREC_TF32X3) r24_gemm_tn_mma<PREC_TF32X3>(K, H, X, nullptr, -1.f, lane);
  else if (prec == PREC_TF32) r24_gemm_tn_mma<PREC_TF32>(K, H, X, nullptr, -1.f, lane);
  else if (prec == PREC_BF16) r24_gemm_tn_mma<PREC_BF16>(K, H, X, nullptr, -1.f, lane);
  else r24_gemm_tn(K, H, X, nullptr, -1.f, lane);
  copy_blk(ap.cK + (size_t)k * BLK, K, lane);
  if (store_h) copy_blk(ap.cH + (size_t)k * BLK, H, lane);
  float* ce = ap.cE + k * 64;
  if (lane < NC) ce[lane] = e;
  so.e = e;
  // arm lanes: scalar Riccati with A = rt_off[2], B = rt_off[0], c = rt_off[1]
  if (lane >= NC && lane < 30) {
    const float Bh = in.rt_off[0], Aa = in.rt_off[2];
    const float Huu = in.rt_diag + Bh * Bh * (*Pa);
    const float Hux = Bh * (*Pa) * Aa;
    const float Hi = 1.f / Huu;
    const float Ka = -Hi * Hux;
    ce[lane] = Ka;
    ce[32 + lane] = Hi;
    ce[32 + lane - NC] = (*Pa) * in.rt_off[1];   // e of the arm lane
    so.e = (*Pa) * in.rt_off[1];
    so.Ka = Ka;
    so.Hi = Hi;
    if (k >= 1) *Pa = in.qt + Aa * Aa * (*Pa) + Hux * Ka;
  }
  if (k >= 1) {
    // P = A^T P A + H_ux^T K
    if (prec == PREC_TF32X3) r24_gemm_tn_mma<PREC_TF32X3>(P, X, K, P, 1.f, lane);
    else if (prec == PREC_TF32) r24_gemm_tn_mma<PREC_TF32>(P, X, K, P, 1.f, lane);
    else if (prec == PREC_BF16) r24_gemm_tn_mma<PREC_BF16>(P, X, K, P, 1.f, lane);
    else r24_gemm_tn(P, X, K, P, 1.f, lane);
    float t[NC];
    if (lane < NC) {
#pragma unroll
      for (int i = 0; i < NC; ++i) t[i] = 0.5f * (P[i * R24 + j] + P[j * R24 + i]);
    }
    __syncwarp();
    if (lane < NC) {
#pragma unroll
      for (int i = 0; i < NC; ++i) P[i * R24 + j] = t[i];
      P[j * R24 + j] += in.qt;
    }
  }
  __syncwarp();
  return so;
}

// ADMM stage inputs: R_t = 2 dt R + sigma I + rho C_u^T diag(cls) C_u
__device__ __forceinline__ StageIn admm_stage_in(const AgentPtrs& ap, int k, float rho, float sigma,
                                                 float* cvec, int lane) {
  const float* md = ap.mdl;
  const float dt = md[M_DT], mu = md[M_MU];
  const float* rc = ap.rcls + k * RS;
  StageIn in;
  in.c = cvec;
  in.rt_off[0] = in.rt_off[1] = in.rt_off[2] = 0.f;
  in.rt_diag = 0.f;
  in.rh = 0.f;
  in.qt = (k >= 1 && lane < 30) ? qt_x(ap, k, lane, rho, sigma) : 0.f;
  if (lane < NC) {
    const int j = lane;
    const int row = j < 12 ? j : j + 8;
    float d = 2.f * dt * md[M_R + j] + sigma + rho * rc[row];
    if (j < 12 && (j % 6) < 3) {
      const int f = j / 6, c = j - 6 * f, p = 12 + 4 * f;
      const float r0 = rho * rc[p], r1 = rho * rc[p + 1], r2 = rho * rc[p + 2], r3 = rho * rc[p + 3];
      if (c == 0) { d += r0 + r1; in.rt_off[2] = mu * (r1 - r0); }
      if (c == 1) { d += r2 + r3; in.rt_off[2] = mu * (r3 - r2); }
      if (c == 2) {
        d += mu * mu * (r0 + r1 + r2 + r3);
        in.rt_off[0] = mu * (r1 - r0);
        in.rt_off[1] = mu * (r3 - r2);
      }
    }
    in.rt_diag = d;
    cvec[lane] = ap.lin[L_STAGE + k * 64 + 32 + lane];
  } else if (lane < 30) {
    in.rt_diag = 2.f * dt * md[M_R + lane] + sigma + rho * rc[lane + 8];
    in.rt_off[0] = dt;     // arm B
    in.rt_off[1] = 0.f;    // arm c
    in.rt_off[2] = 1.f;    // arm A
  }
  __syncwarp();
  return in;
}

template <int PREC>
__device__ __noinline__ void factor_admm(const AgentPtrs& ap, float* sm, int lane, float rho, float sigma,
                                        const LanePat& pat, int prec) {
  const int N = ap.N;
  float* P = sm + S_P;
  float* cvec = sm + S_VEC + V_C * 64;
  const int j = lane < NC ? lane : NC - 1;
  copy_n(sm + S_BV, ap.lin + L_BV, 136 / 4, lane);   // compact B of the ADMM problem
  if (lane < NC) {
    for (int i = 0; i < NC; ++i) P[i * R24 + j] = 0.f;
    P[j * R24 + j] = qt_x(ap, N, j, rho, sigma);
  }
  float Pa = (lane >= NC && lane < 30) ? qt_x(ap, N, lane, rho, sigma) : 0.f;
  __syncwarp();
  for (int k = N - 1; k >= 0; --k) {
    set_stage_A(sm, ap.lin + L_STAGE + k * 64, lane);
    const StageIn in = admm_stage_in(ap, k, rho, sigma, cvec, lane);
    factor_stage<PREC>(ap, sm, lane, k, in, &Pa, pat, prec);
  }
  // the caches were written with generic stores and are read back through
  // the async (TMA) proxy
  fence_proxy_async();
  __syncwarp();
}

// ============================================================ ADMM iteration (A5)
// One OSQP iteration with the equality-constrained KKT solve done by the
// cached Riccati factors (backward linear sweep + forward rollout), then
// relaxation, projection onto [lo, hi] and the dual update, stage by stage.
// The per-stage blocks K_k, H_uu,k^-1 are prefetched one stage ahead into two
// shared-memory buffers with TMA bulk copies (completion on an mbarrier).
// Bounded waits: a wait that gives up (after spin_limit polls) marks the
// pipe timed out for the whole warp; from then on the pipe issues no copy and
// skips every wait, the agent's solve ends with MPC_AGENT_TIMEOUT, and the
// kernel drains the copies still in flight (pipe_drain, bounded too) before
// the warp retires.  `dry` (failure-detection test only) arms the next
// barrier with no copy behind it, so that its wait runs out with nothing in
// flight.
struct Pipe {
  uint64_t* bar;    // kPipeBufs mbarriers, one per shared-memory buffer
  uint32_t st;      // bit b: phase parity of buffer b; bit 8 + b: a copy was issued into
                    // buffer b and not yet waited for; bit 16: timed out; bit 17: dry
  int limit;
  __device__ __forceinline__ bool timed_out() const { return st & PIPE_TIMEOUT_BIT; }
  static constexpr uint32_t PIPE_TIMEOUT_BIT = 1u << 16;
};
constexpr int kPipeBufs = 4;
constexpr uint32_t PIPE_TIMEOUT = Pipe::PIPE_TIMEOUT_BIT, PIPE_DRY = 1u << 17;

__device__ __forceinline__ void pipe_init(Pipe& pp, float* sm, int lane, int limit) {
  pp.bar = reinterpret_cast<uint64_t*>(sm + S_BAR);
  pp.st = 0u;
  pp.limit = limit > 0 ? limit : kSpinLimit;
  if (lane == 0) {
    for (int b = 0; b < kPipeBufs; ++b) mbar_init(pp.bar + b, 1);
    fence_mbar_init();
  }
  __syncwarp();
}
// the next issue of this agent's solve is armed with no copy (test only)
__device__ __forceinline__ void pipe_set_dry(Pipe& pp, bool dry) {
  pp.st = dry ? (pp.st | PIPE_DRY) : (pp.st & ~PIPE_DRY);
}
__device__ __forceinline__ void pipe_issue(Pipe& pp, int b, float* dstK, const float* srcK, float* dstH,
                                           const float* srcH, int lane) {
  if (pp.st & PIPE_TIMEOUT) return;
  const uint32_t bytes = (uint32_t)(BLK * sizeof(float));
  if (pp.st & PIPE_DRY) {
    if (lane == 0) mbar_expect_tx(pp.bar + b, dstH ? 2 * bytes : bytes);
    pp.st &= ~PIPE_DRY;
    return;
  }
  // no proxy fence here: every writer of the caches (factor_admm,
  // polish_solve) fences once after its stores, before the first copy
  if (lane == 0) {
    mbar_expect_tx(pp.bar + b, dstH ? 2 * bytes : bytes);
    tma_load_1d(dstK, srcK, bytes, pp.bar + b);
    if (dstH) tma_load_1d(dstH, srcH, bytes, pp.bar + b);
  }
  pp.st |= 256u << b;
}
__device__ __forceinline__ void pipe_wait(Pipe& pp, int b) {
  if (pp.st & PIPE_TIMEOUT) return;
  // one decision for the whole warp: a lane that gave up times the warp out
  if (!__all_sync(FULL, mbar_wait(pp.bar + b, pp.st >> b & 1u, pp.limit))) {
    pp.st |= PIPE_TIMEOUT;
    return;
  }
  pp.st = (pp.st & ~(256u << b)) ^ (1u << b);
}
// after a timeout: wait (bounded) for the copies still in flight into this
// warp's buffers, so that none lands after the warp has retired
__device__ __forceinline__ void pipe_drain(Pipe& pp) {
  for (int b = 0; b < kPipeBufs; ++b)
    if (pp.st & (256u << b)) {
      mbar_wait(pp.bar + b, pp.st >> b & 1u, pp.limit);
      pp.st &= ~(256u << b);
    }
  __syncwarp();
}
// The four R24 buffers of a pass that reads only K_k (forward rollouts):
// stage k in buffer k mod 4, copied three stages ahead
__device__ __forceinline__ float* kslot(float* sm, int b) {
  return sm + (b == 0 ? S_P : b == 1 ? S_X : b == 2 ? S_H : S_K);
}

// Per-lane global inputs of one stage of the ADMM sweeps.  Each stage's are
// loaded while the previous stage computes (one stage ahead), so a stage
// waits on memory once, for the TMA copy of its blocks, instead of once per
// step that uses a global value.
struct BwdPre {
  float rc0, w0, y0, rc1, w1, y1;   // rows lane and lane + 32 of stage k
  float xr, xk;                     // x_ref,k and x_k (linear term of x_k)
  float rq, wq, yq;                 // joint-box row lane + 26 of stage k - 1 (lanes 12-29)
  float ur, uk;                     // u_ref,k and u_k
  float e, e2;                      // cE_k[lane], cE_k[32 + lane]
  float a[3];                       // lanes 12-21: dA_k entries of the lane's compact A column
};
struct FwdPre {
  float dk, a0, a1, e;              // d_k, dA_k[lane], dA_k[32 + lane] (c_k), arm gain
  float w0, y0, rc0, lo0, hi0;      // row lane of stage k
  float w1, y1, rc1, lo1, hi1;      // row lane + 32
  float uo, xo;                     // u_k and x_{k+1} of the last iterate (relaxation)
};

// store_dy: also write the change of the row multipliers, y_new - y_old, to
// the agent's cEl scratch (free outside a polish), for the primal
// infeasibility test that follows a residual check
__device__ __noinline__ void admm_iteration(const AgentPtrs& ap, float* sm, int lane, float rho,
                                            const SolverParams& prm, Pipe& pp, const LanePat& pat,
                                            bool store_dy = false) {
  // the agent's arrays in registers (a reference to the caller's struct
  // would be re-read after every store)
  const int N = ap.N;
  const float* __restrict__ md = ap.mdl;
  float* __restrict__ X = ap.x; float* __restrict__ U = ap.u;
  float* __restrict__ Wr = ap.w; float* __restrict__ Yr = ap.y;
  const float* __restrict__ XR = ap.xref; const float* __restrict__ UR = ap.uref;
  const float* __restrict__ LO = ap.rlo; const float* __restrict__ HI = ap.rhi;
  const float* __restrict__ RC = ap.rcls; const float* __restrict__ LIN = ap.lin + L_STAGE;
  const float* __restrict__ CE = ap.cE; float* __restrict__ DV = ap.dv;
  float* __restrict__ XT = ap.xt; float* __restrict__ UT = ap.ut; float* __restrict__ EL = ap.cEl;
  const float* CK = ap.cK; const float* CH = ap.cH;
  const float dt = md[M_DT], mu = md[M_MU], sigma = prm.sigma, alpha = prm.alpha;
  float* Ab = sm + S_AB; float* Bm = sm + S_B;
  float* const K0 = sm + S_P; float* const K1 = sm + S_X;
  float* const H0 = sm + S_H; float* const H1 = sm + S_K;
  float* vec = sm + S_VEC;
  float* vS = vec + V_S * 64; float* vH = vec + V_H * 64; float* vX = vec + V_X * 64;
  float* vU = vec + V_U * 64; float* vXN = vec + V_XN * 64; float* vR = vec + V_ROW * 64;
  float* vA = vec + V_D * 64;
  const bool arm = lane >= NC && lane < 30;
  const bool jl = lane >= 12 && lane < 30;      // joint lanes (rate row lane + 8, box row lane + 26)
  const bool r1 = lane < NR - 32;               // the lane owns a second row
  const float twoQ = lane < 30 ? 2.f * dt * md[M_Q + lane] : 0.f;
  const float twoR = lane < 30 ? 2.f * dt * md[M_R + lane] : 0.f;
  // The row algebra of the lane without branches on its index (the lanes of
  // a warp would otherwise run each case in turn), as index and coefficient
  // tables built once per call:
  //  (C_u^T v)_lane = v[t0] + ta (((ts[0] v[tj[0]] + ts[1] v[tj[1]]) + ts[2] v[tj[2]]) + ts[3] v[tj[3]]),
  //  the sums in the order of cuT; index 56 of the row vector is held at zero;
  //  row lane (+ 32 q) of C_u u + C_x x_{k+1} = fmaf(cs1[q], z[ci1[q]], cs0[q] z[ci0[q]])
  //  over z = [u (64) | x_{k+1} (64)], the terms in the order of crow; z[30] = u_30 = 0.
  int t0 = 56, tj[4] = {56, 56, 56, 56};
  float ta = 0.f, ts[4] = {0.f, 0.f, 0.f, 0.f};
  if (lane < 12) {
    const int f = lane / 6, c = lane - 6 * f, pp0 = 12 + 4 * f;
    t0 = lane;
    if (c == 0) { ta = 1.f; tj[0] = pp0; tj[1] = pp0 + 1; ts[0] = 1.f; ts[1] = -1.f; }
    if (c == 1) { ta = 1.f; tj[0] = pp0 + 2; tj[1] = pp0 + 3; ts[0] = 1.f; ts[1] = -1.f; }
    if (c == 2) {
      ta = -mu;
#pragma unroll
      for (int t = 0; t < 4; ++t) { tj[t] = pp0 + t; ts[t] = 1.f; }
    }
  } else if (lane < 30) {
    t0 = lane + 8;
  }
  int ci0[2], ci1[2];
  float cs0[2], cs1[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int r = lane + 32 * q;
    ci0[q] = 30; ci1[q] = 30; cs0[q] = 0.f; cs1[q] = 0.f;
    if (r < 12) { ci0[q] = r; cs0[q] = 1.f; }
    else if (r < 20) {
      const int f = (r - 12) >> 2, t = (r - 12) & 3, bb = 6 * f;
      ci0[q] = bb + (t >> 1); cs0[q] = (t & 1) ? -1.f : 1.f;
      ci1[q] = bb + 2; cs1[q] = -mu;
    } else if (r < 38) { ci0[q] = r - 8; cs0[q] = 1.f; }
    else if (r < NR) { ci0[q] = 64 + r - 26; cs0[q] = 1.f; }
  }
  if (lane >= NR - 32) vR[lane + 32] = 0.f;   // rows 56-63: the zero of the tables
  auto cuT_t = [&](const float* v) -> float {
    const float S = fmaf(ts[3], v[tj[3]], fmaf(ts[2], v[tj[2]], fmaf(ts[1], v[tj[1]], ts[0] * v[tj[0]])));
    return fmaf(ta, S, v[t0]);
  };
  auto crow_t = [&](const float* z, int q) -> float { return fmaf(cs1[q], z[ci1[q]], cs0[q] * z[ci0[q]]); };

  auto load_bwd = [&](int k) {
    BwdPre q;
    const int o = k * RS;
    q.rc0 = RC[o + lane]; q.w0 = Wr[o + lane]; q.y0 = Yr[o + lane];
    q.rc1 = r1 ? RC[o + lane + 32] : 0.f; q.w1 = r1 ? Wr[o + lane + 32] : 0.f; q.y1 = r1 ? Yr[o + lane + 32] : 0.f;
    q.xr = XR[k * VS + lane]; q.xk = X[k * VS + lane];
    const bool hq = jl && k >= 1;
    q.rq = hq ? RC[o - RS + lane + 26] : 0.f;
    q.wq = hq ? Wr[o - RS + lane + 26] : 0.f;
    q.yq = hq ? Yr[o - RS + lane + 26] : 0.f;
    q.ur = UR[k * VS + lane]; q.uk = U[k * VS + lane];
    q.e = CE[k * 64 + lane]; q.e2 = CE[k * 64 + 32 + lane];
    const bool aj = lane >= 12 && lane < NC;
#pragma unroll
    for (int t = 0; t < 3; ++t) q.a[t] = aj ? LIN[k * 64 + t * 10 + (lane - 12)] : 0.f;
    return q;
  };
  auto load_fwd = [&](int k) {
    FwdPre q;
    const int o = k * RS;
    q.dk = DV[k * VS + lane];
    q.a0 = LIN[k * 64 + lane]; q.a1 = LIN[k * 64 + 32 + lane];
    q.e = CE[k * 64 + lane];
    q.w0 = Wr[o + lane]; q.y0 = Yr[o + lane]; q.rc0 = RC[o + lane]; q.lo0 = LO[o + lane]; q.hi0 = HI[o + lane];
    q.w1 = r1 ? Wr[o + lane + 32] : 0.f; q.y1 = r1 ? Yr[o + lane + 32] : 0.f;
    q.rc1 = r1 ? RC[o + lane + 32] : 0.f; q.lo1 = r1 ? LO[o + lane + 32] : 0.f;
    q.hi1 = r1 ? HI[o + lane + 32] : 0.f;
    q.uo = U[k * VS + lane]; q.xo = X[(k + 1) * VS + lane];
    return q;
  };
  // linear term of x_k (k >= 1): -2dt Q xr_k - sigma x_k - C_x^T (rho w - y) of stage k-1
  auto qlin = [&](const BwdPre& q) -> float {
    float v = -twoQ * q.xr - sigma * q.xk;
    if (jl) v -= rho * q.rq * q.wq - q.yq;
    return v;
  };

  // ---- backward sweep: p_k, d_k
  pipe_issue(pp, 0, K0, CK + (size_t)(N - 1) * BLK, H0, CH + (size_t)(N - 1) * BLK, lane);
  float p = 0.f;
  {
    // x_N's linear term: its joint-box row is row lane + 26 of stage N - 1
    const bool hq = jl;
    const float xr = XR[N * VS + lane], xk = X[N * VS + lane];
    const float rq = hq ? RC[(N - 1) * RS + lane + 26] : 0.f;
    const float wq = hq ? Wr[(N - 1) * RS + lane + 26] : 0.f;
    const float yq = hq ? Yr[(N - 1) * RS + lane + 26] : 0.f;
    float v = -twoQ * xr - sigma * xk;
    if (jl) v -= rho * rq * wq - yq;
    p = lane < 30 ? v : 0.f;
  }
  BwdPre cur = load_bwd(N - 1);
  for (int k = N - 1; k >= 0; --k) {
    const int b = (N - 1 - k) & 1;
    float* const Kc = b ? K1 : K0;
    float* const Hc = b ? H1 : H0;
    if (k >= 1)
      pipe_issue(pp, b ^ 1, b ? K0 : K1, CK + (size_t)(k - 1) * BLK, b ? H0 : H1, CH + (size_t)(k - 1) * BLK, lane);
    const BwdPre q = cur;
    if (k >= 1) cur = load_bwd(k - 1);
    if (lane >= 12 && lane < NC) {
      float* av = sm + S_AV + lane * 6;
      av[0] = 1.f;
      av[1] = q.a[0];
      av[2] = q.a[1];
      av[3] = q.a[2];
    }
    __syncwarp();
    vR[lane] = rho * q.rc0 * q.w0 - q.y0;
    if (r1) vR[lane + 32] = rho * q.rc1 * q.w1 - q.y1;
    const float s = (lane < NC ? q.e : 0.f) + p;
    vS[lane] = s;
    __syncwarp();
    float h = 0.f;
    if (lane < 30) {
      const float rlin = -twoR * q.ur - sigma * q.uk - cuT_t(vR);
      h = rlin + (lane < NC ? cc_tv(sm + S_BV, pat.br, vS, lane) : dt * s);
    }
    vH[lane] = h;
    float pn = 0.f;
    if (k >= 1 && lane < 30) pn = qlin(q) + (lane < NC ? cc_tv(sm + S_AV, pat.ar, vS, lane) : s);
    pipe_wait(pp, b);
    __syncwarp();
    // d_k = -H_uu^-1 h and K_k^T h in one pass over the two blocks
    const float2 hk = r24_mtv2(Hc, Kc, vH, lane);
    float d = 0.f;
    if (lane < NC) d = -hk.x;
    else if (arm) d = -q.e2 * h;
    DV[k * VS + lane] = d;
    if (k >= 1) {
      if (lane < NC) pn += hk.y;
      else if (arm) pn += q.e * h;
      p = pn;
    }
    __syncwarp();
  }

  // ---- forward rollout + per-stage relaxation / projection / dual update
  float x = lane < 30 ? X[lane] : 0.f;   // x_0 = x0
  for (int k = 0; k < 3 && k < N; ++k) pipe_issue(pp, k, kslot(sm, k), CK + (size_t)k * BLK, nullptr, nullptr, lane);
  FwdPre fc = load_fwd(0);
  auto row_update = [&](int k, int r, float zt, float wo, float yo, float rc, float lo, float hi) {
    const float wh = alpha * zt + (1.f - alpha) * wo;
    const float rr = rho * rc;
    float wn, yn;
    if (rr > 0.f) {
      wn = fminf(fmaxf(wh + yo / rr, lo), hi);
      yn = yo + rr * (wh - wn);
    } else {
      wn = wh;
      yn = 0.f;
    }
    Wr[k * RS + r] = wn;
    Yr[k * RS + r] = yn;
    if (store_dy) EL[k * 128 + r] = yn - yo;
  };
  for (int k = 0; k < N; ++k) {
    const int b = k & 3;
    float* const Kc = kslot(sm, b);
    // stage k + 3 into the buffer stage k - 1 used (free since its last barrier)
    if (k + 3 < N) pipe_issue(pp, (k + 3) & 3, kslot(sm, (k + 3) & 3), CK + (size_t)(k + 3) * BLK, nullptr, nullptr, lane);
    const FwdPre q = fc;
    if (k + 1 < N) fc = load_fwd(k + 1);
    vX[lane] = x;
    pipe_wait(pp, b);
    vA[lane] = q.a0;
    vA[32 + lane] = q.a1;
    __syncwarp();
    float u = 0.f;
    if (lane < NC) u = r24_mv(Kc, vX, lane) + q.dk;
    else if (arm) u = q.e * x + q.dk;
    vU[lane] = u;
    __syncwarp();
    float xn = 0.f;
    if (lane < NC) xn = ak_mv(Ab, vA, vX, lane) + cm_mv_s(Bm, vU, lane) + vA[32 + lane];
    else if (arm) xn = x + dt * u;
    vXN[lane] = xn;
    XT[(k + 1) * VS + lane] = xn;
    UT[k * VS + lane] = u;
    __syncwarp();
    row_update(k, lane, crow_t(vU, 0), q.w0, q.y0, q.rc0, q.lo0, q.hi0);
    if (r1) row_update(k, lane + 32, crow_t(vU, 1), q.w1, q.y1, q.rc1, q.lo1, q.hi1);
    if (lane < 30) {
      U[k * VS + lane] = alpha * u + (1.f - alpha) * q.uo;
      X[(k + 1) * VS + lane] = alpha * xn + (1.f - alpha) * q.xo;
    }
    x = xn;
    __syncwarp();
  }
}

// ============================================================ residuals (A5 vii)
// Unscaled OSQP residuals of the current iterate: primal |C z - w|_inf over
// constrained rows; dual = stationarity in u after choosing the dynamics
// multipliers that make stationarity in x exact (costate recursion).
// Residuals: rp, rd the inf-norms of the primal and dual residuals; ps, ds
// the global scales (for the rho update); pn, dn the largest residual
// component over its own tolerance eps_abs + eps_rel * (magnitude of the
// terms of that row or stationarity component), the convergence measure
// (<= 1 converged): the components differ by orders of magnitude (forces vs
// joint rates), and one global scale would let the small ones go unchecked.
struct Res { float rp, rd, ps, ds, pn, dn; };
// A polished point must also pass every row and component within its own
// tolerance eps_abs + eps_rel x (magnitude of its terms) (kScaledAccept = 1).
// The magnitude of a stationarity component counts every term that forms it,
// through the costate recursion (sums of absolute values: the scale of its
// FP32 rounding, under 1e-6 of it for the n <= 100 terms here, since
// n 2^-24 < 1e-5).  A correct polish after its refinement step sits at a few
// hundredths of that tolerance (99th percentile over a warm replan); an
// active row whose multiplier has the wrong sign, even one worth only
// 1e-11 of the objective (a flat direction of the cost), lands above it and
// is corrected.
constexpr float kScaledAccept = 1.f;
// Corrections change an active row whose check value exceeds kFixScale times
// its own tolerance; a point that no correction can change (or that of the
// last attempt) is accepted within kScaledLoose times its tolerance (the
// residual bar of 1e-4, absolute plus relative, per component) instead of
// going to ADMM.
constexpr float kFixScale = 1.f;
constexpr float kScaledLoose = 10.f;
// ADMM's own stopping test (its iterate is reported INACCURATE unless a
// polish certifies it) and the threshold of its infeasibility test read the
// scaled residuals of admm_residuals at 10 times the tolerance
constexpr float kAdmmScaledStop = 10.f;

__device__ __noinline__ Res admm_residuals(const AgentPtrs& ap, float* sm, int lane, const SolverParams& prm,
                                           const LanePat& pat) {
  const int N = ap.N;
  const float* md = ap.mdl;
  const float dt = md[M_DT], mu = md[M_MU];
  float* vec = sm + S_VEC;
  float* vU = vec + V_U * 64; float* vXN = vec + V_XN * 64; float* vM = vec + V_S * 64;
  float* vY = vec + V_ROW * 64;
  const float twoQ = lane < 30 ? 2.f * dt * md[M_Q + lane] : 0.f;
  const float twoR = lane < 30 ? 2.f * dt * md[M_R + lane] : 0.f;
  const float* xs = ap.x;
  const float* us = ap.u;
  const float* ys = ap.y;
  const float ea = prm.eps_abs, er = prm.eps_rel;
  float rp = 0.f, ps = 0.f, rd = 0.f, ds = 0.f, pn = 0.f, dn = 0.f;
  for (int k = 0; k < N; ++k) {
    vU[lane] = us[k * VS + lane];
    vXN[lane] = xs[(k + 1) * VS + lane];
    __syncwarp();
    for (int r = lane; r < NR; r += 32) {
      if (ap.rcls[k * RS + r] > 0.f) {
        const float v = crow(vU, vXN, r, mu);
        const float w = ap.w[k * RS + r];
        const float sc = fmaxf(fabsf(v), fabsf(w));
        rp = fmaxf(rp, fabsf(v - w));
        ps = fmaxf(ps, sc);
        pn = fmaxf(pn, fabsf(v - w) / (ea + er * sc));
      }
    }
    __syncwarp();
  }
  auto gx = [&](int k) -> float {   // 2dt Q (x_k - xr_k) + C_x^T y_{k-1}
    float g = twoQ * (xs[k * VS + lane] - ap.xref[k * VS + lane]);
    if (lane >= 12 && lane < 30) g += ys[(k - 1) * RS + lane + 26];
    return g;
  };
  float m = lane < 30 ? gx(N) : 0.f;
  for (int k = N - 1; k >= 0; --k) {
    set_stage_A(sm, ap.lin + L_STAGE + k * 64, lane);
    vM[lane] = m;
    for (int r = lane; r < NR; r += 32) vY[r] = ys[k * RS + r];
    __syncwarp();
    float mn = 0.f;
    if (lane < 30) {
      const float cty = cuT(vY, lane, mu);
      const float gu = twoR * (us[k * VS + lane] - ap.uref[k * VS + lane]) + cty;
      const float btm = lane < NC ? cc_tv(sm + S_BV, pat.br, vM, lane) : dt * m;
      const float ru = gu + btm;
      rd = fmaxf(rd, fabsf(ru));
      const float su = fmaxf(fmaxf(fabsf(twoR * us[k * VS + lane]), fabsf(twoR * ap.uref[k * VS + lane])),
                             fmaxf(fabsf(cty), fabsf(btm)));
      dn = fmaxf(dn, fabsf(ru) / (ea + er * su));
      ds = fmaxf(ds, fmaxf(fabsf(twoR * us[k * VS + lane]), fabsf(twoR * ap.uref[k * VS + lane])));
      ds = fmaxf(ds, fmaxf(fabsf(cty), fabsf(twoQ * xs[(k + 1) * VS + lane])));
      ds = fmaxf(ds, fabsf(twoQ * ap.xref[(k + 1) * VS + lane]));
      if (lane >= 12) ds = fmaxf(ds, fabsf(vY[lane + 26]));
      if (k >= 1) mn = gx(k) + (lane < NC ? cc_tv(sm + S_AV, pat.ar, vM, lane) : m);
    }
    __syncwarp();
    m = mn;
  }
  Res out;
  out.rp = warp_max(rp); out.ps = warp_max(ps); out.rd = warp_max(rd); out.ds = warp_max(ds);
  out.pn = warp_max(pn); out.dn = warp_max(dn);
  return out;
}

// ============================================================ infeasibility (A5 vii)
// OSQP's primal infeasibility certificate (Stellato et al. 2020, Sec. 3.4;
// Banjac et al. 2019): when the constraints admit no point, the change of
// the multipliers over an iteration, dy = y^k - y^(k-1), converges to a
// Farkas certificate.  Here the dynamics rows are eliminated exactly, so
// their multipliers nu are not iterated: they are taken from the costate
// recursion that makes the certificate's x-components vanish,
// m_N = C_x^T dy_(N-1), m_k = C_x^T dy_(k-1) + A_k^T m_(k+1), nu = -m.  The
// problem is declared primal infeasible when the u-components nearly vanish,
// |C_u^T dy_k + B_k^T m_(k+1)|_inf <= eps |dy|_inf, and the support function
// of the constraint set is negative along dy:
// hi^T max(dy, 0) + lo^T min(dy, 0) + e^T nu < -eps |dy|_inf, with
// e^T nu = -(m_0^T x0 + sum_k m_(k+1)^T c_k) and m_0 = A_0^T m_1.
// Reads dy from cEl (written by the preceding admm_iteration).
constexpr float kEpsPrimInf = 1e-4f;   // OSQP's default eps_prim_inf

__device__ __noinline__ bool admm_primal_infeasible(const AgentPtrs& ap, float* sm, int lane, const LanePat& pat) {
  const int N = ap.N;
  const float* md = ap.mdl;
  const float dt = md[M_DT], mu = md[M_MU];
  float* vec = sm + S_VEC;
  float* vM = vec + V_S * 64;
  float* vY = vec + V_ROW * 64;
  const float* dy = ap.cEl;
  float dyn = 0.f, supp = 0.f;
  for (int k = 0; k < N; ++k)
    for (int r = lane; r < NR; r += 32) {
      const float d = dy[k * 128 + r];
      if (ap.rcls[k * RS + r] > 0.f && d != 0.f) {
        dyn = fmaxf(dyn, fabsf(d));
        supp += d > 0.f ? d * ap.rhi[k * RS + r] : d * ap.rlo[k * RS + r];
      }
    }
  dyn = warp_max(dyn);
  supp = warp_sum(supp);
  if (!(dyn > 0.f) || !(supp < INFINITY)) return false;   // no change, or dy leaves an unbounded side
  float m = (lane >= 12 && lane < 30) ? dy[(N - 1) * 128 + lane + 26] : 0.f;
  float ru = 0.f, ex = 0.f;
  for (int k = N - 1; k >= 0; --k) {
    const float* dA = ap.lin + L_STAGE + k * 64;
    set_stage_A(sm, dA, lane);
    vM[lane] = m;
    for (int r = lane; r < NR; r += 32) vY[r] = dy[k * 128 + r];
    __syncwarp();
    float mn = 0.f;
    if (lane < 30) {
      const float btm = lane < NC ? cc_tv(sm + S_BV, pat.br, vM, lane) : dt * m;
      ru = fmaxf(ru, fabsf(cuT(vY, lane, mu) + btm));
      if (lane < NC) ex += m * dA[32 + lane];                 // m_(k+1)^T c_k
      const float atm = lane < NC ? cc_tv(sm + S_AV, pat.ar, vM, lane) : m;
      if (k >= 1) mn = atm + (lane >= 12 ? dy[(k - 1) * 128 + lane + 26] : 0.f);
      else ex += atm * ap.x[lane];                              // m_0^T x0
    }
    __syncwarp();
    m = mn;
  }
  ru = warp_max(ru);
  ex = warp_sum(ex);
  return ru <= kEpsPrimInf * dyn && supp - ex < -kEpsPrimInf * dyn;
}

// ============================================================ polish
// OSQP's solution polishing: active set from (w, y) (row at its lower bound
// when w - lo < -y, at its upper bound when hi - w < y).  Active rows are
// eliminated exactly: u_k = G_k v_k + t_k, and the reduced equality-
// constrained LQ problem is solved by one more Riccati factor + sweep.
// An active joint-box row (on x_{k+1}) eliminates the joint rate of stage k
// through q_{k+1} = q_k + dt qd_k; a joint with both its rate row and its
// joint-box row active at one stage keeps only one of them (a degenerate
// optimum that needs both is left to ADMM).
// Active-set codes: bit 0 lower, bit 1 upper, 3 = equality row.
struct FootAct { int swing, zero, top, tx, ty; };

__device__ void init_active(const AgentPtrs& ap, int lane) {
  for (int k = 0; k < ap.N; ++k) {
    for (int r = lane; r < NR; r += 32) {
      const float lo = ap.rlo[k * RS + r], hi = ap.rhi[k * RS + r];
      const float w = ap.w[k * RS + r], y = ap.y[k * RS + r];
      int a = 0;
      if (lo == hi) a = 3;
      else {
        if (w - lo < -y) a |= 1;
        if (hi - w < y) a |= 2;
      }
      ap.act[k * RS + r] = a;
    }
  }
  __syncwarp();
}

// One stage's per-lane global inputs of a polish pass, loaded together at
// the top of the stage: one memory round trip, where loading each where it
// is used costs one per step (active codes, A_k, bounds, references)
struct StagePre {
  int a0, a1;                      // active-set codes of rows lane and lane + 32
  float dA[3];                     // this lane's entries of the stage-varying A_k block (lanes 12-21)
  float F;                         // force lanes: upper bound of the foot's normal-force row
  float lo_r, hi_r, lo_q, hi_q;    // lanes 12-29: bounds of the joint's rate row and joint-box row
  float uref, ck;                  // u_ref,k and (coupled lanes) the affine term c_k
};
__device__ __forceinline__ StagePre stage_pre(const AgentPtrs& ap, int k, int lane) {
  StagePre p;
  const int* ak = ap.act + k * RS;
  const float* lo = ap.rlo + k * RS;
  const float* hi = ap.rhi + k * RS;
  const float* dA = ap.lin + L_STAGE + k * 64;
  p.a0 = ak[lane];
  p.a1 = lane < NR - 32 ? ak[lane + 32] : 0;
  const bool aj = lane >= 12 && lane < NC;
#pragma unroll
  for (int t = 0; t < 3; ++t) p.dA[t] = aj ? dA[t * 10 + (lane - 12)] : 0.f;
  p.F = lane < 12 ? hi[(lane / 6) * 6 + 2] : 0.f;
  const bool jr = lane >= 12 && lane < 30;
  p.lo_r = jr ? lo[lane + 8] : 0.f;
  p.hi_r = jr ? hi[lane + 8] : 0.f;
  p.lo_q = jr ? lo[lane + 26] : 0.f;
  p.hi_q = jr ? hi[lane + 26] : 0.f;
  p.uref = ap.uref[k * VS + lane];
  p.ck = lane < NC ? dA[32 + lane] : 0.f;
  return p;
}
__device__ __forceinline__ void stage_active_pre(const StagePre& p, int* act, int lane) {
  __syncwarp();
  act[lane] = p.a0;
  if (lane < NR - 32) act[lane + 32] = p.a1;
  __syncwarp();
}
__device__ __forceinline__ void set_stage_A_pre(float* sm, const StagePre& p, int lane) {
  if (lane >= 12 && lane < NC) {
    float* av = sm + S_AV + lane * 6;
    av[0] = 1.f;
    av[1] = p.dA[0];
    av[2] = p.dA[1];
    av[3] = p.dA[2];
  }
  __syncwarp();
}

__device__ __forceinline__ void stage_active(const AgentPtrs& ap, int k, int* act, int lane) {
  __syncwarp();
  for (int r = lane; r < NR; r += 32) act[r] = ap.act[k * RS + r];
  __syncwarp();
}

__device__ __forceinline__ FootAct foot_act(const int* act, int f) {
  FootAct fa;
  const int b = 6 * f, p = 12 + 4 * f;
  fa.swing = act[b + 2] == 3;
  const bool up0 = act[p] & 2, up1 = act[p + 1] & 2, up2 = act[p + 2] & 2, up3 = act[p + 3] & 2;
  fa.zero = !fa.swing && ((act[b + 2] & 1) || (up0 && up1) || (up2 && up3));
  fa.top = !fa.swing && !fa.zero && (act[b + 2] & 2);
  fa.tx = up0 ? 1 : (up1 ? -1 : 0);
  fa.ty = up2 ? 1 : (up3 ? -1 : 0);
  return fa;
}

// The elimination of stage k for input i (< 30).  Force inputs:
// u_i = sum_c gf[c] v_{b+c} + t (row of the foot's 3x3 block G_f); other
// inputs: u_i = g v_i + t + phi x_i with g in {0, 1}.  A joint rate whose
// joint-box row (on x_{k+1}) is active is fixed by q_{k+1} = q_k + dt qdot_k
// = b:  qdot_k = (b - q_k)/dt, i.e. t = b/dt, phi = -1/dt (qbox = 1).
// When the rate row is active as well (a degenerate optimum: the joint rides
// its rate bound onto its limit), the rate keeps its bound t_r and the pair
// fixes q_k = b - dt t_r instead: a constraint on x_k carried to stage k-1,
// where it eliminates that stage's joint rate in the same way (or, if that
// rate is at its bound too, is carried further).  carry_in: the constraint
// on q_{k+1} carried from stage k+1; carry_out: the one passed to stage k-1.
struct Carry { int on; float b; };
struct Elim { float g, t, phi, gf[3]; int qbox; Carry carry_out; };

__device__ __forceinline__ Elim lane_elim(const AgentPtrs& ap, const StagePre& pre, const int* act, int i,
                                          float mu, Carry carry_in) {
  Elim e;
  e.g = 1.f; e.t = 0.f; e.phi = 0.f; e.gf[0] = e.gf[1] = e.gf[2] = 0.f; e.qbox = 0;
  e.carry_out.on = 0; e.carry_out.b = 0.f;
  if (i < 12) {
    const int f = i / 6, c = i - 6 * f;
    const FootAct fa = foot_act(act, f);
    if (fa.swing || fa.zero) { e.g = 0.f; return e; }
    if (c >= 3) return e;                                   // free moment
    e.g = 0.f;
    if (fa.top) {
      const float F = pre.F;
      if (c == 2) e.t = F;
      else {
        const int tt = c == 0 ? fa.tx : fa.ty;
        if (tt) e.t = tt * mu * F;
        else e.gf[c] = 1.f;
      }
    } else {
      if (c == 2) e.gf[2] = 1.f;
      else {
        const int tt = c == 0 ? fa.tx : fa.ty;
        if (tt) e.gf[2] = tt * mu;
        else e.gf[c] = 1.f;
      }
    }
    return e;
  }
  if (i < 30) {
    const int r = i + 8, rq = i + 26;
    const int a = act[r], aq = act[rq];
    int eq = carry_in.on;
    float eb = carry_in.b;
    if (!eq && aq) { eq = 1; eb = (aq & 1) ? pre.lo_q : pre.hi_q; }
    const float dt = ap.mdl[M_DT];
    if (a) {
      e.g = 0.f;
      e.t = (a & 1) ? pre.lo_r : pre.hi_r;
      if (eq) { e.carry_out.on = 1; e.carry_out.b = eb - dt * e.t; }
    } else if (eq) {
      e.g = 0.f;
      e.t = eb / dt;
      e.phi = -1.f / dt;
      e.qbox = 1;
    }
  }
  return e;
}

// Per-stage inputs of the polish factor: compact B_hat = B G (into smem),
// R_hat = G^T D G plus 1 on eliminated inputs, c_hat = c + B t (into cvec),
// r_hat = G^T D (t - u_ref) (per lane), Q_t of x_k with the moved cost of an
// eliminated joint rate, A_hat (identity entry of an eliminated joint).
// uref: this lane's u_ref,k; c_k: this lane's c_k (lanes < 22)
__device__ StageIn polish_stage_in(const AgentPtrs& ap, float* sm, float* cvec, const Elim& el, int lane,
                                   const LanePat& pat, float uref, float c_k) {
  const float* md = ap.mdl;
  const float dt = md[M_DT];
  const float* Bd = sm + S_B;        // dense B (column-major, LDD): compact entry t of column j is
                                     // B(brow(j, t), j); the three force columns of a foot share rows
  float* vec = sm + S_VEC;
  float* gfv = vec + V_T * 64;       // rows of G_f, 3 per force input (indexed 3*i)
  float* gv = vec + V_G * 64;        // g per input
  float* tv = vec + V_D * 64;        // t per input
  float* vD2 = vec + V_H * 64;       // D (t - u_ref)
  const float Dj = lane < 30 ? 2.f * dt * md[M_R + lane] : 0.f;
  if (lane < 30) {
    gv[lane] = el.g;
    tv[lane] = el.t;
    vD2[lane] = Dj * (el.t - uref);
    if (lane < 12) { gfv[lane * 3] = el.gf[0]; gfv[lane * 3 + 1] = el.gf[1]; gfv[lane * 3 + 2] = el.gf[2]; }
  } else {
    tv[lane] = 0.f;
  }
  __syncwarp();
  StageIn in;
  in.c = cvec;
  in.rt_off[0] = in.rt_off[1] = in.rt_off[2] = 0.f;
  in.rt_diag = 0.f;
  in.rh = 0.f;
  // state cost of x_k; an eliminated joint rate moves its cost dt R u^2 onto
  // x_k:  (R/dt) (x_i - b)^2
  in.qt = lane < 30 ? 2.f * dt * md[M_Q + lane] + (el.qbox ? 2.f * md[M_R + lane] / dt : 0.f) : 0.f;
  // A_hat = A + B Phi: the eliminated joint's identity entry vanishes
  if (el.qbox && lane >= 12 && lane < NC) sm[S_AV + lane * 6] = 0.f;
  if (lane < NC) {
    const int j = lane;
    const bool fj = j < 12 && (j % 6) < 3;
    const int b = (j / 6) * 6, c = j - b;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      float v;
      // padding entries (t >= bcnt) read row 0 of B, which is zero (p has no input)
      const int rb = pat.br[t];
      if (fj)
        v = Bd[(b + 0) * LDD + rb] * gfv[(b + 0) * 3 + c] + Bd[(b + 1) * LDD + rb] * gfv[(b + 1) * 3 + c] +
            Bd[(b + 2) * LDD + rb] * gfv[(b + 2) * 3 + c];
      else
        v = Bd[j * LDD + rb] * gv[j];
      sm[S_BV + j * 6 + t] = v;
    }
    if (fj) {
      float d = 0.f, alive = 0.f;
      for (int l = 0; l < 3; ++l) {
        const float g = gfv[(b + l) * 3 + c];
        const float Dl = 2.f * dt * md[M_R + b + l];
        d += g * Dl * g;
        alive = fmaxf(alive, g != 0.f ? 1.f : 0.f);
        for (int r = 0; r < 3; ++r) in.rt_off[r] += gfv[(b + l) * 3 + r] * Dl * g;
      }
      in.rt_diag = d + (1.f - alive);
      in.rh = gfv[(b + 0) * 3 + c] * vD2[b] + gfv[(b + 1) * 3 + c] * vD2[b + 1] + gfv[(b + 2) * 3 + c] * vD2[b + 2];
    } else {
      in.rt_diag = gv[j] * Dj * gv[j] + (1.f - gv[j]);
      in.rh = gv[j] * vD2[j];
    }
    cvec[j] = c_k + cm_mv_s(sm + S_B, tv, lane);   // c_hat
  } else if (lane < 30) {
    const float alive = el.g;
    in.rt_diag = alive * Dj + (1.f - alive);
    in.rt_off[0] = alive * dt;                  // arm B_hat
    in.rt_off[1] = (1.f - alive) * dt * el.t;   // arm c_hat
    in.rt_off[2] = el.qbox ? 0.f : 1.f;         // arm A_hat
    in.rh = alive * vD2[lane];
  }
  __syncwarp();
  return in;
}

// Polish forward pass: v = K x + d, u = G v + t + Phi x, x+ = A x + B u + c
// with the recorded eliminations; a refinement pass re-rolls from the
// previous pass: v = v_old + K (x - x_old) + d' with the correction's
// feed-forward d'.  v is kept (dv) for the next pass.
__device__ __noinline__ void polish_rollout(const AgentPtrs& ap, float* sm, int lane, Pipe& pp, bool refine) {
  const int N = ap.N;
  const float dt = ap.mdl[M_DT];
  float* vec = sm + S_VEC;
  float* vX = vec + V_X * 64; float* vV = vec + V_U * 64; float* vU = vec + V_XN * 64;
  float* vA = vec + V_D * 64;   // the stage's dA_k block and c_k, staged with the stage's other loads
  const bool arm = lane >= NC && lane < 30;
    float x = lane < 30 ? ap.x[lane] : 0.f;
    float xo = x;                                  // previous pass's x_k (x_0 is fixed)
    for (int k = 0; k < 3 && k < N; ++k)
      pipe_issue(pp, k, kslot(sm, k), ap.cK + (size_t)k * BLK, nullptr, nullptr, lane);
    // per-lane global inputs of a stage, loaded one stage ahead (stage k
    // writes dv_k, x_{k+1}, u_k: none of stage k+1's inputs)
    struct RollPre { float4 el; float a0, a1, base, xo_next, e; };
    auto load = [&](int k) {
      RollPre q;
      const float* dA = ap.lin + L_STAGE + k * 64;
      q.el = reinterpret_cast<const float4*>(ap.cEl + k * 128)[lane];
      q.a0 = dA[lane];
      q.a1 = dA[32 + lane];
      q.base = refine ? ap.dv[k * VS + lane] + ap.cD[k * VS + lane] : ap.dv[k * VS + lane];
      q.xo_next = refine ? ap.xt[(k + 1) * VS + lane] : 0.f;
      q.e = ap.cE[k * 64 + lane];
      return q;
    };
    RollPre cur = load(0);
    for (int k = 0; k < N; ++k) {
      const int b = k & 3;
      float* const Kc = kslot(sm, b);
      if (k + 3 < N)
        pipe_issue(pp, (k + 3) & 3, kslot(sm, (k + 3) & 3), ap.cK + (size_t)(k + 3) * BLK, nullptr, nullptr, lane);
      const RollPre q = cur;
      if (k + 1 < N) cur = load(k + 1);
      const float4 el = q.el;
      const float dA0 = q.a0, dA1 = q.a1;
      vX[lane] = refine ? x - xo : x;
      const float base = q.base;
      const float xo_next = q.xo_next;
      pipe_wait(pp, b);
      vA[lane] = dA0;
      vA[32 + lane] = dA1;
      __syncwarp();
      float v = 0.f;
      if (lane < NC) v = r24_mv(Kc, vX, lane) + base;
      else if (arm) v = q.e * vX[lane] + base;
      vV[lane] = v;
      ap.dv[k * VS + lane] = v;
      __syncwarp();
      float u = 0.f;
      if (lane < 12 && (lane % 6) < 3) {
        const int bb = (lane / 6) * 6;
        u = el.x * vV[bb] + el.y * vV[bb + 1] + el.z * vV[bb + 2] + el.w;
      } else if (lane < 30) {
        u = el.x * v + el.w + el.z * x;
      }
      vU[lane] = u;
      vX[lane] = x;
      __syncwarp();
      float xn = 0.f;
      if (lane < NC) xn = ak_mv(sm + S_AB, vA, vX, lane) + cm_mv_s(sm + S_B, vU, lane) + vA[32 + lane];
      else if (arm) xn = x + dt * u;
      ap.xt[(k + 1) * VS + lane] = xn;
      ap.ut[k * VS + lane] = u;
      x = xn;
      xo = xo_next;
      __syncwarp();
    }
}

// One iterative-refinement step of the polish solve: the residual of the
// reduced problem's v-stationarity, R_hat v + r_hat + B_hat^T lam_{k+1}, with
// the costate lam that makes its x-stationarity exact, is the linear term of a
// correction solved with the same factors (K_k, H_uu,k^-1); the rollout then
// applies it through the exact dynamics.
__device__ __noinline__ void polish_refine(const AgentPtrs& ap, float* sm, int lane, const LanePat& pat, Pipe& pp) {
  const int N = ap.N;
  const float* md = ap.mdl;
  const float dt = md[M_DT], mu = md[M_MU];
  float* vec = sm + S_VEC;
  float* cvec = vec + V_C * 64;
  int* act = reinterpret_cast<int*>(vec + V_ACT * 64);
  float* vS = vec + V_S * 64; float* vH = vec + V_H * 64; float* vV = vec + V_U * 64;
  const bool arm = lane >= NC && lane < 30;
  const float twoQ = lane < 30 ? 2.f * dt * md[M_Q + lane] : 0.f;
  float* const K0 = sm + S_P; float* const K1 = sm + S_X;
  float* const H0 = sm + S_H; float* const H1 = sm + S_K;
  float* vR = vec + V_ROW * 64;
  float lam = lane < 30 ? twoQ * (ap.xt[N * VS + lane] - ap.xref[N * VS + lane]) : 0.f;
  float pc = 0.f;
  Carry carry2 = {0, 0.f};
  // per-lane global inputs of a stage, loaded one stage ahead
  struct RefPre { StagePre pre; float v, xr, xt, e, e2; };
  auto load = [&](int k) {
    RefPre q;
    q.pre = stage_pre(ap, k, lane);
    q.v = ap.dv[k * VS + lane];
    q.xr = k >= 1 ? ap.xref[k * VS + lane] : 0.f;
    q.xt = k >= 1 ? ap.xt[k * VS + lane] : 0.f;
    q.e = ap.cE[k * 64 + lane];
    q.e2 = ap.cE[k * 64 + 32 + lane];
    return q;
  };
  pipe_issue(pp, 0, K0, ap.cK + (size_t)(N - 1) * BLK, H0, ap.cH + (size_t)(N - 1) * BLK, lane);
  RefPre cur = load(N - 1);
  for (int k = N - 1; k >= 0; --k) {
    const int b = (N - 1 - k) & 1;
    float* const Kc = b ? K1 : K0;
    float* const Hc = b ? H1 : H0;
    if (k >= 1)
      pipe_issue(pp, b ^ 1, b ? K0 : K1, ap.cK + (size_t)(k - 1) * BLK, b ? H0 : H1,
                 ap.cH + (size_t)(k - 1) * BLK, lane);
    const RefPre q = cur;
    if (k >= 1) cur = load(k - 1);
    const StagePre& pre = q.pre;
    stage_active_pre(pre, act, lane);
    set_stage_A_pre(sm, pre, lane);
    const Elim el = lane_elim(ap, pre, act, lane, mu, carry2);
    carry2 = el.carry_out;
    const StageIn in = polish_stage_in(ap, sm, cvec, el, lane, pat, pre.uref, pre.ck);
    const float v = q.v;
    vV[lane] = v;
    vS[lane] = lam;
    vR[lane] = pc;
    __syncwarp();
    float rv = 0.f, h = 0.f;
    if (lane < 12 && (lane % 6) < 3) {
      const int bb = (lane / 6) * 6, c = lane - bb;
      rv = in.rt_diag * v;
#pragma unroll
      for (int r3 = 0; r3 < 3; ++r3)
        if (r3 != c) rv = fmaf(in.rt_off[r3], vV[bb + r3], rv);
    } else if (lane < 30) {
      rv = in.rt_diag * v;
    }
    if (lane < NC) {
      rv += in.rh + cc_tv(sm + S_BV, pat.br, vS, lane);
      h = rv + cc_tv(sm + S_BV, pat.br, vR, lane);
    } else if (arm) {
      rv += in.rh + in.rt_off[0] * lam;
      h = rv + in.rt_off[0] * pc;
    }
    vH[lane] = h;
    float lamn = 0.f, pcn = 0.f;
    if (k >= 1 && lane < 30) {
      float ql = -twoQ * q.xr;
      if (el.qbox) ql -= 2.f * md[M_R + lane] * el.t;
      lamn = in.qt * q.xt + ql +
             (lane < NC ? cc_tv(sm + S_AV, pat.ar, vS, lane) : (el.qbox ? 0.f : lam));
      pcn = lane < NC ? cc_tv(sm + S_AV, pat.ar, vR, lane) : (el.qbox ? 0.f : pc);
    }
    pipe_wait(pp, b);
    __syncwarp();
    const float2 hk = r24_mtv2(Hc, Kc, vH, lane);
    float d = 0.f;
    if (lane < NC) d = -hk.x;
    else if (arm) d = -q.e2 * h;
    ap.cD[k * VS + lane] = d;
    if (k >= 1) {
      if (lane < NC) pcn += hk.y;
      else if (arm) pcn += q.e * h;
    }
    lam = lamn;
    pc = pcn;
    __syncwarp();
  }
  copy_n(sm + S_BV, ap.lin + L_BV, 136 / 4, lane);
  __syncwarp();
  
  polish_rollout(ap, sm, lane, pp, true);
}

// Factor and solve the reduced problem in one backward pass (the linear
// recursion rides along with the Riccati recursion, since the reduced problem
// is solved once), then roll forward with u = G v + t + Phi x through the
// original dynamics.  The polished primal goes to xt/ut.  Overwrites the
// Riccati caches (the caller refactors if ADMM continues).
template <int PREC>
__device__ __noinline__ bool polish_solve(const AgentPtrs& ap, float* sm, int lane, const LanePat& pat, Pipe& pp,
                                          const SolverParams& prm, int nref, int prec) {
  const int N = ap.N;
  const float* md = ap.mdl;
  const float dt = md[M_DT], mu = md[M_MU];
  float* P = sm + S_P; float* H = sm + S_H; float* K = sm + S_K;
  float* vec = sm + S_VEC;
  float* cvec = vec + V_C * 64;
  int* act = reinterpret_cast<int*>(vec + V_ACT * 64);
  float* vS = vec + V_S * 64; float* vH = vec + V_H * 64;
  const int j = lane < NC ? lane : NC - 1;
  const bool arm = lane >= NC && lane < 30;
  const float twoQ = lane < 30 ? 2.f * dt * md[M_Q + lane] : 0.f;

  // ---- backward: Riccati factor of the reduced problem (cost 2dt Q, 2dt R;
  // no sigma, no rho) and its linear recursion
  if (lane < NC) {
    for (int i = 0; i < NC; ++i) P[i * R24 + j] = 0.f;
    P[j * R24 + j] = 2.f * dt * md[M_Q + j];
  }
  float Pa = arm ? twoQ : 0.f;
  float p = lane < 30 ? -twoQ * ap.xref[N * VS + lane] : 0.f;
  Carry carry = {0, 0.f};
  __syncwarp();
  for (int k = N - 1; k >= 0; --k) {
    const StagePre pre = stage_pre(ap, k, lane);
    const float xr = lane < 30 ? ap.xref[k * VS + lane] : 0.f;   // used after the factor
    stage_active_pre(pre, act, lane);
    set_stage_A_pre(sm, pre, lane);
    const Elim el = lane_elim(ap, pre, act, lane, mu, carry);
    carry = el.carry_out;
    // the stage's elimination, for the forward pass: (g | G_f row 0, G_f row
    // 1, G_f row 2 | phi, t)
    {
      const bool fl = lane < 12 && (lane % 6) < 3;
      reinterpret_cast<float4*>(ap.cEl + k * 128)[lane] =
          make_float4(fl ? el.gf[0] : el.g, el.gf[1], fl ? el.gf[2] : el.phi, el.t);
    }
    const StageIn in = polish_stage_in(ap, sm, cvec, el, lane, pat, pre.uref, pre.ck);
    const StageOut so = factor_stage<PREC>(ap, sm, lane, k, in, &Pa, pat, prec, nref > 0);
    // H (= H_uu^-1) and K of stage k are still in smem
    const float s = p + so.e;
    vS[lane] = s;
    __syncwarp();
    float h = 0.f;
    if (lane < NC) h = in.rh + cc_tv(sm + S_BV, pat.br, vS, lane);
    else if (arm) h = in.rh + el.g * dt * s;
    vH[lane] = h;
    __syncwarp();
    float d = 0.f;
    if (lane < NC) d = -r24_mtv(H, vH, lane);
    else if (arm) d = -so.Hi * h;
    ap.dv[k * VS + lane] = d;
    if (k >= 1) {
      // linear cost of x_k (with the moved cost of an eliminated joint rate)
      float ql = -twoQ * xr;
      if (el.qbox) ql -= 2.f * md[M_R + lane] * el.t;
      if (lane < NC) p = ql + cc_tv(sm + S_AV, pat.ar, vS, lane) + r24_mtv(K, vH, lane);
      else if (arm) p = ql + (el.qbox ? 0.f : s) + so.Ka * h;
    }
    __syncwarp();
  }
  // restore the compact B of the original problem
  copy_n(sm + S_BV, ap.lin + L_BV, 136 / 4, lane);
  fence_proxy_async();   // K_k were written with generic stores; the rollout reads them by TMA
  __syncwarp();

  polish_rollout(ap, sm, lane, pp, false);
  for (int rs = 0; rs < nref; ++rs) polish_refine(ap, sm, lane, pat, pp);
  return !pp.timed_out();
}

// Optimality check of the polished point (xt, ut), one backward pass: KKT
// conditions of the guessed active set (stationarity in the free directions,
// right sign of the multipliers of the active rows, dynamics multipliers from
// the costate recursion) and primal feasibility of every row, each measured
// against its own tolerance (see Res).  With FIX (after a failed check) the
// active set is corrected for a next attempt: active rows whose multiplier
// has the wrong sign by more than tol_d are dropped, rows the point violates
// by more than tol_p are added; a chain of rate-bound stages under a joint
// limit that reaches the given q_0 over-determines q and loses its last rate
// row if the limit is overshot, else the limit row.  Dual and primal
// corrections touch disjoint rows; the stage's conditions are read from the
// copy in act taken before either.  *changed reports whether anything changed.  The thresholds are the tighter
// of the failed check's global tolerances (tol_p, tol_d) and kFixScale
// times the row's or component's own tolerance.
template <bool FIX>
__device__ __noinline__ Res polish_check(const AgentPtrs& ap, float* sm, int lane, const SolverParams& prm,
                                         int* changed, const LanePat& pat, float tol_p = 0.f,
                                         float tol_d = 0.f) {
  const int N = ap.N;
  const float* md = ap.mdl;
  const float dt = md[M_DT], mu = md[M_MU];
  const float ea = prm.eps_abs, er = prm.eps_rel;
  float* vec = sm + S_VEC;
  float* vU = vec + V_U * 64; float* vXN = vec + V_XN * 64; float* vM = vec + V_S * 64;
  float* vG = vec + V_G * 64; float* vT = vec + V_T * 64;
  float* vMa = vec + V_H * 64;   // magnitude of the terms of the costate (sums of absolute values)
  int* act = reinterpret_cast<int*>(vec + V_ACT * 64);
  const float twoQ = lane < 30 ? 2.f * dt * md[M_Q + lane] : 0.f;
  const float twoR = lane < 30 ? 2.f * dt * md[M_R + lane] : 0.f;
  const float* xs = ap.xt;
  const float* us = ap.ut;
  float rp = 0.f, ps = 0.f, rd = 0.f, ds = 0.f, pn = 0.f, dn = 0.f;
  int chg = 0;
  float m = lane < 30 ? twoQ * (xs[N * VS + lane] - ap.xref[N * VS + lane]) : 0.f;
  float ma = lane < 30 ? fabsf(twoQ * xs[N * VS + lane]) + fabsf(twoQ * ap.xref[N * VS + lane]) : 0.f;
  // a chain of stages kc..ke whose joint rate sits at its bound while the
  // joint limit of stage ke is active (see Elim): the limit's multiplier is
  // nu, the multiplier nu' of the constraint carried to stage kc-1, and each
  // rate row's is its own stationarity value minus dt nu; ch_up / ch_lo hold
  // the least / greatest of those values over the chain's rate rows at an
  // upper / lower bound, ch_tol the largest tolerance among them
  int ch_on = 0, ch_ke = 0, ch_side = 0, ch_over = 0;
  float ch_up = 0.f, ch_lo = 0.f, ch_tol = 0.f;
  for (int k = N - 1; k >= 0; --k) {
    // every global input of stage k, loaded together (one memory round trip)
    const StagePre pre = stage_pre(ap, k, lane);
    const float u_k = us[k * VS + lane], x_n = xs[(k + 1) * VS + lane];
    const float xr_n = ap.xref[(k + 1) * VS + lane];
    const float x_k = k >= 1 ? xs[k * VS + lane] : 0.f, xr_k = k >= 1 ? ap.xref[k * VS + lane] : 0.f;
    float rlo[2], rhi[2], rcl[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = lane + 32 * h;
      const bool in = r < NR;
      rlo[h] = in ? ap.rlo[k * RS + r] : 0.f;
      rhi[h] = in ? ap.rhi[k * RS + r] : 0.f;
      rcl[h] = in ? ap.rcls[k * RS + r] : 0.f;
    }
    stage_active_pre(pre, act, lane);
    set_stage_A_pre(sm, pre, lane);
    vM[lane] = m;
    vMa[lane] = ma;
    vU[lane] = u_k;
    vXN[lane] = x_n;
    __syncwarp();
    int* ak = ap.act + k * RS;
    // primal feasibility of the rows of stage k
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = lane + 32 * h;
      if (r >= NR) break;
      const float v = crow(vU, vXN, r, mu);
      const float lo = rlo[h], hi = rhi[h];
      if (rcl[h] > 0.f) ps = fmaxf(ps, fabsf(v));
      const float viol = fmaxf(fmaxf(lo - v, v - hi), 0.f);
      float sc = fabsf(v);
      if (isfinite(lo)) sc = fmaxf(sc, fabsf(lo));
      if (isfinite(hi)) sc = fmaxf(sc, fabsf(hi));
      const float tp = ea + er * sc;
      rp = fmaxf(rp, viol);
      pn = fmaxf(pn, viol / tp);
      if (FIX && viol > fminf(tol_p, kFixScale * tp) && act[r] == 0) {
        ak[r] = (v < lo) ? 1 : 2;
        chg = 1;
      }
    }
    // stationarity of the inputs without their row multipliers, and its tolerance
    float g = 0.f, td = 1.f;
    if (lane < 30) {
      const float u = u_k, ur = pre.uref;
      const float btm = lane < NC ? cc_tv(sm + S_BV, pat.br, vM, lane) : dt * m;
      const float bta = lane < NC ? cc_tv_abs(sm + S_BV, pat.br, vMa, lane) : dt * ma;
      g = twoR * (u - ur) + btm;
      td = ea + er * fmaxf(fmaxf(fabsf(twoR * u), fabsf(twoR * ur)), bta);
      ds = fmaxf(ds, fmaxf(fabsf(twoR * u), fabsf(twoR * ur)));
      ds = fmaxf(ds, fmaxf(fabsf(twoQ * x_n), fabsf(twoQ * xr_n)));
    }
    vG[lane] = g;
    vT[lane] = td;
    __syncwarp();
    // joint rates: input i in 12..29 (row i + 8); multiplier y = -g.  With
    // the joint box of stage k active (row i + 26, on x_{k+1}), the rate is
    // eliminated: its stationarity 2dt R u + dt (m + y_q) = 0 gives the
    // joint-box multiplier y_q, and the costate takes it (m <- m + y_q).
    if (lane >= 12 && lane < 30) {
      const int a = act[lane + 8], aq = act[lane + 26];
      // chain end: the joint limit's multiplier nu and the chain's rate rows
      auto close_chain = [&](float nu, float tol_nu) {
        const float bq = (ch_side & 1) ? fmaxf(nu, 0.f) : fmaxf(-nu, 0.f);
        const float br = fmaxf(fmaxf(dt * nu - ch_up, 0.f), fmaxf(ch_lo - dt * nu, 0.f));
        rd = fmaxf(rd, fmaxf(bq, br));
        dn = fmaxf(dn, fmaxf(bq / tol_nu, br / ch_tol));
        if (FIX && bq > fminf(tol_d, kFixScale * tol_nu)) { ap.act[ch_ke * RS + lane + 26] = 0; chg = 1; }
        if (FIX && br > fminf(tol_d, kFixScale * ch_tol)) { ap.act[ch_ke * RS + lane + 8] = 0; chg = 1; }
        ch_on = 0;
      };
      if (a && (ch_on || aq)) {
        // rate at its bound under a joint limit (own, or carried): the chain
        // goes on to stage k-1; the rate's own stationarity value is -g
        if (!ch_on) {
          ch_on = 1; ch_ke = k; ch_side = aq; ch_up = 3.0e38f; ch_lo = -3.0e38f; ch_tol = 0.f;
          const float qn = vXN[lane];                       // q_{k+1} of this joint
          ch_over = (aq & 1) ? (qn < pre.lo_q) : (qn > pre.hi_q);
        }
        if (a & 2) ch_up = fminf(ch_up, -g);
        else ch_lo = fmaxf(ch_lo, -g);
        ch_tol = fmaxf(ch_tol, td);
        if (k == 0) {
          // q_0 is given: nothing carries the limit further, the chain
          // over-determines q_{ke+1}
          if (FIX) { ap.act[ch_ke * RS + lane + (ch_over ? 8 : 26)] = 0; chg = 1; }
          close_chain(0.f, td);
        }
      } else if (ch_on || aq) {
        // joint rate eliminated by the joint limit (own, or carried to here)
        const float tu = -2.f * md[M_R + lane] * u_k;
        const float yq = tu - m;
        const float tol = ea + er * fmaxf(fabsf(tu), ma);
        if (ch_on) {
          close_chain(yq, tol);
        } else {
          const float bad = (aq & 1) ? fmaxf(yq, 0.f) : fmaxf(-yq, 0.f);   // lower: y_q <= 0; upper: >= 0
          rd = fmaxf(rd, bad);
          dn = fmaxf(dn, bad / tol);
          if (FIX && bad > fminf(tol_d, kFixScale * tol)) { ak[lane + 26] = 0; chg = 1; }
        }
        m += yq;
        ma += fabsf(tu);
      } else {
        float bad;
        if (a & 1) bad = fmaxf(-g, 0.f);           // needs y <= 0 at a lower bound
        else if (a & 2) bad = fmaxf(g, 0.f);       // needs y >= 0 at an upper bound
        else bad = fabsf(g);
        rd = fmaxf(rd, bad);
        dn = fmaxf(dn, bad / td);
        if (FIX && a && bad > fminf(tol_d, kFixScale * td)) { ak[lane + 8] = 0; chg = 1; }
      }
    }
    // feet: lane f in 0..1
    if (lane < 2) {
      const int f = lane, b = 6 * f, p = 12 + 4 * f;
      const FootAct fa = foot_act(act, f);
      const float gx = vG[b], gy = vG[b + 1], gz = vG[b + 2];
      const float tf = fmaxf(fmaxf(vT[b], vT[b + 1]), vT[b + 2]);
      const float thr = fminf(tol_d, kFixScale * tf);
      if (!fa.swing) {
        for (int c = 3; c < 6; ++c) {                                  // free moments
          rd = fmaxf(rd, fabsf(vG[b + c]));
          dn = fmaxf(dn, fabsf(vG[b + c]) / vT[b + c]);
        }
        if (fa.zero) {
          // -g in the normal cone of the pyramid at 0: g . ray >= 0 on its 4 rays
          float worst = 0.f;
          for (int sx = -1; sx <= 1; sx += 2)
            for (int sy = -1; sy <= 1; sy += 2) worst = fmaxf(worst, -(sx * mu * gx + sy * mu * gy + gz));
          rd = fmaxf(rd, worst);
          dn = fmaxf(dn, worst / tf);
          if (FIX && worst > thr) {
            ak[b + 2] &= ~1;
            if ((act[p] & 2) && (act[p + 1] & 2)) { ak[p] = 0; ak[p + 1] = 0; }
            if ((act[p + 2] & 2) && (act[p + 3] & 2)) { ak[p + 2] = 0; ak[p + 3] = 0; }
            chg = 1;
          }
        } else {
          const float ypx = fa.tx ? -fa.tx * gx : 0.f;
          const float ypy = fa.ty ? -fa.ty * gy : 0.f;
          if (fa.tx) {
            rd = fmaxf(rd, fmaxf(-ypx, 0.f));
            dn = fmaxf(dn, fmaxf(-ypx, 0.f) / tf);
            if (FIX && -ypx > thr) { ak[fa.tx > 0 ? p : p + 1] = 0; chg = 1; }
          } else {
            rd = fmaxf(rd, fabsf(gx));
            dn = fmaxf(dn, fabsf(gx) / vT[b]);
          }
          if (fa.ty) {
            rd = fmaxf(rd, fmaxf(-ypy, 0.f));
            dn = fmaxf(dn, fmaxf(-ypy, 0.f) / tf);
            if (FIX && -ypy > thr) { ak[fa.ty > 0 ? p + 2 : p + 3] = 0; chg = 1; }
          } else {
            rd = fmaxf(rd, fabsf(gy));
            dn = fmaxf(dn, fabsf(gy) / vT[b + 1]);
          }
          const float rz = gz - mu * (ypx + ypy);   // = -y_top when f_z sits at its upper bound
          if (fa.top) {
            rd = fmaxf(rd, fmaxf(rz, 0.f));
            dn = fmaxf(dn, fmaxf(rz, 0.f) / tf);
            if (FIX && rz > thr) { ak[b + 2] &= ~2; chg = 1; }
          } else {
            rd = fmaxf(rd, fabsf(rz));
            dn = fmaxf(dn, fabsf(rz) / tf);
          }
        }
      }
    }
    __syncwarp();
    vM[lane] = m;          // costate with the joint-box multipliers of stage k
    vMa[lane] = ma;
    __syncwarp();
    float mn = 0.f, mna = 0.f;
    if (k >= 1 && lane < 30) {
      mn = twoQ * (x_k - xr_k) +
           (lane < NC ? cc_tv(sm + S_AV, pat.ar, vM, lane) : m);
      mna = fabsf(twoQ * x_k) + fabsf(twoQ * xr_k) +
            (lane < NC ? cc_tv_abs(sm + S_AV, pat.ar, vMa, lane) : ma);
    }
    __syncwarp();
    m = mn;
    ma = mna;
  }
  Res out;
  out.rp = warp_max(rp); out.ps = warp_max(ps); out.rd = warp_max(rd); out.ds = warp_max(ds);
  out.pn = warp_max(pn); out.dn = warp_max(dn);
  if (changed) *changed = warp_or(chg);
  return out;
}

// Polish with active-set correction: up to four attempts (eight before any
// ADMM iteration); true when one passes its check, with the polished point copied into (x, u).
// Initial guess from the agent's previous final active set (kept per slot):
// rows that became equalities (a foot switched to swing) are active, rows
// that stopped being equalities start inactive, the rest keep their code.
__device__ void init_active_prev(const AgentPtrs& ap, int lane) {
  for (int k = 0; k < ap.N; ++k) {
    for (int r = lane; r < NR; r += 32) {
      const float lo = ap.rlo[k * RS + r], hi = ap.rhi[k * RS + r];
      int a = ap.act[k * RS + r];
      if (lo == hi) a = 3;
      else if (a == 3) a = 0;
      else {
        if (!isfinite(lo)) a &= ~1;
        if (!isfinite(hi)) a &= ~2;
      }
      ap.act[k * RS + r] = a;
    }
  }
  __syncwarp();
}

// A cold agent's first guess: only the equality rows (swing-foot wrenches).
__device__ void init_active_min(const AgentPtrs& ap, int lane) {
  for (int k = 0; k < ap.N; ++k)
    for (int r = lane; r < NR; r += 32)
      ap.act[k * RS + r] = ap.rlo[k * RS + r] == ap.rhi[k * RS + r] ? 3 : 0;
  __syncwarp();
}

// guess: POLISH_ADMM from ADMM's (w, y); POLISH_PREV the previous replan's
// final active set; POLISH_MIN the equality rows alone (cold agent)
enum : int { POLISH_ADMM = 0, POLISH_PREV = 1, POLISH_MIN = 2 };

// cap > 0: stop after cap reduced solves (the corrections of the last one
// are still applied to the active set, for a later continuation)
template <int PREC>
__device__ __noinline__ bool polish(const AgentPtrs& ap, float* sm, int lane, const SolverParams& prm, Res* res,
                       const LanePat& pat, Pipe& pp, int prec, int guess = POLISH_ADMM, int cap = 0) {
  if (guess == POLISH_PREV) init_active_prev(ap, lane);
  else if (guess == POLISH_MIN) init_active_min(ap, lane);
  else init_active(ap, lane);
  // before any ADMM iteration more corrections pay: the alternative is an
  // ADMM solve
  const int attempts = guess == POLISH_ADMM ? 4 : 8;
  const int stop = cap > 0 && cap < attempts ? cap : attempts;
  const int nref = guess == POLISH_PREV ? prm.refine : prm.refine_admm;
  for (int attempt = 0; attempt < stop; ++attempt) {
    if (!polish_solve<PREC>(ap, sm, lane, pat, pp, prm, nref, prec)) return false;
    const Res pr = polish_check<false>(ap, sm, lane, prm, nullptr, pat);
    const float tol_p = prm.eps_abs + prm.eps_rel * pr.ps;
    const float tol_d = prm.eps_abs + prm.eps_rel * pr.ds;
    const bool base = isfinite(pr.rp) && isfinite(pr.rd) && pr.rp <= tol_p && pr.rd <= tol_d;
    const bool loose = base && pr.pn <= kScaledLoose && pr.dn <= kScaledLoose;
    bool ok = base && pr.pn <= kScaledAccept && pr.dn <= kScaledAccept;
    int changed = 1;
    if (!ok && attempt + 1 < attempts) polish_check<true>(ap, sm, lane, prm, &changed, pat, tol_p, tol_d);
    if (!ok && loose && (!changed || attempt + 1 == attempts)) ok = true;
    if (ok) {
      for (int k = 1; k <= ap.N; ++k) ap.x[k * VS + lane] = ap.xt[k * VS + lane];
      for (int k = 0; k < ap.N; ++k) ap.u[k * VS + lane] = ap.ut[k * VS + lane];
      if (lane == 0) ap.st[T_ATTEMPTS] = attempt + 1;
      __syncwarp();
      *res = pr;
      return true;
    }
    if (attempt + 1 == attempts || !changed) break;
  }
  return false;
}

// ADMM warm start after a failed polish from the previous active set: the
// last polished point (xt, ut) with the row values w = clip(C z) and the row
// multipliers y of its active set (read from the same costate recursion and
// stationarity conditions as the optimality check, projected onto the sign
// each bound allows).  The (x, u, w, y) kept per agent are otherwise those of
// the last replan that ran ADMM, however many replans ago that was.
__device__ __noinline__ void polish_warm_start(const AgentPtrs& ap, float* sm, int lane, const LanePat& pat) {
  const int N = ap.N;
  const float* md = ap.mdl;
  const float dt = md[M_DT], mu = md[M_MU];
  float* vec = sm + S_VEC;
  float* vU = vec + V_U * 64; float* vXN = vec + V_XN * 64; float* vM = vec + V_S * 64;
  float* vG = vec + V_G * 64;
  int* act = reinterpret_cast<int*>(vec + V_ACT * 64);
  const float twoQ = lane < 30 ? 2.f * dt * md[M_Q + lane] : 0.f;
  const float twoR = lane < 30 ? 2.f * dt * md[M_R + lane] : 0.f;
  const float* xs = ap.xt;
  const float* us = ap.ut;
  float m = lane < 30 ? twoQ * (xs[N * VS + lane] - ap.xref[N * VS + lane]) : 0.f;
  int ch_on = 0, ch_ke = 0, ch_side = 0;   // open chain of rate-bound stages under a joint limit
  for (int k = N - 1; k >= 0; --k) {
    stage_active(ap, k, act, lane);
    set_stage_A(sm, ap.lin + L_STAGE + k * 64, lane);
    vM[lane] = m;
    vU[lane] = us[k * VS + lane];
    vXN[lane] = xs[(k + 1) * VS + lane];
    __syncwarp();
    float g = 0.f;
    if (lane < 30)
      g = twoR * (us[k * VS + lane] - ap.uref[k * VS + lane]) +
          (lane < NC ? cc_tv(sm + S_BV, pat.br, vM, lane) : dt * m);
    vG[lane] = g;
    __syncwarp();
    float* yk = ap.y + k * RS;
    float* wk = ap.w + k * RS;
    // joint rate rows (20..37) and joint-box rows (38..55); a chain's
    // multipliers as in the optimality check: the limit takes nu, each rate
    // row its own value minus dt nu
    if (lane >= 12 && lane < 30) {
      const int a = act[lane + 8], aq = act[lane + 26];
      auto close_chain = [&](float nu, int k0) {
        for (int i = k0; i <= ch_ke; ++i) {
          const int ai = ap.act[i * RS + lane + 8];
          const float v = ap.y[i * RS + lane + 8] - dt * nu;
          ap.y[i * RS + lane + 8] = (ai & 1) ? fminf(v, 0.f) : fmaxf(v, 0.f);
        }
        ap.y[ch_ke * RS + lane + 26] = (ch_side & 1) ? fminf(nu, 0.f) : fmaxf(nu, 0.f);
        ch_on = 0;
      };
      if (a && (ch_on || aq)) {
        if (!ch_on) { ch_on = 1; ch_ke = k; ch_side = aq; }
        yk[lane + 8] = -g;
        yk[lane + 26] = 0.f;
        if (k == 0) close_chain(0.f, 0);
      } else if (ch_on || aq) {
        const float v = -2.f * md[M_R + lane] * us[k * VS + lane] - m;
        m += v;
        yk[lane + 8] = 0.f;
        if (ch_on) {
          yk[lane + 26] = 0.f;
          close_chain(v, k + 1);
        } else {
          yk[lane + 26] = (aq & 1) ? fminf(v, 0.f) : fmaxf(v, 0.f);
        }
      } else {
        yk[lane + 8] = (a & 1) ? fminf(-g, 0.f) : ((a & 2) ? fmaxf(-g, 0.f) : 0.f);
        yk[lane + 26] = 0.f;
      }
    }
    // wrench rows (0..11) and friction-pyramid rows (12..19) of foot f
    if (lane < 2) {
      const int f = lane, b = 6 * f, p = 12 + 4 * f;
      const FootAct fa = foot_act(act, f);
      const float gx = vG[b], gy = vG[b + 1], gz = vG[b + 2];
      float yw[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, yp[4] = {0.f, 0.f, 0.f, 0.f};
      if (fa.swing) {
        for (int c = 0; c < 6; ++c) yw[c] = -vG[b + c];    // equality rows
      } else if (fa.zero) {
        yp[0] = fmaxf(-gx, 0.f); yp[1] = fmaxf(gx, 0.f);
        yp[2] = fmaxf(-gy, 0.f); yp[3] = fmaxf(gy, 0.f);
        yw[2] = fminf(-gz + mu * (yp[0] + yp[1] + yp[2] + yp[3]), 0.f);
      } else {
        if (fa.tx) yp[fa.tx > 0 ? 0 : 1] = fmaxf(-fa.tx * gx, 0.f);
        if (fa.ty) yp[fa.ty > 0 ? 2 : 3] = fmaxf(-fa.ty * gy, 0.f);
        const float rz = gz - mu * (yp[0] + yp[1] + yp[2] + yp[3]);
        if (fa.top) yw[2] = fmaxf(-rz, 0.f);
      }
      for (int c = 0; c < 6; ++c) yk[b + c] = yw[c];
      for (int t = 0; t < 4; ++t) yk[p + t] = yp[t];
    }
    for (int r = lane; r < NR; r += 32)
      wk[r] = fminf(fmaxf(crow(vU, vXN, r, mu), ap.rlo[k * RS + r]), ap.rhi[k * RS + r]);
    __syncwarp();
    vM[lane] = m;
    __syncwarp();
    float mn = 0.f;
    if (k >= 1 && lane < 30)
      mn = twoQ * (xs[k * VS + lane] - ap.xref[k * VS + lane]) +
           (lane < NC ? cc_tv(sm + S_AV, pat.ar, vM, lane) : m);
    __syncwarp();
    m = mn;
  }
  for (int k = 1; k <= N; ++k) ap.x[k * VS + lane] = xs[k * VS + lane];
  for (int k = 0; k < N; ++k) ap.u[k * VS + lane] = us[k * VS + lane];
  __syncwarp();
}

// ============================================================ ADMM driver (A5, A6)
// Iterations with a residual check every check_every; OSQP's rho update
// (refactor when the ratio is off by 5x); polish attempts once both residuals
// are within early_polish x the tolerance.  Returns the agent status.
struct Outcome { int status, iters, refac, polished, prec; Res r; };

// Factor precision after a failed polish first: a TF32 or BF16 factor that
// did not give the optimum at once is not trusted for ADMM (an inexact
// factor can make ADMM diverge), so the agent's fallback factors in FP32.
__device__ __forceinline__ int fallback_precision(int p) {
  return (p == PREC_TF32 || p == PREC_BF16) ? PREC_FP32 : p;
}

template <int PREC>
__device__ Outcome admm_solve(const AgentPtrs& ap, float* sm, int lane, const SolverParams& prm, bool factored,
                              Pipe& pp, const LanePat& pat) {
  float rho = *ap.rho;
  Outcome o;
  o.status = MPC_AGENT_MAX_ITER_; o.iters = 0; o.refac = 0; o.polished = 0; o.prec = prm.precision;
  o.r.rp = o.r.rd = o.r.ps = o.r.ds = o.r.pn = o.r.dn = 0.f;
  // polish first: a warm start's previous final active set is usually still
  // right, and a cold agent's optimum has few active rows; a polish from that
  // guess (with its corrections) that passes the KKT check is the optimum,
  // with no ADMM factorisation and no iteration
  if (lane == 0) { ap.st[T_FIRST] = 0; ap.st[T_ATTEMPTS] = 0; }
  if (prm.polish && prm.warm_polish && prm.fixed_iters == 0) {
    Res pr;
    if (polish<PREC>(ap, sm, lane, prm, &pr, pat, pp, o.prec, ap.st[T_WARM] ? POLISH_PREV : POLISH_MIN,
                     prm.defer == 2 || (prm.defer == 3 && !ap.st[T_WARM]) ? 2 : 0)) {
      o.polished = 1;
      o.status = MPC_AGENT_SOLVED_;
      o.r = pr;
      if (lane == 0) ap.st[T_FIRST] = 1;
      return o;
    }
    if (pp.timed_out()) { o.status = MPC_AGENT_TIMEOUT_; return o; }
    // deferred after a capped polish: the corrected active set is kept; a
    // later solve of this agent (same inputs, no flag) continues from it
    if (prm.defer >= 2) { o.status = MPC_AGENT_DEFERRED_; return o; }
    factored = false;   // the polish overwrote the caches
    o.prec = fallback_precision(o.prec);
    polish_warm_start(ap, sm, lane, pat);
    // deferred: the ADMM start is in the warm-start arrays; a later solve of
    // this agent without the polish first runs the ADMM from it
    if (prm.defer == 1) { o.status = MPC_AGENT_DEFERRED_; return o; }
  }
  if (!factored) factor_admm<PREC>(ap, sm, lane, rho, prm.sigma, pat, o.prec);
  const bool fixed = prm.fixed_iters > 0;
  const int max_it = fixed ? prm.fixed_iters : prm.max_iter;
  // polish attempts: the first once both residuals are within early_polish x
  // the tolerance, then again every 100 iterations while they stay there (the
  // active-set guess improves as ADMM proceeds; in FP32 ADMM can plateau just
  // above the tolerance).  The spacing doubles every second attempt, so the
  // attempts cost a bounded share of the iterations; it starts at 20
  // iterations for a warm-started agent (close to its optimum), 100 cold.
  const int polish_every = ap.st[T_WARM] ? 20 : 100;
  int polish_tries = 0, next_polish_it = 0;
  int it = 0;
  for (it = 1; it <= max_it; ++it) {
    const bool check = (!fixed && (it % prm.check_every == 0)) || it == max_it;
    admm_iteration(ap, sm, lane, rho, prm, pp, pat, check && !fixed);
    if (pp.timed_out()) { o.status = MPC_AGENT_TIMEOUT_; break; }
    if (!check) continue;
    o.r = admm_residuals(ap, sm, lane, prm, pat);
    if (!(isfinite(o.r.rp) && isfinite(o.r.rd))) { o.status = MPC_AGENT_NAN_; break; }
    if (fixed) break;
    // OSQP's stopping rule (global scales), and every row and component
    // within kAdmmScaledStop times its own tolerance
    const float tol_p = prm.eps_abs + prm.eps_rel * o.r.ps;
    const float tol_d = prm.eps_abs + prm.eps_rel * o.r.ds;
    if (o.r.rp <= tol_p && o.r.rd <= tol_d && o.r.pn <= kAdmmScaledStop && o.r.dn <= kAdmmScaledStop) {
      o.status = MPC_AGENT_SOLVED_;
      break;
    }
    // a primal residual that stays above its acceptance level: test the
    // last iteration's multiplier change for an infeasibility certificate
    if (o.r.pn > kAdmmScaledStop && admm_primal_infeasible(ap, sm, lane, pat)) {
      o.status = MPC_AGENT_PRIMAL_INFEAS_;
      break;
    }
    if (prm.polish && prm.early_polish > 0.f && polish_tries < 24 && it >= next_polish_it &&
        o.r.rp <= prm.early_polish * tol_p && o.r.rd <= prm.early_polish * tol_d) {
      ++polish_tries;
      next_polish_it = it + (polish_every << (polish_tries >> 1));
      Res pr;
      if (polish<PREC>(ap, sm, lane, prm, &pr, pat, pp, o.prec)) {
        o.polished = 1;
        o.status = MPC_AGENT_SOLVED_;
        o.r = pr;
        break;
      }
      if (pp.timed_out()) { o.status = MPC_AGENT_TIMEOUT_; break; }
      factor_admm<PREC>(ap, sm, lane, rho, prm.sigma, pat, o.prec);   // the polish overwrote the caches
      ++o.refac;
    }
    if (prm.adaptive_rho && it < max_it) {
      const float num = o.r.rp / fmaxf(o.r.ps, 1e-30f);
      const float den = o.r.rd / fmaxf(o.r.ds, 1e-30f);
      float rn = rho * sqrtf(num / fmaxf(den, 1e-30f));
      rn = fminf(fmaxf(rn, 1e-6f), 1e6f);
      if (rn > 5.f * rho || rn < 0.2f * rho) {
        rho = rn;
        factor_admm<PREC>(ap, sm, lane, rho, prm.sigma, pat, o.prec);
        ++o.refac;
      }
    }
  }
  o.iters = it > max_it ? max_it : it;
  if (lane == 0) *ap.rho = rho;
  return o;
}

// ============================================================ torque map (A7)
// q_MPC = x0.q; qdot_MPC = u_0.qdot; qddot = (u_1.qdot - u_0.qdot)/dt;
// tau = K_p (q_MPC - q) + K_d (qdot_MPC - qdot) + [M qddot + h] - J_leg^T W
// (Eqs. rnea, mpc_torque); value = QP objective at the solution.  M qddot + h
// comes from the recursive Newton-Euler algorithm over the agent's kinematic
// tree when it has one (mpc_k_rnea, a kernel of its own after the solve: run
// once per agent inside the persistent kernel its code was always cold in the
// instruction cache, 5x its cost alone), else from the diagonal joint model
// M_j qddot_j + h_j.

// 3-vector helpers of the Newton-Euler recursion
struct V3 { float x, y, z; };
__device__ __forceinline__ V3 v3(float x, float y, float z) { V3 r; r.x = x; r.y = y; r.z = z; return r; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 mv3(const M3& R, V3 a) {
  return v3(R.m[0] * a.x + R.m[1] * a.y + R.m[2] * a.z, R.m[3] * a.x + R.m[4] * a.y + R.m[5] * a.z,
            R.m[6] * a.x + R.m[7] * a.y + R.m[8] * a.z);
}
__device__ __forceinline__ V3 mtv3(const M3& R, V3 a) {   // R^T a
  return v3(R.m[0] * a.x + R.m[3] * a.y + R.m[6] * a.z, R.m[1] * a.x + R.m[4] * a.y + R.m[7] * a.z,
            R.m[2] * a.x + R.m[5] * a.y + R.m[8] * a.z);
}
__device__ __forceinline__ V3 ld3(const float* p) { return v3(p[0], p[1], p[2]); }

// Inverse dynamics of one chain of the tree (joints j0 .. j0+len-1, the
// first hanging off the base) by the recursive Newton-Euler algorithm in
// world coordinates (Luh, Walker and Paul 1980; Featherstone 2008, Ch. 5):
// outward, each link's rotation, angular velocity and acceleration, the
// acceleration of its joint origin and of its centre of mass; inward, the
// force and moment each link transmits to its parent, the joint torque being
// the moment's component along the joint axis.  The base's motion is given:
// rotation Rb, angular velocity wb, angular acceleration dwb and linear
// acceleration ab of its origin, gravity folded into ab as an upward
// acceleration.  tau[t] receives the torque of joint j0 + t.
__device__ __noinline__ void chain_rnea(const float* tr, int j0, int len, const M3& Rb, V3 wb, V3 dwb, V3 ab,
                                        const float* q, const float* qd, const float* qdd, float* tau) {
  // compact loops (not unrolled): this runs once per agent, and unrolled
  // straight-line code here costs more in instruction fetch than in arithmetic
  V3 z[5], d[5], rc[5], F[5], Nm[5];
  M3 R = Rb;
  V3 w = wb, al = dwb, acc = ab;
#pragma unroll 1
  for (int t = 0; t < len; ++t) {
    const float* J = tr + (j0 + t) * TREE_J;
    const V3 ax = ld3(J + TA_AXIS);
    d[t] = mv3(R, ld3(J + TA_OFF));                    // parent origin -> joint origin
    acc = acc + cross(al, d[t]) + cross(w, cross(w, d[t]));
    z[t] = mv3(R, ax);
    const V3 wj = qd[t] * z[t];
    al = al + qdd[t] * z[t] + cross(w, wj);
    w = w + wj;
    // R <- R Rot(ax, q) (Rodrigues): column c of the product is R (Rot e_c)
    float s, c;
    sincosf(q[t], &s, &c);
    const float k = 1.f - c;
    M3 Rn;
#pragma unroll 1
    for (int col = 0; col < 3; ++col) {
      const float e0 = col == 0, e1 = col == 1, e2 = col == 2;
      // Rot e = c e + s (ax x e) + k (ax . e) ax
      const float ad = ax.x * e0 + ax.y * e1 + ax.z * e2;
      const V3 rcol = v3(c * e0 + s * (ax.y * e2 - ax.z * e1) + k * ad * ax.x,
                         c * e1 + s * (ax.z * e0 - ax.x * e2) + k * ad * ax.y,
                         c * e2 + s * (ax.x * e1 - ax.y * e0) + k * ad * ax.z);
      const V3 o = mv3(R, rcol);
      Rn.m[col] = o.x;
      Rn.m[3 + col] = o.y;
      Rn.m[6 + col] = o.z;
    }
    R = Rn;
    const float m = J[TA_MASS];
    rc[t] = mv3(R, ld3(J + TA_COM));                   // joint origin -> centre of mass
    const V3 ac = acc + cross(al, rc[t]) + cross(w, cross(w, rc[t]));
    F[t] = m * ac;
    // N = I_w al + w x (I_w w), I_w = R diag(I) R^T
    const V3 Id = ld3(J + TA_INER);
    const V3 bl = mtv3(R, al), bw = mtv3(R, w);
    const V3 Ial = mv3(R, v3(Id.x * bl.x, Id.y * bl.y, Id.z * bl.z));
    const V3 Iw = mv3(R, v3(Id.x * bw.x, Id.y * bw.y, Id.z * bw.z));
    Nm[t] = Ial + cross(w, Iw);
  }
  V3 f = v3(0.f, 0.f, 0.f), n = v3(0.f, 0.f, 0.f), dn = v3(0.f, 0.f, 0.f);
#pragma unroll 1
  for (int t = len - 1; t >= 0; --t) {
    // moment about joint t's origin: its own link's, plus the child's
    // (transmitted from the child's joint origin, dn = d[t+1] away)
    const V3 nt = Nm[t] + cross(rc[t], F[t]) + n + cross(dn, f);
    f = F[t] + f;
    n = nt;
    dn = d[t];
    tau[t] = dot(z[t], nt);
  }
}

__device__ __noinline__ void torque_map(const AgentPtrs& ap, int lane) {
  const int N = ap.N;
  const float* md = ap.mdl;
  const float dt = md[M_DT];
  // M qddot + h of joint `lane` (lanes 0-17): the diagonal joint model, or,
  // for an agent with a kinematic tree, nothing here: mpc_k_rnea adds the
  // tree's inverse dynamics after the solve
  float inv = 0.f;
  if (md[M_TREE_ON] != 0.f) {
  } else if (lane < 18) {
    inv = md[M_MJ + lane] * ((ap.u[VS + 12 + lane] - ap.u[12 + lane]) / dt) + md[M_HJ + lane];
  }
  if (lane < 18) {
    const int j = lane;
    const float q = ap.inp[I_X0 + 12 + j];
    const float qd0 = ap.u[12 + j];
    float tau = md[M_KP + j] * (q - q) + md[M_KD + j] * (qd0 - ap.inp[I_QD + j]) + inv;
    if (j < 10) {
      const int f = j / 5, jj = j - 5 * f;
      for (int r = 0; r < 6; ++r) tau -= md[M_JLEG + 30 * f + 5 * r + jj] * ap.u[6 * f + r];
    }
    ap.out[O_TAU + j] = tau;
    ap.out[O_QSET + j] = q;
    ap.out[O_QDSET + j] = qd0;
  }
  float v = 0.f;
  if (lane < 30) {
    const float q = md[M_Q + lane], r = md[M_R + lane];
    for (int k = 0; k <= N; ++k) {
      const float e = ap.x[k * VS + lane] - ap.xref[k * VS + lane];
      v = fmaf(dt * q * e, e, v);
    }
    for (int k = 0; k < N; ++k) {
      const float e = ap.u[k * VS + lane] - ap.uref[k * VS + lane];
      v = fmaf(dt * r * e, e, v);
    }
  }
  v = warp_sum(v);
  if (lane == 0) ap.out[O_V] = v;
}

__device__ void mark_status_only(const AgentPtrs& ap, int lane, int status) {
  if (lane < 18) { ap.out[O_TAU + lane] = 0.f; ap.out[O_QSET + lane] = 0.f; ap.out[O_QDSET + lane] = 0.f; }
  if (lane == 0) {
    ap.out[O_V] = 0.f;
    ap.st[T_STATUS] = status;
    ap.st[T_ITERS] = 0; ap.st[T_REFAC] = 0; ap.st[T_POLISHED] = 0;
    *ap.warm = 0;
  }
  __syncwarp();
}

// copy the batch row's inputs into the agent's input record
__device__ __forceinline__ void load_inputs(const Batch& b, int row, const AgentPtrs& ap, int lane) {
  if (lane < 30) ap.inp[I_X0 + lane] = b.x0[(size_t)row * 30 + lane];
  if (lane < 18) ap.inp[I_QD + lane] = b.qd[(size_t)row * 18 + lane];
  if (lane < 4) ap.inp[I_CMD + lane] = b.cmd[(size_t)row * 4 + lane];
  if (lane == 0) ap.inp[I_PHASE] = b.phase[row];
  __syncwarp();
}

__device__ void write_outcome(const AgentPtrs& ap, int lane, const Outcome& o) {
  __syncwarp();
  if (lane == 0) {
    ap.st[T_STATUS] = o.status;
    ap.st[T_ITERS] = o.iters;
    ap.st[T_REFAC] = o.refac;
    ap.st[T_POLISHED] = o.polished;
    ap.out[O_PRIM] = o.r.rp;
    ap.out[O_DUAL] = o.r.rd;
    ap.out[O_PRIM_N] = o.r.pn;
    ap.out[O_DUAL_N] = o.r.dn;
    *ap.warm = (o.status == MPC_AGENT_NAN_ || o.status == MPC_AGENT_TIMEOUT_ ||
                o.status == MPC_AGENT_PRIMAL_INFEAS_) ? 0 : ap.N;
  }
  __syncwarp();
}

// final polish when ADMM ended without an accepted one
template <int PREC>
__device__ void final_polish(const AgentPtrs& ap, float* sm, int lane, const SolverParams& prm, Outcome& o,
                             const LanePat& pat, Pipe& pp) {
  if (!prm.polish || o.polished || o.status == MPC_AGENT_NAN_ || o.status == MPC_AGENT_TIMEOUT_ ||
      o.status == MPC_AGENT_PRIMAL_INFEAS_ || o.status == MPC_AGENT_DEFERRED_)
    return;
  Res pr;
  if (polish<PREC>(ap, sm, lane, prm, &pr, pat, pp, o.prec)) {
    o.polished = 1;
    o.status = MPC_AGENT_SOLVED_;
    o.r = pr;
  } else if (pp.timed_out()) {
    o.status = MPC_AGENT_TIMEOUT_;
  }
}

// SOLVED is kept for a point that passed the polish's KKT check (exact on its
// active set up to rounding); an ADMM iterate that met the stopping test
// without such a check is only as accurate as that test
__device__ __forceinline__ void certify(Outcome& o) {
  if (o.status == MPC_AGENT_SOLVED_ && !o.polished) o.status = MPC_AGENT_INACCURATE_;
}

// An agent whose bounded wait gave up: its outputs are zeroed (the torque
// kernel does the same for the fused form), the copies still in flight into
// the warp's buffers are drained, and the event is counted.  The caller then
// retires the warp: it takes no further agent, so the timed-out barriers are
// never reused.
__device__ void retire_timed_out(const Arena& a, const AgentPtrs& ap, Pipe& pp, int lane) {
  if (lane < 18) { ap.out[O_TAU + lane] = 0.f; ap.out[O_QSET + lane] = 0.f; ap.out[O_QDSET + lane] = 0.f; }
  if (lane == 0) {
    ap.out[O_V] = 0.f;
    atomicAdd(a.fault + F_WAIT_TIMEOUTS, 1);
  }
  pipe_drain(pp);
}

// ============================================================ kernels
extern __shared__ __align__(16) float g_smem[];

// a batch row names a live slot (admitted by mpc_set_models, in range)
__device__ __forceinline__ bool valid_slot(const Arena& a, const Batch& b, int row) {
  const int s = b.ids[row];
  return s >= 0 && s < a.max_agents && a.horizon[s] >= 2 && a.horizon[s] <= a.maxN;
}
__device__ __forceinline__ float* warp_smem() { return g_smem + (threadIdx.x >> 5) * W_FLOATS; }

template <int MINB, int PREC>
__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32, MINB) mpc_k_fused(Arena a, Batch b, SolverParams prm) {
  // persistent: each warp takes the next batch row from the work queue
  // (longest expected solve first) until the queue is empty
  const int lane = threadIdx.x & 31;
  float* sm = warp_smem();
  const LanePat pat = lane_pattern(lane);
  Pipe pp;
  pipe_init(pp, sm, lane, prm.spin_limit);
  int static_row = blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  const int nw = gridDim.x * WARPS_PER_BLOCK;
  for (;;) {
    int idx;
    if (b.counter) {
      idx = 0;
      if (lane == 0) idx = atomicAdd(b.counter, 1);
      idx = __shfl_sync(FULL, idx, 0);
    } else {
      idx = static_row;
      static_row += nw;
    }
    if (idx >= b.n) break;
    const int row = b.order ? b.order[idx] : idx;
    if (!valid_slot(a, b, row)) continue;
    const AgentPtrs ap = agent_ptrs(a, b.ids[row]);
    pipe_set_dry(pp, b.ids[row] == prm.wait_test_slot);
    if (prm.split) {
      // set up by mpc_k_setup (the torque map follows in mpc_k_torque)
      if (ap.st[T_STATUS] == MPC_AGENT_NAN_) continue;
      load_lin(ap, sm, lane);
    } else {
      load_inputs(b, row, ap, lane);
      if (!setup_agent(ap, sm, lane, prm)) { mark_status_only(ap, lane, MPC_AGENT_NAN_); continue; }
    }
    Outcome o = admm_solve<PREC>(ap, sm, lane, prm, false, pp, pat);
    final_polish<PREC>(ap, sm, lane, prm, o, pat, pp);
    certify(o);
    write_outcome(ap, lane, o);
    if (o.status == MPC_AGENT_TIMEOUT_) {
      retire_timed_out(a, ap, pp, lane);
      break;
    }
    if (!prm.split) torque_map(ap, lane);
    __syncwarp();
  }
}

template <int MINB>
__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32, MINB) mpc_k_setup(Arena a, Batch b, SolverParams prm) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  if (row >= b.n || !valid_slot(a, b, row)) return;
  float* sm = warp_smem();
  const AgentPtrs ap = agent_ptrs(a, b.ids[row]);
  load_inputs(b, row, ap, lane);
  if (!setup_agent(ap, sm, lane, prm)) mark_status_only(ap, lane, MPC_AGENT_NAN_);
  else if (lane == 0) ap.st[T_STATUS] = MPC_AGENT_MAX_ITER_;
}

// Set-up of the fused form: the same per-agent work as mpc_k_setup, with a
// per-warp shared-memory window that starts at S_AB (set-up never touches the
// factor blocks below it): half the shared memory per warp, so about 20
// warps per SM instead of the solve kernels' 12 hide its memory latency
constexpr int W_SETUP = W_FLOATS - S_AB;
__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32) mpc_k_setup_lean(Arena a, Batch b, SolverParams prm) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  if (row >= b.n || !valid_slot(a, b, row)) return;
  // offsets from S_AB on land in this warp's window; nothing below S_AB is addressed
  float* sm = g_smem + (threadIdx.x >> 5) * W_SETUP - S_AB;
  const AgentPtrs ap = agent_ptrs(a, b.ids[row]);
  load_inputs(b, row, ap, lane);
  if (!setup_agent(ap, sm, lane, prm)) mark_status_only(ap, lane, MPC_AGENT_NAN_);
  else if (lane == 0) ap.st[T_STATUS] = MPC_AGENT_MAX_ITER_;
}

template <int MINB, int PREC>
__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32, MINB) mpc_k_factor(Arena a, Batch b, SolverParams prm) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  if (row >= b.n || !valid_slot(a, b, row)) return;
  float* sm = warp_smem();
  const AgentPtrs ap = agent_ptrs(a, b.ids[row]);
  if (ap.st[T_STATUS] == MPC_AGENT_NAN_) return;
  load_lin(ap, sm, lane);
  factor_admm<PREC>(ap, sm, lane, *ap.rho, prm.sigma, lane_pattern(lane), prm.precision);
}

template <int MINB, int PREC>
__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32, MINB) mpc_k_admm(Arena a, Batch b, SolverParams prm) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  if (row >= b.n || !valid_slot(a, b, row)) return;
  float* sm = warp_smem();
  const AgentPtrs ap = agent_ptrs(a, b.ids[row]);
  if (ap.st[T_STATUS] == MPC_AGENT_NAN_) return;
  load_lin(ap, sm, lane);
  const LanePat pat = lane_pattern(lane);
  Pipe pp;
  pipe_init(pp, sm, lane, prm.spin_limit);
  pipe_set_dry(pp, b.ids[row] == prm.wait_test_slot);
  const Outcome o = admm_solve<PREC>(ap, sm, lane, prm, true, pp, pat);
  write_outcome(ap, lane, o);
  if (o.status == MPC_AGENT_TIMEOUT_) retire_timed_out(a, ap, pp, lane);
}

template <int MINB, int PREC>
__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32, MINB) mpc_k_polish(Arena a, Batch b, SolverParams prm) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  if (row >= b.n || !valid_slot(a, b, row)) return;
  float* sm = warp_smem();
  const AgentPtrs ap = agent_ptrs(a, b.ids[row]);
  Outcome o;
  o.status = ap.st[T_STATUS];
  o.iters = ap.st[T_ITERS];
  o.refac = ap.st[T_REFAC];
  o.polished = ap.st[T_POLISHED];
  o.r.rp = ap.out[O_PRIM];
  o.r.rd = ap.out[O_DUAL];
  o.r.pn = ap.out[O_PRIM_N];
  o.r.dn = ap.out[O_DUAL_N];
  o.r.ps = o.r.ds = 0.f;
  o.prec = prm.warm_polish && prm.fixed_iters == 0 ? fallback_precision(prm.precision) : prm.precision;
  if (o.polished || o.status == MPC_AGENT_NAN_ || o.status == MPC_AGENT_TIMEOUT_ ||
      o.status == MPC_AGENT_PRIMAL_INFEAS_)
    return;
  if (!prm.polish) {
    certify(o);
    if (lane == 0) ap.st[T_STATUS] = o.status;
    return;
  }
  load_lin(ap, sm, lane);
  copy_n(sm + S_BV, ap.lin + L_BV, 136 / 4, lane);
  Pipe pp;
  pipe_init(pp, sm, lane, prm.spin_limit);
  final_polish<PREC>(ap, sm, lane, prm, o, lane_pattern(lane), pp);
  certify(o);
  if (o.polished) write_outcome(ap, lane, o);
  else if (lane == 0) ap.st[T_STATUS] = o.status;
  if (o.status == MPC_AGENT_TIMEOUT_) {
    write_outcome(ap, lane, o);
    retire_timed_out(a, ap, pp, lane);
  }
}

__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32) mpc_k_torque(Arena a, Batch b) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  if (row >= b.n || !valid_slot(a, b, row)) return;
  const AgentPtrs ap = agent_ptrs(a, b.ids[row]);
  const int st = ap.st[T_STATUS];
  if (st == MPC_AGENT_NAN_ || st == MPC_AGENT_TIMEOUT_ || st == MPC_AGENT_DEFERRED_) {
    // a failed or deferred solve leaves no torques: zeroed outputs, as the status says
    if (lane < 18) { ap.out[O_TAU + lane] = 0.f; ap.out[O_QSET + lane] = 0.f; ap.out[O_QDSET + lane] = 0.f; }
    if (lane == 0) ap.out[O_V] = 0.f;
    return;
  }
  torque_map(ap, lane);
}

}  // namespace

// ============================================================ variant launcher
// One translation unit instantiates one register-cap variant.
// Inverse dynamics of the agents' kinematic trees (Eq. rnea), added to the
// torques of the solve: four threads per agent, one per chain (left leg,
// right leg, left arm, right arm); the base moves as the MPC predicts
// (orientation and angular velocity of x0, accelerations (x_1 - x_0)/dt of
// its twist).  Agents without a tree, or whose solve failed (non-finite or
// timed out), are left alone.
static __global__ void __launch_bounds__(128) mpc_k_rnea(Arena a, Batch b) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = gt >> 2, c = gt & 3;
  if (row >= b.n || !valid_slot(a, b, row)) return;
  const AgentPtrs ap = agent_ptrs(a, b.ids[row]);
  const float* md = ap.mdl;
  if (md[M_TREE_ON] == 0.f) return;
  const int status = ap.st[T_STATUS];
  if (status == MPC_AGENT_NAN_ || status == MPC_AGENT_TIMEOUT_ || status == MPC_AGENT_DEFERRED_) return;
  const int j0 = c < 2 ? 5 * c : 10 + 4 * (c - 2), len = c < 2 ? 5 : 4;
  const float dt = md[M_DT], idt = 1.f / dt;
  const float* x0 = ap.inp + I_X0;
  const float* x1 = ap.x + VS;
  const float cr = cosf(x0[3]), sr = sinf(x0[3]), cp = cosf(x0[4]), sp = sinf(x0[4]);
  const float cy = cosf(x0[5]), sy = sinf(x0[5]);
  const M3 Rb = {{cy * cp, cy * sp * sr - sy * cr, cy * sp * cr + sy * sr,
                  sy * cp, sy * sp * sr + cy * cr, sy * sp * cr - cy * sr,
                  -sp, cp * sr, cp * cr}};
  const V3 wb = v3(x0[9], x0[10], x0[11]);
  const V3 dwb = v3((x1[9] - x0[9]) * idt, (x1[10] - x0[10]) * idt, (x1[11] - x0[11]) * idt);
  const V3 ab = v3((x1[6] - x0[6]) * idt, (x1[7] - x0[7]) * idt, (x1[8] - x0[8]) * idt + GRAV);
  float q[5], qd[5], qdd[5], tl[5];
  for (int t = 0; t < len; ++t) {
    q[t] = x0[12 + j0 + t];
    qd[t] = ap.u[12 + j0 + t];
    qdd[t] = (ap.u[VS + 12 + j0 + t] - qd[t]) * idt;
  }
  chain_rnea(md + M_TREE, j0, len, Rb, wb, dwb, ab, q, qd, qdd, tl);
  for (int t = 0; t < len; ++t) ap.out[O_TAU + j0 + t] += tl[t];
}

template <int MINB, int PREC>
cudaError_t configure_smem() {
  const int bytes = (int)smem_bytes_per_block();
  void (*ks[])(Arena, Batch, SolverParams) = {mpc_k_fused<MINB, PREC>, mpc_k_setup<MINB>, mpc_k_factor<MINB, PREC>,
                                              mpc_k_admm<MINB, PREC>, mpc_k_polish<MINB, PREC>};
  for (auto k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int MINB, int PREC>
cudaError_t launch_prec(const Arena& a, const Batch& b, const SolverParams& prm, int form, int grid_fused,
                        cudaStream_t st, int* launches) {
  // one-time set-up per device (also done before any stream capture by a
  // call with n = 0): smem opt-in and the resident grid of the persistent kernel
  static int configured = -1, resident = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t smem = smem_bytes_per_block();
  if (configured != dev) {
    cudaError_t e = configure_smem<MINB, PREC>();
    if (e != cudaSuccess) return e;
    int nsm = 0, per_sm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mpc_k_fused<MINB, PREC>, WARPS_PER_BLOCK * 32, smem);
    resident = nsm * (per_sm > 0 ? per_sm : 1);
    configured = dev;
  }
  if (b.n <= 0) return cudaSuccess;
  const int blocks = (b.n + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
  const dim3 thr(WARPS_PER_BLOCK * 32);
  if (form == 1) {
    // resident grid: the persistent warps drain the work queue.  Split:
    // the once-per-agent set-up and torque map run as kernels of their own
    // around it, where every warp runs the same code (inside the persistent
    // kernel that code was cold in the instruction cache for each agent)
    int g = b.counter ? resident : blocks;
    if (grid_fused > 0 && grid_fused < g) g = grid_fused;
    if (g > blocks) g = blocks;
    if (prm.split) {
      mpc_k_setup_lean<<<blocks, thr, WARPS_PER_BLOCK * W_SETUP * sizeof(float), st>>>(a, b, prm);
      if (launches) *launches += 1;
    }
    mpc_k_fused<MINB, PREC><<<g, thr, smem, st>>>(a, b, prm);
    if (launches) *launches += 1;
    if (prm.split) {
      mpc_k_torque<<<blocks, thr, 0, st>>>(a, b);
      if (launches) *launches += 1;
    }
  } else if (form == 2) {
    // the paper's literal solve: f_init / f_param / linearisation, then the
    // KKT system's block LDL^T and the OSQP iterations on it, then the torque map
    mpc_k_setup_lean<<<blocks, thr, WARPS_PER_BLOCK * W_SETUP * sizeof(float), st>>>(a, b, prm);
    cudaError_t e = launch_ldl(a, b, prm, st, launches);
    if (e != cudaSuccess) return e;
    mpc_k_torque<<<blocks, thr, 0, st>>>(a, b);
    if (launches) *launches += 2;
  } else {
    mpc_k_setup<MINB><<<blocks, thr, smem, st>>>(a, b, prm);
    mpc_k_factor<MINB, PREC><<<blocks, thr, smem, st>>>(a, b, prm);
    mpc_k_admm<MINB, PREC><<<blocks, thr, smem, st>>>(a, b, prm);
    mpc_k_polish<MINB, PREC><<<blocks, thr, smem, st>>>(a, b, prm);
    mpc_k_torque<<<blocks, thr, 0, st>>>(a, b);
    if (launches) *launches += 5;
  }
  if (prm.trees) {
    mpc_k_rnea<<<(b.n * 4 + 127) / 128, 128, 0, st>>>(a, b);
    if (launches) *launches += 1;
  }
  return cudaGetLastError();
}

// Kernel variants: the minimum resident blocks per SM given to the compiler
// (register cap), each in three builds: the FP32 factor only, the split-TF32
// tensor-core factor only, or the factor precision read at run time (TF32 /
// BF16 / FP64 paths).
template <int MINB>
cudaError_t launch_variant(const Arena& a, const Batch& b, const SolverParams& prm, int form, int grid_fused,
                           cudaStream_t st, int* launches) {
  if (prm.precision == PREC_FP32) return launch_prec<MINB, PREC_FP32>(a, b, prm, form, grid_fused, st, launches);
  if (prm.precision == PREC_TF32X3) return launch_prec<MINB, PREC_TF32X3>(a, b, prm, form, grid_fused, st, launches);
  return launch_prec<MINB, PREC_ANY>(a, b, prm, form, grid_fused, st, launches);
}

}  // namespace mpc
