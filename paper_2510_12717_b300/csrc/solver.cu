// Kernels of the batched MPC solver (sm_103a).  One warp per agent.
//
// Two launch forms of the same device steps:
//   plain : mpc_k_setup -> mpc_k_factor -> mpc_k_admm -> mpc_k_polish -> mpc_k_torque,
//           one launch per step, all intermediates in the global arenas;
//   fused : mpc_k_fused runs every step of an agent in one warp, keeping the
//           constant stage matrices in shared memory between steps.
#include "solver_dev.cuh"
#include "solver.h"

namespace mpc {

// ============================================================ small helpers
__device__ __forceinline__ float qt_x(const AgentPtrs& ap, int k, int i, float rho, float sigma, bool with_rows) {
  // diagonal of the x_k block of the ADMM KKT matrix (k >= 1): 2 dt Q + sigma
  // + rho on the joint-box row of stage k-1
  const float* md = ap.mdl;
  float v = 2.f * md[M_DT] * md[M_Q + i] + sigma;
  if (with_rows && i >= 12 && i < 30) v += rho * ap.rcls[(k - 1) * RS + i + 26];
  return v;
}

// A_k x (rows) or A_k^T x (columns) for the coupled block: A_base + dA_k,
// dA_k nonzero only in rows 9-11 (w) x columns 12-21 (leg joints).
template <bool T>
__device__ __forceinline__ float ak_mv(const float* Ab, const float* dA, const float* v, int lane) {
  float r = wmv<T>(Ab, v, lane);
  if (!T) {
    if (lane >= 9 && lane < 12) {
      const float* row = dA + (lane - 9) * 10;
#pragma unroll
      for (int c = 0; c < 10; ++c) r = fmaf(row[c], v[12 + c], r);
    }
  } else {
    if (lane >= 12 && lane < 22) {
      const int c = lane - 12;
      r = fmaf(dA[c], v[9], fmaf(dA[10 + c], v[10], fmaf(dA[20 + c], v[11], r)));
    }
  }
  return r;
}

// ============================================================ setup (A1, A2)
// Contact schedule, references, bounds (f_param), analytic linearisation
// about x0 and u_ref (f_KKT Jacobians), warm or cold start (f_init).
// Returns false (agent marked NaN) when an input is not finite.
__device__ bool setup_agent(const AgentPtrs& ap, float* sm, int lane, const SolverParams& prm) {
  const int N = ap.N;
  const float* md = ap.mdl;
  float* vec = sm + W_VEC;
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
  // stage bounds: lane k writes the 56 rows of stage k
  if (lane < N) {
    const int f = flags[lane];
    float* lo = ap.rlo + lane * RS;
    float* hi = ap.rhi + lane * RS;
    float* cl = ap.rcls + lane * RS;
    for (int i = 0; i < 2; ++i) {
      const int b = 6 * i, p = 12 + 4 * i;
      const bool stance = (f >> i) & 1;
      for (int c = 0; c < 6; ++c) {
        if (stance) {
          const bool z = (c == 2);
          lo[b + c] = z ? 0.f : -INFINITY;
          hi[b + c] = z ? fzmax : INFINITY;
          cl[b + c] = z ? 1.f : 0.f;
        } else {
          lo[b + c] = 0.f;
          hi[b + c] = 0.f;
          cl[b + c] = 1000.f;
        }
      }
      for (int t = 0; t < 4; ++t) {
        lo[p + t] = -INFINITY;
        hi[p + t] = stance ? 0.f : INFINITY;
        cl[p + t] = stance ? 1.f : 0.f;
      }
    }
    for (int j = 0; j < 18; ++j) {
      lo[20 + j] = -qdmax; hi[20 + j] = qdmax; cl[20 + j] = 1.f;
      lo[38 + j] = -qlim;  hi[38 + j] = qlim;  cl[38 + j] = 1.f;
    }
  }

  // references: desired trajectory (Eqs. des_traj_1..5) and force split
  const float dt = md[M_DT];
  const float ch = ap.inp[I_CMD], cvx = ap.inp[I_CMD + 1], cvy = ap.inp[I_CMD + 2], cwz = ap.inp[I_CMD + 3];
  for (int k = 0; k <= N; ++k) {
    const float yaw = xbar[5] + ((float)k * dt) * cwz;
    float v = 0.f;
    if (lane == 2) v = ch;
    else if (lane == 5) v = yaw;
    else if (lane == 6) v = cosf(yaw) * cvx - sinf(yaw) * cvy;
    else if (lane == 7) v = sinf(yaw) * cvx + cosf(yaw) * cvy;
    else if (lane == 11) v = cwz;
    else if (lane >= 12 && lane < 30) v = md[M_QNOM + lane - 12];
    ap.xref[k * VS + lane] = v;
  }
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
  // B = dt f_u: lane j fills column j
  float* Ab = sm + W_ABASE;
  float* Bm = sm + W_B;
  if (lane < NC) {
    const int j = lane;
    for (int i = 0; i < NC; ++i) {
      float a = (i == j) ? 1.f : 0.f;
      if (i < 3 && j == i + 6) a += dt;
      if (i >= 3 && i < 6 && j >= 3 && j < 6) a += dt * m3(dE, i - 3, j - 3);
      if (i >= 3 && i < 6 && j >= 9 && j < 12) a += dt * m3(Einv, i - 3, j - 9);
      if (i >= 9 && i < 12 && j >= 9 && j < 12) a += dt * m3(gyro, i - 9, j - 9);
      Ab[j * LD + i] = a;
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
      Bm[j * LD + i] = b;
    }
  }
  __syncwarp();
  // stash A_base and B for the separate-kernel form
  wcopy_block(ap.lin + L_ABASE, Ab, lane);
  wcopy_block(ap.lin + L_B, Bm, lane);

  // per stage: dA_k = dt dw/dq_leg (depends on the stance forces of u_ref_k)
  // and c_k = x0 + dt f(x0, u_ref_k) - A_k x0 - B u_ref_k
  for (int k = 0; k < N; ++k) {
    float* st = ap.lin + L_STAGE + k * 64;
    const float FL = ap.uref[k * VS + 2], FR = ap.uref[k * VS + 8];
    if (lane < 30) {
      const int r = lane / 10, col = lane - 10 * r, f = col / 5, j = col - 5 * f;
      const float F = f ? FR : FL;
      const float jr0 = md[M_JLEG + 30 * f + 0 * 5 + j], jr1 = md[M_JLEG + 30 * f + 1 * 5 + j];
      st[lane] = dt * F * (m3(Iwi, r, 0) * jr1 - m3(Iwi, r, 1) * jr0);
    }
    __syncwarp();
    if (lane < NC) {
      const int i = lane;
      float f0 = 0.f;
      if (i < 3) f0 = xbar[6 + i];
      else if (i < 6) f0 = m3(Einv, i - 3, 0) * w0 + m3(Einv, i - 3, 1) * w1 + m3(Einv, i - 3, 2) * w2;
      else if (i < 9) f0 = (i == 8) ? (FL + FR) * invm - GRAV : 0.f;
      else if (i < 12) {
        // I_w^-1 (r_L x f_L + r_R x f_R - w x I_w w) with f = (0, 0, F)
        const float t0 = rl[0][1] * FL + rl[1][1] * FR - (w1 * Iww2 - w2 * Iww1);
        const float t1 = -rl[0][0] * FL - rl[1][0] * FR - (w2 * Iww0 - w0 * Iww2);
        const float t2 = -(w0 * Iww1 - w1 * Iww0);
        const int r = i - 9;
        f0 = m3(Iwi, r, 0) * t0 + m3(Iwi, r, 1) * t1 + m3(Iwi, r, 2) * t2;
      }
      const float Ax = ak_mv<false>(Ab, st, xbar, lane);
      const float Bu = Bm[2 * LD + i] * FL + Bm[8 * LD + i] * FR;
      st[32 + i] = xbar[i] + dt * f0 - Ax - Bu;
    }
    __syncwarp();
  }

  // warm or cold start (f_init: the current pose repeated over the horizon,
  // everything else zero; duals zero)
  const bool warm = prm.warm_start && (*ap.warm == N);
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

// ============================================================ factor (A3, A4)
// Assembles the stage blocks of the ADMM KKT system (P + sigma I + rho C^T C
// with the dynamics as exact constraints) and runs the backward Riccati
// recursion.  Caches per stage: K_k, H_uu,k^-1, e_k = P_{k+1} c_k (coupled),
// scalar gain and inverse for the arm lanes.
__device__ void factor_admm(const AgentPtrs& ap, float* sm, int lane, float rho, float sigma) {
  const int N = ap.N;
  const float* md = ap.mdl;
  const float dt = md[M_DT], mu = md[M_MU];
  float* Ab = sm + W_ABASE; float* Bm = sm + W_B; float* P = sm + W_P; float* Ak = sm + W_AK;
  float* PA = sm + W_PA; float* PB = sm + W_PB; float* H = sm + W_H; float* X = sm + W_X;
  float* K = sm + W_K;
  float* vT = sm + W_VEC + V_T * 64;
  const int j = lane < NC ? lane : NC - 1;

  // P_N = diag(Qt_N)
  if (lane < NC) {
    for (int i = 0; i < NC; ++i) P[j * LD + i] = 0.f;
    P[j * LD + j] = qt_x(ap, N, j, rho, sigma, true);
  }
  float Pa = (lane >= NC && lane < 30) ? qt_x(ap, N, lane, rho, sigma, true) : 0.f;
  __syncwarp();

  for (int k = N - 1; k >= 0; --k) {
    const float* dA = ap.lin + L_STAGE + k * 64;
    const float* rc = ap.rcls + k * RS;
    // A_k = A_base + dA_k
    if (lane < NC) {
      for (int i = 0; i < NC; ++i) {
        float a = Ab[j * LD + i];
        if (i >= 9 && i < 12 && j >= 12) a += dA[(i - 9) * 10 + (j - 12)];
        Ak[j * LD + i] = a;
      }
    }
    __syncwarp();
    wgemm<false, false>(PA, P, Ak, nullptr, 1.f, lane);
    wgemm<false, false>(PB, P, Bm, nullptr, 1.f, lane);
    // R_tilde_k into H: 2 dt R + sigma + rho C_u^T diag(cls) C_u
    if (lane < NC) {
      for (int i = 0; i < NC; ++i) H[j * LD + i] = 0.f;
      const int row = j < 12 ? j : j + 8;
      float d = 2.f * dt * md[M_R + j] + sigma + rho * rc[row];
      if (j < 12) {
        const int f = j / 6, c = j - 6 * f, b = 6 * f, p = 12 + 4 * f;
        const float r0 = rho * rc[p], r1 = rho * rc[p + 1], r2 = rho * rc[p + 2], r3 = rho * rc[p + 3];
        if (c == 0) { d += r0 + r1; H[j * LD + b + 2] = mu * (r1 - r0); }
        if (c == 1) { d += r2 + r3; H[j * LD + b + 2] = mu * (r3 - r2); }
        if (c == 2) {
          d += mu * mu * (r0 + r1 + r2 + r3);
          H[j * LD + b] = mu * (r1 - r0);
          H[j * LD + b + 1] = mu * (r3 - r2);
        }
      }
      H[j * LD + j] = d;
    }
    __syncwarp();
    wgemm<true, false>(H, Bm, PB, H, 1.f, lane);     // H_uu = R_tilde + B^T P B
    wgemm<true, false>(X, Bm, PA, nullptr, 1.f, lane);  // H_ux = B^T P A
    winv(H, lane);
    wgemm<false, false>(K, H, X, nullptr, -1.f, lane);  // K = -H_uu^-1 H_ux
    if (lane < NC) vT[lane] = dA[32 + lane];
    __syncwarp();
    const float e = wmv<false>(P, vT, lane);
    wcopy_block(ap.cK + (size_t)k * MB, K, lane);
    wcopy_block(ap.cH + (size_t)k * MB, H, lane);
    float* ce = ap.cE + k * 64;
    if (lane < NC) ce[lane] = e;
    // arms: scalar Riccati, A = 1, B = dt, c = 0
    float Ka = 0.f, Hux = 0.f;
    if (lane >= NC && lane < 30) {
      const float Rt = 2.f * dt * md[M_R + lane] + sigma + rho * rc[lane + 8];
      const float Huu = Rt + dt * dt * Pa;
      Hux = dt * Pa;
      const float Hi = 1.f / Huu;
      Ka = -Hi * Hux;
      ce[lane] = Ka;
      ce[32 + lane] = Hi;
    }
    if (k >= 1) {
      wgemm<true, false>(PB, Ak, PA, nullptr, 1.f, lane);   // A^T P A
      wgemm<true, false>(P, X, K, PB, 1.f, lane);           // + H_ux^T K
      float t[NC];
      if (lane < NC) {
#pragma unroll
        for (int i = 0; i < NC; ++i) t[i] = 0.5f * (P[j * LD + i] + P[i * LD + j]);
      }
      __syncwarp();
      if (lane < NC) {
#pragma unroll
        for (int i = 0; i < NC; ++i) P[j * LD + i] = t[i];
        P[j * LD + j] += qt_x(ap, k, j, rho, sigma, true);
      }
      if (lane >= NC && lane < 30) Pa = qt_x(ap, k, lane, rho, sigma, true) + Pa + Hux * Ka;
      __syncwarp();
    }
  }
}

// ============================================================ ADMM iteration (A5)
// One OSQP iteration with the equality-constrained KKT solve done by the
// cached Riccati factors (backward linear sweep + forward rollout), then
// relaxation, projection onto [lo, hi] and the dual update, stage by stage.
__device__ void admm_iteration(const AgentPtrs& ap, float* sm, int lane, float rho, const SolverParams& prm) {
  const int N = ap.N;
  const float* md = ap.mdl;
  const float dt = md[M_DT], mu = md[M_MU], sigma = prm.sigma, alpha = prm.alpha;
  float* Ab = sm + W_ABASE; float* Bm = sm + W_B; float* K = sm + W_K; float* H = sm + W_H;
  float* vec = sm + W_VEC;
  float* vS = vec + V_S * 64; float* vH = vec + V_H * 64; float* vX = vec + V_X * 64;
  float* vU = vec + V_U * 64; float* vXN = vec + V_XN * 64; float* vR = vec + V_ROW * 64;
  const bool arm = lane >= NC && lane < 30;
  const float twoQ = lane < 30 ? 2.f * dt * md[M_Q + lane] : 0.f;
  const float twoR = lane < 30 ? 2.f * dt * md[M_R + lane] : 0.f;

  // ---- backward sweep: p_k, d_k
  // linear term of x_N: -2dt Q xr_N - sigma x_N - C_x^T (rho w - y) of stage N-1
  auto qlin = [&](int k) -> float {   // k >= 1
    float v = -twoQ * ap.xref[k * VS + lane] - sigma * ap.x[k * VS + lane];
    if (lane >= 12 && lane < 30) {
      const int r = lane + 26;
      v -= rho * ap.rcls[(k - 1) * RS + r] * ap.w[(k - 1) * RS + r] - ap.y[(k - 1) * RS + r];
    }
    return v;
  };
  float p = lane < 30 ? qlin(N) : 0.f;
  for (int k = N - 1; k >= 0; --k) {
    const float* ce = ap.cE + k * 64;
    const float* dA = ap.lin + L_STAGE + k * 64;
    wcopy_block(K, ap.cK + (size_t)k * MB, lane);
    wcopy_block(H, ap.cH + (size_t)k * MB, lane);
    for (int r = lane; r < NR; r += 32)
      vR[r] = rho * ap.rcls[k * RS + r] * ap.w[k * RS + r] - ap.y[k * RS + r];
    const float s = (lane < NC ? ce[lane] : 0.f) + p;
    vS[lane] = s;
    __syncwarp();
    float h = 0.f;
    if (lane < 30) {
      const float rlin = -twoR * ap.uref[k * VS + lane] - sigma * ap.u[k * VS + lane] - cuT(vR, lane, mu);
      h = rlin + (lane < NC ? wmv<true>(Bm, vS, lane) : dt * s);
    }
    vH[lane] = h;
    __syncwarp();
    float d = 0.f;
    if (lane < NC) d = -wmv<false>(H, vH, lane);
    else if (arm) d = -ce[32 + lane] * h;
    ap.dv[k * VS + lane] = d;
    if (k >= 1) {
      float pn = 0.f;
      if (lane < NC) pn = qlin(k) + ak_mv<true>(Ab, dA, vS, lane) + wmv<true>(K, vH, lane);
      else if (arm) pn = qlin(k) + s + ce[lane] * h;
      p = pn;
    }
    __syncwarp();
  }

  // ---- forward rollout + per-stage relaxation / projection / dual update
  float x = lane < 30 ? ap.x[lane] : 0.f;   // x_0 = x0
  for (int k = 0; k < N; ++k) {
    const float* ce = ap.cE + k * 64;
    const float* dA = ap.lin + L_STAGE + k * 64;
    wcopy_block(K, ap.cK + (size_t)k * MB, lane);
    vX[lane] = x;
    __syncwarp();
    float u = 0.f;
    if (lane < NC) u = wmv<false>(K, vX, lane) + ap.dv[k * VS + lane];
    else if (arm) u = ce[lane] * x + ap.dv[k * VS + lane];
    vU[lane] = u;
    __syncwarp();
    float xn = 0.f;
    if (lane < NC) xn = ak_mv<false>(Ab, dA, vX, lane) + wmv<false>(Bm, vU, lane) + dA[32 + lane];
    else if (arm) xn = x + dt * u;
    vXN[lane] = xn;
    ap.xt[(k + 1) * VS + lane] = xn;
    ap.ut[k * VS + lane] = u;
    __syncwarp();
    for (int r = lane; r < NR; r += 32) {
      const float zt = crow(vU, vXN, r, mu);
      const float wo = ap.w[k * RS + r], yo = ap.y[k * RS + r];
      const float wh = alpha * zt + (1.f - alpha) * wo;
      const float rr = rho * ap.rcls[k * RS + r];
      float wn, yn;
      if (rr > 0.f) {
        wn = fminf(fmaxf(wh + yo / rr, ap.rlo[k * RS + r]), ap.rhi[k * RS + r]);
        yn = yo + rr * (wh - wn);
      } else {
        wn = wh;
        yn = 0.f;
      }
      ap.w[k * RS + r] = wn;
      ap.y[k * RS + r] = yn;
    }
    if (lane < 30) {
      ap.u[k * VS + lane] = alpha * u + (1.f - alpha) * ap.u[k * VS + lane];
      ap.x[(k + 1) * VS + lane] = alpha * xn + (1.f - alpha) * ap.x[(k + 1) * VS + lane];
    }
    x = xn;
    __syncwarp();
  }
}

// ============================================================ residuals (A5 vii)
// Unscaled OSQP residuals of the current iterate: primal |C z - w|_inf over
// constrained rows; dual = stationarity in u after choosing the dynamics
// multipliers that make stationarity in x exact (costate recursion).
struct Res { float rp, rd, ps, ds; };

__device__ Res admm_residuals(const AgentPtrs& ap, float* sm, int lane, const float* xs, const float* us,
                              const float* ys, bool with_y) {
  const int N = ap.N;
  const float* md = ap.mdl;
  const float dt = md[M_DT], mu = md[M_MU];
  float* Ab = sm + W_ABASE; float* Bm = sm + W_B;
  float* vec = sm + W_VEC;
  float* vU = vec + V_U * 64; float* vXN = vec + V_XN * 64; float* vM = vec + V_S * 64;
  float* vY = vec + V_ROW * 64;
  const float twoQ = lane < 30 ? 2.f * dt * md[M_Q + lane] : 0.f;
  const float twoR = lane < 30 ? 2.f * dt * md[M_R + lane] : 0.f;
  float rp = 0.f, ps = 0.f, rd = 0.f, ds = 0.f;
  // primal
  for (int k = 0; k < N; ++k) {
    vU[lane] = us[k * VS + lane];
    vXN[lane] = xs[(k + 1) * VS + lane];
    __syncwarp();
    for (int r = lane; r < NR; r += 32) {
      if (ap.rcls[k * RS + r] > 0.f) {
        const float v = crow(vU, vXN, r, mu);
        const float w = ap.w[k * RS + r];
        rp = fmaxf(rp, fabsf(v - w));
        ps = fmaxf(ps, fmaxf(fabsf(v), fabsf(w)));
      }
    }
    __syncwarp();
  }
  // dual: costate backward
  auto gx = [&](int k) -> float {   // 2dt Q (x_k - xr_k) + C_x^T y_{k-1}
    float g = twoQ * (xs[k * VS + lane] - ap.xref[k * VS + lane]);
    if (with_y && lane >= 12 && lane < 30) g += ys[(k - 1) * RS + lane + 26];
    return g;
  };
  float m = lane < 30 ? gx(N) : 0.f;
  for (int k = N - 1; k >= 0; --k) {
    const float* dA = ap.lin + L_STAGE + k * 64;
    vM[lane] = m;
    for (int r = lane; r < NR; r += 32) vY[r] = with_y ? ys[k * RS + r] : 0.f;
    __syncwarp();
    if (lane < 30) {
      const float cty = cuT(vY, lane, mu);
      const float gu = twoR * (us[k * VS + lane] - ap.uref[k * VS + lane]) + cty;
      const float ru = gu + (lane < NC ? wmv<true>(Bm, vM, lane) : dt * m);
      rd = fmaxf(rd, fabsf(ru));
      ds = fmaxf(ds, fmaxf(fabsf(twoR * us[k * VS + lane]), fabsf(twoR * ap.uref[k * VS + lane])));
      ds = fmaxf(ds, fmaxf(fabsf(cty), fabsf(twoQ * xs[(k + 1) * VS + lane])));
      ds = fmaxf(ds, fabsf(twoQ * ap.xref[(k + 1) * VS + lane]));
      if (lane >= 12) ds = fmaxf(ds, fabsf(vY[lane + 26]));
    }
    float mn = 0.f;
    if (k >= 1 && lane < 30) mn = gx(k) + (lane < NC ? ak_mv<true>(Ab, dA, vM, lane) : m);
    __syncwarp();
    m = mn;
  }
  Res out;
  out.rp = warp_max(rp); out.ps = warp_max(ps); out.rd = warp_max(rd); out.ds = warp_max(ds);
  return out;
}

// ============================================================ ADMM driver (A5, A6)
// Returns the agent status; fills iteration / refactor counts and residuals.
__device__ int admm_solve(const AgentPtrs& ap, float* sm, int lane, const SolverParams& prm, bool factored,
                          int* iters_out, int* refac_out, Res* res_out) {
  float rho = *ap.rho;
  if (!factored) factor_admm(ap, sm, lane, rho, prm.sigma);
  int refac = 0, status = MPC_AGENT_MAX_ITER_, it = 0;
  const bool fixed = prm.fixed_iters > 0;
  const int max_it = fixed ? prm.fixed_iters : prm.max_iter;
  Res r = {0.f, 0.f, 0.f, 0.f};
  for (it = 1; it <= max_it; ++it) {
    admm_iteration(ap, sm, lane, rho, prm);
    const bool check = (!fixed && (it % prm.check_every == 0)) || it == max_it;
    if (!check) continue;
    r = admm_residuals(ap, sm, lane, ap.x, ap.u, ap.y, true);
    if (!(isfinite(r.rp) && isfinite(r.rd))) { status = MPC_AGENT_NAN_; break; }
    if (fixed) break;
    if (r.rp <= prm.eps_abs + prm.eps_rel * r.ps && r.rd <= prm.eps_abs + prm.eps_rel * r.ds) {
      status = MPC_AGENT_SOLVED_;
      break;
    }
    if (prm.adaptive_rho && it < max_it) {
      const float num = r.rp / fmaxf(r.ps, 1e-30f);
      const float den = r.rd / fmaxf(r.ds, 1e-30f);
      float rn = rho * sqrtf(num / fmaxf(den, 1e-30f));
      rn = fminf(fmaxf(rn, 1e-6f), 1e6f);
      if (rn > 5.f * rho || rn < 0.2f * rho) {
        rho = rn;
        factor_admm(ap, sm, lane, rho, prm.sigma);
        ++refac;
      }
    }
  }
  if (it > max_it) it = max_it;
  if (lane == 0) *ap.rho = rho;
  *iters_out = it;
  *refac_out = refac;
  *res_out = r;
  return status;
}

// ============================================================ polish (NEXT-2 of OSQP)
// Active-set guess from (w, y) as in OSQP's polish: row i is at its lower
// bound when w_i - lo_i < -y_i, at its upper bound when hi_i - w_i < y_i.
// The active rows are eliminated exactly: u_k = G_k v_k + t_k, and the
// reduced equality-constrained LQ problem is solved by one more Riccati
// factor + sweep.  Joint-box (state) rows are not handled: if any is active
// the polish is skipped.

// Per-stage active-set description built by every lane from smem rows.
struct FootAct { int swing, zero, top, tx, ty; };

// Initial guess of every stage's active set, stored in the agent's act array
// (code: bit 0 at lower bound, bit 1 at upper bound, 3 = equality row).
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

// stage k's active-set codes into shared memory
__device__ __forceinline__ void stage_active(const AgentPtrs& ap, int k, int* act, int lane) {
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

// Row i of G (u = G v + t) for u index i < 22 and t_i, dead_i; lane writes
// G(i, j) for the j of its block into G (column-major, zeroed by the caller).
__device__ __forceinline__ void gamma_row(const AgentPtrs& ap, int k, const int* act, int i, float mu,
                                          float* G, float* t, float* dead) {
  float ti = 0.f, di = 0.f;
  if (i < 12) {
    const int f = i / 6, c = i - 6 * f, b = 6 * f;
    const FootAct fa = foot_act(act, f);
    if (fa.swing || fa.zero) {
      di = 1.f;
    } else if (c >= 3) {
      G[i * LD + i] = 1.f;
    } else if (fa.top) {
      const float F = ap.rhi[k * RS + b + 2];
      if (c == 2) { ti = F; di = 1.f; }
      else {
        const int tt = c == 0 ? fa.tx : fa.ty;
        if (tt) { ti = tt * mu * F; di = 1.f; }
        else G[i * LD + i] = 1.f;
      }
    } else {
      if (c == 2) G[i * LD + i] = 1.f;
      else {
        const int tt = c == 0 ? fa.tx : fa.ty;
        if (tt) { G[(b + 2) * LD + i] = tt * mu; di = 1.f; }
        else G[i * LD + i] = 1.f;
      }
    }
  } else {
    const int r = i + 8;
    const int a = act[r];
    if (a & 1) { ti = ap.rlo[k * RS + r]; di = 1.f; }
    else if (a & 2) { ti = ap.rhi[k * RS + r]; di = 1.f; }
    else G[i * LD + i] = 1.f;
  }
  t[i] = ti;
  dead[i] = di;
}

// arm lane: (t, dead) of its joint-rate row
__device__ __forceinline__ void arm_gamma(const AgentPtrs& ap, int k, const int* act, int lane, float* t, float* dead) {
  const int r = lane + 8;
  const int a = act[r];
  *t = 0.f; *dead = 0.f;
  if (a & 1) { *t = ap.rlo[k * RS + r]; *dead = 1.f; }
  else if (a & 2) { *t = ap.rhi[k * RS + r]; *dead = 1.f; }
}


// Factor and solve the reduced problem; the polished primal goes to xt/ut.
__device__ bool polish_solve(const AgentPtrs& ap, float* sm, int lane) {
  const int N = ap.N;
  const float* md = ap.mdl;
  const float dt = md[M_DT], mu = md[M_MU];
  float* Ab = sm + W_ABASE; float* Bm = sm + W_B; float* P = sm + W_P; float* Ak = sm + W_AK;
  float* PA = sm + W_PA; float* PB = sm + W_PB; float* H = sm + W_H; float* X = sm + W_X;
  float* K = sm + W_K;
  float* vec = sm + W_VEC;
  float* vT = vec + V_T * 64; float* vD = vec + V_G * 64; float* vC = vec + V_MISC * 64;
  int* act = reinterpret_cast<int*>(vec + V_LO * 64);
  const int j = lane < NC ? lane : NC - 1;
  const bool arm = lane >= NC && lane < 30;
  const float twoQ = lane < 30 ? 2.f * dt * md[M_Q + lane] : 0.f;
  const float twoR = lane < 30 ? 2.f * dt * md[M_R + lane] : 0.f;

  // state (joint-box) rows active anywhere -> no polish
  int qact = 0;
  for (int k = 0; k < N; ++k) {
    stage_active(ap, k, act, lane);
    for (int r = lane; r < NR; r += 32) qact |= (r >= 38 && act[r] != 0);
    __syncwarp();
  }
  if (warp_or(qact)) return false;

  // ---- factor of the reduced problem (cost 2dt Q, 2dt R; no sigma, no rho)
  if (lane < NC) {
    for (int i = 0; i < NC; ++i) P[j * LD + i] = 0.f;
    P[j * LD + j] = 2.f * dt * md[M_Q + j];
  }
  float Pa = arm ? twoQ : 0.f;
  __syncwarp();
  for (int k = N - 1; k >= 0; --k) {
    const float* dA = ap.lin + L_STAGE + k * 64;
    float* cc = ap.cC + k * 64;
    float* ce = ap.cE + k * 64;
    stage_active(ap, k, act, lane);
    if (lane < NC) for (int i = 0; i < NC; ++i) X[j * LD + i] = 0.f;
    __syncwarp();
    if (lane < NC) gamma_row(ap, k, act, lane, mu, X, vT, vD);
    float ta = 0.f, da = 0.f;
    if (arm) arm_gamma(ap, k, act, lane, &ta, &da);
    __syncwarp();
    // B_hat = B G -> PB ; D G -> PA ; R_hat = G^T D G + diag(dead) -> H
    wgemm<false, false>(PB, Bm, X, nullptr, 1.f, lane);
    if (lane < NC) for (int i = 0; i < NC; ++i) PA[j * LD + i] = 2.f * dt * md[M_R + i] * X[j * LD + i];
    __syncwarp();
    wgemm<true, false>(H, X, PA, nullptr, 1.f, lane);
    if (lane < NC) {
      H[j * LD + j] += vD[j];
      vC[lane] = twoR * (vT[lane] - ap.uref[k * VS + lane]);
    }
    __syncwarp();
    // c_hat = c + B t ; r_hat = G^T 2dt R (t - u_ref)
    if (lane < NC) {
      cc[lane] = dA[32 + lane] + wmv<false>(Bm, vT, lane);
      cc[32 + lane] = wmv<true>(X, vC, lane);
    } else if (arm) {
      cc[lane] = da > 0.f ? dt * ta : 0.f;
      cc[32 + lane] = 0.f;
    }
    __syncwarp();
    // X <- B_hat (G is no longer needed); keep a copy for the sweep
    if (lane < NC) for (int i = 0; i < NC; ++i) X[j * LD + i] = PB[j * LD + i];
    __syncwarp();
    wcopy_block(ap.cB + (size_t)k * MB, X, lane);
    if (lane < NC) {
      for (int i = 0; i < NC; ++i) {
        float a = Ab[j * LD + i];
        if (i >= 9 && i < 12 && j >= 12) a += dA[(i - 9) * 10 + (j - 12)];
        Ak[j * LD + i] = a;
      }
    }
    __syncwarp();
    wgemm<false, false>(PA, P, Ak, nullptr, 1.f, lane);   // P A
    wgemm<false, false>(PB, P, X, nullptr, 1.f, lane);    // P B_hat
    wgemm<true, false>(H, X, PB, H, 1.f, lane);           // H_uu = R_hat + B_hat^T P B_hat
    wgemm<true, false>(PB, X, PA, nullptr, 1.f, lane);    // H_ux
    winv(H, lane);
    wgemm<false, false>(K, H, PB, nullptr, -1.f, lane);
    if (lane < NC) vT[lane] = cc[lane];
    __syncwarp();
    const float e = wmv<false>(P, vT, lane);
    wcopy_block(ap.cK + (size_t)k * MB, K, lane);
    wcopy_block(ap.cH + (size_t)k * MB, H, lane);
    if (lane < NC) ce[lane] = e;
    float Ka = 0.f, Hux = 0.f;
    if (arm) {
      const float Bh = da > 0.f ? 0.f : dt;
      const float Rt = da > 0.f ? 1.f : twoR;
      const float Huu = Rt + Bh * Bh * Pa;
      Hux = Bh * Pa;
      const float Hi = 1.f / Huu;
      Ka = -Hi * Hux;
      ce[lane] = Ka;
      ce[32 + lane] = Hi;
      ce[32 + lane - NC] = Pa * cc[lane];   // e of the arm lane
    }
    if (k >= 1) {
      wgemm<true, false>(X, Ak, PA, nullptr, 1.f, lane);   // A^T P A
      wgemm<true, false>(P, PB, K, X, 1.f, lane);          // + H_ux^T K
      float t[NC];
      if (lane < NC) {
#pragma unroll
        for (int i = 0; i < NC; ++i) t[i] = 0.5f * (P[j * LD + i] + P[i * LD + j]);
      }
      __syncwarp();
      if (lane < NC) {
#pragma unroll
        for (int i = 0; i < NC; ++i) P[j * LD + i] = t[i];
        P[j * LD + j] += 2.f * dt * md[M_Q + j];
      }
      if (arm) Pa = twoQ + Pa + Hux * Ka;
    }
    __syncwarp();
  }

  // ---- backward sweep of the reduced problem
  float* vS = vec + V_S * 64; float* vH = vec + V_H * 64; float* vX = vec + V_X * 64;
  float* vV = vec + V_U * 64;
  float p = lane < 30 ? -twoQ * ap.xref[N * VS + lane] : 0.f;
  for (int k = N - 1; k >= 0; --k) {
    const float* ce = ap.cE + k * 64;
    const float* cc = ap.cC + k * 64;
    const float* dA = ap.lin + L_STAGE + k * 64;
    stage_active(ap, k, act, lane);
    float ta = 0.f, da = 0.f;
    if (arm) arm_gamma(ap, k, act, lane, &ta, &da);
    wcopy_block(K, ap.cK + (size_t)k * MB, lane);
    wcopy_block(H, ap.cH + (size_t)k * MB, lane);
    wcopy_block(X, ap.cB + (size_t)k * MB, lane);
    const float s = p + (lane < NC ? ce[lane] : (arm ? ce[32 + lane - NC] : 0.f));
    vS[lane] = s;
    __syncwarp();
    float h = 0.f;
    if (lane < NC) h = cc[32 + lane] + wmv<true>(X, vS, lane);
    else if (arm) h = cc[32 + lane] + (da > 0.f ? 0.f : dt) * s;
    vH[lane] = h;
    __syncwarp();
    float d = 0.f;
    if (lane < NC) d = -wmv<false>(H, vH, lane);
    else if (arm) d = -ce[32 + lane] * h;
    ap.dv[k * VS + lane] = d;
    if (k >= 1) {
      const float ql = lane < 30 ? -twoQ * ap.xref[k * VS + lane] : 0.f;
      if (lane < NC) p = ql + ak_mv<true>(Ab, dA, vS, lane) + wmv<true>(K, vH, lane);
      else if (arm) p = ql + s + ce[lane] * h;
    }
    __syncwarp();
  }
  // ---- forward rollout, u = G v + t
  float x = lane < 30 ? ap.x[lane] : 0.f;
  for (int k = 0; k < N; ++k) {
    const float* ce = ap.cE + k * 64;
    const float* cc = ap.cC + k * 64;
    const float* dA = ap.lin + L_STAGE + k * 64;
    stage_active(ap, k, act, lane);
    if (lane < NC) for (int i = 0; i < NC; ++i) PA[j * LD + i] = 0.f;
    __syncwarp();
    if (lane < NC) gamma_row(ap, k, act, lane, mu, PA, vT, vD);
    float ta = 0.f, da = 0.f;
    if (arm) arm_gamma(ap, k, act, lane, &ta, &da);
    wcopy_block(K, ap.cK + (size_t)k * MB, lane);
    wcopy_block(X, ap.cB + (size_t)k * MB, lane);
    vX[lane] = x;
    __syncwarp();
    float v = 0.f;
    if (lane < NC) v = wmv<false>(K, vX, lane) + ap.dv[k * VS + lane];
    else if (arm) v = ce[lane] * x + ap.dv[k * VS + lane];
    vV[lane] = v;
    __syncwarp();
    float xn = 0.f, u = 0.f;
    if (lane < NC) {
      xn = ak_mv<false>(Ab, dA, vX, lane) + wmv<false>(X, vV, lane) + cc[lane];
      u = wmv<false>(PA, vV, lane) + vT[lane];
    } else if (arm) {
      xn = x + (da > 0.f ? 0.f : dt) * v + cc[lane];
      u = da > 0.f ? ta : v;
    }
    ap.xt[(k + 1) * VS + lane] = xn;
    ap.ut[k * VS + lane] = u;
    x = xn;
    __syncwarp();
  }
  return true;
}

// Optimality check of the polished point (xt, ut): primal feasibility of
// every row, and KKT conditions of the guessed active set (stationarity in
// the free directions, right sign of the multipliers of the active rows),
// with the dynamics multipliers from the costate recursion.  When `fix` is
// set the active set is corrected for a next attempt: rows the point
// violates are added, active rows whose multiplier has the wrong sign are
// dropped; *changed reports whether anything changed.
__device__ Res polish_check(const AgentPtrs& ap, float* sm, int lane, const SolverParams& prm, bool fix,
                            int* changed) {
  const int N = ap.N;
  const float* md = ap.mdl;
  const float dt = md[M_DT], mu = md[M_MU];
  float* Ab = sm + W_ABASE; float* Bm = sm + W_B;
  float* vec = sm + W_VEC;
  float* vU = vec + V_U * 64; float* vXN = vec + V_XN * 64; float* vM = vec + V_S * 64;
  float* vG = vec + V_G * 64;
  const float twoQ = lane < 30 ? 2.f * dt * md[M_Q + lane] : 0.f;
  const float twoR = lane < 30 ? 2.f * dt * md[M_R + lane] : 0.f;
  const float* xs = ap.xt;
  const float* us = ap.ut;
  float rp = 0.f, ps = 0.f, rd = 0.f, ds = 0.f;
  int chg = 0;
  // scales first (they set the tolerances)
  float m = lane < 30 ? twoQ * (xs[N * VS + lane] - ap.xref[N * VS + lane]) : 0.f;
  for (int k = 0; k < N; ++k) {
    if (lane < 30) {
      ds = fmaxf(ds, fmaxf(fabsf(twoR * us[k * VS + lane]), fabsf(twoR * ap.uref[k * VS + lane])));
      ds = fmaxf(ds, fmaxf(fabsf(twoQ * xs[(k + 1) * VS + lane]), fabsf(twoQ * ap.xref[(k + 1) * VS + lane])));
    }
    vU[lane] = us[k * VS + lane];
    vXN[lane] = xs[(k + 1) * VS + lane];
    __syncwarp();
    for (int r = lane; r < NR; r += 32)
      if (ap.rcls[k * RS + r] > 0.f) ps = fmaxf(ps, fabsf(crow(vU, vXN, r, mu)));
    __syncwarp();
  }
  ps = warp_max(ps);
  ds = warp_max(ds);
  const float tol_p = prm.eps_abs + prm.eps_rel * ps;
  const float tol_d = prm.eps_abs + prm.eps_rel * ds;
  // dual conditions, costate backward
  int* act = reinterpret_cast<int*>(vec + V_LO * 64);
  for (int k = N - 1; k >= 0; --k) {
    const float* dA = ap.lin + L_STAGE + k * 64;
    stage_active(ap, k, act, lane);
    vM[lane] = m;
    __syncwarp();
    float g = 0.f;
    if (lane < 30)
      g = twoR * (us[k * VS + lane] - ap.uref[k * VS + lane]) + (lane < NC ? wmv<true>(Bm, vM, lane) : dt * m);
    vG[lane] = g;
    __syncwarp();
    int* ak = ap.act + k * RS;
    // joint rates: lane i in 12..29 (row i + 8); y = -g
    if (lane >= 12 && lane < 30) {
      const int a = act[lane + 8];
      float bad = 0.f;
      if (a & 1) bad = fmaxf(-g, 0.f);         // needs y <= 0 at a lower bound
      else if (a & 2) bad = fmaxf(g, 0.f);     // needs y >= 0 at an upper bound
      else rd = fmaxf(rd, fabsf(g));
      rd = fmaxf(rd, bad);
      if (fix && bad > tol_d) { ak[lane + 8] = 0; chg = 1; }
    }
    // feet: lane f in 0..1
    if (lane < 2) {
      const int f = lane, b = 6 * f, p = 12 + 4 * f;
      const FootAct fa = foot_act(act, f);
      const float gx = vG[b], gy = vG[b + 1], gz = vG[b + 2];
      if (!fa.swing) {
        for (int c = 3; c < 6; ++c) rd = fmaxf(rd, fabsf(vG[b + c]));   // free moments
        if (fa.zero) {
          // -g in the normal cone of the pyramid at 0: g . ray >= 0 on its 4 rays
          float worst = 0.f;
          for (int sx = -1; sx <= 1; sx += 2)
            for (int sy = -1; sy <= 1; sy += 2)
              worst = fmaxf(worst, -(sx * mu * gx + sy * mu * gy + gz));
          rd = fmaxf(rd, worst);
          if (fix && worst > tol_d) {
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
            if (fix && -ypx > tol_d) { ak[fa.tx > 0 ? p : p + 1] = 0; chg = 1; }
          } else rd = fmaxf(rd, fabsf(gx));
          if (fa.ty) {
            rd = fmaxf(rd, fmaxf(-ypy, 0.f));
            if (fix && -ypy > tol_d) { ak[fa.ty > 0 ? p + 2 : p + 3] = 0; chg = 1; }
          } else rd = fmaxf(rd, fabsf(gy));
          const float rz = gz - mu * (ypx + ypy);   // = -y_top when f_z sits at its upper bound
          if (fa.top) {
            rd = fmaxf(rd, fmaxf(rz, 0.f));
            if (fix && rz > tol_d) { ak[b + 2] &= ~2; chg = 1; }
          } else rd = fmaxf(rd, fabsf(rz));
        }
      }
    }
    float mn = 0.f;
    if (k >= 1 && lane < 30)
      mn = twoQ * (xs[k * VS + lane] - ap.xref[k * VS + lane]) + (lane < NC ? ak_mv<true>(Ab, dA, vM, lane) : m);
    __syncwarp();
    m = mn;
  }
  // primal feasibility of every row (after the dual pass, so that the dual
  // conditions are read on the active set the point was solved with)
  for (int k = 0; k < N; ++k) {
    vU[lane] = us[k * VS + lane];
    vXN[lane] = xs[(k + 1) * VS + lane];
    __syncwarp();
    for (int r = lane; r < NR; r += 32) {
      const float v = crow(vU, vXN, r, mu);
      const float lo = ap.rlo[k * RS + r], hi = ap.rhi[k * RS + r];
      const float viol = fmaxf(fmaxf(lo - v, v - hi), 0.f);
      rp = fmaxf(rp, viol);
      if (fix && viol > tol_p && ap.act[k * RS + r] == 0) {
        ap.act[k * RS + r] = (v < lo) ? 1 : 2;
        chg = 1;
      }
    }
    __syncwarp();
  }
  Res out;
  out.rp = warp_max(rp); out.ps = ps; out.rd = warp_max(rd); out.ds = ds;
  if (changed) *changed = warp_or(chg);
  return out;
}

// Polish with active-set correction: up to four attempts; returns true and
// leaves the polished point in (x, u) when one passes its check.
__device__ bool polish(const AgentPtrs& ap, float* sm, int lane, const SolverParams& prm, Res* res) {
  init_active(ap, lane);
  for (int attempt = 0; attempt < 4; ++attempt) {
    if (!polish_solve(ap, sm, lane)) return false;
    int changed = 0;
    const Res pr = polish_check(ap, sm, lane, prm, true, &changed);
    const bool ok = isfinite(pr.rp) && isfinite(pr.rd) && pr.rp <= prm.eps_abs + prm.eps_rel * pr.ps &&
                    pr.rd <= prm.eps_abs + prm.eps_rel * pr.ds;
    if (ok) {
      for (int k = 1; k <= ap.N; ++k) ap.x[k * VS + lane] = ap.xt[k * VS + lane];
      for (int k = 0; k < ap.N; ++k) ap.u[k * VS + lane] = ap.ut[k * VS + lane];
      __syncwarp();
      *res = pr;
      return true;
    }
    if (!changed) return false;
  }
  return false;
}

// ============================================================ torque map (A7)
// q_MPC = x0.q; qdot_MPC = u_0.qdot; qddot = (u_1.qdot - u_0.qdot)/dt;
// tau = K_p (q_MPC - q) + K_d (qdot_MPC - qdot) + M qddot + h - J_leg^T W
// (Eqs. rnea, mpc_torque); value = QP objective at the solution.
__device__ void torque_map(const AgentPtrs& ap, int lane) {
  const int N = ap.N;
  const float* md = ap.mdl;
  const float dt = md[M_DT];
  if (lane < 18) {
    const int j = lane;
    const float q = ap.inp[I_X0 + 12 + j];
    const float qd0 = ap.u[12 + j];
    const float qd1 = ap.u[VS + 12 + j];
    float tau = md[M_KP + j] * (q - q) + md[M_KD + j] * (qd0 - ap.inp[I_QD + j])
              + md[M_MJ + j] * ((qd1 - qd0) / dt) + md[M_HJ + j];
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

__device__ void mark_nan(const AgentPtrs& ap, int lane) {
  if (lane < 18) { ap.out[O_TAU + lane] = 0.f; ap.out[O_QSET + lane] = 0.f; ap.out[O_QDSET + lane] = 0.f; }
  if (lane == 0) {
    ap.out[O_V] = 0.f;
    ap.st[T_STATUS] = MPC_AGENT_NAN_;
    ap.st[T_ITERS] = 0; ap.st[T_REFAC] = 0; ap.st[T_POLISHED] = 0;
    *ap.warm = 0;
  }
}

// copy the batch row's inputs into the agent's input record
__device__ __forceinline__ void load_inputs(const Batch& b, int row, const AgentPtrs& ap, int lane) {
  if (lane < 30) ap.inp[I_X0 + lane] = b.x0[(size_t)row * 30 + lane];
  if (lane < 18) ap.inp[I_QD + lane] = b.qd[(size_t)row * 18 + lane];
  if (lane < 4) ap.inp[I_CMD + lane] = b.cmd[(size_t)row * 4 + lane];
  if (lane == 0) ap.inp[I_PHASE] = b.phase[row];
  __syncwarp();
}

// load the constant stage matrices (A_base, B) of the agent into smem
__device__ __forceinline__ void load_lin(const AgentPtrs& ap, float* sm, int lane) {
  wcopy_block(sm + W_ABASE, ap.lin + L_ABASE, lane);
  wcopy_block(sm + W_B, ap.lin + L_B, lane);
  __syncwarp();
}

// ADMM + polish + status bookkeeping for one agent (factor already done when
// `factored`)
__device__ void solve_agent(const AgentPtrs& ap, float* sm, int lane, const SolverParams& prm, bool factored) {
  int iters = 0, refac = 0;
  Res r;
  int status = admm_solve(ap, sm, lane, prm, factored, &iters, &refac, &r);
  int polished = 0;
  if (status != MPC_AGENT_NAN_ && prm.polish) {
    Res pr;
    if (polish(ap, sm, lane, prm, &pr)) {
      polished = 1;
      r.rp = pr.rp; r.rd = pr.rd;
      status = MPC_AGENT_SOLVED_;
    }
  }
  __syncwarp();
  if (lane == 0) {
    ap.st[T_STATUS] = status;
    ap.st[T_ITERS] = iters;
    ap.st[T_REFAC] = refac;
    ap.st[T_POLISHED] = polished;
    ap.out[O_PRIM] = r.rp;
    ap.out[O_DUAL] = r.rd;
    *ap.warm = (status == MPC_AGENT_NAN_) ? 0 : ap.N;
  }
  __syncwarp();
}

// ============================================================ kernels
extern __shared__ __align__(16) float g_smem[];

// a batch row names a live slot (admitted by mpc_set_models, in range)
__device__ __forceinline__ bool valid_slot(const Arena& a, const Batch& b, int row) {
  const int s = b.ids[row];
  return s >= 0 && s < a.max_agents && a.horizon[s] >= 2 && a.horizon[s] <= a.maxN;
}

__device__ __forceinline__ float* warp_smem() { return g_smem + (threadIdx.x >> 5) * W_FLOATS; }

__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32) mpc_k_fused(Arena a, Batch b, SolverParams prm) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  const int nw = gridDim.x * WARPS_PER_BLOCK;
  float* sm = warp_smem();
  for (int row = gw; row < b.n; row += nw) {
    if (!valid_slot(a, b, row)) continue;
    const AgentPtrs ap = agent_ptrs(a, b.ids[row]);
    load_inputs(b, row, ap, lane);
    if (!setup_agent(ap, sm, lane, prm)) { mark_nan(ap, lane); continue; }
    solve_agent(ap, sm, lane, prm, false);
    torque_map(ap, lane);
    __syncwarp();
  }
}

__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32) mpc_k_setup(Arena a, Batch b, SolverParams prm) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  if (row >= b.n || !valid_slot(a, b, row)) return;
  float* sm = warp_smem();
  const AgentPtrs ap = agent_ptrs(a, b.ids[row]);
  load_inputs(b, row, ap, lane);
  const bool ok = setup_agent(ap, sm, lane, prm);
  if (!ok) mark_nan(ap, lane);
  else if (lane == 0) ap.st[T_STATUS] = MPC_AGENT_MAX_ITER_;
}

__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32) mpc_k_factor(Arena a, Batch b, SolverParams prm) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  if (row >= b.n || !valid_slot(a, b, row)) return;
  float* sm = warp_smem();
  const AgentPtrs ap = agent_ptrs(a, b.ids[row]);
  if (ap.st[T_STATUS] == MPC_AGENT_NAN_) return;
  load_lin(ap, sm, lane);
  factor_admm(ap, sm, lane, *ap.rho, prm.sigma);
}

__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32) mpc_k_admm(Arena a, Batch b, SolverParams prm) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  if (row >= b.n || !valid_slot(a, b, row)) return;
  float* sm = warp_smem();
  const AgentPtrs ap = agent_ptrs(a, b.ids[row]);
  if (ap.st[T_STATUS] == MPC_AGENT_NAN_) return;
  load_lin(ap, sm, lane);
  SolverParams p2 = prm;
  p2.polish = 0;
  solve_agent(ap, sm, lane, p2, true);
}

__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32) mpc_k_polish(Arena a, Batch b, SolverParams prm) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  if (row >= b.n || !valid_slot(a, b, row)) return;
  float* sm = warp_smem();
  const AgentPtrs ap = agent_ptrs(a, b.ids[row]);
  if (ap.st[T_STATUS] == MPC_AGENT_NAN_ || !prm.polish) return;
  load_lin(ap, sm, lane);
  Res pr;
  if (polish(ap, sm, lane, prm, &pr) && lane == 0) {
    ap.st[T_STATUS] = MPC_AGENT_SOLVED_;
    ap.st[T_POLISHED] = 1;
    ap.out[O_PRIM] = pr.rp;
    ap.out[O_DUAL] = pr.rd;
  }
}

__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32) mpc_k_torque(Arena a, Batch b) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  if (row >= b.n || !valid_slot(a, b, row)) return;
  const AgentPtrs ap = agent_ptrs(a, b.ids[row]);
  if (ap.st[T_STATUS] == MPC_AGENT_NAN_) return;
  torque_map(ap, lane);
}

// gather per-slot outputs of a batch into caller buffers
__global__ void mpc_k_gather(Arena a, int n, const int* ids, float* tau, float* qset, float* qdset,
                             float* value, int* status) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = t / 32, lane = t & 31;
  if (row >= n) return;
  const int s = ids[row];
  if (s < 0 || s >= a.max_agents || a.horizon[s] < 2) {   // not a live slot
    if (lane < 18) {
      if (tau) tau[(size_t)row * 18 + lane] = 0.f;
      if (qset) qset[(size_t)row * 18 + lane] = 0.f;
      if (qdset) qdset[(size_t)row * 18 + lane] = 0.f;
    }
    if (lane == 0) {
      if (value) value[row] = 0.f;
      if (status) status[row] = -1;
    }
    return;
  }
  const float* o = a.out + (size_t)s * OUT_F;
  if (lane < 18) {
    if (tau) tau[(size_t)row * 18 + lane] = o[O_TAU + lane];
    if (qset) qset[(size_t)row * 18 + lane] = o[O_QSET + lane];
    if (qdset) qdset[(size_t)row * 18 + lane] = o[O_QDSET + lane];
  }
  if (lane == 0) {
    if (value) value[row] = o[O_V];
    if (status) status[row] = a.stat[(size_t)s * ST_I + T_STATUS];
  }
}

// ============================================================ host launchers
static int g_smem_configured = -1;

static cudaError_t configure_smem() {
  const int bytes = WARPS_PER_BLOCK * W_FLOATS * (int)sizeof(float);
  cudaError_t e;
  void (*ks[])(Arena, Batch, SolverParams) = {mpc_k_fused, mpc_k_setup, mpc_k_factor, mpc_k_admm, mpc_k_polish};
  for (auto k : ks) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

size_t smem_bytes_per_block() { return (size_t)WARPS_PER_BLOCK * W_FLOATS * sizeof(float); }

cudaError_t launch_solve(const Arena& a, const Batch& b, const SolverParams& prm, int form, int grid_fused,
                         cudaStream_t st, int* launches) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (g_smem_configured != dev) {
    cudaError_t e = configure_smem();
    if (e != cudaSuccess) return e;
    g_smem_configured = dev;
  }
  if (b.n <= 0) return cudaSuccess;
  const size_t smem = smem_bytes_per_block();
  const int blocks = (b.n + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
  const dim3 thr(WARPS_PER_BLOCK * 32);
  if (form == 1) {
    const int g = grid_fused > 0 ? (grid_fused < blocks ? grid_fused : blocks) : blocks;
    mpc_k_fused<<<g, thr, smem, st>>>(a, b, prm);
    if (launches) *launches += 1;
  } else {
    mpc_k_setup<<<blocks, thr, smem, st>>>(a, b, prm);
    mpc_k_factor<<<blocks, thr, smem, st>>>(a, b, prm);
    mpc_k_admm<<<blocks, thr, smem, st>>>(a, b, prm);
    mpc_k_polish<<<blocks, thr, smem, st>>>(a, b, prm);
    mpc_k_torque<<<blocks, thr, 0, st>>>(a, b);
    if (launches) *launches += 5;
  }
  return cudaGetLastError();
}

cudaError_t launch_gather(const Arena& a, int n, const int* ids, float* tau, float* qset, float* qdset,
                          float* value, int* status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  const int blocks = (n * 32 + threads - 1) / threads;
  mpc_k_gather<<<blocks, threads, 0, st>>>(a, n, ids, tau, qset, qdset, value, status);
  return cudaGetLastError();
}

}  // namespace mpc
