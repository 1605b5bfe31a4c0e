// Device code of the batched MPC solver: one warp solves one agent.
//
// Lane i (< 30) owns index i of the state x and the input u (layout in
// arena.h).  Lanes 0-21 carry the coupled base+leg block, whose stage
// matrices are dense 22x22 blocks kept column-major with stride LD = 23 in
// shared memory (an odd stride makes both row and column walks bank-conflict
// free); lanes 22-29 carry the eight decoupled arm joints as scalars.
//
// Paper mapping (Alg. 1):
//   f_init/f_param    -> setup_agent()   contact schedule, references, bounds,
//                                        warm or cold start
//   f_KKT             -> setup_agent()   linearisation (analytic Jacobians)
//                        factor()        per-stage KKT blocks (assembly)
//   cuDSS_fac         -> factor()        backward Riccati recursion
//   cuDSS_solve       -> sweep()         backward/forward linear sweeps
//   f_ADMM            -> admm_*()        relaxation, projection, dual update,
//                                        residuals, rho update
//   line search       -> alpha = 1 (the solution is the final iterate)
//   f_RNEA + PD law   -> torque_map()
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include "arena.h"

namespace mpc {

constexpr float GRAV = 9.81f;
constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------- smem map
// per-warp shared workspace (floats)
enum : int {
  W_ABASE = 0, W_B = MB, W_P = 2 * MB, W_AK = 3 * MB, W_PA = 4 * MB, W_PB = 5 * MB,
  W_H = 6 * MB, W_X = 7 * MB, W_K = 8 * MB, W_VEC = 9 * MB, NVEC = 16,
  W_FLOATS = 9 * MB + NVEC * 64
};
// vector slots inside W_VEC (64 floats each)
enum : int { V_S = 0, V_H = 1, V_X = 2, V_U = 3, V_XN = 4, V_ROW = 5, V_ROW2 = 6,
             V_T = 7, V_G = 8, V_MISC = 9, V_FLAGS = 10, V_LO = 11, V_HI = 12, V_CLS = 13 };

struct AgentPtrs {
  const float* mdl;
  const double* sch;
  int N;
  float *x, *u, *w, *y, *rho;
  int* warm;
  float *inp, *xref, *uref, *rlo, *rhi, *rcls, *lin, *cK, *cH, *cE, *cB, *cC, *xt, *ut, *dv;
  int* act;
  float* out;
  int* st;
};

__device__ __forceinline__ AgentPtrs agent_ptrs(const Arena& a, int s) {
  AgentPtrs p;
  const int n = a.maxN;
  p.mdl = a.model + (size_t)s * MODEL_F;
  p.sch = a.sched + (size_t)s * SCHED_D;
  p.N = a.horizon[s];
  p.x = a.xs + (size_t)s * (n + 1) * VS;
  p.u = a.us + (size_t)s * n * VS;
  p.w = a.ws + (size_t)s * n * RS;
  p.y = a.ys + (size_t)s * n * RS;
  p.rho = a.rho + s;
  p.warm = a.warm_valid + s;
  p.inp = a.inp + (size_t)s * IN_F;
  p.xref = a.xref + (size_t)s * (n + 1) * VS;
  p.uref = a.uref + (size_t)s * n * VS;
  p.rlo = a.rlo + (size_t)s * n * RS;
  p.rhi = a.rhi + (size_t)s * n * RS;
  p.rcls = a.rcls + (size_t)s * n * RS;
  p.lin = a.lin + (size_t)s * lin_floats(n);
  p.cK = a.cK + (size_t)s * n * MB;
  p.cH = a.cH + (size_t)s * n * MB;
  p.cE = a.cE + (size_t)s * n * 64;
  p.cB = a.cB + (size_t)s * n * MB;
  p.cC = a.cC + (size_t)s * n * 64;
  p.xt = a.xt + (size_t)s * (n + 1) * VS;
  p.ut = a.ut + (size_t)s * n * VS;
  p.dv = a.dv + (size_t)s * n * VS;
  p.act = a.act + (size_t)s * n * RS;
  p.out = a.out + (size_t)s * OUT_F;
  p.st = a.stat + (size_t)s * ST_I;
  return p;
}

// ------------------------------------------------------- warp reductions
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}
__device__ __forceinline__ int warp_or(int v) { return __any_sync(FULL, v); }

// ------------------------------------------------- dense 22x22 warp algebra
// Block element (i, j) sits at j*LD + i.  Lanes >= NC compute on a clamped
// index and never store.

// C = op(A) op(B) (+ Cadd).  C must not alias A or B; Cadd may alias C.
template <bool TA, bool TB>
__device__ __forceinline__ void wgemm(float* C, const float* A, const float* B,
                                      const float* Cadd, float alpha, int lane) {
  const int i = lane < NC ? lane : NC - 1;
  float acc[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) acc[j] = 0.f;
#pragma unroll 2
  for (int k = 0; k < NC; ++k) {
    const float a = TA ? A[i * LD + k] : A[k * LD + i];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const float b = TB ? B[k * LD + j] : B[j * LD + k];
      acc[j] = fmaf(a, b, acc[j]);
    }
  }
  __syncwarp();
  if (lane < NC) {
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      float v = alpha * acc[j];
      if (Cadd) v += Cadd[j * LD + i];
      C[j * LD + i] = v;
    }
  }
  __syncwarp();
}

// y_i = sum_j op(M)(i, j) v_j for the lane's row i (< NC)
template <bool TM>
__device__ __forceinline__ float wmv(const float* M, const float* v, int lane) {
  const int i = lane < NC ? lane : NC - 1;
  float a0 = 0.f, a1 = 0.f;
#pragma unroll
  for (int j = 0; j < NC; j += 2) {
    a0 = fmaf(TM ? M[i * LD + j] : M[j * LD + i], v[j], a0);
    a1 = fmaf(TM ? M[i * LD + j + 1] : M[(j + 1) * LD + i], v[j + 1], a1);
  }
  return a0 + a1;
}

// In-place inverse of a symmetric positive definite block by Gauss-Jordan
// elimination without pivoting; lane j updates column j.
__device__ __forceinline__ void winv(float* H, int lane) {
  const int j = lane < NC ? lane : NC - 1;
  for (int p = 0; p < NC; ++p) {
    float col[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) col[i] = H[p * LD + i];
    const float rowp = H[j * LD + p];
    const float inv = 1.f / col[p];
    __syncwarp();
    if (lane < NC) {
      if (j == p) {
#pragma unroll
        for (int i = 0; i < NC; ++i) H[j * LD + i] = (i == p) ? inv : -col[i] * inv;
      } else {
        const float rp = rowp * inv;
#pragma unroll
        for (int i = 0; i < NC; ++i)
          H[j * LD + i] = (i == p) ? rp : fmaf(-col[i], rp, H[j * LD + i]);
      }
    }
    __syncwarp();
  }
}

// copy a 22x22 block (MB floats) between memories, whole warp
__device__ __forceinline__ void wcopy_block(float* dst, const float* src, int lane) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
  float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int t = lane; t < MB / 4; t += 32) d4[t] = s4[t];
}

// ----------------------------------------------------------- row algebra
// Stage rows (paper Eq. mpc_formulation constraints, row layout as in the
// include file): 0-11 wrench box, 12-19 friction pyramid, 20-37 joint-rate
// box, 38-55 joint box on x_{k+1}.

// (C_u^T v)_i for u index i, v = 56 row values
__device__ __forceinline__ float cuT(const float* v, int i, float mu) {
  if (i < 12) {
    const int f = i / 6, c = i - 6 * f, p = 12 + 4 * f;
    float r = v[i];
    if (c == 0) r += v[p] - v[p + 1];
    else if (c == 1) r += v[p + 2] - v[p + 3];
    else if (c == 2) r -= mu * (v[p] + v[p + 1] + v[p + 2] + v[p + 3]);
    return r;
  }
  return i < 30 ? v[i + 8] : 0.f;
}
// (C_x^T v)_i for x index i
__device__ __forceinline__ float cxT(const float* v, int i) {
  return (i >= 12 && i < 30) ? v[i + 26] : 0.f;
}
// row value r of C_u u + C_x xn
__device__ __forceinline__ float crow(const float* u, const float* xn, int r, float mu) {
  if (r < 12) return u[r];
  if (r < 20) {
    const int f = (r - 12) >> 2, t = (r - 12) & 3, b = 6 * f;
    const float fz = u[b + 2];
    switch (t) {
      case 0: return u[b] - mu * fz;
      case 1: return -u[b] - mu * fz;
      case 2: return u[b + 1] - mu * fz;
      default: return -u[b + 1] - mu * fz;
    }
  }
  if (r < 38) return u[r - 8];
  return xn[r - 26];
}

// ------------------------------------------------------------ 3x3 helpers
struct M3 { float m[9]; };
__device__ __forceinline__ float m3(const M3& a, int r, int c) { return a.m[3 * r + c]; }
__device__ __forceinline__ M3 mul3(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q)
      c.m[3 * r + q] = a.m[3 * r] * b.m[q] + a.m[3 * r + 1] * b.m[3 + q] + a.m[3 * r + 2] * b.m[6 + q];
  return c;
}
__device__ __forceinline__ M3 skew3(float x, float y, float z) {
  M3 s = {{0.f, -z, y, z, 0.f, -x, -y, x, 0.f}};
  return s;
}

}  // namespace mpc
