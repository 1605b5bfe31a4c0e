// Device code of the batched MPC solver: one warp solves one agent.
//
// Lane i (< 30) owns index i of the state x and the input u (layout in
// arena.h).  Lanes 0-21 carry the coupled base+leg block; lanes 22-29 the
// eight decoupled arm joints as scalar problems.
//
// Dense 22x22 blocks (Riccati P, H_uu^-1, H_ux, K) are row-major with stride
// 24 ("R24"): element (i, j) at i*24 + j.  A lane reading M(k, lane) walks
// consecutive banks, and a row M(k, 0..23) is 16-byte aligned so it can be
// broadcast with float4 loads.  The stage matrices A_k and B are sparse with
// a fixed pattern (the model's block structure); they are kept as compact
// columns (at most 6 nonzeros per column, values in shared memory, row
// indices known at compile time), plus one dense column-major copy (stride
// 23) of A_base and B for the row-oriented products of the forward rollout.
//
// Paper mapping (Alg. 1):
//   f_init/f_param    -> setup_agent()   contact schedule, references, bounds,
//                                        warm or cold start
//   f_KKT             -> setup_agent()   linearisation (analytic Jacobians)
//                        factor()        per-stage KKT blocks (assembly)
//   cuDSS_fac         -> factor()        backward Riccati recursion
//   cuDSS_solve       -> sweep           backward/forward linear sweeps
//   f_ADMM            -> admm_*()        relaxation, projection, dual update,
//                                        residuals, rho update
//   line search       -> alpha = 1 (the solution is the final iterate)
//   f_RNEA + PD law   -> torque_map()
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include "arena.h"

namespace mpc {

constexpr float GRAV = 9.81f;
constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------- smem map
// per-warp shared workspace (floats); R24 blocks are BLK floats
enum : int {
  S_P = 0, S_H = BLK, S_X = 2 * BLK, S_K = 3 * BLK,     // factor blocks / sweep double buffers
  S_AB = 4 * BLK,                                        // dense A_base, column-major LD = 23
  S_B = S_AB + 512,                                      // dense B (or B_hat), column-major LD = 23
  S_AV = S_B + 512,                                      // compact A_k columns: 22 x 6
  S_BV = S_AV + 136,                                     // compact B columns: 22 x 6
  S_VEC = S_BV + 136,                                    // 12 vectors of 64
  S_BAR = S_VEC + 12 * 64,                               // 4 mbarriers (32 bytes)
  W_FLOATS = S_BAR + 8
};
enum : int { V_S = 0, V_H = 1, V_X = 2, V_U = 3, V_XN = 4, V_ROW = 5, V_T = 6, V_G = 7,
             V_C = 8, V_FLAGS = 9, V_ACT = 10, V_D = 11 };
constexpr int LDD = 23;   // stride of the dense column-major copies

struct AgentPtrs {
  const float* mdl;
  const double* sch;
  int N;
  float *x, *u, *w, *y, *rho;
  int* warm;
  float *inp, *xref, *uref, *rlo, *rhi, *rcls, *lin, *cK, *cH, *cE, *cEl, *cD, *xt, *ut, *dv;
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
  p.cK = a.cK + (size_t)s * n * BLK;
  p.cH = a.cH + (size_t)s * n * BLK;
  p.cE = a.cE + (size_t)s * n * 64;
  p.cEl = a.cEl + (size_t)s * n * 128;
  p.cD = a.cD + (size_t)s * n * VS;
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

// ------------------------------------------------- sparsity of A_k and B
// Compact column j holds the nonzero rows of column j, at most 6.
//   A = I + dt f_x:  p <- v, Theta <- Theta (pitch, yaw columns), Theta <- w,
//                    w <- w (gyroscopic), w <- leg joints (contact dependent)
//   B = dt f_u:      v, w <- foot forces; w <- foot moments; q_leg <- qdot_leg
// (polish's B_hat = B G keeps the same pattern: G mixes forces within a foot)
__host__ __device__ constexpr int acnt(int j) { return j < 4 ? 1 : j < 6 ? 3 : j < 9 ? 2 : j < 12 ? 6 : 4; }
__host__ __device__ constexpr int arow(int j, int t) {
  return j < 4 ? j : j < 6 ? 3 + t : j < 9 ? (t == 0 ? j : j - 6) : j < 12 ? (t < 3 ? 3 + t : 6 + t)
                                                                          : (t == 0 ? j : 8 + t);
}
__host__ __device__ constexpr int bcnt(int j) { return j < 12 ? ((j % 6) < 3 ? 6 : 3) : 1; }
__host__ __device__ constexpr int brow(int j, int t) {
  return j < 12 ? ((j % 6) < 3 ? 6 + t : 9 + t) : j;
}

// ------------------------------------------------- dense R24 warp algebra
// C = alpha * A^T B (+ Cadd):  lane i computes row i of C.  A(k, i) is read by
// the lane (consecutive banks), B(k, 0..21) is broadcast with float4 loads.
// C may alias Cadd but not A or B.
__device__ __forceinline__ void r24_gemm_tn(float* C, const float* A, const float* B, const float* Cadd,
                                            float alpha, int lane) {
  // one pass of 22 accumulators (two passes of 12 re-read A and computed the
  // padding columns: 1.3 % slower on the warm replan, 3 % faster in the ADMM
  // iterations); the two padding columns (22, 23) of C are written as zero
  // (row-vector products read them)
  const int i = lane < NC ? lane : NC - 1;
  float4 out[6];
  {
    float acc[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = 0.f;
#pragma unroll 2
    for (int k = 0; k < NC; ++k) {
      const float a = A[k * R24 + i];
      const float4* b4 = reinterpret_cast<const float4*>(B + k * R24);
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        const float4 b = b4[m];
        acc[4 * m + 0] = fmaf(a, b.x, acc[4 * m + 0]);
        acc[4 * m + 1] = fmaf(a, b.y, acc[4 * m + 1]);
        acc[4 * m + 2] = fmaf(a, b.z, acc[4 * m + 2]);
        acc[4 * m + 3] = fmaf(a, b.w, acc[4 * m + 3]);
      }
      const float2 b2 = *reinterpret_cast<const float2*>(B + k * R24 + 20);
      acc[20] = fmaf(a, b2.x, acc[20]);
      acc[21] = fmaf(a, b2.y, acc[21]);
    }
#pragma unroll
    for (int m = 0; m < 5; ++m)
      out[m] = make_float4(alpha * acc[4 * m], alpha * acc[4 * m + 1], alpha * acc[4 * m + 2], alpha * acc[4 * m + 3]);
    out[5] = make_float4(alpha * acc[20], alpha * acc[21], 0.f, 0.f);
  }
  __syncwarp();
  if (lane < NC) {
    float4* c4 = reinterpret_cast<float4*>(C + i * R24);
    const float4* d4 = reinterpret_cast<const float4*>(Cadd + i * R24);
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      float4 v = out[m];
      if (Cadd) {
        const float4 d = d4[m];
        v.x += d.x; v.y += d.y;
        if (m < 5) { v.z += d.z; v.w += d.w; }   // columns 22, 23 stay zero
      }
      c4[m] = v;
    }
  }
  __syncwarp();
}

// y_i = sum_j M(j, i) v_j  (M^T v; for symmetric M this is M v)
__device__ __forceinline__ float r24_mtv(const float* M, const float* v, int lane) {
  const int i = lane < NC ? lane : NC - 1;
  float a0 = 0.f, a1 = 0.f;
#pragma unroll
  for (int j = 0; j < NC; j += 2) {
    a0 = fmaf(M[j * R24 + i], v[j], a0);
    a1 = fmaf(M[(j + 1) * R24 + i], v[j + 1], a1);
  }
  return a0 + a1;
}
// (M1^T v)_i and (M2^T v)_i in one pass: four independent sums, each matrix's
// in the order of r24_mtv (same results, half the dependent chain)
__device__ __forceinline__ float2 r24_mtv2(const float* M1, const float* M2, const float* v, int lane) {
  const int i = lane < NC ? lane : NC - 1;
  float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
#pragma unroll
  for (int j = 0; j < NC; j += 2) {
    const float v0 = v[j], v1 = v[j + 1];
    a0 = fmaf(M1[j * R24 + i], v0, a0);
    a1 = fmaf(M1[(j + 1) * R24 + i], v1, a1);
    b0 = fmaf(M2[j * R24 + i], v0, b0);
    b1 = fmaf(M2[(j + 1) * R24 + i], v1, b1);
  }
  return make_float2(a0 + a1, b0 + b1);
}
// y_i = sum_j M(i, j) v_j  (row of the lane, float4 loads)
__device__ __forceinline__ float r24_mv(const float* M, const float* v, int lane) {
  const int i = lane < NC ? lane : NC - 1;
  const float4* m4 = reinterpret_cast<const float4*>(M + i * R24);
  const float4* v4 = reinterpret_cast<const float4*>(v);
  float a0 = 0.f, a1 = 0.f;
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    const float4 a = m4[m], b = v4[m];
    a0 = fmaf(a.x, b.x, a0); a1 = fmaf(a.y, b.y, a1);
    a0 = fmaf(a.z, b.z, a0); a1 = fmaf(a.w, b.w, a1);
  }
  return a0 + a1;
}

// In-place inverse of a symmetric positive definite R24 block by the sweep
// operator (Goodnight 1979) on 2 x 2 pivot blocks: sweeping the index pair
// S = {k, k+1} with B = M_SS maps
//   M_SS <- -B^-1,  M_iS <- M_iS B^-1,  M_Sj <- B^-1 M_Sj,
//   M_ij <- M_ij - M_iS B^-1 M_Sj   (i, j outside S),
// keeps M symmetric, and equals sweeping k and then k+1 one at a time; after
// all eleven pairs M holds -M^-1.  Lane j keeps column j in registers; the
// columns k and k+1 every lane needs are, by symmetry, the rows k and k+1 of
// the lanes' own columns: one shared-memory write per lane and row, double
// buffered in sc (2 buffers x 2 rows x 32 floats, 16-byte aligned), and one
// warp barrier per pair.  A pair writes the next pair's rows first, into the
// other buffer, which every lane finished reading at the pair before.
__device__ __forceinline__ void r24_inv(float* H, float* sc, int lane) {
  const int j = lane < NC ? lane : NC - 1;
  float h[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) h[i] = H[i * R24 + j];
  sc[lane] = h[0];
  sc[32 + lane] = h[1];
#pragma unroll
  for (int r = 0; r < NC / 2; ++r) {
    const int k = 2 * r;
    __syncwarp();
    const float* V0 = sc + (r & 1) * 64;   // column k
    const float* V1 = V0 + 32;             // column k + 1
    const float a = V0[k], b = V0[k + 1], c = V1[k + 1];
    // the pivot block of an SPD matrix is SPD, its determinant well away from
    // 0: the fast reciprocal (2 ulp) is ample
    const float id = __fdividef(1.f, fmaf(a, c, -b * b));
    const bool s0 = j == k, s1 = j == k + 1, in = s0 || s1;
    // lanes outside S: y = B^-1 M_Sj; lanes in S: their new entries are
    // M_iS B^-1 e_j (their old column is dropped: keep = 0)
    float y0 = id * fmaf(c, h[k], -b * h[k + 1]);
    float y1 = id * fmaf(a, h[k + 1], -b * h[k]);
    if (s0) { y0 = -id * c; y1 = id * b; }
    if (s1) { y0 = id * b; y1 = -id * a; }
    const float keep = in ? 0.f : 1.f;
    // the next pair's rows first
    if (r + 1 < NC / 2) {
      float* N0 = sc + ((r + 1) & 1) * 64;
      h[k + 2] = fmaf(-V0[k + 2], y0, fmaf(-V1[k + 2], y1, keep * h[k + 2]));
      h[k + 3] = fmaf(-V0[k + 3], y0, fmaf(-V1[k + 3], y1, keep * h[k + 3]));
      N0[lane] = h[k + 2];
      N0[32 + lane] = h[k + 3];
    }
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      if (i == k || i == k + 1 || i == k + 2 || i == k + 3) continue;
      h[i] = fmaf(-V0[i], y0, fmaf(-V1[i], y1, keep * h[i]));
    }
    // M_SS <- -B^-1 on the lanes in S, M_Sj <- B^-1 M_Sj elsewhere
    if (s0) { h[k] = -id * c; h[k + 1] = id * b; }
    else if (s1) { h[k] = id * b; h[k + 1] = -id * a; }
    else { h[k] = y0; h[k + 1] = y1; }
  }
  if (lane < NC) {
#pragma unroll
    for (int i = 0; i < NC; ++i) H[i * R24 + j] = -h[i];
  }
  __syncwarp();
}

// The same inverse with the sweep in FP64 (the stage Schur complement where
// conditioning needs it); H in and out stays FP32.  sc: 2 x 32 doubles
// (16-byte aligned).  A pivot reads the row back element by element, so the
// row is not held in registers twice.
static __device__ __noinline__ void r24_inv_f64(float* H, double* sc, int lane) {
  const int j = lane < NC ? lane : NC - 1;
  double h[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) h[i] = (double)H[i * R24 + j];
  sc[lane] = h[0];
#pragma unroll
  for (int p = 0; p < NC; ++p) {
    __syncwarp();
    const double* v = sc + (p & 1) * 32;
    const double inv = 1.0 / v[p];
    double* nxt = sc + ((p + 1) & 1) * 32;
    if (j == p) {
      if (p + 1 < NC) { h[p + 1] = -h[p + 1] * inv; nxt[lane] = h[p + 1]; }
#pragma unroll
      for (int i = 0; i < NC; ++i)
        if (i != p && i != p + 1) h[i] = -h[i] * inv;
      h[p] = inv;
    } else {
      const double rp = h[p] * inv;
      if (p + 1 < NC) { h[p + 1] = fma(-v[p + 1], rp, h[p + 1]); nxt[lane] = h[p + 1]; }
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        if (i == p || i == p + 1) continue;
        const double ci = i < p ? -v[i] : v[i];
        h[i] = fma(-ci, rp, h[i]);
      }
      h[p] = rp;
    }
  }
  if (lane < NC) {
#pragma unroll
    for (int i = 0; i < NC; ++i) H[i * R24 + j] = (float)h[i];
  }
  __syncwarp();
}

// ------------------------------------------------- tensor-core R24 products
// C = alpha * A^T B (+ Cadd) for the 22 x 22 blocks on the warp's tensor
// cores (mma.sync), FP32 accumulation: M = 22 padded to 32 (two m16 tiles),
// N = 22 padded to 24 (three n8 tiles), K = 22 padded to 24 (TF32, k8) or 32
// (BF16, k16).  Padding reads as zero; the padding columns of C are written
// as zero.  Fragment layouts (PTX ISA, mma.m16n8k8 .tf32 / m16n8k16 .bf16):
// g = lane / 4, t = lane % 4;  C: (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1).
// PREC_TF32X3: error-compensated split TF32 (Ootomo and Yokota, 2022): each
// operand x = hi + lo with hi = tf32(x) and lo = tf32(x - hi), and
// A B = A_hi B_hi + A_hi B_lo + A_lo B_hi (the A_lo B_lo term, 2^-22 of the
// product, is dropped): three mma per tile, FP32-level accuracy.
enum : int { PREC_FP32 = 0, PREC_TF32 = 1, PREC_BF16 = 2, PREC_FP64 = 3, PREC_TF32X3 = 4 };
// kernel specialisation: PREC_FP32 compiles the FP32 factor only; PREC_ANY
// reads the precision at run time
constexpr int PREC_ANY = -1;

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// the split of TF32X3: hi = tf32(x), lo = tf32(x - hi)
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
// A^T(m, k) = A[k][m] and B(k, n) with the 22 x 22 bounds applied
__device__ __forceinline__ float r24_at(const float* A, int k, int m) {
  return (k < NC && m < NC) ? A[k * R24 + m] : 0.f;
}

template <int P>
__device__ __noinline__ void r24_gemm_tn_mma(float* C, const float* A, const float* B, const float* Cadd,
                                             float alpha, int lane) {
  const int g = lane >> 2, t = lane & 3;
  float acc[2][3][4];
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 3; ++ni)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[mi][ni][c] = 0.f;
  if (P == PREC_TF32X3) {
#pragma unroll
    for (int k0 = 0; k0 < 24; k0 += 8) {
      uint32_t ah[2][4], al[2][4], bh[3][2], bl[3][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int m = 16 * mi + g;
        split_tf32(r24_at(A, k0 + t, m), ah[mi][0], al[mi][0]);
        split_tf32(r24_at(A, k0 + t, m + 8), ah[mi][1], al[mi][1]);
        split_tf32(r24_at(A, k0 + t + 4, m), ah[mi][2], al[mi][2]);
        split_tf32(r24_at(A, k0 + t + 4, m + 8), ah[mi][3], al[mi][3]);
      }
#pragma unroll
      for (int ni = 0; ni < 3; ++ni) {
        const int n = 8 * ni + g;
        split_tf32(r24_at(B, k0 + t, n), bh[ni][0], bl[ni][0]);
        split_tf32(r24_at(B, k0 + t + 4, n), bh[ni][1], bl[ni][1]);
      }
      // the small terms first, then the leading one
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 3; ++ni) {
          asm volatile(
              "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};"
              : "+f"(acc[mi][ni][0]), "+f"(acc[mi][ni][1]), "+f"(acc[mi][ni][2]), "+f"(acc[mi][ni][3])
              : "r"(al[mi][0]), "r"(al[mi][1]), "r"(al[mi][2]), "r"(al[mi][3]), "r"(bh[ni][0]), "r"(bh[ni][1]));
          asm volatile(
              "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};"
              : "+f"(acc[mi][ni][0]), "+f"(acc[mi][ni][1]), "+f"(acc[mi][ni][2]), "+f"(acc[mi][ni][3])
              : "r"(ah[mi][0]), "r"(ah[mi][1]), "r"(ah[mi][2]), "r"(ah[mi][3]), "r"(bl[ni][0]), "r"(bl[ni][1]));
          asm volatile(
              "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};"
              : "+f"(acc[mi][ni][0]), "+f"(acc[mi][ni][1]), "+f"(acc[mi][ni][2]), "+f"(acc[mi][ni][3])
              : "r"(ah[mi][0]), "r"(ah[mi][1]), "r"(ah[mi][2]), "r"(ah[mi][3]), "r"(bh[ni][0]), "r"(bh[ni][1]));
        }
    }
  } else if (P == PREC_TF32) {
#pragma unroll
    for (int k0 = 0; k0 < 24; k0 += 8) {
      uint32_t a[2][4], b[3][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int m = 16 * mi + g;
        a[mi][0] = to_tf32(r24_at(A, k0 + t, m));
        a[mi][1] = to_tf32(r24_at(A, k0 + t, m + 8));
        a[mi][2] = to_tf32(r24_at(A, k0 + t + 4, m));
        a[mi][3] = to_tf32(r24_at(A, k0 + t + 4, m + 8));
      }
#pragma unroll
      for (int ni = 0; ni < 3; ++ni) {
        const int n = 8 * ni + g;
        b[ni][0] = to_tf32(r24_at(B, k0 + t, n));
        b[ni][1] = to_tf32(r24_at(B, k0 + t + 4, n));
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 3; ++ni)
          asm volatile(
              "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};"
              : "+f"(acc[mi][ni][0]), "+f"(acc[mi][ni][1]), "+f"(acc[mi][ni][2]), "+f"(acc[mi][ni][3])
              : "r"(a[mi][0]), "r"(a[mi][1]), "r"(a[mi][2]), "r"(a[mi][3]), "r"(b[ni][0]), "r"(b[ni][1]));
    }
  } else {
#pragma unroll
    for (int k0 = 0; k0 < 32; k0 += 16) {
      uint32_t a[2][4], b[3][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int m = 16 * mi + g;
        a[mi][0] = pack_bf16(r24_at(A, k0 + 2 * t, m), r24_at(A, k0 + 2 * t + 1, m));
        a[mi][1] = pack_bf16(r24_at(A, k0 + 2 * t, m + 8), r24_at(A, k0 + 2 * t + 1, m + 8));
        a[mi][2] = pack_bf16(r24_at(A, k0 + 2 * t + 8, m), r24_at(A, k0 + 2 * t + 9, m));
        a[mi][3] = pack_bf16(r24_at(A, k0 + 2 * t + 8, m + 8), r24_at(A, k0 + 2 * t + 9, m + 8));
      }
#pragma unroll
      for (int ni = 0; ni < 3; ++ni) {
        const int n = 8 * ni + g;
        b[ni][0] = pack_bf16(r24_at(B, k0 + 2 * t, n), r24_at(B, k0 + 2 * t + 1, n));
        b[ni][1] = pack_bf16(r24_at(B, k0 + 2 * t + 8, n), r24_at(B, k0 + 2 * t + 9, n));
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 3; ++ni)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};"
              : "+f"(acc[mi][ni][0]), "+f"(acc[mi][ni][1]), "+f"(acc[mi][ni][2]), "+f"(acc[mi][ni][3])
              : "r"(a[mi][0]), "r"(a[mi][1]), "r"(a[mi][2]), "r"(a[mi][3]), "r"(b[ni][0]), "r"(b[ni][1]));
    }
  }
  __syncwarp();
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 3; ++ni)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int row = 16 * mi + g + ((c & 2) ? 8 : 0);
        const int col = 8 * ni + 2 * t + (c & 1);
        if (row < NC) {
          float v = 0.f;
          if (col < NC) v = alpha * acc[mi][ni][c] + (Cadd ? Cadd[row * R24 + col] : 0.f);
          C[row * R24 + col] = v;
        }
      }
  __syncwarp();
}

// dense column-major (LDD) mat-vec, lane row i: sum_j M(i, j) v_j
__device__ __forceinline__ float cm_mv(const float* M, const float* v, int lane) {
  const int i = lane < NC ? lane : NC - 1;
  float a0 = 0.f, a1 = 0.f;
#pragma unroll
  for (int j = 0; j < NC; j += 2) {
    a0 = fmaf(M[j * LDD + i], v[j], a0);
    a1 = fmaf(M[(j + 1) * LDD + i], v[j + 1], a1);
  }
  return a0 + a1;
}

// the same product for a matrix with the sparsity of A_base and B (rows 0-11
// have their nonzeros in columns 0-11, rows 12-21 only on the diagonal):
// the structural zeros are skipped, the nonzero terms accumulate in the same
// two sums (even / odd columns) in the same order, so the result equals
// cm_mv's
__device__ __forceinline__ float cm_mv_s(const float* M, const float* v, int lane) {
  const int i = lane < NC ? lane : NC - 1;
  float a0 = 0.f, a1 = 0.f;
#pragma unroll
  for (int j = 0; j < 12; j += 2) {
    a0 = fmaf(M[j * LDD + i], v[j], a0);
    a1 = fmaf(M[(j + 1) * LDD + i], v[j + 1], a1);
  }
  const float m = i >= 12 ? M[i * LDD + i] : 0.f;
  if (i & 1) a1 = fmaf(m, v[i], a1);
  else a0 = fmaf(m, v[i], a0);
  return a0 + a1;
}

// compact-column transposed products for the lane's own column i:
// (A^T v)_i = sum_t A(arow(i,t), i) v[arow(i,t)]; runtime lane, so the
// pattern is read from per-lane registers filled by load_pattern().
struct LanePat { int ar[6], br[6]; };
__device__ __forceinline__ LanePat lane_pattern(int lane) {
  LanePat p;
  const int j = lane < NC ? lane : 0;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    p.ar[t] = t < acnt(j) ? arow(j, t) : 0;
    p.br[t] = t < bcnt(j) ? brow(j, t) : 0;
  }
  return p;
}
__device__ __forceinline__ float cc_tv(const float* val, const int* rows, const float* v, int lane) {
  const int j = lane < NC ? lane : 0;
  float a = 0.f;
#pragma unroll
  for (int t = 0; t < 6; ++t) a = fmaf(val[j * 6 + t], v[rows[t]], a);
  return a;
}

// the same product with the absolute values of the matrix (v >= 0): the
// magnitude of the terms that form (A^T v)_i
__device__ __forceinline__ float cc_tv_abs(const float* val, const int* rows, const float* v, int lane) {
  const int j = lane < NC ? lane : 0;
  float a = 0.f;
#pragma unroll
  for (int t = 0; t < 6; ++t) a = fmaf(fabsf(val[j * 6 + t]), v[rows[t]], a);
  return a;
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

// ------------------------------------------------- TMA bulk copies (1D)
// cp.async.bulk global -> shared, completion counted on an mbarrier.  Waits
// are bounded: after a given number of polls (SolverParams.spin_limit,
// kSpinLimit by default, arena.h) the wait gives up and reports it.

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// returns false if the phase did not complete within `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, int limit) {
  uint32_t done = 0;
  for (int it = 0; it < limit; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace mpc
