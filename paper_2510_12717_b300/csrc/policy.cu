// Residual policy and joint-torque blending after the MPC solve (paper Sec. IV
// "Residual Architecture" and "Blending Strategy", Eq. joint-torque): per
// agent the observation o = [p, theta, q_j, omega, v, qdot_j, phi(5), V_MPC]
// in R^54, an MLP of three 256-wide ELU layers to leg actions a in R^10, and
// tau = tau_MPC + lambda (K_p (a + q_hat - q) - K_d qdot) on the leg joints.
//
// The MLP is a batched dense contraction, run on the tensor cores: a block
// takes 32 agents (two m16 tiles, sharing every weight fragment) through every layer with mma.m16n8k16 bf16
// (FP32 accumulation), its four warps splitting each layer's 256 outputs
// (64 columns each); a layer's inputs are bfloat16 rows in the block's shared
// memory, its weights bfloat16 in global memory transposed to [out][in] so
// that a B fragment (two consecutive k of one column) is one 32-bit load; the
// epilogue adds the bias, applies ELU and writes the next layer's bfloat16
// inputs.
#include <cuda_bf16.h>
#include <stdint.h>
#include "solver_dev.cuh"
#include "policy.h"

namespace mpc {
namespace {

constexpr int PA_LD = 264;                 // bf16 row stride of the activations (256 + 8)
constexpr int PA_ROWS = 32;                // agents per block (two m16 tiles)
constexpr int PA_MT = PA_ROWS / 16;
constexpr int PA_WARPS = 4;                // each takes 64 of a layer's 256 outputs
constexpr int PA_BYTES = 2 * PA_ROWS * PA_LD * 2;        // two activation buffers

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float* c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// out[16 x 64-column slice] = act(in[16 x K] W + b) for one warp; K a
// multiple of 16 (compile-time, so the loops unroll and the weight loads run
// ahead); the block synchronises before the next layer reads out
template <bool ELU, int K>
__device__ __forceinline__ void dense_layer(const __nv_bfloat16* in, __nv_bfloat16* out, const __nv_bfloat16* WT,
                                            const float* bias, int n0, int lane) {
  const int g = lane >> 2, t = lane & 3;
  float acc[PA_MT][8][4];
#pragma unroll
  for (int m = 0; m < PA_MT; ++m)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[m][j][0] = acc[m][j][1] = acc[m][j][2] = acc[m][j][3] = 0.f;
#pragma unroll
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[PA_MT][4];
#pragma unroll
    for (int m = 0; m < PA_MT; ++m) {
      const __nv_bfloat16* r0 = in + (16 * m + g) * PA_LD + k0 + 2 * t;
      a[m][0] = ld32(r0);
      a[m][1] = ld32(r0 + 8 * PA_LD);
      a[m][2] = ld32(r0 + 8);
      a[m][3] = ld32(r0 + 8 * PA_LD + 8);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const __nv_bfloat16* w = WT + (size_t)(n0 + 8 * j + g) * K + k0 + 2 * t;
      const uint32_t b0 = ld32(w), b1 = ld32(w + 8);
#pragma unroll
      for (int m = 0; m < PA_MT; ++m) mma_bf16(acc[m][j], a[m][0], a[m][1], a[m][2], a[m][3], b0, b1);
    }
  }
#pragma unroll
  for (int m = 0; m < PA_MT; ++m)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = n0 + 8 * j + 2 * t;
      float v[4] = {acc[m][j][0] + bias[col], acc[m][j][1] + bias[col + 1], acc[m][j][2] + bias[col],
                    acc[m][j][3] + bias[col + 1]};
      if (ELU) {
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = v[c] > 0.f ? v[c] : expm1f(v[c]);
      }
      __nv_bfloat16* o = out + (16 * m + g) * PA_LD + col;
      *reinterpret_cast<__nv_bfloat162*>(o) = __floats2bfloat162_rn(v[0], v[1]);
      *reinterpret_cast<__nv_bfloat162*>(o + 8 * PA_LD) = __floats2bfloat162_rn(v[2], v[3]);
    }
}

// observation entry c of agent ap (see the header)
__device__ __forceinline__ float obs_entry(const AgentPtrs& ap, int c) {
  const float* x0 = ap.inp + I_X0;
  if (c < 6) return x0[c];                              // p, theta
  if (c < 24) return x0[12 + (c - 6)];                  // q_j
  if (c < 27) return x0[9 + (c - 24)];                  // omega
  if (c < 30) return x0[6 + (c - 27)];                  // v
  if (c < 48) return ap.inp[I_QD + (c - 30)];           // qdot_j (measured)
  const float ph = ap.inp[I_PHASE];
  if (c == 48) return ph;
  if (c == 53) return ap.out[O_V];
  const int f = (c - 49) >> 1;
  float s, co;
  sincospif(2.f * (ph + (float)ap.sch[S_OFF + f]), &s, &co);
  return ((c - 49) & 1) ? co : s;
}

__global__ void __launch_bounds__(PA_WARPS * 32) mpc_k_policy(Arena a, int n, const int* ids, PolicyDev pol,
                                                              float* tau, float* act) {
  extern __shared__ __align__(16) uint8_t psm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * PA_ROWS;
  __nv_bfloat16* bufA = reinterpret_cast<__nv_bfloat16*>(psm);
  __nv_bfloat16* bufB = bufA + PA_ROWS * PA_LD;
  // layer-1 input: the observations, zero-padded to K = 64 (and rows past n)
  for (int idx = threadIdx.x; idx < PA_ROWS * POL_K1; idx += PA_WARPS * 32) {
    const int r = idx / POL_K1, c = idx - r * POL_K1;
    float v = 0.f;
    if (row0 + r < n && c < POL_OBS) v = obs_entry(agent_ptrs(a, ids[row0 + r]), c);
    bufA[r * PA_LD + c] = __float2bfloat16_rn(v);
  }
  __syncthreads();
  const int n0 = 64 * warp;
  dense_layer<true, POL_K1>(bufA, bufB, pol.W1, pol.b1, n0, lane);
  __syncthreads();
  dense_layer<true, POL_HID>(bufB, bufA, pol.W2, pol.b2, n0, lane);
  __syncthreads();
  dense_layer<true, POL_HID>(bufA, bufB, pol.W3, pol.b3, n0, lane);
  __syncthreads();
  // output layer: N = 16 (10 actions + zero padding), FP32 result; warp w
  // sums the k range [64 w, 64 w + 64), the partial sums meet in shared memory
  const int g = lane >> 2, t = lane & 3;
  float acc[PA_MT][2][4];
#pragma unroll
  for (int m = 0; m < PA_MT; ++m)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[m][j][0] = acc[m][j][1] = acc[m][j][2] = acc[m][j][3] = 0.f;
#pragma unroll
  for (int k0 = 64 * warp; k0 < 64 * warp + 64; k0 += 16) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const __nv_bfloat16* w = pol.W4 + (size_t)(8 * j + g) * POL_HID + k0 + 2 * t;
      const uint32_t b0 = ld32(w), b1 = ld32(w + 8);
#pragma unroll
      for (int m = 0; m < PA_MT; ++m) {
        const __nv_bfloat16* r0 = bufB + (16 * m + g) * PA_LD + k0 + 2 * t;
        mma_bf16(acc[m][j], ld32(r0), ld32(r0 + 8 * PA_LD), ld32(r0 + 8), ld32(r0 + 8 * PA_LD + 8), b0, b1);
      }
    }
  }
  float* part = reinterpret_cast<float*>(bufA);         // [4 warps][PA_ROWS x 16]
  float* pw = part + warp * PA_ROWS * 16;
#pragma unroll
  for (int m = 0; m < PA_MT; ++m)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int col = 8 * j + 2 * t, r = 16 * m + g;
      pw[r * 16 + col] = acc[m][j][0];
      pw[r * 16 + col + 1] = acc[m][j][1];
      pw[(r + 8) * 16 + col] = acc[m][j][2];
      pw[(r + 8) * 16 + col + 1] = acc[m][j][3];
    }
  __syncthreads();
  // blend (Eq. joint-torque) on the legs; arms keep the MPC torque
  for (int idx = threadIdx.x; idx < PA_ROWS * 18; idx += PA_WARPS * 32) {
    const int r = idx / 18, j = idx - r * 18;
    if (row0 + r >= n) continue;
    const AgentPtrs ap = agent_ptrs(a, ids[row0 + r]);
    float out = ap.out[O_TAU + j];
    if (j < POL_ACT) {
      const int P = PA_ROWS * 16;
      const float aj = part[r * 16 + j] + part[P + r * 16 + j] + part[2 * P + r * 16 + j] +
                       part[3 * P + r * 16 + j] + pol.b4[j];
      const float q = ap.inp[I_X0 + 12 + j], qd = ap.inp[I_QD + j];
      const float res = ap.mdl[M_KP + j] * (aj + ap.mdl[M_QNOM + j] - q) - ap.mdl[M_KD + j] * qd;
      out = fmaf(pol.lambda, res, out);
      if (act) act[(size_t)(row0 + r) * POL_ACT + j] = aj;
    }
    if (tau) tau[(size_t)(row0 + r) * 18 + j] = out;
  }
}

}  // namespace

size_t policy_smem_bytes() { return (size_t)PA_BYTES; }

cudaError_t launch_policy(const Arena& a, int n, const int* ids, const PolicyDev& pol, float* tau, float* act,
                          cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(mpc_k_policy, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)policy_smem_bytes());
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int blocks = (n + PA_ROWS - 1) / PA_ROWS;
  mpc_k_policy<<<blocks, PA_WARPS * 32, policy_smem_bytes(), st>>>(a, n, ids, pol, tau, act);
  return cudaGetLastError();
}

}  // namespace mpc
