// Residual policy and joint-torque blending after the MPC solve (paper Sec. IV
// "Residual Architecture" and "Blending Strategy", Eq. joint-torque): per
// agent the observation o = [p, theta, q_j, omega, v, qdot_j, phi(5), V_MPC]
// in R^54, an MLP of three 256-wide ELU layers to leg actions a in R^10, and
// tau = tau_MPC + lambda (K_p (a + q_hat - q) - K_d qdot) on the leg joints.
//
// The MLP is a batched dense contraction, run on the tensor cores: one warp
// takes 16 agents (one m16 tile) through every layer with mma.m16n8k16 bf16
// (FP32 accumulation); a layer's inputs are bfloat16 rows in the warp's
// shared memory, its weights bfloat16 in global memory transposed to
// [out][in] so that a B fragment (two consecutive k of one column) is one
// 32-bit load; the epilogue adds the bias, applies ELU and writes the next
// layer's bfloat16 inputs.
#include <cuda_bf16.h>
#include <stdint.h>
#include "solver_dev.cuh"
#include "policy.h"

namespace mpc {
namespace {

constexpr int PA_LD = 264;                 // bf16 row stride of the activations (256 + 8)
constexpr int PA_ROWS = 16;                // agents per warp
constexpr int PA_WARPS = 4;
constexpr int PA_WARP_BYTES = 2 * PA_ROWS * PA_LD * 2;   // two activation buffers

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float* c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// out[16 x N] = act(in[16 x K] W + b) for one warp; K a multiple of 16, N of 64
template <bool ELU>
__device__ __forceinline__ void dense_layer(const __nv_bfloat16* in, __nv_bfloat16* out, const __nv_bfloat16* WT,
                                            const float* bias, int K, int N, int lane) {
  const int g = lane >> 2, t = lane & 3;
  for (int n0 = 0; n0 < N; n0 += 64) {
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
      const uint32_t a0 = ld32(in + g * PA_LD + k0 + 2 * t);
      const uint32_t a1 = ld32(in + (g + 8) * PA_LD + k0 + 2 * t);
      const uint32_t a2 = ld32(in + g * PA_LD + k0 + 2 * t + 8);
      const uint32_t a3 = ld32(in + (g + 8) * PA_LD + k0 + 2 * t + 8);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const __nv_bfloat16* w = WT + (size_t)(n0 + 8 * j + g) * K + k0 + 2 * t;
        mma_bf16(acc[j], a0, a1, a2, a3, ld32(w), ld32(w + 8));
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = n0 + 8 * j + 2 * t;
      float v[4] = {acc[j][0] + bias[col], acc[j][1] + bias[col + 1], acc[j][2] + bias[col], acc[j][3] + bias[col + 1]};
      if (ELU) {
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = v[c] > 0.f ? v[c] : expm1f(v[c]);
      }
      *reinterpret_cast<__nv_bfloat162*>(out + g * PA_LD + col) = __floats2bfloat162_rn(v[0], v[1]);
      *reinterpret_cast<__nv_bfloat162*>(out + (g + 8) * PA_LD + col) = __floats2bfloat162_rn(v[2], v[3]);
    }
  }
  __syncwarp();
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
  const int row0 = (blockIdx.x * PA_WARPS + warp) * PA_ROWS;
  if (row0 >= n) return;
  __nv_bfloat16* bufA = reinterpret_cast<__nv_bfloat16*>(psm + warp * PA_WARP_BYTES);
  __nv_bfloat16* bufB = bufA + PA_ROWS * PA_LD;
  // layer-1 input: the observations, zero-padded to K = 64 (and rows past n)
  for (int idx = lane; idx < PA_ROWS * POL_K1; idx += 32) {
    const int r = idx / POL_K1, c = idx - r * POL_K1;
    float v = 0.f;
    if (row0 + r < n && c < POL_OBS) v = obs_entry(agent_ptrs(a, ids[row0 + r]), c);
    bufA[r * PA_LD + c] = __float2bfloat16_rn(v);
  }
  __syncwarp();
  dense_layer<true>(bufA, bufB, pol.W1, pol.b1, POL_K1, POL_HID, lane);
  dense_layer<true>(bufB, bufA, pol.W2, pol.b2, POL_HID, POL_HID, lane);
  dense_layer<true>(bufA, bufB, pol.W3, pol.b3, POL_HID, POL_HID, lane);
  // output layer: N = 16 (10 actions + zero padding), FP32 result
  const int g = lane >> 2, t = lane & 3;
  float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  for (int k0 = 0; k0 < POL_HID; k0 += 16) {
    const uint32_t a0 = ld32(bufB + g * PA_LD + k0 + 2 * t);
    const uint32_t a1 = ld32(bufB + (g + 8) * PA_LD + k0 + 2 * t);
    const uint32_t a2 = ld32(bufB + g * PA_LD + k0 + 2 * t + 8);
    const uint32_t a3 = ld32(bufB + (g + 8) * PA_LD + k0 + 2 * t + 8);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const __nv_bfloat16* w = pol.W4 + (size_t)(8 * j + g) * POL_HID + k0 + 2 * t;
      mma_bf16(acc[j], a0, a1, a2, a3, ld32(w), ld32(w + 8));
    }
  }
  float* stage = reinterpret_cast<float*>(bufA);        // 16 x 16 actions
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int col = 8 * j + 2 * t;
    stage[g * 16 + col] = acc[j][0] + pol.b4[col];
    stage[g * 16 + col + 1] = acc[j][1] + pol.b4[col + 1];
    stage[(g + 8) * 16 + col] = acc[j][2] + pol.b4[col];
    stage[(g + 8) * 16 + col + 1] = acc[j][3] + pol.b4[col + 1];
  }
  __syncwarp();
  // blend (Eq. joint-torque) on the legs; arms keep the MPC torque
  for (int idx = lane; idx < PA_ROWS * 18; idx += 32) {
    const int r = idx / 18, j = idx - r * 18;
    if (row0 + r >= n) continue;
    const AgentPtrs ap = agent_ptrs(a, ids[row0 + r]);
    float out = ap.out[O_TAU + j];
    if (j < POL_ACT) {
      const float aj = stage[r * 16 + j];
      const float q = ap.inp[I_X0 + 12 + j], qd = ap.inp[I_QD + j];
      const float res = ap.mdl[M_KP + j] * (aj + ap.mdl[M_QNOM + j] - q) - ap.mdl[M_KD + j] * qd;
      out = fmaf(pol.lambda, res, out);
      if (act) act[(size_t)(row0 + r) * POL_ACT + j] = aj;
    }
    if (tau) tau[(size_t)(row0 + r) * 18 + j] = out;
  }
}

}  // namespace

size_t policy_smem_bytes() { return (size_t)PA_WARPS * PA_WARP_BYTES; }

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
  const int rows_per_block = PA_WARPS * PA_ROWS;
  const int blocks = (n + rows_per_block - 1) / rows_per_block;
  mpc_k_policy<<<blocks, PA_WARPS * 32, policy_smem_bytes(), st>>>(a, n, ids, pol, tau, act);
  return cudaGetLastError();
}

}  // namespace mpc
