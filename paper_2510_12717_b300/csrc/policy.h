// Residual policy: device weights and the launch of the policy kernel.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include "arena.h"

namespace mpc {

constexpr int POL_OBS = 54, POL_K1 = 64, POL_HID = 256, POL_ACT = 10, POL_N4 = 16;

// bfloat16 weights transposed to [out][in] (in padded to 64 for layer 1, out
// padded to 16 for layer 4, padding zero); FP32 biases (b4 padded to 16)
struct PolicyDev {
  const __nv_bfloat16 *W1, *W2, *W3, *W4;
  const float *b1, *b2, *b3, *b4;
  float lambda;
};

size_t policy_smem_bytes();
cudaError_t launch_policy(const Arena& a, int n, const int* ids, const PolicyDev& pol, float* tau, float* act,
                          cudaStream_t st);

}  // namespace mpc
