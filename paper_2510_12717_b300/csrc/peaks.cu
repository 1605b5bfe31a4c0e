// Arithmetic-throughput microbenchmarks: the measured ceilings of the units
// the solve runs on (FP32 FMA for the Riccati factor and sweeps, FP64 FMA for
// the Schur inverse, mma.sync TF32 / BF16 for the reduced-precision stage
// products and the residual policy).  Each kernel keeps every warp busy with
// independent dependency chains on one unit only, so its rate is that unit's
// issue limit at the clock the GPU runs while the kernel runs.
#include <cuda_runtime.h>
#include <stdint.h>
#include "mpcgpu.h"

namespace {

constexpr int kChains = 8;     // independent accumulators per thread (FMA)
constexpr int kUnroll = 16;    // FMAs per chain per loop trip
constexpr int kMmaAcc = 4;     // independent mma accumulators per warp

template <typename T>
__global__ void __launch_bounds__(256) k_peak_fma(T* out, int trips) {
  T a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = T(threadIdx.x + c) * T(1e-3);
  const T m = T(0.999999), s = T(1e-7);
  for (int it = 0; it < trips; ++it) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, s);
  }
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

__device__ __forceinline__ void mma_tf32(float* c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16(float* c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// BF16 = false: m16n8k8 TF32 (2048 FLOP per mma); true: m16n8k16 BF16 (4096)
template <bool BF16>
__global__ void __launch_bounds__(256) k_peak_mma(float* out, int trips) {
  // small operands (0x3c00 pairs are about 1/128 in either format), so the
  // accumulators stay finite however long the loop runs
  const uint32_t a = 0x3c003c00u + (threadIdx.x & 3), b = 0x3c003c00u;
  float c[kMmaAcc][4];
#pragma unroll
  for (int i = 0; i < kMmaAcc; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0.f;
  for (int it = 0; it < trips; ++it) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r)
#pragma unroll
      for (int i = 0; i < kMmaAcc; ++i) {
        if (BF16) mma_bf16(c[i], a, a, a, a, b, b);
        else mma_tf32(c[i], a, a, a, a, b, b);
      }
  }
  float acc = 0.f;
#pragma unroll
  for (int i = 0; i < kMmaAcc; ++i) acc += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace

extern "C" mpc_status mpc_measure_peak(int32_t kind, void* stream, double* tflops, double* ms) {
  if (!tflops || kind < MPC_PEAK_FP32_FMA || kind > MPC_PEAK_BF16_MMA_SYNC) return MPC_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return MPC_ERR_CUDA;
  const int threads = 256, blocks = sms * 8;           // 64 warps per SM: every scheduler saturated
  const int trips = kind == MPC_PEAK_FP64_FMA ? 64 : 2048;
  void* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) return MPC_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&]() {
    switch (kind) {
      case MPC_PEAK_FP32_FMA: k_peak_fma<float><<<blocks, threads, 0, st>>>((float*)out, trips); break;
      case MPC_PEAK_FP64_FMA: k_peak_fma<double><<<blocks, threads, 0, st>>>((double*)out, trips); break;
      case MPC_PEAK_TF32_MMA_SYNC: k_peak_mma<false><<<blocks, threads, 0, st>>>((float*)out, trips); break;
      default: k_peak_mma<true><<<blocks, threads, 0, st>>>((float*)out, trips); break;
    }
  };
  const int reps = 5;
  launch();                                            // warm-up (clocks ramp, module load)
  cudaEventRecord(e0, st);
  for (int r = 0; r < reps; ++r) launch();
  cudaEventRecord(e1, st);
  cudaError_t err = cudaEventSynchronize(e1);
  float t = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || t <= 0.f) return MPC_ERR_CUDA;
  const double per_launch_ms = t / reps;
  const double units = (double)blocks * threads * trips * kUnroll;
  double flop;
  if (kind == MPC_PEAK_FP32_FMA || kind == MPC_PEAK_FP64_FMA)
    flop = units * kChains * 2.0;
  else
    flop = units / 32.0 * kMmaAcc * (kind == MPC_PEAK_TF32_MMA_SYNC ? 2048.0 : 4096.0);
  *tflops = flop / (per_launch_ms * 1e-3) / 1e12;
  if (ms) *ms = per_launch_ms;
  return MPC_OK;
}
