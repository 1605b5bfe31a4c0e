// Host-side dispatch of the solver kernels and the output gather.
#include "solver_dev.cuh"
#include "solver.h"

namespace mpc {

size_t smem_bytes_per_block() { return (size_t)WARPS_PER_BLOCK * W_FLOATS * sizeof(float); }

// Work queue of the persistent kernel: batch rows sorted by expected solve
// cost, longest first (a longest-processing-time-first list schedule, so
// the slow agents do not finish last).  Cost = N * (previous iterations + 10),
// from the agent's last solve when its warm start is valid.  Counting sort
// over 256 cost buckets in one block; resets the queue counter.
constexpr int kBuckets = 256;

__global__ void __launch_bounds__(1024) mpc_k_order(Arena a, Batch b, int* order) {
  __shared__ int hist[kBuckets];
  __shared__ int base[kBuckets];
  for (int t = threadIdx.x; t < kBuckets; t += blockDim.x) hist[t] = 0;
  __syncthreads();
  auto bucket = [&](int row) -> int {
    const int s = b.ids[row];
    if (s < 0 || s >= a.max_agents) return 0;
    const int N = a.horizon[s];
    if (N < 2 || N > a.maxN) return 0;
    const int prev = (a.warm_valid[s] == N) ? a.stat[(size_t)s * ST_I + T_ITERS] : 30;
    const int key = N * (min(max(prev, 0), 4000) + 10);
    return kBuckets - 1 - min(kBuckets - 1, key >> 4);   // descending cost
  };
  for (int r = threadIdx.x; r < b.n; r += blockDim.x) atomicAdd(&hist[bucket(r)], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int t = 0; t < kBuckets; ++t) { base[t] = acc; acc += hist[t]; }
    *b.counter = 0;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < b.n; r += blockDim.x) order[atomicAdd(&base[bucket(r)], 1)] = r;
}

cudaError_t launch_solve(const Arena& a, const Batch& b, const SolverParams& prm, int form, int grid_fused,
                         cudaStream_t st, int* launches, int variant) {
  // queue buffers: the batch's own (one per ticket, so batches on different
  // streams do not share them) or the arena's
  int* ord = b.order ? const_cast<int*>(b.order) : a.order;
  int* cnt = b.counter ? b.counter : a.counter;
  Batch bb = b;
  bb.order = nullptr;
  bb.counter = nullptr;
  if (form == 1 && b.n > 0 && ord && cnt && b.n <= a.max_agents) {
    mpc_k_order<<<1, 1024, 0, st>>>(a, Batch{b.n, b.ids, b.x0, b.qd, b.cmd, b.phase, nullptr, cnt}, ord);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (launches) *launches += 1;
    bb.order = ord;
    bb.counter = cnt;
  }
  if (variant == 2) return launch_variant<3>(a, bb, prm, form, grid_fused, st, launches);
  return launch_variant<2>(a, bb, prm, form, grid_fused, st, launches);
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


cudaError_t launch_gather(const Arena& a, int n, const int* ids, float* tau, float* qset, float* qdset,
                          float* value, int* status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  const int blocks = (n * 32 + threads - 1) / threads;
  mpc_k_gather<<<blocks, threads, 0, st>>>(a, n, ids, tau, qset, qdset, value, status);
  return cudaGetLastError();
}

}  // namespace mpc
