// Host-visible interface of the solver kernels (used by the C ABI layer).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include "arena.h"

namespace mpc {

constexpr int WARPS_PER_BLOCK = 4;

// per-agent status codes (same values as mpc_agent_status in the public header)
constexpr int MPC_AGENT_SOLVED_ = 0;
constexpr int MPC_AGENT_MAX_ITER_ = 1;
constexpr int MPC_AGENT_PRIMAL_INFEAS_ = 2;
constexpr int MPC_AGENT_NAN_ = 4;
constexpr int MPC_AGENT_TIMEOUT_ = 5;
constexpr int MPC_AGENT_INACCURATE_ = 6;
constexpr int MPC_AGENT_DEFERRED_ = 7;

size_t smem_bytes_per_block();

// Enqueue the whole hot path for a batch.  form 0 = plain (five step
// kernels), 1 = fused (one kernel; grid_fused > 0 caps its grid), 2 =
// literal (set-up, block LDL^T factor, OSQP iterations, torque map).  variant:
// register cap of the solver kernels, 1 = 2 blocks/SM, 2 = 3 blocks/SM.
// *launches is incremented by the number of kernels enqueued.
cudaError_t launch_solve(const Arena& a, const Batch& b, const SolverParams& prm, int form, int grid_fused,
                         cudaStream_t st, int* launches, int variant);

template <int MINB>
cudaError_t launch_variant(const Arena& a, const Batch& b, const SolverParams& prm, int form, int grid_fused,
                           cudaStream_t st, int* launches);

// Literal form (MPC_FORM_LDL): the block LDL^T factor of the full KKT system
// and the OSQP iterations on it (ldl.cu), between the set-up kernel and the
// torque map.
cudaError_t launch_ldl(const Arena& a, const Batch& b, const SolverParams& prm, cudaStream_t st, int* launches);

cudaError_t launch_gather(const Arena& a, int n, const int* ids, float* tau, float* qset, float* qdset,
                          float* value, int* status, cudaStream_t st);

}  // namespace mpc
