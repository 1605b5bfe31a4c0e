// Solver kernels, variant 1: at least 2 resident blocks per SM.
#include "solver_impl.cuh"

namespace mpc {
template cudaError_t launch_variant<2>(const Arena&, const Batch&, const SolverParams&, int, int, cudaStream_t,
                                          int*);
}  // namespace mpc
