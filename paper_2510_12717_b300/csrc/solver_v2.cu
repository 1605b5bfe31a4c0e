// Solver kernels, variant 2: at least 3 resident blocks per SM.
#include "solver_impl.cuh"

namespace mpc {
template cudaError_t launch_variant<3>(const Arena&, const Batch&, const SolverParams&, int, int, cudaStream_t,
                                          int*);
}  // namespace mpc
