// Whole-solve cooperative kernels in float arithmetic (solve_fused_launch.cuh).
#include "solve_fused_launch.cuh"

namespace etp {
template int fused_max_steps<float>(int, int, int, size_t*);
template cudaError_t launch_fused_solve<float>(etp_ctx*, const FusedSolve<float>&, int, int, size_t, int);
}  // namespace etp
