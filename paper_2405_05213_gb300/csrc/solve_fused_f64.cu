// Whole-solve cooperative kernels in double arithmetic (solve_fused_launch.cuh).
#include "solve_fused_launch.cuh"

namespace etp {
template int fused_max_steps<double>(int, int, int, size_t*);
template cudaError_t launch_fused_solve<double>(etp_ctx*, const FusedSolve<double>&, int, int, size_t, int);
}  // namespace etp
