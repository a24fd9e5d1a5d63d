// Whole-solve cooperative kernels in float arithmetic (solve_fused_launch.cuh).
#include "solve_fused_launch.cuh"

namespace etp {
template FusedPlan fused_plan<float>(int, int, int, int64_t, int);
template cudaError_t launch_fused_solve<float>(etp_ctx*, const FusedSolve<float>&, int, int, const FusedPlan&);
}  // namespace etp
