// Whole-solve cooperative kernels in double arithmetic (solve_fused_launch.cuh).
#include "solve_fused_launch.cuh"

namespace etp {
template FusedPlan fused_plan<double>(int, int, int, int64_t, int);
template cudaError_t launch_fused_solve<double>(etp_ctx*, const FusedSolve<double>&, int, int, const FusedPlan&);
}  // namespace etp
