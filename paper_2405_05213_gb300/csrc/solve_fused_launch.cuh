// Launches of the whole-solve cooperative kernel (solve_fused.cuh) for Q1
// meshes on a uniform box, per (precision, material, frozen-state count).
// Instantiated per precision in solve_fused_f{32,64}.cu (parallel compiles).
#pragma once

#include <algorithm>
#include <mutex>

#include "etp_host.cuh"
#include "solve_fused.cuh"

namespace etp {

namespace fused_detail {

constexpr size_t kSmemPerBlock = 227 * 1024;

struct FusedInfo {
  const void* fn = nullptr;
  size_t static_smem = 0;
};

template <typename T, int KIND, int NS>
FusedInfo fused_info() {
  static FusedInfo info;
  static std::once_flag once;
  std::call_once(once, [] {
    info.fn = (const void*)k_krylov_solve_fused<T, KIND, NS>;
    cudaFuncAttributes a{};
    if (cudaFuncGetAttributes(&a, k_krylov_solve_fused<T, KIND, NS>) == cudaSuccess) info.static_smem = a.sharedSizeBytes;
    cudaFuncSetAttribute(k_krylov_solve_fused<T, KIND, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(kSmemPerBlock - info.static_smem));
    cudaGetLastError();
  });
  return info;
}

template <typename T>
FusedInfo fused_lookup(int kind, int ns) {
#define ETP_FUSED_CASE(K_, N_) \
  if (kind == K_ && ns == N_) return fused_info<T, K_, N_>();
  ETP_FUSED_CASE(MAT_LINEAR, 0)
  ETP_FUSED_CASE(MAT_NEOHOOKE, 1) ETP_FUSED_CASE(MAT_NEOHOOKE, 2)
  ETP_FUSED_CASE(MAT_MOONEY_RIVLIN, 1) ETP_FUSED_CASE(MAT_MOONEY_RIVLIN, 2)
  ETP_FUSED_CASE(MAT_SVK, 1) ETP_FUSED_CASE(MAT_SVK, 2)
  ETP_FUSED_CASE(MAT_YEOH, 1) ETP_FUSED_CASE(MAT_YEOH, 2)
#undef ETP_FUSED_CASE
  return FusedInfo{};
}

}  // namespace fused_detail

// Largest column count the fused kernel can step to within `cap` (its shared
// memory holds the Gram-Schmidt tiles of every step up to it), 0 if none.
template <typename T>
int fused_max_steps(int kind, int ns, int cap, size_t* dyn_smem) {
  const fused_detail::FusedInfo info = fused_detail::fused_lookup<T>(kind, ns);
  if (!info.fn) return 0;
  size_t need = 1024;
  int j_end = 0;
  for (int j = 1; j <= cap; ++j) {
    const size_t s = std::max(need, cgs_smem_bytes<T>(j, pk_tile_rows<T>(j)));
    if (info.static_smem + s > fused_detail::kSmemPerBlock) break;
    need = s;
    j_end = j;
  }
  *dyn_smem = need;
  return j_end;
}

// Cooperative launch of one fused solve on `grid_max` blocks at most (fewer if
// fewer are co-resident with this much shared memory).
template <typename T>
cudaError_t launch_fused_solve(etp_ctx* ctx, const FusedSolve<T>& f, int kind, int ns, size_t dyn_smem,
                               int grid_max) {
  const fused_detail::FusedInfo info = fused_detail::fused_lookup<T>(kind, ns);
  if (!info.fn) return cudaErrorInvalidValue;
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, info.fn, 128, dyn_smem) != cudaSuccess || bps < 1) {
    cudaGetLastError();
    return cudaErrorCooperativeLaunchTooLarge;
  }
  const int grid = std::max(1, std::min(grid_max, std::min(bps, 2) * ctx->num_sms));
  FusedSolve<T> args = f;
  void* argv[] = {(void*)&args};
  return cudaLaunchCooperativeKernel(info.fn, dim3(grid), dim3(128), argv, dyn_smem, ctx->stream);
}

}  // namespace etp
