// Launches of the whole-solve cooperative kernel (solve_fused.cuh) for Q1
// meshes on a uniform box, per (precision, material, frozen-state count).
// Instantiated per precision in solve_fused_f{32,64}.cu (parallel compiles).
#pragma once

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

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

// Launch plan of one fused solve over vectors of L rows: the last column
// count it steps to (within cap), its grid, dynamic shared memory and the
// offsets of the partial-sum copy area. Preferred: one tile per block for
// every step (the tiles of V stay in shared memory), on two blocks per SM with
// the tile rows of the first step; else the two-stage tile pipeline. j_end = 0
// if neither fits.
template <typename T>
FusedPlan fused_plan_uncached(int kind, int ns, int cap, int64_t L, int num_sms) {
  FusedPlan plan;
  const fused_detail::FusedInfo info = fused_detail::fused_lookup<T>(kind, ns);
  if (!info.fn) return plan;
  int dev = 0, sm_bytes = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaGetLastError();
  // one tile per block on 2 blocks per SM
  const int tr = pk_tile_rows<T>(1, L);
  const int64_t ntiles = pk_ntiles(L, tr);
  const int64_t half = (int64_t)sm_bytes / 2 - reserved - (int64_t)info.static_smem;
  if (ntiles <= 2 * (int64_t)num_sms && half > 0) {
    // the tile area of every step up to j_end, with room left for the copy of
    // the partial sums of up to 32 columns
    int j_end = 0;
    for (int j = 1; j <= cap; ++j) {
      if (pk_tile_rows<T>(j, L) != tr) break;
      const size_t area = ((size_t)(j + 1) * (tr + 1) * sizeof(T) + 15) / 16 * 16;
      const size_t red = ntiles <= kPkRedundantTiles ? pk_red_bytes(L, std::min(j, 32), tr) : 0;
      if ((int64_t)(area + red) > half) break;
      j_end = j;
    }
    while (j_end >= 1) {
      const size_t area = ((size_t)(j_end + 1) * (tr + 1) * sizeof(T) + 15) / 16 * 16;
      size_t red = 0;
      if (ntiles <= kPkRedundantTiles) red = std::min<size_t>((size_t)half - area, pk_red_bytes(L, j_end, tr)) / 16 * 16;
      int bps = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, info.fn, 128, area + red) == cudaSuccess && bps >= 2) {
        plan.j_end = j_end;
        plan.dyn = std::max<size_t>(area + red, 1024);
        plan.red_off = (uint32_t)area;
        plan.red_bytes = (uint32_t)red;
        plan.grid = 2 * num_sms;
        return plan;
      }
      cudaGetLastError();
      j_end -= 8;  // the occupancy estimate above was too generous: shrink and retry
    }
  }
  // two-stage pipeline over several tiles per block
  size_t need = 1024;
  int j_end = 0;
  for (int j = 1; j <= cap; ++j) {
    const size_t sz = std::max(need, pk_tile_bytes<T>(j, pk_tile_rows<T>(j, L)));
    if (info.static_smem + sz > fused_detail::kSmemPerBlock) break;
    need = sz;
    j_end = j;
  }
  if (j_end < 1) return plan;
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, info.fn, 128, need) != cudaSuccess || bps < 1) {
    cudaGetLastError();
    return plan;
  }
  plan.j_end = j_end;
  plan.dyn = need;
  plan.red_off = (uint32_t)need;
  plan.red_bytes = 0;
  plan.grid = std::min(bps, 2) * num_sms;
  return plan;
}

// The plan, cached per (material, frozen states, capacity, rows, SMs): it is
// asked for at every solve and takes occupancy queries.
template <typename T>
FusedPlan fused_plan(int kind, int ns, int cap, int64_t L, int num_sms) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int64_t, int>, FusedPlan> cache;
  const auto key = std::make_tuple(kind, ns, cap, L, num_sms);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  const FusedPlan plan = fused_plan_uncached<T>(kind, ns, cap, L, num_sms);
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = plan;
  return plan;
}

// Cooperative launch of one fused solve with its plan.
template <typename T>
cudaError_t launch_fused_solve(etp_ctx* ctx, const FusedSolve<T>& f, int kind, int ns, const FusedPlan& plan) {
  const fused_detail::FusedInfo info = fused_detail::fused_lookup<T>(kind, ns);
  if (!info.fn) return cudaErrorInvalidValue;
  FusedSolve<T> args = f;
  args.pk.red_off = plan.red_off;
  args.pk.red_bytes = plan.red_bytes;
  void* argv[] = {(void*)&args};
  return cudaLaunchCooperativeKernel(info.fn, dim3(plan.grid), dim3(128), argv, plan.dyn, ctx->stream);
}

}  // namespace etp
