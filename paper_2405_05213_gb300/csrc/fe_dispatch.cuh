// Launch dispatch for the element apply and the frozen-coefficient build:
// picks the (order, precision, material, geometry, frozen-state count)
// instance. Instantiated per (order, precision) in fe_q{1,2}_f{32,64}.cu so
// the heavy template code compiles in parallel.
#pragma once

#include <algorithm>
#include <atomic>

#include "fe_kernels.cuh"

namespace etp {

// grid > 0 replaces the default grid of a Q1 pass (autotuned; elements are
// independent, so the result does not depend on it).
template <int P, typename T>
cudaError_t launch_elem_apply(const ApplyParams<T>& p, int kind, bool box, int ns, int num_sms, cudaStream_t st,
                              int grid);
template <int P, typename T>
cudaError_t launch_frozen_build(const FrozenBuildParams<T>& p, int kind, bool box, cudaStream_t st);
template <int P, typename T>
cudaError_t launch_elem_apply_batch(ElemBatch<T>& b, int kind, bool box, int ns, int num_sms, cudaStream_t st);

// Element apply: Q1, one wave of resident blocks whose teams loop over the
// elements; Q2, one block per block of elements.
#define ETP_APPLY_CASE(KIND_, BOX_, NS_)                                                       \
  if (kind == KIND_ && box == BOX_ && ns == NS_) {                                             \
    static std::atomic<int> bps{0};                                                            \
    if (bps.load() == 0) {                                                                     \
      int n = 0;                                                                               \
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_elem_apply<P, T, KIND_, BOX_, NS_>, \
                                                        ElemTraits<P>::BLOCK, 0) != cudaSuccess || \
          n < 1)                                                                               \
        n = 1;                                                                                 \
      bps.store(n);                                                                            \
    }                                                                                          \
    const int64_t wave = (int64_t)bps.load() * num_sms;                                         \
    ApplyParams<T> q = p;                                                                      \
    unsigned g = (unsigned)(P == 1 ? std::min<int64_t>(nblocks, grid > 0 ? (int64_t)grid : wave) : nblocks); \
    if (P == 1 && grid <= 0 && nblocks < wave) { /* small mesh: fewer elements per block */    \
      q.epb = (int)((p.n_elems + wave - 1) / wave);                                            \
      g = (unsigned)((p.n_elems + q.epb - 1) / q.epb);                                         \
    }                                                                                          \
    k_elem_apply<P, T, KIND_, BOX_, NS_><<<g, ElemTraits<P>::BLOCK, 0, st>>>(q);               \
    return cudaGetLastError();                                                                 \
  }

#define ETP_APPLY_KIND(KIND_)    \
  ETP_APPLY_CASE(KIND_, true, 1)  \
  ETP_APPLY_CASE(KIND_, true, 2)  \
  ETP_APPLY_CASE(KIND_, false, 1) \
  ETP_APPLY_CASE(KIND_, false, 2)

// Batched element apply: one wave of resident blocks shared out in
// proportion to the meshes' element blocks (Q1, whose teams loop), or one
// block per block of elements (Q2).
#define ETP_APPLY_BATCH_CASE(KIND_, BOX_, NS_)                                                 \
  if (kind == KIND_ && box == BOX_ && ns == NS_) {                                             \
    static std::atomic<int> bps{0};                                                            \
    if (bps.load() == 0) {                                                                     \
      int n = 0;                                                                               \
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_elem_apply_batch<P, T, KIND_, BOX_, NS_>, \
                                                        ElemTraits<P>::BLOCK, 0) != cudaSuccess || \
          n < 1)                                                                               \
        n = 1;                                                                                 \
      bps.store(n);                                                                            \
    }                                                                                          \
    const int64_t wave = (int64_t)bps.load() * num_sms;                                        \
    int64_t total = 0;                                                                         \
    for (int i = 0; i < b.n; ++i) total += (b.item[i].n_elems + ElemTraits<P>::EPB - 1) / ElemTraits<P>::EPB; \
    b.off[0] = 0;                                                                              \
    for (int i = 0; i < b.n; ++i) {                                                            \
      const int64_t nbk = std::max<int64_t>(1, (b.item[i].n_elems + ElemTraits<P>::EPB - 1) / ElemTraits<P>::EPB); \
      const int64_t share = P == 1 ? std::min<int64_t>(nbk, std::max<int64_t>(1, (wave * nbk + total - 1) / std::max<int64_t>(total, 1))) : nbk; \
      b.off[i + 1] = b.off[i] + (int)share;                                                    \
    }                                                                                          \
    k_elem_apply_batch<P, T, KIND_, BOX_, NS_><<<(unsigned)b.off[b.n], ElemTraits<P>::BLOCK, 0, st>>>(b); \
    return cudaGetLastError();                                                                 \
  }

#define ETP_APPLY_BATCH_KIND(KIND_)    \
  ETP_APPLY_BATCH_CASE(KIND_, true, 1)  \
  ETP_APPLY_BATCH_CASE(KIND_, true, 2)  \
  ETP_APPLY_BATCH_CASE(KIND_, false, 1) \
  ETP_APPLY_BATCH_CASE(KIND_, false, 2)

#define ETP_BUILD_CASE(KIND_, BOX_)                                                        \
  if (kind == KIND_ && box == BOX_) {                                                      \
    k_frozen_build<P, T, KIND_, BOX_><<<nblocks, ElemTraits<P>::BLOCK, 0, st>>>(p);        \
    return cudaGetLastError();                                                             \
  }

#define ETP_DEFINE_LAUNCH_ELEM_APPLY(P_, T_)                                                      \
  template <>                                                                                     \
  cudaError_t launch_elem_apply<P_, T_>(const ApplyParams<T_>& p, int kind, bool box, int ns,     \
                                        int num_sms, cudaStream_t st, int grid) {                 \
    constexpr int P = P_;                                                                         \
    using T = T_;                                                                                 \
    if (p.n_elems == 0) return cudaSuccess;                                                       \
    const int64_t nblocks = (p.n_elems + ElemTraits<P>::EPB - 1) / ElemTraits<P>::EPB;            \
    ETP_APPLY_CASE(MAT_LINEAR, true, 0)                                                           \
    ETP_APPLY_CASE(MAT_LINEAR, false, 0)                                                          \
    ETP_APPLY_KIND(MAT_NEOHOOKE)                                                                  \
    ETP_APPLY_KIND(MAT_MOONEY_RIVLIN)                                                             \
    ETP_APPLY_KIND(MAT_SVK)                                                                       \
    ETP_APPLY_KIND(MAT_YEOH)                                                                      \
    ETP_APPLY_CASE(MAT_SVK_TANGENT, true, 1)                                                      \
    ETP_APPLY_CASE(MAT_SVK_TANGENT, false, 1)                                                     \
    if constexpr (sizeof(T) == 8) { /* consistent tangents of the FP64 Newmark-beta step */       \
      ETP_APPLY_CASE(MAT_NH_TANGENT, true, 1)                                                     \
      ETP_APPLY_CASE(MAT_NH_TANGENT, false, 1)                                                    \
      ETP_APPLY_CASE(MAT_MR_TANGENT, true, 1)                                                     \
      ETP_APPLY_CASE(MAT_MR_TANGENT, false, 1)                                                    \
      ETP_APPLY_CASE(MAT_YEOH_TANGENT, true, 1)                                                   \
      ETP_APPLY_CASE(MAT_YEOH_TANGENT, false, 1)                                                  \
    }                                                                                             \
    return cudaErrorInvalidValue;                                                                 \
  }                                                                                               \
  template <>                                                                                     \
  cudaError_t launch_frozen_build<P_, T_>(const FrozenBuildParams<T_>& p, int kind, bool box,     \
                                          cudaStream_t st) {                                      \
    constexpr int P = P_;                                                                         \
    using T = T_;                                                                                 \
    if (p.n_elems == 0) return cudaSuccess;                                                       \
    const unsigned nblocks = (unsigned)((p.n_elems + ElemTraits<P>::EPB - 1) / ElemTraits<P>::EPB); \
    ETP_BUILD_CASE(MAT_NEOHOOKE, true)                                                            \
    ETP_BUILD_CASE(MAT_NEOHOOKE, false)                                                           \
    ETP_BUILD_CASE(MAT_MOONEY_RIVLIN, true)                                                       \
    ETP_BUILD_CASE(MAT_MOONEY_RIVLIN, false)                                                      \
    ETP_BUILD_CASE(MAT_SVK, true)                                                                 \
    ETP_BUILD_CASE(MAT_SVK, false)                                                                \
    ETP_BUILD_CASE(MAT_YEOH, true)                                                                \
    ETP_BUILD_CASE(MAT_YEOH, false)                                                               \
    return cudaErrorInvalidValue;                                                                 \
  }                                                                                               \
  template <>                                                                                     \
  cudaError_t launch_elem_apply_batch<P_, T_>(ElemBatch<T_> & b, int kind, bool box, int ns,      \
                                              int num_sms, cudaStream_t st) {                     \
    constexpr int P = P_;                                                                         \
    using T = T_;                                                                                 \
    if (b.n < 1 || b.n > kMaxBatch) return cudaErrorInvalidValue;                                 \
    ETP_APPLY_BATCH_CASE(MAT_LINEAR, true, 0)                                                     \
    ETP_APPLY_BATCH_CASE(MAT_LINEAR, false, 0)                                                    \
    ETP_APPLY_BATCH_KIND(MAT_NEOHOOKE)                                                            \
    ETP_APPLY_BATCH_KIND(MAT_MOONEY_RIVLIN)                                                       \
    ETP_APPLY_BATCH_KIND(MAT_SVK)                                                                 \
    ETP_APPLY_BATCH_KIND(MAT_YEOH)                                                                \
    return cudaErrorInvalidValue;                                                                 \
  }

}  // namespace etp
