// Launch dispatch for the element apply: picks the (order, precision, material,
// geometry, frozen-state count) instance. Instantiated per (order, precision)
// in fe_q{1,2}_f{32,64}.cu so the heavy template code compiles in parallel.
#pragma once

#include "fe_kernels.cuh"

namespace etp {

template <int P, typename T>
cudaError_t launch_elem_apply(const ApplyParams<T>& p, int kind, bool box, int ns, cudaStream_t st);

#define ETP_APPLY_CASE(KIND_, BOX_, NS_)                                                     \
  if (kind == KIND_ && box == BOX_ && ns == NS_) {                                           \
    k_elem_apply<P, T, KIND_, BOX_, NS_><<<grid, ElemTraits<P>::BLOCK, 0, st>>>(p);          \
    return cudaGetLastError();                                                               \
  }

#define ETP_APPLY_KIND(KIND_)   \
  ETP_APPLY_CASE(KIND_, true, 1) \
  ETP_APPLY_CASE(KIND_, true, 2) \
  ETP_APPLY_CASE(KIND_, false, 1) \
  ETP_APPLY_CASE(KIND_, false, 2)

#define ETP_DEFINE_LAUNCH_ELEM_APPLY(P_, T_)                                                    \
  template <>                                                                                   \
  cudaError_t launch_elem_apply<P_, T_>(const ApplyParams<T_>& p, int kind, bool box, int ns,   \
                                        cudaStream_t st) {                                      \
    constexpr int P = P_;                                                                       \
    using T = T_;                                                                               \
    if (p.n_elems == 0) return cudaSuccess;                                                     \
    const unsigned grid = (unsigned)((p.n_elems + ElemTraits<P>::EPB - 1) / ElemTraits<P>::EPB); \
    ETP_APPLY_CASE(MAT_LINEAR, true, 0)                                                         \
    ETP_APPLY_CASE(MAT_LINEAR, false, 0)                                                        \
    ETP_APPLY_KIND(MAT_NEOHOOKE)                                                                \
    ETP_APPLY_KIND(MAT_MOONEY_RIVLIN)                                                           \
    ETP_APPLY_KIND(MAT_SVK)                                                                     \
    ETP_APPLY_KIND(MAT_YEOH)                                                                    \
    return cudaErrorInvalidValue;                                                               \
  }

}  // namespace etp
