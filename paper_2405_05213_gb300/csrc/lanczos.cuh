// Energy-inner-product Lanczos for linear materials (Section 4.3 notes that a
// symmetric operator admits a Lanczos process; Section 5.2, Eq. "energyExpr",
// gives the energy this inner product measures).
//
// With H_bar symmetric positive definite (linear elasticity, P = 0), A =
// [[0, I], [-H_bar, 0]] is skew-adjoint in <w, w'>_E = u^T H_bar u' + v^T v':
// <A w, w'>_E = -<w, A w'>_E. An Arnoldi process in that inner product gives a
// skew-symmetric tridiagonal T_m (zero diagonal), so the basis obeys the
// three-term recurrence
//     beta_j v_{j+1} = A v_j + beta_{j-1} v_{j-1},   beta_j = ||.||_E,
// and exp(tau A) w ~= ||w||_E V_m exp(tau T_m) e_1. The E-norm of a candidate
// w = [w_u; w_v] needs H_bar w_u, which is exactly the bottom half of the next
// operator apply (A w = [w_v; -H_bar w_u]); so each step costs one apply, an
// axpy pass and one two-term dot pass, instead of the O(j) Gram-Schmidt passes.
// Columns are stored raw with their scale in coef[SCALE] (as the Arnoldi
// columns): v_j = s_j V_j.
#pragma once

#include <type_traits>

#include "krylov_kernels.cuh"

namespace etp {

// V_next = s_z * z + c * V_prev (c = beta_{j-1} s_{j-1}; V_prev may be null when
// c = 0), where z = A V_j (raw column) and s_z = s_j its scale.
template <typename T>
static __global__ void __launch_bounds__(256) k_lanczos_form(int64_t L, const T* __restrict__ z,
                                                            const T* __restrict__ V_prev, T* __restrict__ V_next,
                                                            const double* __restrict__ coef, int j,
                                                            const double* __restrict__ betas, const KState* ks) {
  if (ks->stop) return;
  const double sz = coef[COEF_SCALE * COEF_STRIDE + (j - 1)];
  const double c = (j >= 2) ? betas[j - 2] * coef[COEF_SCALE * COEF_STRIDE + (j - 2)] : 0.0;
  const T szt = (T)sz, ct = (T)c;
  // 16-byte vectors (L is a multiple of 768 rows, the columns start on 256-byte boundaries)
  using V4 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int W = 16 / (int)sizeof(T);
  const V4* z4 = reinterpret_cast<const V4*>(z);
  const V4* p4 = reinterpret_cast<const V4*>(V_prev);
  V4* o4 = reinterpret_cast<V4*>(V_next);
  const int64_t n4 = L / W;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n4; r += (int64_t)gridDim.x * blockDim.x) {
    V4 a = z4[r];
    T* av = reinterpret_cast<T*>(&a);
    if (j >= 2) {
      V4 b = p4[r];
      const T* bv = reinterpret_cast<const T*>(&b);
#pragma unroll
      for (int k = 0; k < W; ++k) av[k] = szt * av[k] + ct * bv[k];
    } else {
#pragma unroll
      for (int k = 0; k < W; ++k) av[k] = szt * av[k];
    }
    o4[r] = a;
  }
}

// E-norm squared of the raw column X from zx = A X: X_u . (-zx_bot) + X_v . X_v
// (X_v = zx_top), summed per block then by the last block. With `init` the
// column is the start vector: ks->beta = ||w||_E and its scale 1/||w||_E are
// set. Otherwise the Hessenberg (tridiagonal) column j-1 is written:
// H[j-2, j-1] = -beta_{j-1}, H[j, j-1] = beta_j, zeros elsewhere, the scale of
// column j is 1/beta_j, and a happy breakdown (beta_j <= 1e-14 ||T_j||_F) or a
// non-finite / negative norm stops the process.
template <typename T>
static __global__ void __launch_bounds__(256) k_lanczos_norm(int64_t L, const T* __restrict__ X,
                                                            const T* __restrict__ zx, double* partials,
                                                            unsigned int* counter, double* coef, double* betas,
                                                            double* H, int ldH, int j, int init, KState* ks) {
  __shared__ double s_red[32];
  if (ks->stop) return;
  const int64_t half = L / 2;
  // two sums: u . H u (a >= 0) and v . v (b >= 0); running sums in the column
  // precision with the rounding error carried (float-float for FP32 columns)
  T ah = T(0), al = T(0), bh = T(0), bl = T(0);
  using V4 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int W = 16 / (int)sizeof(T);
  const V4* x4 = reinterpret_cast<const V4*>(X);
  const V4* zt4 = reinterpret_cast<const V4*>(zx);
  const V4* zb4 = reinterpret_cast<const V4*>(zx + half);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < half / W; r += (int64_t)gridDim.x * blockDim.x) {
    const V4 xu4 = x4[r], hb4 = zb4[r], xv4 = zt4[r];
    const T* xu = reinterpret_cast<const T*>(&xu4);
    const T* hb = reinterpret_cast<const T*>(&hb4);
    const T* xv = reinterpret_cast<const T*>(&xv4);
    T pa = T(0), pb = T(0);  // W products summed plainly, then carried in the running pair
#pragma unroll
    for (int k = 0; k < W; ++k) {
      pa -= xu[k] * hb[k];
      pb += xv[k] * xv[k];
    }
    acc_add(ah, al, pa);
    acc_add(bh, bl, pb);
  }
  const double sa = block_sum(pair_value(ah, al), s_red);
  const double sb = block_sum(pair_value(bh, bl), s_red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sa;
    partials[2 * blockIdx.x + 1] = sb;
  }
  if (!elect_last_block(counter)) return;
  double ta = 0.0, tb = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
    ta += __ldcg(partials + 2 * k);
    tb += __ldcg(partials + 2 * k + 1);
  }
  ta = block_sum(ta, s_red);
  tb = block_sum(tb, s_red);
  if (threadIdx.x == 0) {
    *counter = 0u;
    const double n2 = ta + tb;
    const bool bad = !isfinite(n2) || ta < -1e-6 * fabs(tb) - 1e-300;
    const double bn = (n2 > 0.0) ? sqrt(n2) : 0.0;
    if (init) {
      ks->beta = bn;
      if (bad) {
        ks->err |= KERR_NONFINITE;
        ks->stop = 1;
      } else if (bn == 0.0) {
        ks->stop = 1;
      }
      coef[COEF_SCALE * COEF_STRIDE + 0] = bn > 0.0 ? 1.0 / bn : 0.0;
    } else {
      const int col = j - 1;
      for (int i = 0; i <= j; ++i) H[i + (int64_t)col * ldH] = 0.0;
      if (j >= 2) H[(j - 2) + (int64_t)col * ldH] = -betas[j - 2];
      H[j + (int64_t)col * ldH] = bn;
      betas[j - 1] = bn;
      const double hn2 = ks->hnorm2 + 2.0 * bn * bn;
      if (bad) {
        ks->err |= KERR_NONFINITE;
        ks->stop = 1;
      } else if (bn <= 1e-14 * sqrt(ks->hnorm2 + bn * bn)) {
        ks->breakdown_j = j;
        ks->stop = 1;
      } else {
        coef[COEF_SCALE * COEF_STRIDE + j] = 1.0 / bn;
      }
      ks->hnorm2 = hn2;
    }
  }
}

}  // namespace etp
