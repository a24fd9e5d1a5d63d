// Arnoldi vector kernels (Section 4.3): classical Gram-Schmidt with one
// reorthogonalisation pass (CGS2), the start vector, the state update
// w_new = ||w|| V_m exp(tau H_m) e_1, and state/field conversions.
//
// Basis columns are stored unnormalised: column i holds v_i / s_i and
// coef[SCALE + i] = s_i, so normalising a new column costs nothing.
// Reductions: per-block partial sums, then the last block to finish sums them
// in block order (deterministic for a fixed grid).
#pragma once

#include "etp_internal.cuh"

namespace etp {

// offsets into the per-solve coefficient buffer (each kMaxCap + 1 doubles)
constexpr int COEF_H1 = 0;
constexpr int COEF_H2 = 1;
constexpr int COEF_G = 2;
constexpr int COEF_SCALE = 3;
// the two-pass form of the bulk kernels (cgs_bulk.cuh) keeps more per-solve state:
constexpr int COEF_A = 4;     // reorthogonalisation coefficients a of the candidate column
constexpr int COEF_D = 5;     // update coefficients of the next candidate
constexpr int COEF_HT = 6;    // first-pass Hessenberg coefficients of the current column
constexpr int COEF_MISC = 7;  // scalars: MISC_R, MISC_SU, MISC_EU
constexpr int COEF_SCALE2 = 8;  // the column scales as float-float pairs (persistent step, FP32 tiles)
constexpr int COEF_NUM = 9;
constexpr int COEF_STRIDE = kMaxCap + 1;
constexpr int MISC_R = 0;   // norm r of the candidate after reorthogonalisation
constexpr int MISC_SU = 1;  // scale of the candidate's stored column
constexpr int MISC_EU = 2;  // coefficient of the candidate in the next candidate's update
constexpr int MISC_ONE = 3;  // 1.0 (scale of raw columns applied as they are)

template <typename T>
struct CgsParams {
  int64_t L;            // rows (multiple of 128)
  T* V;                 // basis, column stride L
  int j;                // columns in use
  T* z;                 // work vector
  T* vout;              // UPD_NORM: new basis column j
  double* coef;
  double* partials;     // [grid][j] or [grid]
  unsigned int* counter;
  KState* ks;
  double* H;            // Hessenberg, column-major
  int ldH;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block of one double per thread (blockDim.x multiple of 32, <= 1024).
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    r = warp_sum(r);
  }
  return r;  // valid in thread 0
}

// Running sum (hi, lo): float-float with Knuth's TwoSum for float (the
// rounding error of every addition is carried in lo; FP64 arithmetic runs at a
// small fraction of the FP32 rate on this GPU), plain double for double.
__device__ __forceinline__ void acc_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += e;
}
__device__ __forceinline__ void acc_add(double& hi, double& lo, double x) {
  (void)lo;
  hi += x;
}
// (hi, lo) += (h2, l2)
template <typename T>
__device__ __forceinline__ void acc_add_pair(T& hi, T& lo, T h2, T l2) {
  acc_add(hi, lo, h2);
  lo += l2;
}
template <typename T>
__device__ __forceinline__ void warp_allsum_pair(T& hi, T& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const T l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    acc_add_pair(hi, lo, h2, l2);
  }
}
// Block partial slots are 8 bytes: (hi, lo) floats, or one double.
__device__ __forceinline__ void store_partial(double* slot, float hi, float lo) {
  *reinterpret_cast<float2*>(slot) = make_float2(hi, lo);
}
__device__ __forceinline__ void store_partial(double* slot, double hi, double lo) { *slot = hi + lo; }
__device__ __forceinline__ void load_partial(const double* slot, float& hi, float& lo) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(slot));
  hi = v.x;
  lo = v.y;
}
__device__ __forceinline__ void load_partial(const double* slot, double& hi, double& lo) {
  hi = __ldcg(slot);
  lo = 0.0;
}
template <typename T>
__device__ __forceinline__ double pair_value(T hi, T lo) {
  return (double)hi + (double)lo;
}
// A double as the float-float pair (hi, lo) in one 8-byte slot.
__device__ __forceinline__ void store_scale_pair(double* slot, double s) {
  const float hi = (float)s;
  store_partial(slot, hi, (float)(s - (double)hi));
}

// Last-block-done election (threadFenceReduction pattern).
__device__ __forceinline__ bool elect_last_block(unsigned int* counter) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int v = atomicAdd(counter, 1u);
    s_last = (v == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// Asynchronous global -> shared copy of one element (sm_80+ cp.async, L1-allocating).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem_dst, const T* gmem_src) {
  const unsigned int s = (unsigned int)__cvta_generic_to_shared(smem_dst);
  if (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
// 16-byte global -> shared copy through L2 only (data other blocks wrote in this launch).
__device__ __forceinline__ void cp_async16_cg(double* smem_dst, const double* gmem_src) {
  const unsigned int s = (unsigned int)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

// Work split of a tile's dot products for j <= 128 columns (the persistent
// step): thread t takes column t % j and row segment t / j of the tile
// (segments of whole 16-row chunks), so every thread works even when j is
// small. Returns false for idle threads.
template <int TR>
__device__ __forceinline__ bool cgs_segment(int j, int t, int& col, int& r_lo, int& r_hi) {
  const int S = 128 / j;                    // segments per column
  const int seg = t / j;
  if (seg >= S) return false;
  col = t % j;
  const int chunks = TR / 16;
  const int per = (chunks + S - 1) / S;     // chunks per segment
  r_lo = seg * per * 16;
  r_hi = min(TR, (seg + 1) * per * 16);
  return r_lo < r_hi;
}


// V_0 = w (unnormalised), beta = ||w||, reset the solve state.
template <typename T>
static __global__ void __launch_bounds__(256) k_init_basis(int64_t L, const double* __restrict__ w, T* __restrict__ V0,
                                                    double* partials, unsigned int* counter, double* coef,
                                                    KState* ks) {
  __shared__ double s_red[32];
  double acc = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < L; r += (int64_t)gridDim.x * blockDim.x) {
    const double x = w[r];
    V0[r] = (T)x;
    acc += x * x;
  }
  const double s = block_sum(acc, s_red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
  if (!elect_last_block(counter)) return;
  double n2 = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) n2 += __ldcg(partials + b);
  n2 = block_sum(n2, s_red);
  if (threadIdx.x == 0) {
    const double beta = sqrt(n2);
    ks->beta = beta;
    ks->breakdown_j = 0;
    ks->found_m = -1;
    ks->eps = 0.0;
    ks->hnorm2 = 0.0;
    ks->converged = 0;
    ks->err = isfinite(beta) ? 0 : KERR_NONFINITE;
    ks->stop = (beta == 0.0 || !isfinite(beta)) ? 1 : 0;
    coef[COEF_SCALE * COEF_STRIDE + 0] = beta > 0.0 ? 1.0 / beta : 0.0;
    store_scale_pair(coef + COEF_SCALE2 * COEF_STRIDE, beta > 0.0 ? 1.0 / beta : 0.0);
    coef[COEF_MISC * COEF_STRIDE + MISC_R] = 1.0;  // the first candidate is q_1 itself
    coef[COEF_MISC * COEF_STRIDE + MISC_ONE] = 1.0;
    *counter = 0u;
  }
}

// w_out = e_0 w_old + beta sum_{i>=1} e_i s_i V_i ; optional frozen displacement
// u* = w_out_top / sqrt(m) for the corrector.
template <typename T>
static __global__ void __launch_bounds__(256) k_combine(int64_t L, int64_t nn_pad, const double* __restrict__ w_old,
                                                 const T* __restrict__ V, const double* __restrict__ e,
                                                 const double* __restrict__ coef, const KState* __restrict__ ks,
                                                 double* __restrict__ w_out, T* __restrict__ ustar,
                                                 const T* __restrict__ minvsqrt) {
  __shared__ double s_a[kMaxCap];
  __shared__ float s_af[kMaxCap];
  const int m = ks->found_m;
  const double beta = ks->beta;
  for (int i = threadIdx.x; i < kMaxCap; i += blockDim.x) {
    s_a[i] = (i < m) ? (i == 0 ? e[0] : beta * e[i] * coef[COEF_SCALE * COEF_STRIDE + i]) : 0.0;
    s_af[i] = (float)s_a[i];
  }
  __syncthreads();
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < L; r += (int64_t)gridDim.x * blockDim.x) {
    double out = 0.0;
    if (m > 0) {
      if (sizeof(T) == 8) {
        out = s_a[0] * w_old[r];
        for (int i = 1; i < m; ++i) out += s_a[i] * (double)V[(int64_t)i * L + r];
      } else {
        // groups of 8 FP32 products, accumulated without rounding loss in float-float
        float hi = 0.f, lo = 0.f;
        int i = 1;
        while (i < m) {
          const int iend = min(i + 8, m);
          float part = 0.f;
          for (int k = i; k < iend; ++k) part = fmaf(s_af[k], (float)V[(int64_t)k * L + r], part);
          acc_add(hi, lo, part);
          i = iend;
        }
        out = fma(s_a[0], w_old[r], (double)hi + (double)lo);
      }
    }
    w_out[r] = out;
    if (ustar && r < 3 * nn_pad) {
      if (sizeof(T) == 8) ustar[r] = (T)(out * (double)minvsqrt[r % nn_pad]);
      else ustar[r] = (T)((float)out * (float)minvsqrt[r % nn_pad]);
    }
  }
}

// u* = w_top / sqrt(m) in the apply precision.
template <typename T>
static __global__ void k_extract_u(int64_t nn_pad, const double* __restrict__ w, const T* __restrict__ minvsqrt,
                            T* __restrict__ ustar) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < 3 * nn_pad) ustar[r] = (T)(w[r] * (double)minvsqrt[r % nn_pad]);
}

// w_bar = [sqrt(m) u; sqrt(m) v] from node-major physical fields; fixed DOFs -> 0.
static __global__ void k_state_from_uv(int64_t n_nodes, int64_t nn_pad, const double* __restrict__ u,
                                const double* __restrict__ v, const double* __restrict__ msqrt,
                                const uint8_t* __restrict__ fixed, double* __restrict__ w) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn_pad) return;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double a = 0.0, b = 0.0;
    if (n < n_nodes && !(fixed[n] & (1 << c))) {
      a = msqrt[n] * u[3 * n + c];
      b = msqrt[n] * v[3 * n + c];
    }
    w[c * nn_pad + n] = a;
    w[(3 + c) * nn_pad + n] = b;
  }
}

static __global__ void k_uv_from_state(int64_t n_nodes, int64_t nn_pad, const double* __restrict__ w,
                                const double* __restrict__ minvsqrt, double* __restrict__ u,
                                double* __restrict__ v) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (u) u[3 * n + c] = w[c * nn_pad + n] * minvsqrt[n];
    if (v) v[3 * n + c] = w[(3 + c) * nn_pad + n] * minvsqrt[n];
  }
}

// x . y over [0, n) into out[0], FP64 (two-stage: partials then last block)
static __global__ void __launch_bounds__(256) k_dot64(int64_t n, const double* __restrict__ x,
                                               const double* __restrict__ y, double* partials,
                                               unsigned int* counter, double* out) {
  __shared__ double s_red[32];
  double acc = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    acc += x[r] * y[r];
  const double s = block_sum(acc, s_red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
  if (!elect_last_block(counter)) return;
  double t = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(partials + b);
  t = block_sum(t, s_red);
  if (threadIdx.x == 0) {
    *out = t;
    *counter = 0u;
  }
}

// sum of squares of x[0..n) into out[0] (two-stage: partials then last block)
static __global__ void __launch_bounds__(256) k_sumsq(int64_t n, const double* __restrict__ x, double* partials,
                                               unsigned int* counter, double* out) {
  __shared__ double s_red[32];
  double acc = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    acc += x[r] * x[r];
  const double s = block_sum(acc, s_red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
  if (!elect_last_block(counter)) return;
  double t = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(partials + b);
  t = block_sum(t, s_red);
  if (threadIdx.x == 0) {
    *out = t;
    *counter = 0u;
  }
}

}  // namespace etp
