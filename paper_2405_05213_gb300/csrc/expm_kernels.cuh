// Small dense exponential of the Hessenberg matrix, FP64 (Section 4.3).
//
// The paper evaluates exp(H_m) by a Taylor series when ||H_m|| <= 1 and by
// scaling and squaring otherwise. Here: B = tau H_j / 2^s with
// s = max(0, ceil(log2 ||tau H_j||_1)) so that ||B||_1 <= 1; T_18(B), the
// degree-18 Taylor polynomial (truncation error below e/19! ~ 2e-17 for
// ||B|| <= 1), is evaluated by the Paterson-Stockmeyer scheme with powers
// B, B^2, B^3, B^4 (seven matrix products); then s squarings.
//
// Every matrix product is one launch spread over the whole GPU (FP64
// throughput per SM is small on this part, so one product per SM would be far
// slower). Several candidate sizes j (a window of Arnoldi steps) are evaluated
// in the same launches; each candidate owns six ld x ld matrices of workspace:
// B, B^2, B^3, B^4, R0, R1.
#pragma once

#include "etp_internal.cuh"
#include "krylov_kernels.cuh"

namespace etp {

constexpr int EXPM_TAYLOR_DEG = 18;
constexpr int EXPM_NMAT = 6;
enum : int { XM_B = 0, XM_P2 = 1, XM_P3 = 2, XM_P4 = 3, XM_R0 = 4, XM_R1 = 5 };

struct ExpmParams {
  const double* H;   // Hessenberg, column-major, leading dimension ldH
  int ldH;
  int j0;            // candidate c has size j0 + c
  int ncand;
  double tau;
  double* ws;        // workspace: ncand * 6 * ld * ld
  int ld;
  int* s_arr;        // per-candidate scaling exponent, -1 = candidate invalid
  const KState* ks;  // may be null (standalone use)
  double coef[EXPM_TAYLOR_DEG + 1];  // 1/k!
};

__device__ __forceinline__ double* xm(const ExpmParams& p, int cand, int which) {
  return p.ws + ((size_t)cand * EXPM_NMAT + which) * (size_t)p.ld * p.ld;
}

// largest valid candidate size (a breakdown at j_b leaves H valid up to j_b)
__device__ __forceinline__ bool cand_valid(const ExpmParams& p, int j) {
  if (!p.ks) return true;
  const int jb = p.ks->breakdown_j;
  if (p.ks->beta == 0.0 || (p.ks->err != 0)) return false;
  return jb == 0 || j <= jb;
}

// scaling exponent and B = tau H_j / 2^s of candidate `cand` (one block)
__device__ __forceinline__ void expm_prep_cand(const ExpmParams& p, int cand) {
  const int j = p.j0 + cand;
  __shared__ double s_colmax[256];
  __shared__ int s_s;
  if (!cand_valid(p, j)) {
    if (threadIdx.x == 0) p.s_arr[cand] = -1;
    return;
  }
  // column sums of |tau H_j|: warp w sums columns w, w+8, ... with lanes over rows
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double mx = 0.0;
  for (int c = warp; c < j; c += nw) {
    double s = 0.0;
    for (int r = lane; r < j; r += 32) s += fabs(p.tau * p.H[r + (size_t)c * p.ldH]);
    s = warp_sum(s);
    mx = fmax(mx, s);
  }
  if (lane == 0) s_colmax[warp] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < nw; ++i) m = fmax(m, s_colmax[i]);
    int s = 0;
    if (m > 1.0) s = (int)ceil(log2(m));
    if (!isfinite(m)) s = 0;
    s_s = s;
    p.s_arr[cand] = s;
  }
  __syncthreads();
  const int s = s_s;
  double* B = xm(p, cand, XM_B);
  for (int idx = threadIdx.x; idx < j * j; idx += blockDim.x) {
    const int r = idx % j, c = idx / j;
    B[r + (size_t)c * p.ld] = ldexp(p.tau * p.H[r + (size_t)c * p.ldH], -s);
  }
}

static __global__ void __launch_bounds__(256) k_expm_prep(ExpmParams p) { expm_prep_cand(p, blockIdx.x); }

// Matrix-product stages. stage 0: P2 = B B. stage 1: P3 = P2 B (z=0), P4 = P2 P2 (z=1).
// stage 2 (k = Horner index 3..0): R_out = C_k + P4 R_in, C_k = sum_r c_{4k+r} B^r,
// R_in = C_4 = c16 I + c17 B + c18 B^2 when k = 3.
// stage 3 (k = squaring index): R_out = R_in R_in for candidates with s > k.
// One entry (idx = r + c j) of a stage product of candidate `cand`; `z`
// selects the product of stage 1. Matrix reads go through L2 (ld.global.cg):
// the single-launch check writes them in earlier stages of the same kernel.
__device__ __forceinline__ void expm_mm_entry(const ExpmParams& p, int cand, int idx, int z, int stage, int k) {
  const int j = p.j0 + cand;
  const int s = __ldcg(p.s_arr + cand);
  if (s < 0) return;
  if (idx >= j * j) return;
  const int r = idx % j, c = idx / j;
  const int ld = p.ld;
  const double* B = xm(p, cand, XM_B);
  const double* P2 = xm(p, cand, XM_P2);
  const double* P3 = xm(p, cand, XM_P3);
  const double* P4 = xm(p, cand, XM_P4);
  if (stage == 0 || stage == 1) {
    const double *X, *Y;
    double* O;
    if (stage == 0) { X = B; Y = B; O = xm(p, cand, XM_P2); }
    else if (z == 0) { X = P2; Y = B; O = xm(p, cand, XM_P3); }
    else { X = P2; Y = P2; O = xm(p, cand, XM_P4); }
    double acc = 0.0;
    for (int t = 0; t < j; ++t) acc += __ldcg(X + r + (size_t)t * ld) * __ldcg(Y + t + (size_t)c * ld);
    O[r + (size_t)c * ld] = acc;
    return;
  }
  if (stage == 2) {
    // ping-pong: k=3 -> R0, k=2 -> R1, k=1 -> R0, k=0 -> R1
    const double* Rin = (k == 2 || k == 0) ? xm(p, cand, XM_R0) : xm(p, cand, XM_R1);
    double* Rout = (k == 3 || k == 1) ? xm(p, cand, XM_R0) : xm(p, cand, XM_R1);
    const double* cf = p.coef;
    double acc = 0.0;
    if (k == 3) {
      for (int t = 0; t < j; ++t) {
        const size_t tc = t + (size_t)c * ld;
        const double c4 = (t == c ? cf[16] : 0.0) + cf[17] * __ldcg(B + tc) + cf[18] * __ldcg(P2 + tc);
        acc += __ldcg(P4 + r + (size_t)t * ld) * c4;
      }
    } else {
      for (int t = 0; t < j; ++t) acc += __ldcg(P4 + r + (size_t)t * ld) * __ldcg(Rin + t + (size_t)c * ld);
    }
    const size_t rc = r + (size_t)c * ld;
    const double ck = (r == c ? cf[4 * k] : 0.0) + cf[4 * k + 1] * __ldcg(B + rc) + cf[4 * k + 2] * __ldcg(P2 + rc) +
                      cf[4 * k + 3] * __ldcg(P3 + rc);
    Rout[rc] = ck + acc;
    return;
  }
  // stage 3: squaring k
  if (k >= s) return;
  const double* Rin = (k % 2 == 0) ? xm(p, cand, XM_R1) : xm(p, cand, XM_R0);
  double* Rout = (k % 2 == 0) ? xm(p, cand, XM_R0) : xm(p, cand, XM_R1);
  double acc = 0.0;
  for (int t = 0; t < j; ++t) acc += __ldcg(Rin + r + (size_t)t * ld) * __ldcg(Rin + t + (size_t)c * ld);
  Rout[r + (size_t)c * ld] = acc;
}

static __global__ void __launch_bounds__(64) k_expm_mm(ExpmParams p, int stage, int k) {
  expm_mm_entry(p, blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.z, stage, k);
}

__device__ __forceinline__ const double* expm_result(const ExpmParams& p, int cand) {
  const int s = __ldcg(p.s_arr + cand);
  return (s % 2 == 0) ? xm(p, cand, XM_R1) : xm(p, cand, XM_R0);
}

// Pick the Krylov size: the smallest candidate j with
// eps_j = beta tau h_{j+1,j} |[exp(tau H_j)]_{j,1}| <= tol beta (Eq. "subspace
// error estimate"), or a happy breakdown; with target > 0 only j = target.
// On success: ks->found_m, eps, converged, stop; e = first column of exp(tau H_m).
// If nothing passes and last_window, the largest candidate is taken (not converged).
__device__ __forceinline__ void expm_select_block(const ExpmParams& p, KState* ks, double tol, int target,
                                                  int last_window, double* e_out) {
  __shared__ int s_pick;
  __shared__ double s_eps;
  __shared__ int s_conv;
  if (threadIdx.x == 0) {
    int pick = -1;
    double eps_pick = 0.0;
    int conv = 0;
    const double beta = ks->beta;
    if (beta == 0.0) {
      ks->found_m = 0; ks->eps = 0.0; ks->converged = 1; ks->stop = 1;
    } else if (ks->err == 0) {
      int last_valid = -1;
      for (int c = 0; c < p.ncand; ++c) {
        const int j = p.j0 + c;
        if (__ldcg(p.s_arr + c) < 0) continue;
        last_valid = c;
        const bool brk = (ks->breakdown_j == j);
        const double* E = expm_result(p, c);
        const double h = p.H[j + (size_t)(j - 1) * p.ldH];
        const double eps = brk ? 0.0 : beta * p.tau * h * fabs(__ldcg(E + j - 1));
        const bool ok = brk || (target > 0 ? (j == target) : (eps <= tol * beta));
        if (ok) { pick = c; eps_pick = eps; conv = 1; break; }
      }
      if (pick < 0 && last_window && last_valid >= 0) {
        pick = last_valid;
        const int j = p.j0 + pick;
        const double* E = expm_result(p, pick);
        eps_pick = beta * p.tau * p.H[j + (size_t)(j - 1) * p.ldH] * fabs(__ldcg(E + j - 1));
        conv = (target > 0) ? 1 : 0;
      }
      if (pick >= 0) {
        ks->found_m = p.j0 + pick;
        ks->eps = eps_pick;
        ks->converged = conv;
        ks->stop = 1;
      }
    }
    s_pick = pick;
    s_eps = eps_pick;
    s_conv = conv;
  }
  __syncthreads();
  if (s_pick >= 0) {
    const int j = p.j0 + s_pick;
    const double* E = expm_result(p, s_pick);
    for (int i = threadIdx.x; i < j; i += blockDim.x) e_out[i] = __ldcg(E + i);
  }
}

static __global__ void k_expm_select(ExpmParams p, KState* ks, double tol, int target, int last_window,
                              double* e_out) {
  expm_select_block(p, ks, tol, target, last_window, e_out);
}

// Checks of several trajectories at once (ragged batches): candidate c of the
// whole launch belongs to item i with cand_off[i] <= c < cand_off[i+1]; the
// per-candidate arithmetic is the single launch's.
constexpr int kMaxExpmBatch = 64;
struct ExpmBatch {
  int n;
  int cand_off[kMaxExpmBatch + 1];
  ExpmParams item[kMaxExpmBatch];
};
struct ExpmSelect {
  KState* ks;
  double tol;
  int last_window;
  double* e_out;
  KState* ks_copy;  // receives the state after the selection (one staging array for all items)
};
struct ExpmSelectBatch {
  ExpmSelect sel[kMaxExpmBatch];
};

__device__ __forceinline__ int expm_batch_item(const ExpmBatch& b, int c) {
  int i = 0;
  while (i + 1 < b.n && c >= b.cand_off[i + 1]) ++i;
  return i;
}

static __global__ void __launch_bounds__(256) k_expm_prep_batch(const __grid_constant__ ExpmBatch b) {
  const int i = expm_batch_item(b, blockIdx.x);
  expm_prep_cand(b.item[i], blockIdx.x - b.cand_off[i]);
}

static __global__ void __launch_bounds__(64) k_expm_mm_batch(const __grid_constant__ ExpmBatch b, int stage, int k) {
  const int i = expm_batch_item(b, blockIdx.y);
  expm_mm_entry(b.item[i], blockIdx.y - b.cand_off[i], blockIdx.x * blockDim.x + threadIdx.x, blockIdx.z, stage, k);
}

static __global__ void k_expm_select_batch(const __grid_constant__ ExpmBatch b,
                                           const __grid_constant__ ExpmSelectBatch s) {
  const ExpmSelect& q = s.sel[blockIdx.x];
  expm_select_block(b.item[blockIdx.x], q.ks, q.tol, 0, q.last_window, q.e_out);
  __syncthreads();
  if (threadIdx.x == 0 && q.ks_copy) *q.ks_copy = *q.ks;
}

// Standalone: copy the first column of the result of candidate 0.
static __global__ void k_expm_first_column(ExpmParams p, double* out) {
  const int j = p.j0;
  const double* E = expm_result(p, 0);
  for (int i = threadIdx.x; i < j; i += blockDim.x) out[i] = E[i];
}

}  // namespace etp
