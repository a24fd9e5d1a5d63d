// Newmark-beta (beta = 1/4, gamma = 1/2, average acceleration), the paper's
// comparison integrator (Section 6), on the GPU for linear materials, in the
// mass-scaled variables of the propagator (u_bar = M^{1/2} u, v_bar, a_bar):
//
//   u_pred = u + dt v + dt^2 (1/2 - beta) a,   v_pred = v + (1 - gamma) dt a,
//   (I + beta dt^2 H_bar) a_new = -H_bar u_pred,
//   u = u_pred + beta dt^2 a_new,              v = v_pred + gamma dt a_new,
//
// with H_bar = M^{-1/2} K M^{-1/2} applied matrix-free by the propagator's
// FP64 element pass and node gather (z = A x gives -H_bar x_top in its bottom
// half), and the SPD system solved by conjugate gradients warm-started from
// the previous acceleration. The state stays in the trajectory's FP64 w_bar,
// so etp_energy, etp_state_get and the propagator's steps see the same state.
#include <math.h>

#include <algorithm>

#include "etp_host.cuh"
#include "krylov_kernels.cuh"

namespace etp {
namespace {

constexpr double kNmBeta = 0.25, kNmGamma = 0.5;

// Device scalars of the CG iteration (one cache line each is not needed).
enum : int { NS_RR = 0, NS_PQ = 1, NS_RRNEW = 2, NS_BB = 3, NS_ONE = 4, NS_NUM = 8 };

// Two-stage sum of per-thread values over the grid into *out (partials, then
// the last block in block order: deterministic for a fixed grid).
__device__ __forceinline__ void grid_sum(double acc, double* partials, unsigned int* counter, double* out) {
  __shared__ double s_red[32];
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

// Predictors (top and bottom halves of w_bar, n = 3 nn_pad rows each); the
// displacement predictor is also written to the apply input X (top half).
static __global__ void __launch_bounds__(256) k_nm_predict(int64_t n, const double* __restrict__ w,
                                                           const double* __restrict__ a, double dt,
                                                           double* __restrict__ wt, double* __restrict__ X) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const double u = w[r], v = w[n + r], ar = a[r];
    const double up = u + dt * v + dt * dt * (0.5 - kNmBeta) * ar;
    wt[r] = up;
    wt[n + r] = v + (1.0 - kNmGamma) * dt * ar;
    X[r] = up;
  }
}

// After the apply of u_pred: b = -H_bar u_pred (Z bottom) -> R, ||b||^2; the
// warm start x = a_prev -> Xs and the apply input X.
static __global__ void __launch_bounds__(256) k_nm_rhs(int64_t n, const double* __restrict__ Zb,
                                                       const double* __restrict__ a, double* __restrict__ R,
                                                       double* __restrict__ Xs, double* __restrict__ X,
                                                       double* partials, unsigned int* counter, double* S) {
  double acc = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const double b = Zb[r];
    R[r] = b;
    Xs[r] = a[r];
    X[r] = a[r];
    acc += b * b;
  }
  grid_sum(acc, partials, counter, S + NS_BB);
}

// After the apply of x0: r = b - (x0 + c H_bar x0) = R - Xs + c Zb; p = r (X
// top); rr = r.r.
static __global__ void __launch_bounds__(256) k_nm_res0(int64_t n, const double* __restrict__ Zb, double c,
                                                        const double* __restrict__ Xs, double* __restrict__ R,
                                                        double* __restrict__ X, double* partials,
                                                        unsigned int* counter, double* S) {
  double acc = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const double rv = R[r] - Xs[r] + c * Zb[r];
    R[r] = rv;
    X[r] = rv;
    acc += rv * rv;
  }
  grid_sum(acc, partials, counter, S + NS_RR);
}

// After the apply of p: q = p + c H_bar p = p - c Zb -> Q; pq = p.q.
static __global__ void __launch_bounds__(256) k_nm_pq(int64_t n, const double* __restrict__ X,
                                                      const double* __restrict__ Zb, double c, double* __restrict__ Q,
                                                      double* partials, unsigned int* counter, double* S) {
  double acc = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const double p = X[r];
    const double q = p - c * Zb[r];
    Q[r] = q;
    acc += p * q;
  }
  grid_sum(acc, partials, counter, S + NS_PQ);
}

// alpha = rr / pq; x += alpha p; r -= alpha q; rr' = r.r into S[i_new].
static __global__ void __launch_bounds__(256) k_nm_update(int64_t n, const double* __restrict__ X,
                                                          const double* __restrict__ Q, double* __restrict__ Xs,
                                                          double* __restrict__ R, double* partials,
                                                          unsigned int* counter, double* S, int i_old, int i_new) {
  const double pq = S[NS_PQ];
  const double alpha = pq != 0.0 ? S[i_old] / pq : 0.0;  // r = 0 exactly: nothing left to do
  double acc = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    Xs[r] += alpha * X[r];
    const double rv = R[r] - alpha * Q[r];
    R[r] = rv;
    acc += rv * rv;
  }
  grid_sum(acc, partials, counter, S + i_new);
}

// p = r + (rr' / rr) p (the apply input X).
static __global__ void __launch_bounds__(256) k_nm_dir(int64_t n, const double* __restrict__ R, double* __restrict__ X,
                                                       const double* S, int i_old, int i_new) {
  const double beta = S[i_old] != 0.0 ? S[i_new] / S[i_old] : 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    X[r] = R[r] + beta * X[r];
}

// u = u_pred + beta dt^2 a_new, v = v_pred + gamma dt a_new (in wt).
static __global__ void __launch_bounds__(256) k_nm_final(int64_t n, const double* __restrict__ Xs, double dt,
                                                         double* __restrict__ wt) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const double an = Xs[r];
    wt[r] += kNmBeta * dt * dt * an;
    wt[n + r] += kNmGamma * dt * an;
  }
}

// a = -H_bar u (Z bottom) for the initial acceleration.
static __global__ void __launch_bounds__(256) k_nm_copy(int64_t n, const double* __restrict__ src,
                                                        double* __restrict__ dst) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    dst[r] = src[r];
}

}  // namespace

// Workspace of the Newmark path (FP64, allocated at the first Newmark step):
// X, Z (Krylov-layout vectors of L rows: apply input / output), the current
// acceleration A, the CG vectors Xs (new acceleration), R, Q (3 nn_pad rows
// each), the element terms (n_elems * nen * 3) and the device scalars.
struct NmWork {
  double *X, *Z, *A, *Xs, *R, *Q, *Ye, *S;
};

static NmWork nm_work(etp_traj* t) {
  const int64_t L = t->L, n = L / 2;
  double* b = (double*)t->d_nm;
  NmWork w;
  w.X = b;
  w.Z = w.X + L;
  w.A = w.Z + L;
  w.Xs = w.A + n;
  w.R = w.Xs + n;
  w.Q = w.R + n;
  w.S = w.Q + n;
  w.Ye = w.S + NS_NUM;
  return w;
}

size_t newmark_work_bytes(const etp_traj* t) {
  const int64_t L = t->L, n = L / 2;
  return sizeof(double) * ((size_t)(2 * L + 4 * n + NS_NUM) + (size_t)3 * t->mesh->nen * t->mesh->n_elems);
}

// z = A x in FP64 for the Krylov-layout vector X (scale 1): Z bottom = -H_bar X_top.
static etp_status nm_apply(etp_traj* t, const NmWork& w) {
  FrozenSet fz;
  return apply_A<double>(t->mesh, w.X, w.S + NS_ONE, fz, w.Ye, w.Z, nullptr, nullptr, true);
}

}  // namespace etp

using namespace etp;

extern "C" etp_status etp_newmark_step(etp_traj* t, double dt, double tol, int* iters_out) {
  if (!t) return fail(ETP_ERR_INVALID, "null trajectory");
  if (!(dt > 0) || !isfinite(dt)) return fail(ETP_ERR_INVALID, "dt must be positive and finite");
  if (!(tol > 0) || !(tol < 1)) return fail(ETP_ERR_INVALID, "tol must be in (0, 1)");
  etp_mesh* m = t->mesh;
  if (m->kind != MAT_LINEAR) return fail(ETP_ERR_INVALID, "the GPU Newmark step covers linear materials");
  if (t->has_load) return fail(ETP_ERR_INVALID, "the GPU Newmark step covers P = 0");
  etp_ctx* ctx = m->ctx;
  cudaStream_t st = ctx->stream;
  ETP_CUDA_TRY(cudaSetDevice(ctx->device));
  if (!t->d_nm) {
    const size_t bytes = newmark_work_bytes(t);
    ETP_TRY(dalloc((char**)&t->d_nm, bytes));
    ETP_CUDA_TRY(cudaMemsetAsync(t->d_nm, 0, bytes, st));
    const double one = 1.0;
    ETP_CUDA_TRY(cudaMemcpyAsync(nm_work(t).S + NS_ONE, &one, sizeof(double), cudaMemcpyHostToDevice, st));
    ETP_CUDA_TRY(cudaStreamSynchronize(st));
    t->nm_valid = false;
  }
  const NmWork w = nm_work(t);
  const int64_t L = t->L, n = L / 2;
  const unsigned grid = (unsigned)std::min<int64_t>(4 * ctx->num_sms, (n + 255) / 256);
  double* part = t->d_partials;
  unsigned int* cnt = t->d_counter + 8;
  double* h = reinterpret_cast<double*>(reinterpret_cast<char*>(t->h_ks) + 2048);  // pinned scalars
  const double* Zb = w.Z + n;
  auto read_scalars = [&]() -> etp_status {
    ETP_CUDA_TRY(cudaMemcpyAsync(h, w.S, sizeof(double) * NS_NUM, cudaMemcpyDeviceToHost, st));
    ETP_CUDA_TRY(cudaStreamSynchronize(st));
    return ETP_OK;
  };
  auto blas = [&](double) { ctx->launches++; };  // vector kernels of the CG (counted, not timed)
  if (!t->nm_valid) {  // a_0 = -H_bar u_0 (M a + K u = 0)
    k_nm_copy<<<grid, 256, 0, st>>>(n, t->d_w, w.X);
    ETP_TRY(nm_apply(t, w));
    k_nm_copy<<<grid, 256, 0, st>>>(n, Zb, w.A);
    ETP_CUDA_TRY(cudaGetLastError());
    t->nm_valid = true;
  }
  const double c = kNmBeta * dt * dt;
  k_nm_predict<<<grid, 256, 0, st>>>(n, t->d_w, w.A, dt, t->d_wtmp, w.X);
  blas(8.0 * 6.0 * n);
  ETP_TRY(nm_apply(t, w));
  k_nm_rhs<<<grid, 256, 0, st>>>(n, Zb, w.A, w.R, w.Xs, w.X, part, cnt, w.S);
  blas(8.0 * 5.0 * n);
  ETP_TRY(nm_apply(t, w));
  k_nm_res0<<<grid, 256, 0, st>>>(n, Zb, c, w.Xs, w.R, w.X, part, cnt, w.S);
  blas(8.0 * 5.0 * n);
  ETP_CUDA_TRY(cudaGetLastError());
  ETP_TRY(read_scalars());
  const double target = tol * tol * std::max(h[NS_BB], h[NS_RR]);
  int iters = 0, i_old = NS_RR, i_new = NS_RRNEW;
  bool conv = !(h[NS_RR] > target);
  const int max_iters = 20000;
  // the residual is read every kNmCheck iterations (one host synchronisation
  // each); iterations past convergence only refine the solution
  constexpr int kNmCheck = 4;
  while (!conv && iters < max_iters) {
    for (int k = 0; k < kNmCheck; ++k) {
      ETP_TRY(nm_apply(t, w));
      k_nm_pq<<<grid, 256, 0, st>>>(n, w.X, Zb, c, w.Q, part, cnt, w.S);
      k_nm_update<<<grid, 256, 0, st>>>(n, w.X, w.Q, w.Xs, w.R, part, cnt, w.S, i_old, i_new);
      k_nm_dir<<<grid, 256, 0, st>>>(n, w.R, w.X, w.S, i_old, i_new);
      blas(8.0 * 13.0 * n);
      std::swap(i_old, i_new);
      ++iters;
    }
    ETP_CUDA_TRY(cudaGetLastError());
    ETP_TRY(read_scalars());
    const double rr = h[i_old];  // the newest residual norm (roles swapped after the update)
    if (!isfinite(rr)) return fail(ETP_ERR_NONFINITE, "non-finite residual in the Newmark solve");
    if (rr <= target) conv = true;
  }
  if (iters_out) *iters_out = iters;
  if (!conv) return fail(ETP_ERR_NOT_CONVERGED, "Newmark CG did not reach tol");
  k_nm_final<<<grid, 256, 0, st>>>(n, w.Xs, dt, t->d_wtmp);
  k_nm_copy<<<grid, 256, 0, st>>>(n, w.Xs, w.A);
  blas(8.0 * 7.0 * n);
  ETP_CUDA_TRY(cudaGetLastError());
  std::swap(t->d_w, t->d_wtmp);
  t->steps++;
  ETP_CUDA_TRY(cudaStreamSynchronize(st));
  return ETP_OK;
}
