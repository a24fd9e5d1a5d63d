// Newmark-beta (beta = 1/4, gamma = 1/2, average acceleration), the paper's
// comparison integrator (Section 6), on the GPU, in the mass-scaled variables
// of the propagator (u_bar = M^{1/2} u, v_bar, a_bar). Linear materials:
//
//   u_pred = u + dt v + dt^2 (1/2 - beta) a,   v_pred = v + (1 - gamma) dt a,
//   (I + beta dt^2 H_bar) a_new = -H_bar u_pred,
//   u = u_pred + beta dt^2 a_new,              v = v_pred + gamma dt a_new,
//
// with H_bar = M^{-1/2} K M^{-1/2} applied matrix-free by the propagator's
// FP64 element pass and node gather (z = A x gives -H_bar x_top in its bottom
// half), and the SPD system solved by conjugate gradients warm-started from
// the previous acceleration. Nonlinear materials: Newton iterations on
// a + R_bar(u_pred + beta dt^2 a) = 0, the residual from the secant apply
// (H(u) u = R(u)), the corrections by CG with the consistent tangent operator
// of the material (MAT_*_TANGENT on the iterate's stored coefficients). The
// state stays in the trajectory's FP64 w_bar, so etp_energy, etp_state_get and
// the propagator's steps see the same state.
#include <math.h>

#include <algorithm>
#include <cstdlib>
#include <string>

#include "etp_host.cuh"
#include "krylov_kernels.cuh"

namespace etp {
namespace {

constexpr double kNmBeta = 0.25, kNmGamma = 0.5;

// Device scalars of the CG iteration (one cache line each is not needed).
enum : int { NS_RR = 0, NS_PQ = 1, NS_RRNEW = 2, NS_BB = 3, NS_ONE = 4, NS_AA = 5, NS_RR0 = 6, NS_NUM = 8 };

// Two-stage sum of per-thread values over the grid into *out (partials, then
// the last block in block order: deterministic for a fixed grid).
// out2 (nullable) receives a second copy of the sum.
__device__ __forceinline__ void grid_sum(double acc, double* partials, unsigned int* counter, double* out,
                                         double* out2 = nullptr) {
  __shared__ double s_red[32];
  const double s = block_sum(acc, s_red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
  if (!elect_last_block(counter)) return;
  double t = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(partials + b);
  t = block_sum(t, s_red);
  if (threadIdx.x == 0) {
    *out = t;
    if (out2) *out2 = t;
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
  grid_sum(acc, partials, counter, S + NS_RR, S + NS_RR0);
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

// Newton iterate of a nonlinear step: u_bar = u_pred + c a_bar into the apply
// input X (top half) and the physical frozen state u* = M^{-1/2} u_bar (SoA).
static __global__ void __launch_bounds__(256) k_nm_newton_u(int64_t n, int64_t nn_pad, const double* __restrict__ up,
                                                            const double* __restrict__ an, double c,
                                                            const double* __restrict__ minvsqrt,
                                                            double* __restrict__ X, double* __restrict__ us) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const double u = up[r] + c * an[r];
    X[r] = u;
    us[r] = u * minvsqrt[r % nn_pad];
  }
}

// Newton right-hand side b = -(a + R_bar(u)) = Zb - a (Zb = -R_bar(u) from the
// secant apply, H(u) u = R(u)) -> R; zero start for the CG (Xs = 0); ||b||^2
// and ||a||^2 (two reductions: partials at [0, grid) and [grid, 2 grid)).
static __global__ void __launch_bounds__(256) k_nm_newton_rhs(int64_t n, const double* __restrict__ Zb,
                                                              const double* __restrict__ an, double* __restrict__ R,
                                                              double* __restrict__ Xs, double* partials,
                                                              unsigned int* counter, double* S) {
  double accb = 0.0, acca = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const double a = an[r];
    const double b = Zb[r] - a;
    R[r] = b;
    Xs[r] = 0.0;
    accb += b * b;
    acca += a * a;
  }
  grid_sum(accb, partials, counter, S + NS_BB);
  __syncthreads();
  grid_sum(acca, partials + gridDim.x, counter + 1, S + NS_AA);
}

// r = b for a zero start: p = r (X top), rr = r.r.
static __global__ void __launch_bounds__(256) k_nm_zero_start(int64_t n, const double* __restrict__ R,
                                                              double* __restrict__ X, double* partials,
                                                              unsigned int* counter, double* S) {
  double acc = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const double v = R[r];
    X[r] = v;
    acc += v * v;
  }
  grid_sum(acc, partials, counter, S + NS_RR, S + NS_RR0);
}

// a += dx (Newton update).
static __global__ void __launch_bounds__(256) k_nm_add(int64_t n, const double* __restrict__ dx, double* __restrict__ a) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    a[r] += dx[r];
}

// a = -H_bar u (Z bottom) for the initial acceleration.
static __global__ void __launch_bounds__(256) k_nm_copy(int64_t n, const double* __restrict__ src,
                                                        double* __restrict__ dst) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    dst[r] = src[r];
}

}  // namespace

// Workspace of the Newmark path (FP64, allocated at the first Newmark step):
// the stored coefficients of the Newton iterate (nonlinear only, first:
// its planes start on 16-byte boundaries), X, Z (Krylov-layout vectors of L
// rows: apply input / output), the current acceleration A, the CG vectors Xs,
// R, Q, the Newton iterate An and frozen state Us (3 nn_pad rows each), the
// device scalars and the element terms (n_elems * nen * 3).
struct NmWork {
  double *Fz, *X, *Z, *A, *Xs, *R, *Q, *An, *Us, *S, *Ye;
};

static size_t nm_fz_doubles(const etp_traj* t) {
  return t->mesh->kind == MAT_LINEAR ? 0 : frozen_buffer_bytes(t->mesh, sizeof(double)) / sizeof(double);
}

static NmWork nm_work(etp_traj* t) {
  const int64_t L = t->L, n = L / 2;
  double* b = (double*)t->d_nm;
  NmWork w;
  w.Fz = b;
  w.X = w.Fz + nm_fz_doubles(t);
  w.Z = w.X + L;
  w.A = w.Z + L;
  w.Xs = w.A + n;
  w.R = w.Xs + n;
  w.Q = w.R + n;
  w.An = w.Q + n;
  w.Us = w.An + n;
  w.S = w.Us + n;
  w.Ye = w.S + NS_NUM;
  return w;
}

size_t newmark_work_bytes(const etp_traj* t) {
  const int64_t L = t->L, n = L / 2;
  return sizeof(double) * (nm_fz_doubles(t) + (size_t)(2 * L + 6 * n + NS_NUM) +
                           (size_t)3 * t->mesh->nen * t->mesh->n_elems);
}

// z = A x in FP64 for the Krylov-layout vector X (scale 1): Z bottom =
// -H_bar X_top, with H = K (linear), the secant H(u*) or the consistent tangent.
static etp_status nm_apply(etp_traj* t, const NmWork& w, const FrozenSet& fz, int kind) {
  return apply_A<double>(t->mesh, w.X, w.S + NS_ONE, fz, w.Ye, w.Z, nullptr, nullptr, true, kind);
}

// Launch geometry, reduction scratch and pinned scalars of the Newmark kernels.
struct NmRun {
  etp_traj* t;
  NmWork w;
  int64_t n;
  unsigned grid;
  cudaStream_t st;
  double* part;
  unsigned int* cnt;
  double* h;  // pinned mirror of the device scalars
  etp_status read() {
    ETP_CUDA_TRY(cudaMemcpyAsync(h, w.S, sizeof(double) * NS_NUM, cudaMemcpyDeviceToHost, st));
    ETP_CUDA_TRY(cudaStreamSynchronize(st));
    return ETP_OK;
  }
};

// Conjugate gradients for (I + c H_bar_op) x = b: b in R, the start x0 in Xs
// (zero_start: x0 = 0, else x0 also in X top); H_bar_op = -(apply of kind)
// bottom half. On return Xs = x with ||r|| <= tol max(||b||, ||r0||); the
// residual is read every kNmCheck iterations (iterations past convergence only
// refine); the blocks of kNmCheck iterations run as a captured CUDA graph.
static etp_status nm_cg(NmRun& q, const FrozenSet& fz, int kind, double c, double tol, bool zero_start,
                        int* iters_out) {
  const NmWork& w = q.w;
  const double* Zb = w.Z + q.n;
  etp_ctx* ctx = q.t->mesh->ctx;
  if (zero_start) {
    k_nm_zero_start<<<q.grid, 256, 0, q.st>>>(q.n, w.R, w.X, q.part, q.cnt, w.S);
  } else {
    ETP_TRY(nm_apply(q.t, w, fz, kind));
    k_nm_res0<<<q.grid, 256, 0, q.st>>>(q.n, Zb, c, w.Xs, w.R, w.X, q.part, q.cnt, w.S);
  }
  ctx->launches++;
  ETP_CUDA_TRY(cudaGetLastError());
  // no synchronisation before the first block: its residual norms (||b||, ||r0||
  // kept in NS_BB / NS_RR0) are read with the first block's result
  int iters = 0;
  bool conv = false;
  constexpr int kNmCheck = 4;
  const int max_iters = 20000;
  etp_traj* t = q.t;
  // one block of kNmCheck iterations; its launches and their arguments are the
  // same for every block (the scalar slots return to their roles after an even
  // number of iterations), so it is captured once into a CUDA graph per
  // (operator kind, c) and replayed (not while event profiling is on)
  auto block = [&]() -> etp_status {
    int a = NS_RR, b = NS_RRNEW;
    for (int k = 0; k < kNmCheck; ++k) {
      ETP_TRY(nm_apply(t, w, fz, kind));
      k_nm_pq<<<q.grid, 256, 0, q.st>>>(q.n, w.X, Zb, c, w.Q, q.part, q.cnt, w.S);
      k_nm_update<<<q.grid, 256, 0, q.st>>>(q.n, w.X, w.Q, w.Xs, w.R, q.part, q.cnt, w.S, a, b);
      k_nm_dir<<<q.grid, 256, 0, q.st>>>(q.n, w.R, w.X, w.S, a, b);
      ctx->launches += 3;
      std::swap(a, b);
    }
    ETP_CUDA_TRY(cudaGetLastError());
    return ETP_OK;
  };
  // (capture needs a created stream: not the legacy default stream)
  const bool use_graph = !ctx->profiling && q.st != nullptr && !ctx->no_graphs;
  if (use_graph && (!t->nm_exec || t->nm_exec_kind != kind || t->nm_exec_c != c)) {
    if (t->nm_exec) cudaGraphExecDestroy((cudaGraphExec_t)t->nm_exec);
    t->nm_exec = nullptr;
    cudaGraph_t g = nullptr;
    ETP_CUDA_TRY(cudaStreamBeginCapture(q.st, cudaStreamCaptureModeThreadLocal));
    const etp_status bs = block();
    const cudaError_t ec = cudaStreamEndCapture(q.st, &g);
    if (bs != ETP_OK) {
      if (g) cudaGraphDestroy(g);
      return bs;
    }
    if (ec != cudaSuccess) return fail(ETP_ERR_CUDA, std::string("CG block capture: ") + cudaGetErrorString(ec));
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return fail(ETP_ERR_CUDA, std::string("CG block graph: ") + cudaGetErrorString(ei));
    t->nm_exec = ex;
    t->nm_exec_kind = kind;
    t->nm_exec_c = c;
  }
  while (!conv && iters < max_iters) {
    if (use_graph) {
      ETP_CUDA_TRY(cudaGraphLaunch((cudaGraphExec_t)t->nm_exec, q.st));
      ctx->launches += 5 * kNmCheck;  // the kernels the graph runs
    } else {
      ETP_TRY(block());
    }
    iters += kNmCheck;
    ETP_CUDA_TRY(cudaGetLastError());
    ETP_TRY(q.read());
    const double target = tol * tol * std::max(q.h[NS_BB], q.h[NS_RR0]);
    const double rr = q.h[NS_RR];  // the newest residual norm (an even number of iterations per block)
    if (!isfinite(rr)) return fail(ETP_ERR_NONFINITE, "non-finite residual in the Newmark solve");
    if (rr <= target) conv = true;
  }
  if (iters_out) *iters_out += iters;
  if (!conv) return fail(ETP_ERR_NOT_CONVERGED, "Newmark CG did not reach tol");
  return ETP_OK;
}

// Stored coefficients of the material at the frozen state w.Us (FP64).
static etp_status nm_frozen(NmRun& q, FrozenSet* fz) {
  FrozenSet one;
  one.count = 1;
  one.u[0] = q.w.Us;
  void* buf[1] = {q.w.Fz};
  ETP_TRY(build_frozen<double>(q.t->mesh, one, buf, &q.t->d_ks->err));
  *fz = one;
  return ETP_OK;
}

// Acceleration of the current state: a = -H_bar u (linear) or -R_bar(u)
// (nonlinear, through the secant identity H(u) u = R(u)).
static etp_status nm_accel0(NmRun& q) {
  etp_traj* t = q.t;
  etp_mesh* m = t->mesh;
  FrozenSet fz;
  if (m->kind == MAT_LINEAR) {
    k_nm_copy<<<q.grid, 256, 0, q.st>>>(q.n, t->d_w, q.w.X);
  } else {
    k_nm_newton_u<<<q.grid, 256, 0, q.st>>>(q.n, m->nn_pad, t->d_w, q.w.A, 0.0, m->d_minvsqrt64, q.w.X, q.w.Us);
    ETP_TRY(nm_frozen(q, &fz));
  }
  ETP_TRY(nm_apply(t, q.w, fz, m->kind));
  k_nm_copy<<<q.grid, 256, 0, q.st>>>(q.n, q.w.Z + q.n, q.w.A);
  ETP_CUDA_TRY(cudaGetLastError());
  return ETP_OK;
}

}  // namespace etp

using namespace etp;

extern "C" etp_status etp_newmark_step(etp_traj* t, double dt, double tol, int* iters_out) {
  if (!t) return fail(ETP_ERR_INVALID, "null trajectory");
  if (!(dt > 0) || !isfinite(dt)) return fail(ETP_ERR_INVALID, "dt must be positive and finite");
  if (!(tol > 0) || !(tol < 1)) return fail(ETP_ERR_INVALID, "tol must be in (0, 1)");
  etp_mesh* m = t->mesh;
  if (m->kind != MAT_LINEAR && tangent_kind(m->kind) < 0)
    return fail(ETP_ERR_INVALID, "no consistent tangent for this material");
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
  NmRun q;
  q.t = t;
  q.w = nm_work(t);
  q.n = t->L / 2;
  q.grid = (unsigned)std::min<int64_t>(4 * ctx->num_sms, (q.n + 255) / 256);
  q.st = st;
  q.part = t->d_partials;
  q.cnt = t->d_counter + 8;
  q.h = reinterpret_cast<double*>(reinterpret_cast<char*>(t->h_ks) + 2048);  // pinned scalars
  const NmWork& w = q.w;
  const double* Zb = w.Z + q.n;
  if (!t->nm_valid) {
    ETP_TRY(nm_accel0(q));
    t->nm_valid = true;
  }
  const double c = kNmBeta * dt * dt;
  int iters = 0;
  k_nm_predict<<<q.grid, 256, 0, st>>>(q.n, t->d_w, w.A, dt, t->d_wtmp, w.X);
  ctx->launches++;
  const double* a_new = w.Xs;
  if (m->kind == MAT_LINEAR) {
    FrozenSet fz;
    ETP_TRY(nm_apply(t, w, fz, MAT_LINEAR));
    k_nm_rhs<<<q.grid, 256, 0, st>>>(q.n, Zb, w.A, w.R, w.Xs, w.X, q.part, q.cnt, w.S);
    ctx->launches++;
    ETP_TRY(nm_cg(q, fz, MAT_LINEAR, c, tol, false, &iters));
  } else {
    // Newton on a + R_bar(u_pred + c a) = 0 from the previous acceleration, each
    // correction solved with the consistent tangent: (I + c H_bar_T(u)) da = -F
    k_nm_copy<<<q.grid, 256, 0, st>>>(q.n, w.A, w.An);
    bool conv = false;
    for (int it = 0; it < 30 && !conv; ++it) {
      k_nm_newton_u<<<q.grid, 256, 0, st>>>(q.n, m->nn_pad, t->d_wtmp, w.An, c, m->d_minvsqrt64, w.X, w.Us);
      FrozenSet fz;
      ETP_TRY(nm_frozen(q, &fz));
      ETP_TRY(nm_apply(t, w, fz, m->kind));  // Z bottom = -R_bar(u)
      k_nm_newton_rhs<<<q.grid, 256, 0, st>>>(q.n, Zb, w.An, w.R, w.Xs, q.part, q.cnt, w.S);
      ctx->launches += 2;
      ETP_CUDA_TRY(cudaGetLastError());
      ETP_TRY(q.read());
      const double fnorm = sqrt(q.h[NS_BB]);
      if (!isfinite(fnorm)) return fail(ETP_ERR_NONFINITE, "non-finite Newton residual in the Newmark step");
      if (fnorm <= tol * sqrt(q.h[NS_AA])) {  // relative Newton residual
        conv = true;
        break;
      }
      ETP_TRY(nm_cg(q, fz, tangent_kind(m->kind), c, tol, true, &iters));
      k_nm_add<<<q.grid, 256, 0, st>>>(q.n, w.Xs, w.An);
      ctx->launches++;
    }
    if (!conv) return fail(ETP_ERR_NOT_CONVERGED, "Newton iterations of the Newmark step did not converge");
    a_new = w.An;
  }
  if (iters_out) *iters_out = iters;
  k_nm_final<<<q.grid, 256, 0, st>>>(q.n, a_new, dt, t->d_wtmp);
  k_nm_copy<<<q.grid, 256, 0, st>>>(q.n, a_new, w.A);
  ctx->launches += 2;
  ETP_CUDA_TRY(cudaGetLastError());
  std::swap(t->d_w, t->d_wtmp);
  t->steps++;
  return ETP_OK;  // stream-ordered: the next call or read-back waits for it
}
