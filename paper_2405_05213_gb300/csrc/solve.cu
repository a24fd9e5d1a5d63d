// Krylov solve exp(tau A) w (Section 4.3) on the device: Arnoldi with CGS2,
// windowed a-priori estimate checks, and the state combine.
#include <math.h>

#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "arnoldi_pk.cuh"
#include "cgs_bulk.cuh"
#include "etp_host.cuh"
#include "expm_kernels.cuh"
#include "krylov_kernels.cuh"
#include "lanczos.cuh"
#include "solve_fused.cuh"

namespace etp {

// Autotuned launch shapes (etp_autotune), process-wide, read before the
// built-in rules: Gram-Schmidt tile shapes keyed by (bytes per scalar, pass,
// rows, probed column count) and Q1 element-pass grids keyed by (order, bytes
// per scalar, material, geometry, frozen states, elements).
struct BulkCfgT {
  int tr = 0, ns = 0, occ = 0;
};
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int64_t, int>, BulkCfgT> g_cgs_tuned;
static std::map<std::tuple<int, int, int, int, int, int64_t>, int> g_elem_tuned;

// Tuned shape for j columns: the one probed at the smallest tuned column count
// >= j (its tiles fit for j too: shared memory grows with j).
static bool tuned_cgs(int s, int mode, int64_t L, int j, BulkCfgT* out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_cgs_tuned.lower_bound(std::make_tuple(s, mode, L, j));
  if (it == g_cgs_tuned.end() || std::get<0>(it->first) != s || std::get<1>(it->first) != mode ||
      std::get<2>(it->first) != L)
    return false;
  *out = it->second;
  return true;
}

static int tuned_elem_grid(const etp_mesh* m, int s, int ns) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_elem_tuned.find(std::make_tuple(m->order, s, m->kind, m->is_box ? 1 : 0, ns, m->n_elems));
  return it == g_elem_tuned.end() ? 0 : it->second;
}

cudaEvent_t take_event(etp_ctx* ctx) {
  if (ctx->event_pool.empty()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  cudaEvent_t e = ctx->event_pool.back();
  ctx->event_pool.pop_back();
  return e;
}

ProfScope::ProfScope(etp_ctx* c, int k, double by, double fl) : ctx(c), cls(k), bytes(by), flops(fl) {
  ctx->launches++;
  if (!ctx->profiling) return;
  a = take_event(ctx);
  b = take_event(ctx);
  if (a) cudaEventRecord(a, ctx->stream);
}

ProfScope::~ProfScope() {
  if (!ctx->profiling || !a || !b) return;
  cudaEventRecord(b, ctx->stream);
  ctx->records.push_back(ProfRecord{a, b, cls, bytes, flops});
}

// Algorithmic flops of one element pass (FMA = 2, other operations 1), counted
// from the formulation: per Gauss point the reference-gradient products and the
// gradients of x and of each frozen state over the element's nodes, the secant
// stress per frozen state (frozen coefficients + P_lin; per material below) and
// the dV scaling; per node the sum over Gauss points of P : grad N. General
// geometry adds the J^-1 products.
// Algorithmic flops (FMA = 2) of one element apply: per Gauss point the
// gradient of x (Q1: 18 per node; Q2: sum-factorised, below), the secant stress
// of each frozen state from its stored coefficients (with the rebuild of the
// fields not stored), the weight (9); the scatter P : grad N (Q1: 18 per node
// and point). General geometry adds the J^-T mapping. Shape-function values
// are tabulated, not counted.
static double plin_flops(int kind) {
  switch (kind) {
    case MAT_LINEAR: return 30.0;
    case MAT_NEOHOOKE: return 288.0;
    case MAT_MOONEY_RIVLIN: return 487.0;
    case MAT_SVK: return 192.0;
    case MAT_SVK_TANGENT: return 252.0;
    case MAT_NH_TANGENT:
    case MAT_MR_TANGENT:
    case MAT_YEOH_TANGENT: return 1500.0;  // dual-number P(F): about three times its value
    default: return 308.0;  // Yeoh
  }
}
// Flops of one element pass: the method's contractions (gradient, secant
// stress of every frozen state, scatter). The rebuild of C*^-1, P_e(D*) and E*
// from the stored fields (NH/Yeoh 123, MR 135 per point and state) is not
// counted: it is what this layout trades for bytes, not work of the method.
static double elem_apply_flops(const etp_mesh* m, int ns) {
  const double nen = m->nen, nq = m->nq;
  const double states = (m->kind == MAT_LINEAR) ? 1.0 : (double)ns;
  const double stress = states * plin_flops(m->kind) + 9.0;
  if (m->order == 2) {
    // sum-factorised gradient and scatter: three 3-point passes each (1944 FMA
    // per element each way); general geometry maps G and P by J^-T per point
    const double geo = m->is_box ? 0.0 : 36.0;
    return (2.0 * 3888.0 + nq * (stress + geo)) * (double)m->n_elems;
  }
  const double geo = m->is_box ? 0.0 : 15.0;
  const double per_q = nen * (18.0 + geo) + stress;
  const double per_e = nq * per_q + nen * nq * (18.0 + geo);
  return per_e * (double)m->n_elems;
}
// Frozen coefficients of one state: grad u* (18 per node) and F*, C*^-1, P_e
// and the material factors per Gauss point.
static double frozen_build_flops(const etp_mesh* m) {
  double prep = 0.0;
  switch (m->kind) {
    case MAT_NEOHOOKE: prep = 180.0; break;
    case MAT_MOONEY_RIVLIN: prep = 203.0; break;
    case MAT_SVK: prep = 30.0; break;
    default: prep = 194.0; break;  // Yeoh
  }
  const double geo = m->is_box ? 0.0 : 15.0;
  return (double)m->n_elems * m->nq * (m->nen * (18.0 + geo) + prep);
}

size_t frozen_buffer_bytes(const etp_mesh* m, size_t s) {
  return (size_t)frozen_nf_of(m->kind) * (size_t)frozen_stride(m->n_elems, m->nq) * s;
}

template <typename T>
etp_status build_frozen(etp_mesh* m, FrozenSet& fz, void* const* bufs, int* err) {
  if (m->kind == MAT_LINEAR) return ETP_OK;
  etp_ctx* ctx = m->ctx;
  const bool f64 = sizeof(T) == 8;
  for (int k = 0; k < fz.count; ++k) {
    FrozenBuildParams<T> p{};
    p.n_elems = m->n_elems;
    p.nn_pad = m->nn_pad;
    p.conn = m->d_conn;
    p.geo = f64 ? (const T*)m->d_geo64 : (const T*)m->d_geo32;
    for (int d = 0; d < 3; ++d) p.hinv[d] = m->is_box ? (T)(2.0 / m->box_h[d]) : T(0);
    p.us = (const T*)fz.u[k];
    for (int i = 0; i < kMaxParams; ++i) p.prm[i] = (T)m->params[i];
    p.fz = (T*)bufs[k];
    p.err = err;
    const double s = sizeof(T);
    ProfScope ps(ctx, KC_FROZEN,
                 3.0 * m->n_nodes * s + 4.0 * m->nen * m->n_elems + (double)frozen_buffer_bytes(m, sizeof(T)),
                 frozen_build_flops(m));
    cudaError_t e = (m->order == 1) ? launch_frozen_build<1, T>(p, m->kind, m->is_box, ctx->stream)
                                    : launch_frozen_build<2, T>(p, m->kind, m->is_box, ctx->stream);
    if (e != cudaSuccess) return fail(ETP_ERR_CUDA, std::string("frozen build: ") + cudaGetErrorString(e));
    fz.data[k] = bufs[k];
  }
  return ETP_OK;
}
template etp_status build_frozen<float>(etp_mesh*, FrozenSet&, void* const*, int*);
template etp_status build_frozen<double>(etp_mesh*, FrozenSet&, void* const*, int*);

// The lexicographic-box incidences of a Q1 box mesh (none otherwise).
static BoxInc mesh_box_inc(const etp_mesh* m) {
  BoxInc b;
  if (m->order == 1 && m->is_box) {
    b.nx = m->box_n[0];
    b.ny = m->box_n[1];
    b.nz = m->box_n[2];
  }
  return b;
}

template <typename T>
ApplyParams<T> make_apply_params(const etp_mesh* m, const T* x, const double* xscale, const FrozenSet& fz, T* Ye,
                                 const int* stop) {
  const bool f64 = sizeof(T) == 8;
  ApplyParams<T> p{};
  p.n_elems = m->n_elems;
  p.nn_pad = m->nn_pad;
  p.conn = m->d_conn;
  p.x = x;
  p.xscale = xscale;
  p.minvsqrt = f64 ? (const T*)m->d_minvsqrt64 : (const T*)m->d_minvsqrt32;
  p.geo = f64 ? (const T*)m->d_geo64 : (const T*)m->d_geo32;
  for (int d = 0; d < 3; ++d) p.hinv[d] = m->is_box ? (T)(2.0 / m->box_h[d]) : T(0);
  p.dvbox = m->is_box ? (T)(m->box_h[0] * m->box_h[1] * m->box_h[2] / 8.0) : T(0);
  p.escale = m->d_escale;
  p.fz0 = (const T*)fz.data[0];
  p.fz1 = (const T*)fz.data[1];
  p.c0 = (T)fz.c[0];
  p.c1 = (T)fz.c[1];
  for (int i = 0; i < kMaxParams; ++i) p.prm[i] = (T)m->params[i];
  p.Ye = Ye;
  p.stop = stop;
  p.qtab = f64 ? (const T*)m->d_qtab64 : nullptr;  // FP32 computes them faster than it loads them
  return p;
}
template ApplyParams<float> make_apply_params<float>(const etp_mesh*, const float*, const double*, const FrozenSet&,
                                                     float*, const int*);
template ApplyParams<double> make_apply_params<double>(const etp_mesh*, const double*, const double*,
                                                       const FrozenSet&, double*, const int*);

// Algorithmic bytes of one element pass: x, the stored coefficients of ns
// frozen states, the element outputs, connectivity, element scales.
double elem_apply_bytes(const etp_mesh* m, int ns, size_t s) {
  const double N = 3.0 * (double)m->n_nodes;
  return N * s + ns * (double)frozen_buffer_bytes(m, s) + 3.0 * m->nen * m->n_elems * s + 4.0 * m->nen * m->n_elems +
         (m->d_escale ? 4.0 * m->n_elems : 0.0);
}
double elem_apply_flops_of(const etp_mesh* m, int ns) { return elem_apply_flops(m, ns); }

template <typename T>
etp_status apply_A(etp_mesh* m, const T* x, const double* xscale, const FrozenSet& fz, T* Ye, T* z,
                   const int* stop, const T* pbar, bool gather, int kind_override) {
  etp_ctx* ctx = m->ctx;
  const ApplyParams<T> p = make_apply_params<T>(m, x, xscale, fz, Ye, stop);
  const int kind = kind_override >= 0 ? kind_override : m->kind;
  const int ns = (kind == MAT_LINEAR) ? 0 : fz.count;
  if (kind != MAT_LINEAR && ns == 0) return fail(ETP_ERR_INVALID, "nonlinear apply needs a frozen state");
  if (kind != MAT_LINEAR && (!fz.data[0] || (ns > 1 && !fz.data[1])))
    return fail(ETP_ERR_INVALID, "nonlinear apply needs the stored frozen coefficients");
  const double s = sizeof(T);
  const double N = 3.0 * (double)m->n_nodes;
  {
    ProfScope ps(ctx, KC_ELEM, elem_apply_bytes(m, ns, sizeof(T)), elem_apply_flops(m, ns));
    const int grid = tuned_elem_grid(m, (int)sizeof(T), ns);
    cudaError_t e = (m->order == 1)
                        ? launch_elem_apply<1, T>(p, kind, m->is_box, ns, ctx->num_sms, ctx->stream, grid)
                        : launch_elem_apply<2, T>(p, kind, m->is_box, ns, ctx->num_sms, ctx->stream, grid);
    if (e != cudaSuccess) return fail(ETP_ERR_CUDA, std::string("element apply: ") + cudaGetErrorString(e));
  }
  if (!gather) return ETP_OK;
  {
    // x (bottom half) read, z written, the element contributions and their incidence read once
    ProfScope ps(ctx, KC_GATHER, 3.0 * N * s + (3.0 * s + 4.0) * m->nen * m->n_elems + 4.0 * (m->n_nodes + 1));
    const unsigned grid = (unsigned)((m->nn_pad + 255) / 256);
    k_gather_apply<T><<<grid, 256, 0, ctx->stream>>>(m->n_nodes, m->nn_pad, m->d_inc_ptr, m->d_inc_idx,
                                                     mesh_box_inc(m), Ye,
                                                     p.minvsqrt, m->d_fixed, x + 3 * m->nn_pad, xscale, z,
                                                     stop, pbar, pbar ? x + 3 * m->nn_pad - 1 : nullptr);
    ETP_CUDA_TRY(cudaGetLastError());
  }
  return ETP_OK;
}

template etp_status apply_A<float>(etp_mesh*, const float*, const double*, const FrozenSet&, float*, float*,
                                   const int*, const float*, bool, int);
template etp_status apply_A<double>(etp_mesh*, const double*, const double*, const FrozenSet&, double*, double*,
                                    const int*, const double*, bool, int);

// Parameters of the persistent Arnoldi step j of trajectory t (z = A v_j from
// the element terms in t->d_Ye, then the CGS2 passes against columns 0..j-1).
template <typename T>
PkParams<T> make_pk_params(etp_traj* t, int j, const T* pbar) {
  etp_mesh* m = t->mesh;
  const int64_t L = t->L;
  T* V = (T*)t->d_V;
  const T* x = V + (int64_t)(j - 1) * L;
  PkParams<T> q{};
  q.n_nodes = m->n_nodes;
  q.nn_pad = m->nn_pad;
  q.inc_ptr = m->d_inc_ptr;
  q.inc_idx = m->d_inc_idx;
  q.box = mesh_box_inc(m);
  q.Ye = (const T*)t->d_Ye;
  q.minvsqrt = sizeof(T) == 8 ? (const T*)m->d_minvsqrt64 : (const T*)m->d_minvsqrt32;
  q.fixed = m->d_fixed;
  q.xb = x + 3 * m->nn_pad;
  q.xscale = t->d_coef + COEF_SCALE * COEF_STRIDE + (j - 1);
  q.c.L = L;
  q.c.V = V;
  q.c.j = j;
  q.c.z = (T*)t->d_z;
  q.c.vout = V + (int64_t)j * L;
  q.c.coef = t->d_coef;
  q.c.partials = t->d_partials;
  q.c.counter = t->d_counter;
  q.c.ks = t->d_ks;
  q.c.H = t->d_H;
  q.c.ldH = t->m_cap + 1;
  q.pbar = pbar;
  q.xi = pbar ? x + 3 * m->nn_pad - 1 : nullptr;
  q.bar = t->d_counter + 1;  // words 1-3
  q.spin_limit = m->ctx->pk_spin_limit ? m->ctx->pk_spin_limit : kBarrierSpinLimit;
  return q;
}
template PkParams<float> make_pk_params<float>(etp_traj*, int, const float*);
template PkParams<double> make_pk_params<double>(etp_traj*, int, const double*);

// Shared memory per SM, reserved shared memory per block and a kernel's static
// shared memory (cached per kernel).
struct PkSmemInfo {
  int64_t sm_bytes = 0, reserved = 0, stat = 0;
};
static PkSmemInfo pk_smem_info(const void* fn) {
  static std::mutex mu;
  static std::map<const void*, PkSmemInfo> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(fn);
  if (it != cache.end()) return it->second;
  int dev = 0, sm_bytes = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaFuncAttributes a{};
  cudaFuncGetAttributes(&a, fn);
  cudaGetLastError();
  PkSmemInfo r{sm_bytes, reserved, (int64_t)a.sharedSizeBytes};
  cache[fn] = r;
  return r;
}

// Co-resident blocks per SM (1 or 2) of a persistent-step kernel (128 threads
// of at most 128 registers: shared memory is the limit) with this much dynamic
// shared memory. Arithmetic, not an occupancy query: the batched launches ask
// with a different size almost every time.
int pk_blocks_per_sm(const void* fn, size_t smem) {
  const PkSmemInfo i = pk_smem_info(fn);
  return ((int64_t)smem + i.stat + i.reserved) * 2 <= i.sm_bytes ? 2 : 1;
}

// Dynamic shared memory a block of this persistent-step kernel can have with
// two blocks per SM.
size_t pk_two_per_sm_smem(const void* fn) {
  const PkSmemInfo i = pk_smem_info(fn);
  const int64_t v = i.sm_bytes / 2 - i.reserved - i.stat;
  return v > 0 ? (size_t)v / 16 * 16 : 0;
}

// Allow a persistent-step kernel all the dynamic shared memory a block can
// have beside its static shared memory.
void pk_allow_smem(const void* fn) {
  cudaFuncAttributes a{};
  if (cudaFuncGetAttributes(&a, fn) == cudaSuccess)
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(227 * 1024 - a.sharedSizeBytes));
  cudaGetLastError();
}

// Persistent Arnoldi step (gather + CGS2) as one cooperative launch: one block
// per tile while the tiles fit the co-resident blocks (at most two per SM).
template <typename T, int TR>
static cudaError_t launch_pk_tr(etp_traj* t, const PkParams<T>& p) {
  etp_ctx* ctx = t->mesh->ctx;
  static std::once_flag once;
  std::call_once(once, [] { pk_allow_smem((const void*)k_arnoldi_step_pk<T, TR>); });
  PkParams<T> args = p;
  size_t smem = pk_step_smem<T>(p.c.L, p.c.j, TR, args);
  const int64_t ntiles = pk_ntiles(p.c.L, TR);
  // the copy of the partial sums only where it keeps two blocks per SM (or one suffices)
  const size_t two = pk_two_per_sm_smem((const void*)k_arnoldi_step_pk<T, TR>);
  if (ntiles > ctx->num_sms && smem > two && args.red_off <= two) {
    args.red_bytes = 0;
    smem = std::max<size_t>(args.red_off, 1024);
  }
  const int bps = pk_blocks_per_sm((const void*)k_arnoldi_step_pk<T, TR>, smem);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)bps * ctx->num_sms, ntiles));
  void* argv[] = {(void*)&args};
  return cudaLaunchCooperativeKernel((const void*)k_arnoldi_step_pk<T, TR>, dim3(grid), dim3(128), argv, smem,
                                     ctx->stream);
}

template <typename T>
static cudaError_t launch_pk(etp_traj* t, const PkParams<T>& p) {
  switch (pk_tile_rows<T>(p.c.j, p.c.L)) {
    case 256: return launch_pk_tr<T, 256>(t, p);
    case 128: return launch_pk_tr<T, 128>(t, p);
    case 64: return launch_pk_tr<T, 64>(t, p);
    default: return launch_pk_tr<T, 32>(t, p);
  }
}

// Bytes of per-tile partial sums the persistent step needs for every column
// count up to m_cap (0 for vectors that use the bulk passes).
size_t pk_partials_bytes(int64_t L, int m_cap, int precision) {
  if (L > kPkMaxRows) return 0;
  int64_t most = 0;
  for (int j = 1; j <= m_cap; ++j) {
    const int tr = precision == ETP_PREC_FP64 ? pk_tile_rows<double>(j, L) : pk_tile_rows<float>(j, L);
    most = std::max(most, pk_partials_count(L, j, tr));
  }
  return sizeof(double) * (size_t)most;
}

// The persistent step pays off where launch and reduction latency dominate.
static bool use_persistent(const etp_traj* t) {
  return !t->mesh->ctx->no_persistent && t->mesh->ctx->cooperative && t->L <= kPkMaxRows;
}

static double taylor_coef(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= i;
  return 1.0 / f;
}

etp_status run_expm_window(etp_ctx* ctx, const double* H, int ldH, int j0, int j1, double tau, double* ws, int ld,
                           int* s_arr, const KState* ks, int* h_s) {
  ExpmParams p{};
  p.H = H;
  p.ldH = ldH;
  p.j0 = j0;
  p.ncand = j1 - j0 + 1;
  p.tau = tau;
  p.ws = ws;
  p.ld = ld;
  p.s_arr = s_arr;
  p.ks = ks;
  for (int k = 0; k <= EXPM_TAYLOR_DEG; ++k) p.coef[k] = taylor_coef(k);
  ProfScope ps(ctx, KC_EXPM, 0.0);
  cudaStream_t st = ctx->stream;
  k_expm_prep<<<p.ncand, 256, 0, st>>>(p);
  ETP_CUDA_TRY(cudaGetLastError());
  ETP_CUDA_TRY(cudaMemcpyAsync(h_s, s_arr, sizeof(int) * p.ncand, cudaMemcpyDeviceToHost, st));
  const unsigned gx = (unsigned)((j1 * j1 + 63) / 64);
  k_expm_mm<<<dim3(gx, p.ncand, 1), 64, 0, st>>>(p, 0, 0);
  k_expm_mm<<<dim3(gx, p.ncand, 2), 64, 0, st>>>(p, 1, 0);
  for (int k = 3; k >= 0; --k) k_expm_mm<<<dim3(gx, p.ncand, 1), 64, 0, st>>>(p, 2, k);
  ETP_CUDA_TRY(cudaGetLastError());
  ETP_CUDA_TRY(cudaStreamSynchronize(st));
  int smax = 0;
  for (int c = 0; c < p.ncand; ++c) smax = std::max(smax, h_s[c]);
  for (int k = 0; k < smax; ++k) k_expm_mm<<<dim3(gx, p.ncand, 1), 64, 0, st>>>(p, 3, k);
  ETP_CUDA_TRY(cudaGetLastError());
  ctx->launches += 6 + smax;
  return ETP_OK;
}

// One a-priori check (Eq. "subspace error estimate") in ONE cooperative
// launch: scaling and B of every candidate size, the Paterson-Stockmeyer
// products, the squarings (their number read from the scaling exponents on
// the device, no host round trip) and the selection, with bounded barriers
// between the stages. The per-entry arithmetic is the multi-launch check's
// (expm_prep_cand / expm_mm_entry / expm_select_block), so the results are the
// same bits.
struct ExpmCoop {
  ExpmParams p;
  KState* ks;
  double tol;
  int target, last_window;
  double* e_out;
  unsigned int* bar;  // three counter words of the grid barrier
};

static __global__ void __launch_bounds__(64) k_expm_window_coop(const __grid_constant__ ExpmCoop q) {
  GridBar gb = make_grid_bar(q.bar, &q.ks->err, (int)gridDim.x);
  expm_window_stages(q.p, blockIdx.x, gridDim.x, gb);
  if (blockIdx.x == 0) expm_select_block(q.p, q.ks, q.tol, q.target, q.last_window, q.e_out);
}

static cudaError_t launch_expm_window_coop(etp_ctx* ctx, const ExpmCoop& q) {
  static std::mutex mu;
  static int bps = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (bps == 0) {
      int n = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_expm_window_coop, 64, 0) != cudaSuccess || n < 1) n = 1;
      bps = std::min(n, 8);
    }
  }
  const int jmax = q.p.j0 + q.p.ncand - 1;
  const int64_t need = std::max<int64_t>(q.p.ncand, ((int64_t)jmax * jmax * q.p.ncand + 63) / 64);
  const int grid = (int)std::min<int64_t>(need, (int64_t)bps * ctx->num_sms);
  ExpmCoop args = q;
  void* argv[] = {(void*)&args};
  return cudaLaunchCooperativeKernel((const void*)k_expm_window_coop, dim3(grid), dim3(64), argv, 0, ctx->stream);
}

// Tile shape of a Gram-Schmidt pass (rows per tile, pipeline stages, blocks
// per SM) for j columns, chosen once per j: the largest tile that fits (large
// tiles need no column-group combine and fewer barriers per byte; measured on
// the 12.8M-DOF slab, 1024-row tiles at one block per SM beat 256-row tiles at
// two), with the fewest stages that keep 64 KB of copies in flight per SM,
// else as many stages as fit. The choice depends on j only, so the grid and
// the reduction order are reproducible.
struct BulkCfg {
  int tr = 0, ns = 0, occ = 0;
  size_t smem = 0;
};

constexpr size_t kBulkSmemMax = 220 * 1024;

template <typename T, int MODE, int KA>
static BulkCfg cgs_bulk_config(int j) {
  static std::mutex mu;
  static BulkCfg cache[kMaxCap + 1];
  static bool attr_set = false;
  std::lock_guard<std::mutex> lock(mu);
  if (!attr_set) {
    cudaFuncSetAttribute(k_cgs_bulk<T, MODE, KA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBulkSmemMax);
    attr_set = true;
  }
  BulkCfg& c = cache[j];
  if (c.tr) return c;
  const int trs[] = {1024, 512, 256, 128, 64};
  for (int tr : trs) {
    BulkCfg best;
    size_t best_fly = 0;
    for (int ns = 2; ns <= kBulkMaxStages; ++ns) {
      const size_t smem = cgs_bulk_smem_bytes<T>(j, tr, ns, MODE);
      if (smem > kBulkSmemMax) break;
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cgs_bulk<T, MODE, KA>, kBulkThreads, smem) !=
          cudaSuccess)
        occ = 0;
      occ = std::min(occ, kCgsMaxBlocksPerSm);
      if (occ < 1) break;
      const size_t fly = (size_t)occ * (size_t)(j + 1) * tr * sizeof(T) * (size_t)(ns - 1);
      if (fly > best_fly) {
        best_fly = fly;
        best = BulkCfg{tr, ns, occ, smem};
      }
      if (fly >= (size_t)64 * 1024) break;
    }
    if (best.tr) {
      c = best;
      break;
    }
  }
  if (!c.tr) {  // nothing with two stages fits: one stage of the smallest tile
    const size_t smem = cgs_bulk_smem_bytes<T>(j, 64, 1, MODE);
    int occ = 0;
    if (smem <= kBulkSmemMax &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cgs_bulk<T, MODE, KA>, kBulkThreads, smem) ==
            cudaSuccess &&
        occ >= 1)
      c = BulkCfg{64, 1, std::min(occ, kCgsMaxBlocksPerSm), smem};
  }
  cudaGetLastError();  // an occupancy query that failed leaves no sticky error
  return c;
}

template <typename T, int MODE, int KA>
static cudaError_t launch_cgs_ka(etp_traj* t, const CgsParams<T>& p) {
  BulkCfg c = cgs_bulk_config<T, MODE, KA>(p.j);  // also sets the kernel's shared-memory limit
  BulkCfgT u;
  if (tuned_cgs((int)sizeof(T), MODE, p.L, p.j, &u)) {
    const size_t smem = cgs_bulk_smem_bytes<T>(p.j, u.tr, u.ns, MODE);
    if (smem <= kBulkSmemMax) c = BulkCfg{u.tr, u.ns, u.occ, smem};
  }
  if (!c.tr) return cudaErrorInvalidConfiguration;
  const int64_t ntiles = (p.L + c.tr - 1) / c.tr;
  const int grid = (int)std::min<int64_t>(ntiles, (int64_t)c.occ * t->mesh->ctx->num_sms);
  k_cgs_bulk<T, MODE, KA><<<grid, kBulkThreads, c.smem, t->mesh->ctx->stream>>>(p, c.tr, c.ns);
  return cudaGetLastError();
}

// Column slots per warp: 8 (j <= 64, the common case) or 32 (j <= 256).
template <typename T, int MODE>
static cudaError_t launch_cgs(etp_traj* t, const CgsParams<T>& p) {
  if (p.j <= 8 * (kBulkThreads / 32)) return launch_cgs_ka<T, MODE, 8>(t, p);
  return launch_cgs_ka<T, MODE, 32>(t, p);
}

static int window_size(const etp_traj* t) {
  if (t->mesh->ctx->krylov_window > 0) return t->mesh->ctx->krylov_window;
  if (t->L >= (int64_t)4 << 20) return 1;
  return 2;
}

// Stored frozen coefficients of a solve's frozen states (per midpoint-history
// slot: a state already built and unchanged since is reused); fzb receives fz
// with its data pointers set. Call after the solve state is reset, so an
// inverted point found here is kept in the state.
template <typename T>
etp_status prepare_frozen(etp_traj* t, const FrozenSet& fz, FrozenSet* fzb_out) {
  etp_mesh* m = t->mesh;
  FrozenSet fzb = fz;
  if (m->kind != MAT_LINEAR && fz.count > 0) {
    const size_t need = frozen_buffer_bytes(m, sizeof(T));
    if (t->fz_bytes < need || t->fz_version != m->material_version) {
      for (bool& v : t->fz_valid) v = false;
      t->fz_version = m->material_version;
    }
    if (t->fz_bytes < need) {
      for (auto& b : t->d_fz) { dfree(b); b = nullptr; }
      t->fz_bytes = 0;
      for (auto& b : t->d_fz) ETP_TRY(dalloc((char**)&b, need));
      t->fz_bytes = need;
    }
    for (int k = 0; k < fz.count; ++k) {
      const int sl = fz.slot[k];
      if (sl < 0 || sl > 2) return fail(ETP_ERR_INVALID, "frozen state without a history slot");
      if (!t->fz_valid[sl]) {
        FrozenSet one;
        one.count = 1;
        one.u[0] = fz.u[k];
        void* buf[1] = {t->d_fz[sl]};
        ETP_TRY(build_frozen<T>(m, one, buf, &t->d_ks->err));
        t->fz_valid[sl] = true;
      }
      fzb.data[k] = t->d_fz[sl];
    }
  }
  *fzb_out = fzb;
  return ETP_OK;
}
template etp_status prepare_frozen<float>(etp_traj*, const FrozenSet&, FrozenSet*);
template etp_status prepare_frozen<double>(etp_traj*, const FrozenSet&, FrozenSet*);

template <typename T>
static etp_status solve_impl(etp_traj* t, double tau, const double* w_in, double* w_out, const FrozenSet& fz,
                             double tol, int m_fixed, T* ustar_out, SolveResult* res, int kind) {
  etp_mesh* m = t->mesh;
  etp_ctx* ctx = m->ctx;
  cudaStream_t st = ctx->stream;
  const int64_t L = t->L;
  T* V = (T*)t->d_V;
  T* z = (T*)t->d_z;
  const double s = sizeof(T);
  const int red_grid = 2 * ctx->num_sms;
  {
    ProfScope ps(ctx, KC_OTHER, (double)L * (8.0 + s));
    k_init_basis<T><<<red_grid, 256, 0, st>>>(L, w_in, V, t->d_partials, t->d_counter, t->d_coef, t->d_ks);
    ETP_CUDA_TRY(cudaGetLastError());
  }
  const T* pbar = t->has_load ? (const T*)t->d_pbar : nullptr;  // constant external load
  // the frozen state is fixed for the whole solve: its coefficients are built
  // once here (after the solve state is reset, so an inverted point is kept)
  FrozenSet fzb;
  ETP_TRY(prepare_frozen<T>(t, fz, &fzb));
  // energy-inner-product Lanczos (linear materials without load): the start
  // column's E-norm from one apply; ks->beta and its scale become ||w||_E
  const bool lz = t->krylov == ETP_KRYLOV_LANCZOS_ENERGY;
  double* betas = t->d_coef + COEF_D * COEF_STRIDE;
  const double* one = t->d_coef + COEF_MISC * COEF_STRIDE + MISC_ONE;
  if (lz) {
    if (m->kind != MAT_LINEAR || pbar)
      return fail(ETP_ERR_INVALID, "the energy Lanczos process needs a linear material without load");
    ETP_TRY(apply_A<T>(m, V, one, fzb, (T*)t->d_Ye, z, &t->d_ks->stop, nullptr, true));
    ProfScope ps(ctx, KC_LANCZOS, 1.5 * (double)L * s);
    k_lanczos_norm<T><<<4 * ctx->num_sms, 256, 0, st>>>(L, V, z, t->d_partials, t->d_counter, t->d_coef, betas, t->d_H,
                                               t->m_cap + 1, 0, 1, t->d_ks);
    ETP_CUDA_TRY(cudaGetLastError());
  }
  const int cap = m_fixed > 0 ? m_fixed : t->m_cap;
  // Check schedule. Every size 1..m is checked, in ascending order, so the
  // selected m is the smallest passing one (Eq. "subspace error estimate")
  // whatever the schedule. The first checkpoint is one below the previous
  // solve's m of this kind (at it for short vectors, where an Arnoldi step costs
  // less than a check and m mostly repeats): all sizes up to it are evaluated
  // in one batched launch set (the products of the small exponential are
  // launch-bound, so many candidates cost about one), then every W steps.
  const int W = window_size(t);
  const int hint = t->m_hint[kind & 1];
  const bool pk = !lz && use_persistent(t);
  int next_check = m_fixed > 0 ? cap : std::min(cap, hint >= 2 ? (pk ? hint : hint - 1) : 8);
  int* d_stop = &t->d_ks->stop;
  int done = 0, win_start = 1;
  bool found = false, failed = false;
  // Short vectors on a Q1 box: the whole solve in one cooperative launch (as far
  // as its shared memory reaches; a fixed m only if all of it), one host
  // synchronisation; same bits as the launch-per-step loop below, which takes
  // over if the solve is not done by then.
  if (pk && m->order == 1 && m->is_box && !ctx->no_fused && ctx->pk_spin_limit == 0) {
    const int ns = (m->kind == MAT_LINEAR) ? 0 : fzb.count;
    const FusedPlan plan = fused_plan<T>(m->kind, ns, cap, L, ctx->num_sms);
    int j_end = plan.j_end;
    if (m_fixed > 0 && j_end < cap) j_end = 0;
    if (j_end >= 1) {
      FusedSolve<T> f{};
      const double* scale = t->d_coef + COEF_SCALE * COEF_STRIDE;
      f.ap = make_apply_params<T>(m, V, scale, fzb, (T*)t->d_Ye, d_stop);
      // a small mesh spread over every block of the launch (FP64 arithmetic is slow per SM)
      f.ap.epb = (int)std::min<int64_t>(ElemTraits<1>::EPB, std::max<int64_t>(1, (m->n_elems + plan.grid - 1) / plan.grid));
      f.pk = make_pk_params<T>(t, 1, pbar);
      f.pk.spin_limit = kBarrierSpinLimit;  // the test hook's lower limit applies to the per-step kernel only
      f.ex.H = t->d_H; f.ex.ldH = t->m_cap + 1; f.ex.tau = tau; f.ex.ws = t->d_expm_ws; f.ex.ld = t->m_cap;
      f.ex.s_arr = (int*)t->d_red; f.ex.ks = t->d_ks;
      for (int k = 0; k <= EXPM_TAYLOR_DEG; ++k) f.ex.coef[k] = taylor_coef(k);
      f.ks = t->d_ks;
      f.V = V;
      f.scale = scale;
      f.j_end = j_end;
      f.cap = cap;
      f.first_check = std::min(j_end, next_check);
      f.W = W;
      f.m_fixed = m_fixed;
      f.tol = tol;
      f.e_out = t->d_y;
      {
        ProfScope ps(ctx, KC_FUSED, (double)j_end * (elem_apply_bytes(m, ns, sizeof(T)) + 9.0 * m->n_nodes * s) +
                                        (double)j_end * (3.0 * j_end / 2.0 + 5.0) * L * s);
        // every SM: the small exponentials of the checks are FP64 products, spread over the GPU
        ETP_CUDA_TRY(launch_fused_solve<T>(ctx, f, m->kind, ns, plan));
      }
      ctx->launches++;
      ETP_CUDA_TRY(cudaMemcpyAsync(t->h_ks, t->d_ks, sizeof(KState), cudaMemcpyDeviceToHost, st));
      ETP_CUDA_TRY(cudaStreamSynchronize(st));
      if (t->h_ks->err) failed = true;
      else if (t->h_ks->found_m >= 0) found = true;
      done = j_end;
      win_start = j_end + 1;
      next_check = std::min(cap, j_end + W);
    }
  }
  while (done < cap && !found && !failed) {
    const int jend = next_check;
    for (int j = done + 1; j <= jend; ++j) {
      if (lz) {
        // v_{j+1} from A v_j + beta_{j-1} v_{j-1} (raw column j), its apply, its E-norm
        T* col = V + (int64_t)j * L;
        {
          ProfScope ps(ctx, KC_LANCZOS, (j >= 2 ? 3.0 : 2.0) * (double)L * s);
          k_lanczos_form<T><<<8 * ctx->num_sms, 256, 0, st>>>(L, z, j >= 2 ? V + (int64_t)(j - 2) * L : nullptr,
                                                              col, t->d_coef, j, betas, t->d_ks);
          ETP_CUDA_TRY(cudaGetLastError());
        }
        ETP_TRY(apply_A<T>(m, col, one, fzb, (T*)t->d_Ye, z, d_stop, nullptr, true));
        ProfScope ps(ctx, KC_LANCZOS, 1.5 * (double)L * s);
        k_lanczos_norm<T><<<4 * ctx->num_sms, 256, 0, st>>>(L, col, z, t->d_partials, t->d_counter, t->d_coef, betas,
                                                   t->d_H, t->m_cap + 1, j, 0, t->d_ks);
        ETP_CUDA_TRY(cudaGetLastError());
        continue;
      }
      const T* x = V + (int64_t)(j - 1) * L;
      const double* xscale = t->d_coef + COEF_SCALE * COEF_STRIDE + (j - 1);
      if (pk) {
        ETP_TRY(apply_A<T>(m, x, xscale, fzb, (T*)t->d_Ye, z, d_stop, pbar, false));
        const PkParams<T> q = make_pk_params<T>(t, j, pbar);
        ProfScope ps(ctx, KC_FUSED, 3.0 * 3.0 * m->n_nodes * s + (double)(3 * j + 5) * L * s);
        ETP_CUDA_TRY(launch_pk<T>(t, q));
        continue;
      }
      ETP_TRY(apply_A<T>(m, x, xscale, fzb, (T*)t->d_Ye, z, d_stop, pbar));
      CgsParams<T> p{};
      p.L = L;
      p.V = V;
      p.j = j;
      p.z = z;
      p.vout = V + (int64_t)j * L;
      p.coef = t->d_coef;
      p.partials = t->d_partials;
      p.counter = t->d_counter;
      p.ks = t->d_ks;
      p.H = t->d_H;
      p.ldH = t->m_cap + 1;
      // two passes per step (cgs_bulk.cuh): dots with z, then q_j and the next
      // candidate from the same staged tiles with their dots
      {
        ProfScope ps(ctx, KC_DOT, (double)(j + 1) * L * s);
        ETP_CUDA_TRY((launch_cgs<T, BULK_DOT>(t, p)));
      }
      {
        ProfScope ps(ctx, KC_UPD_DOT, (double)(j + 3) * L * s);
        ETP_CUDA_TRY((launch_cgs<T, BULK_UPD>(t, p)));
      }
    }
    done = jend;
    int target = 0;
    int lo = win_start, hi = done;
    if (m_fixed > 0) {
      // learn whether a breakdown ended the process early
      ETP_CUDA_TRY(cudaMemcpyAsync(t->h_ks, t->d_ks, sizeof(KState), cudaMemcpyDeviceToHost, st));
      ETP_CUDA_TRY(cudaStreamSynchronize(st));
      if (t->h_ks->err) { failed = true; break; }
      const int jb = t->h_ks->breakdown_j;
      lo = hi = target = (jb > 0 ? jb : cap);
      if (t->h_ks->beta == 0.0) lo = hi = target = 1;
    }
    for (int j0 = lo; j0 <= hi && !found && !failed; j0 += kMaxCand) {
      const int j1 = std::min(hi, j0 + kMaxCand - 1);
      ExpmParams q{};
      q.H = t->d_H; q.ldH = t->m_cap + 1; q.j0 = j0; q.ncand = j1 - j0 + 1; q.tau = tau;
      q.ws = t->d_expm_ws; q.ld = t->m_cap; q.s_arr = (int*)t->d_red; q.ks = t->d_ks;
      if (ctx->cooperative && !ctx->no_coop_expm) {
        // the whole check in one launch (no host read of the scaling exponents)
        for (int k = 0; k <= EXPM_TAYLOR_DEG; ++k) q.coef[k] = taylor_coef(k);
        ExpmCoop c{q, t->d_ks, tol, target, (j1 >= cap) ? 1 : 0, t->d_y, t->d_counter + 10};  // words 10-12
        ProfScope ps(ctx, KC_EXPM, 0.0);
        ETP_CUDA_TRY(launch_expm_window_coop(ctx, c));
      } else {
        ETP_TRY(run_expm_window(ctx, t->d_H, t->m_cap + 1, j0, j1, tau, t->d_expm_ws, t->m_cap,
                                (int*)t->d_red, t->d_ks, (int*)(t->h_ks + 1)));
        ProfScope ps(ctx, KC_EXPM, 0.0);
        k_expm_select<<<1, 128, 0, st>>>(q, t->d_ks, tol, target, (j1 >= cap) ? 1 : 0, t->d_y);
        ETP_CUDA_TRY(cudaGetLastError());
      }
      ETP_CUDA_TRY(cudaMemcpyAsync(t->h_ks, t->d_ks, sizeof(KState), cudaMemcpyDeviceToHost, st));
      ETP_CUDA_TRY(cudaStreamSynchronize(st));
      if (t->h_ks->err) failed = true;
      else if (t->h_ks->found_m >= 0) found = true;
    }
    win_start = done + 1;
    next_check = std::min(cap, done + W);
  }
  const KState& ks = *t->h_ks;
  if (ks.err & KERR_TIMEOUT) {
    // a barrier or a copy wait gave up: reset the reduction and barrier words
    // so the next solve starts clean
    cudaMemsetAsync(t->d_counter, 0, 16 * sizeof(unsigned int), st);
    return fail(ETP_ERR_TIMEOUT, "a bounded wait of the Arnoldi step timed out");
  }
  if (ks.err & KERR_INVERTED) return fail(ETP_ERR_INVERTED_ELEMENT, "det F <= 0 at a Gauss point of the frozen state");
  if (ks.err) return fail(ETP_ERR_NONFINITE, "non-finite value in the Krylov process");
  if (!found) return fail(ETP_ERR_INVALID, "Krylov solve ended without a selected size");
  {
    ProfScope ps(ctx, KC_COMBINE, (double)std::max(ks.found_m - 1, 0) * L * s + 2.0 * L * 8.0);
    const T* minv = sizeof(T) == 8 ? (const T*)m->d_minvsqrt64 : (const T*)m->d_minvsqrt32;
    k_combine<T><<<4 * ctx->num_sms, 256, 0, st>>>(L, m->nn_pad, w_in, V, t->d_y, t->d_coef, t->d_ks, w_out,
                                                   ustar_out, minv);
    ETP_CUDA_TRY(cudaGetLastError());
  }
  res->m = ks.found_m;
  res->eps = ks.eps;
  res->beta = ks.beta;
  res->converged = ks.converged != 0;
  t->last_m = ks.found_m;
  if (m_fixed == 0 && ks.found_m > 0) t->m_hint[kind & 1] = ks.found_m;
  return ETP_OK;
}

etp_status krylov_solve(etp_traj* t, double tau, const double* w_in, double* w_out, const FrozenSet& fz,
                        double tol, int m_fixed, void* ustar_out, SolveResult* res, int kind) {
  if (t->prec == ETP_PREC_FP64)
    return solve_impl<double>(t, tau, w_in, w_out, fz, tol, m_fixed, (double*)ustar_out, res, kind);
  return solve_impl<float>(t, tau, w_in, w_out, fz, tol, m_fixed, (float*)ustar_out, res, kind);
}

// ---------------------------------------------------------------- autotuner
// Times `reps` launches (after one untimed) of every candidate on the
// trajectory's own buffers; returns the fastest candidate's index. `launch(c)`
// issues candidate c. The solve state is zeroed before every launch so that
// no pass skips its work.
template <typename F>
static int time_candidates(etp_traj* t, int n_cand, int reps, F launch, float* best_ms) {
  cudaStream_t st = t->mesh->ctx->stream;
  std::vector<cudaEvent_t> ev(2 * reps);
  for (auto& e : ev) cudaEventCreate(&e);
  int best = -1;
  float best_t = 0.f;
  for (int c = 0; c < n_cand; ++c) {
    bool ok = true;
    for (int r = 0; r <= reps; ++r) {
      cudaMemsetAsync(t->d_ks, 0, sizeof(KState), st);
      if (r > 0) cudaEventRecord(ev[2 * (r - 1)], st);
      if (launch(c) != cudaSuccess) ok = false;
      if (r > 0) cudaEventRecord(ev[2 * (r - 1) + 1], st);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess || !ok) {
      cudaGetLastError();
      continue;
    }
    float tmin = 1e30f;
    for (int r = 0; r < reps; ++r) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[2 * r], ev[2 * r + 1]);
      tmin = std::min(tmin, ms);
    }
    if (best < 0 || tmin < best_t) {
      best = c;
      best_t = tmin;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (best_ms) *best_ms = best_t;
  return best;
}

template <typename T, int MODE, int KA>
static int tune_cgs_probe(etp_traj* t, int j, int reps) {
  etp_ctx* ctx = t->mesh->ctx;
  (void)cgs_bulk_config<T, MODE, KA>(j);  // shared-memory limit of the kernel
  CgsParams<T> p{};
  p.L = t->L;
  p.V = (T*)t->d_V;
  p.j = j;
  p.z = (T*)t->d_z;
  p.vout = (T*)t->d_V + (int64_t)j * t->L;
  p.coef = t->d_coef;
  p.partials = t->d_partials;
  p.counter = t->d_counter;
  p.ks = t->d_ks;
  p.H = t->d_H;
  p.ldH = t->m_cap + 1;
  std::vector<BulkCfg> cand;
  for (int tr : {1024, 512, 256, 128, 64})
    for (int ns = 2; ns <= kBulkMaxStages; ++ns) {
      const size_t smem = cgs_bulk_smem_bytes<T>(j, tr, ns, MODE);
      if (smem > kBulkSmemMax) continue;
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cgs_bulk<T, MODE, KA>, kBulkThreads, smem) !=
          cudaSuccess)
        occ = 0;
      occ = std::min(occ, kCgsMaxBlocksPerSm);
      if (occ < 1) continue;
      cand.push_back(BulkCfg{tr, ns, occ, smem});
      if (occ > 1) cand.push_back(BulkCfg{tr, ns, std::max(1, occ / 2), smem});
    }
  cudaGetLastError();
  if (cand.empty()) return 0;
  auto launch = [&](int c) {
    const BulkCfg& b = cand[c];
    const int64_t ntiles = (p.L + b.tr - 1) / b.tr;
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)b.occ * ctx->num_sms);
    k_cgs_bulk<T, MODE, KA><<<grid, kBulkThreads, b.smem, ctx->stream>>>(p, b.tr, b.ns);
    return cudaGetLastError();
  };
  const int best = time_candidates(t, (int)cand.size(), reps, launch, nullptr);
  if (best < 0) return 0;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_cgs_tuned[std::make_tuple((int)sizeof(T), MODE, t->L, j)] = BulkCfgT{cand[best].tr, cand[best].ns, cand[best].occ};
  return 1;
}

template <typename T>
static int tune_elem(etp_traj* t, int reps) {
  etp_mesh* m = t->mesh;
  etp_ctx* ctx = m->ctx;
  if (m->order != 1) return 0;  // Q2 passes take one block per block of elements
  int tuned = 0;
  const std::vector<int> states = m->kind == MAT_LINEAR ? std::vector<int>{0} : std::vector<int>{1, 2};
  for (int ns : states) {
    FrozenSet fz;
    fz.count = ns;
    fz.data[0] = t->d_fz[0];
    fz.data[1] = t->d_fz[1];
    fz.c[0] = 1.75;
    fz.c[1] = -0.75;
    const ApplyParams<T> p =
        make_apply_params<T>(m, (const T*)t->d_V, t->d_coef + COEF_SCALE * COEF_STRIDE, fz, (T*)t->d_Ye, nullptr);
    const int64_t nblocks = (m->n_elems + ElemTraits<1>::EPB - 1) / ElemTraits<1>::EPB;
    std::vector<int> grids = {0};  // the built-in rule: one wave of resident blocks
    for (int k : {1, 2, 3, 4, 6, 8, 12, 16})
      if ((int64_t)k * ctx->num_sms <= nblocks) grids.push_back(k * ctx->num_sms);
    auto launch = [&](int c) {
      return launch_elem_apply<1, T>(p, m->kind, m->is_box, ns, ctx->num_sms, ctx->stream, grids[c]);
    };
    // at least 7 timed launches per grid (one launch is ~1 ms at 12.8M DOFs; near-ties are common)
    const int best = time_candidates(t, (int)grids.size(), std::max(reps, 7), launch, nullptr);
    if (best < 0) continue;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_elem_tuned[std::make_tuple(m->order, (int)sizeof(T), m->kind, m->is_box ? 1 : 0, ns, m->n_elems)] = grids[best];
    ++tuned;
  }
  return tuned;
}

template <typename T>
static etp_status autotune_impl(etp_traj* t, int reps, int* n_out) {
  etp_ctx* ctx = t->mesh->ctx;
  cudaStream_t st = ctx->stream;
  // defined contents for the timed passes (the workspace is scratch between steps)
  ETP_CUDA_TRY(cudaMemsetAsync(t->d_V, 0, sizeof(T) * (size_t)t->L * (t->m_cap + 1), st));
  ETP_CUDA_TRY(cudaMemsetAsync(t->d_z, 0, sizeof(T) * (size_t)t->L, st));
  ETP_CUDA_TRY(cudaMemsetAsync(t->d_coef, 0, sizeof(double) * COEF_NUM * COEF_STRIDE, st));
  int n = tune_elem<T>(t, reps);
  if (!use_persistent(t)) {
    std::vector<int> probes;
    // every column count up to 32 (the common Krylov sizes), then coarser
    for (int j = 1; j <= 32; ++j)
      if (j <= t->m_cap) probes.push_back(j);
    for (int j : {40, 48, 56, 64, 96, 128, 192, 256})
      if (j <= t->m_cap) probes.push_back(j);
    if (probes.empty() || probes.back() != t->m_cap) probes.push_back(t->m_cap);
    for (int j : probes) {
      if (j <= 8 * (kBulkThreads / 32)) {
        n += tune_cgs_probe<T, BULK_DOT, 8>(t, j, reps);
        n += tune_cgs_probe<T, BULK_UPD, 8>(t, j, reps);
      } else {
        n += tune_cgs_probe<T, BULK_DOT, 32>(t, j, reps);
        n += tune_cgs_probe<T, BULK_UPD, 32>(t, j, reps);
      }
    }
  }
  // leave the solve state as a fresh trajectory has it
  ETP_CUDA_TRY(cudaMemsetAsync(t->d_ks, 0, sizeof(KState), st));
  ETP_CUDA_TRY(cudaMemsetAsync(t->d_counter, 0, sizeof(unsigned int) * 16, st));
  ETP_CUDA_TRY(cudaMemsetAsync(t->d_coef, 0, sizeof(double) * COEF_NUM * COEF_STRIDE, st));
  ETP_CUDA_TRY(cudaStreamSynchronize(st));
  if (n_out) *n_out = n;
  return ETP_OK;
}

}  // namespace etp

extern "C" etp_status etp_autotune(etp_traj* t, int reps, int* n_configs) {
  using namespace etp;
  if (!t) return fail(ETP_ERR_INVALID, "null trajectory");
  if (reps < 1 || reps > 100) return fail(ETP_ERR_INVALID, "reps must be in 1..100");
  ETP_CUDA_TRY(cudaSetDevice(t->mesh->ctx->device));
  return t->prec == ETP_PREC_FP64 ? autotune_impl<double>(t, reps, n_configs)
                                  : autotune_impl<float>(t, reps, n_configs);
}
