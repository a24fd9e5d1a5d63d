// C ABI of libetp (include/etp.h): contexts, meshes, materials, trajectories,
// the time step (Sections 3-4), energy (Section 5.2), checkpoints, diagnostics.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cstdlib>
#include <string>
#include <vector>

#include "etp_host.cuh"
#include "expm_kernels.cuh"
#include "fe_setup_kernels.cuh"
#include "krylov_kernels.cuh"

namespace etp {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

etp_status fail(etp_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

// Detect a uniform lexicographic box: coordinates on a tensor grid with equal
// spacing per axis and the connectivity of the lexicographic generator.
static bool detect_box(etp_mesh* m) {
  const int p = m->order;
  const int64_t nn = m->n_nodes;
  const double* X = m->h_coords.data();
  std::vector<double> xs, ys, zs;
  for (int64_t n = 0; n < nn; ++n) {
    if (X[3 * n + 1] == X[1] && X[3 * n + 2] == X[2]) xs.push_back(X[3 * n]);
  }
  const int64_t NX = (int64_t)xs.size();
  if (NX < 2 || nn % NX) return false;
  for (int64_t n = 0; n < nn; n += NX) {
    if (X[3 * n + 2] == X[2]) ys.push_back(X[3 * n + 1]);
  }
  const int64_t NY = (int64_t)ys.size();
  if (NY < 2 || nn % (NX * NY)) return false;
  const int64_t NZ = nn / (NX * NY);
  if (NZ < 2) return false;
  for (int64_t k = 0; k < NZ; ++k) zs.push_back(X[3 * (k * NX * NY) + 2]);
  if ((NX - 1) % p || (NY - 1) % p || (NZ - 1) % p) return false;
  const double hx = (xs.back() - xs[0]) / (NX - 1), hy = (ys.back() - ys[0]) / (NY - 1),
               hz = (zs.back() - zs[0]) / (NZ - 1);
  if (!(hx > 0 && hy > 0 && hz > 0)) return false;
  auto tol = [](double h) { return 1e-12 * std::max(1.0, fabs(h)); };
  for (int64_t k = 0; k < NZ; ++k)
    for (int64_t j = 0; j < NY; ++j)
      for (int64_t i = 0; i < NX; ++i) {
        const int64_t n = i + NX * (j + NY * k);
        if (fabs(X[3 * n] - (xs[0] + i * hx)) > tol(xs.back()) || fabs(X[3 * n + 1] - (ys[0] + j * hy)) > tol(ys.back()) ||
            fabs(X[3 * n + 2] - (zs[0] + k * hz)) > tol(zs.back()))
          return false;
      }
  const int64_t nx = (NX - 1) / p, ny = (NY - 1) / p, nz = (NZ - 1) / p;
  if (nx * ny * nz != m->n_elems) return false;
  const int p1 = p + 1;
  for (int64_t ek = 0; ek < nz; ++ek)
    for (int64_t ej = 0; ej < ny; ++ej)
      for (int64_t ei = 0; ei < nx; ++ei) {
        const int64_t e = ei + nx * (ej + ny * ek);
        for (int c = 0; c < p1; ++c)
          for (int b = 0; b < p1; ++b)
            for (int a = 0; a < p1; ++a) {
              const int64_t n = (p * ei + a) + NX * ((p * ej + b) + NY * (p * ek + c));
              if (m->h_conn[e * m->nen + a + p1 * (b + p1 * c)] != n) return false;
            }
      }
  m->box_n[0] = (int)nx; m->box_n[1] = (int)ny; m->box_n[2] = (int)nz;
  m->box_h[0] = hx * p; m->box_h[1] = hy * p; m->box_h[2] = hz * p;  // element edge lengths
  return true;
}

}  // namespace etp

using namespace etp;

extern "C" {

const char* etp_last_error(void) { return g_err.c_str(); }

const char* etp_version(void) { return "etp 0.1 (sm_103a)"; }

etp_status etp_ctx_create(int device, void* cuda_stream, etp_ctx** out) {
  if (!out) return fail(ETP_ERR_INVALID, "out is null");
  *out = nullptr;
  int ndev = 0;
  ETP_CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(ETP_ERR_INVALID, "no such CUDA device");
  ETP_CUDA_TRY(cudaSetDevice(device));
  etp_ctx* c = new etp_ctx();
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
  c->cooperative = coop != 0;
  c->no_persistent = std::getenv("ETP_NO_PERSISTENT") != nullptr;
  c->no_fused = std::getenv("ETP_NO_FUSED_SOLVE") != nullptr;
  c->no_coop_expm = std::getenv("ETP_NO_COOP_EXPM") != nullptr;
  if (const char* s = std::getenv("ETP_KRYLOV_WINDOW")) {
    const int w = atoi(s);
    if (w >= 1 && w <= 8) c->krylov_window = w;
  }
  c->no_graphs = std::getenv("ETP_NO_GRAPHS") != nullptr;
  *out = c;
  return ETP_OK;
}

etp_status etp_debug_spin_limit(etp_ctx* c, uint64_t polls) {
  if (!c) return fail(ETP_ERR_INVALID, "null context");
  c->pk_spin_limit = polls;
  return ETP_OK;
}

void etp_ctx_destroy(etp_ctx* c) {
  if (!c) return;
  for (auto& r : c->records) { cudaEventDestroy(r.start); cudaEventDestroy(r.stop); }
  for (auto e : c->event_pool) cudaEventDestroy(e);
  dfree(c->expm_ws);
  dfree(c->d_chk_s);
  dfree(c->d_chk_ks);
  if (c->h_chk_s) cudaFreeHost(c->h_chk_s);
  if (c->h_chk_ks) cudaFreeHost(c->h_chk_ks);
  delete c;
}

etp_status etp_mesh_create(etp_ctx* ctx, int order, int64_t n_nodes, const double* coords, int64_t n_elems,
                           const int32_t* conn, int64_t n_fixed, const int32_t* fixed_dofs, etp_mesh** out) {
  if (!ctx || !out) return fail(ETP_ERR_INVALID, "null context or out");
  *out = nullptr;
  if (order != 1 && order != 2) return fail(ETP_ERR_INVALID, "order must be 1 or 2");
  if (n_nodes <= 0 || n_elems <= 0 || !coords || !conn) return fail(ETP_ERR_INVALID, "empty mesh");
  if (n_nodes > (int64_t)INT32_MAX / 3) return fail(ETP_ERR_INVALID, "too many nodes");
  if (n_fixed < 0 || (n_fixed > 0 && !fixed_dofs)) return fail(ETP_ERR_INVALID, "bad fixed DOF list");
  ETP_CUDA_TRY(cudaSetDevice(ctx->device));
  etp_mesh* m = new etp_mesh();
  m->ctx = ctx;
  m->order = order;
  m->nen = (order + 1) * (order + 1) * (order + 1);
  m->nq = m->nen;
  m->n_nodes = n_nodes;
  m->n_elems = n_elems;
  // at least one padding node: its last top-half row carries the augmented
  // entry of a loaded state (etp_load_set)
  m->nn_pad = round_up(n_nodes + 1, 128);
  if ((int64_t)m->nen * n_elems > (int64_t)INT32_MAX) { delete m; return fail(ETP_ERR_INVALID, "too many elements"); }
  m->h_coords.assign(coords, coords + 3 * n_nodes);
  m->h_conn.assign(conn, conn + m->nen * n_elems);
  for (int64_t i = 0; i < m->nen * n_elems; ++i)
    if (conn[i] < 0 || conn[i] >= n_nodes) { delete m; return fail(ETP_ERR_INVALID, "connectivity out of range"); }
  m->h_fixed.assign(n_nodes, 0);
  for (int64_t i = 0; i < n_fixed; ++i) {
    const int32_t d = fixed_dofs[i];
    if (d < 0 || d >= 3 * n_nodes) { delete m; return fail(ETP_ERR_INVALID, "fixed DOF out of range"); }
    m->h_fixed[d / 3] |= (uint8_t)(1u << (d % 3));
  }
  m->is_box = detect_box(m) && !std::getenv("ETP_FORCE_GENERAL_GEOMETRY");
  // node -> (element, local node) incidence, ascending
  std::vector<int32_t> ptr(n_nodes + 1, 0), idx((size_t)m->nen * n_elems);
  for (int64_t i = 0; i < m->nen * n_elems; ++i) ptr[conn[i] + 1]++;
  for (int64_t n = 0; n < n_nodes; ++n) ptr[n + 1] += ptr[n];
  std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
  for (int64_t i = 0; i < m->nen * n_elems; ++i) idx[fill[conn[i]]++] = (int32_t)i;
  etp_status s = ETP_OK;
  auto cleanup = [&](etp_status st) { etp_mesh_destroy(m); return st; };
  if ((s = dalloc(&m->d_conn, sizeof(int32_t) * m->nen * n_elems)) != ETP_OK) return cleanup(s);
  if ((s = dalloc(&m->d_inc_ptr, sizeof(int32_t) * (n_nodes + 1))) != ETP_OK) return cleanup(s);
  if ((s = dalloc(&m->d_inc_idx, sizeof(int32_t) * idx.size())) != ETP_OK) return cleanup(s);
  if ((s = dalloc(&m->d_fixed, n_nodes)) != ETP_OK) return cleanup(s);
  cudaStream_t st = ctx->stream;
  cudaMemcpyAsync(m->d_conn, conn, sizeof(int32_t) * m->nen * n_elems, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(m->d_inc_ptr, ptr.data(), sizeof(int32_t) * (n_nodes + 1), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(m->d_inc_idx, idx.data(), sizeof(int32_t) * idx.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(m->d_fixed, m->h_fixed.data(), n_nodes, cudaMemcpyHostToDevice, st);
  if (order == 1) {  // the element pass's lane constants, once per mesh
    if ((s = dalloc(&m->d_qtab64, sizeof(double) * 8 * 48)) != ETP_OK) return cleanup(s);
    double h[3];
    for (int d = 0; d < 3; ++d) h[d] = m->is_box ? 2.0 / m->box_h[d] : 0.0;
    if (m->is_box) k_q1_lane_table<double, true><<<1, 32, 0, st>>>(h[0], h[1], h[2], m->d_qtab64);
    else k_q1_lane_table<double, false><<<1, 32, 0, st>>>(0.0, 0.0, 0.0, m->d_qtab64);
  }
  if (!m->is_box) {
    double* d_coords = nullptr;
    int* d_err = nullptr;
    if ((s = dalloc(&d_coords, sizeof(double) * 3 * n_nodes)) != ETP_OK) return cleanup(s);
    if ((s = dalloc(&d_err, sizeof(int))) != ETP_OK) { dfree(d_coords); return cleanup(s); }
    if ((s = dalloc(&m->d_geo64, sizeof(double) * 10 * m->nq * n_elems)) != ETP_OK ||
        (s = dalloc(&m->d_geo32, sizeof(float) * 10 * m->nq * n_elems)) != ETP_OK) {
      dfree(d_coords); dfree(d_err);
      return cleanup(s);
    }
    cudaMemcpyAsync(d_coords, coords, sizeof(double) * 3 * n_nodes, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(d_err, 0, sizeof(int), st);
    const int64_t nthreads = n_elems * m->nq;
    const unsigned grid = (unsigned)((nthreads + 127) / 128);
    if (order == 1) k_geometry<1><<<grid, 128, 0, st>>>(n_elems, d_coords, m->d_conn, m->d_geo64, m->d_geo32, d_err);
    else k_geometry<2><<<grid, 128, 0, st>>>(n_elems, d_coords, m->d_conn, m->d_geo64, m->d_geo32, d_err);
    int herr = 0;
    cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    dfree(d_coords);
    dfree(d_err);
    if (e != cudaSuccess) return cleanup(fail(ETP_ERR_CUDA, cudaGetErrorString(e)));
    if (herr) return cleanup(fail(ETP_ERR_INVALID, "element with det J <= 0 in the reference configuration"));
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cleanup(fail(ETP_ERR_CUDA, cudaGetErrorString(e)));
  *out = m;
  return ETP_OK;
}

void etp_mesh_destroy(etp_mesh* m) {
  if (!m) return;
  dfree(m->d_conn); dfree(m->d_inc_ptr); dfree(m->d_inc_idx); dfree(m->d_fixed);
  dfree(m->d_geo64); dfree(m->d_geo32); dfree(m->d_escale); dfree(m->d_qtab64);
  dfree(m->d_msqrt); dfree(m->d_minvsqrt64); dfree(m->d_minvsqrt32);
  delete m;
}

etp_status etp_material_set(etp_mesh* m, int kind, const double* params, int n_params, double rho,
                            const float* elem_scale) {
  if (!m) return fail(ETP_ERR_INVALID, "null mesh");
  static const int need[5] = {2, 2, 3, 2, 4};
  if (kind < 0 || kind > 4) return fail(ETP_ERR_INVALID, "unknown material kind");
  if (!params || n_params < need[kind] || n_params > kMaxParams) return fail(ETP_ERR_INVALID, "wrong parameter count");
  if (!(rho > 0)) return fail(ETP_ERR_INVALID, "density must be positive");
  for (int i = 0; i < n_params; ++i)
    if (!isfinite(params[i])) return fail(ETP_ERR_INVALID, "non-finite material parameter");
  if (kind == MAT_YEOH && params[3] == 0.0) return fail(ETP_ERR_INVALID, "Yeoh D1 must be non-zero");
  etp_ctx* ctx = m->ctx;
  ETP_CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  m->kind = kind;
  for (int i = 0; i < kMaxParams; ++i) m->params[i] = i < n_params ? params[i] : 0.0;
  m->rho = rho;
  dfree(m->d_escale);
  if (elem_scale) {
    ETP_TRY(dalloc(&m->d_escale, sizeof(float) * m->n_elems));
    ETP_CUDA_TRY(cudaMemcpyAsync(m->d_escale, elem_scale, sizeof(float) * m->n_elems, cudaMemcpyHostToDevice, st));
  }
  dfree(m->d_msqrt); dfree(m->d_minvsqrt64); dfree(m->d_minvsqrt32);
  ETP_TRY(dalloc(&m->d_msqrt, sizeof(double) * m->nn_pad));
  ETP_TRY(dalloc(&m->d_minvsqrt64, sizeof(double) * m->nn_pad));
  ETP_TRY(dalloc(&m->d_minvsqrt32, sizeof(float) * m->nn_pad));
  double *d_coords = nullptr, *d_mc = nullptr, *d_mass = nullptr;
  int* d_err = nullptr;
  etp_status s = ETP_OK;
  if ((s = dalloc(&d_coords, sizeof(double) * 3 * m->n_nodes)) != ETP_OK ||
      (s = dalloc(&d_mc, sizeof(double) * m->nen * m->n_elems)) != ETP_OK ||
      (s = dalloc(&d_mass, sizeof(double) * m->n_nodes)) != ETP_OK || (s = dalloc(&d_err, sizeof(int))) != ETP_OK) {
    dfree(d_coords); dfree(d_mc); dfree(d_mass); dfree(d_err);
    return s;
  }
  cudaMemcpyAsync(d_coords, m->h_coords.data(), sizeof(double) * 3 * m->n_nodes, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(d_err, 0, sizeof(int), st);
  const double box_det = m->box_h[0] * m->box_h[1] * m->box_h[2] / 8.0;
  const int64_t nt = m->nen * m->n_elems;
  const unsigned grid = (unsigned)((nt + 127) / 128);
  if (m->order == 1)
    k_mass_contrib<1><<<grid, 128, 0, st>>>(m->n_elems, d_coords, m->d_conn, rho, m->is_box, box_det, d_mc, d_err);
  else
    k_mass_contrib<2><<<grid, 128, 0, st>>>(m->n_elems, d_coords, m->d_conn, rho, m->is_box, box_det, d_mc, d_err);
  k_gather_scalar<<<(unsigned)((m->n_nodes + 255) / 256), 256, 0, st>>>(m->n_nodes, m->d_inc_ptr, m->d_inc_idx, d_mc,
                                                                         d_mass);
  k_mass_finish<<<(unsigned)((m->nn_pad + 255) / 256), 256, 0, st>>>(m->n_nodes, m->nn_pad, d_mass, m->d_msqrt,
                                                                     m->d_minvsqrt64, m->d_minvsqrt32);
  m->h_mass.resize(m->n_nodes);
  int herr = 0;
  cudaMemcpyAsync(m->h_mass.data(), d_mass, sizeof(double) * m->n_nodes, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  dfree(d_coords); dfree(d_mc); dfree(d_mass); dfree(d_err);
  if (e != cudaSuccess) return fail(ETP_ERR_CUDA, cudaGetErrorString(e));
  if (herr) return fail(ETP_ERR_INVALID, "element with det J <= 0 at a node");
  for (int64_t n = 0; n < m->n_nodes; ++n)
    if (!(m->h_mass[n] > 0)) return fail(ETP_ERR_INVALID, "node with zero mass (not attached to an element)");
  m->material_ready = true;
  m->material_version += 1;
  return ETP_OK;
}

static etp_status upload_uv(etp_traj* t, const double* u, const double* v, int on_device, double* w_dst) {
  etp_mesh* m = t->mesh;
  cudaStream_t st = m->ctx->stream;
  const size_t nb = sizeof(double) * 3 * m->n_nodes;
  double *du = nullptr, *dv = nullptr;
  if (on_device) {
    du = (double*)u;
    dv = (double*)v;
  } else {
    // stage through the combine scratch (the Arnoldi work vector is large enough)
    ETP_TRY(dalloc(&du, nb));
    etp_status s = dalloc(&dv, nb);
    if (s != ETP_OK) { dfree(du); return s; }
    cudaMemcpyAsync(du, u, nb, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dv, v, nb, cudaMemcpyHostToDevice, st);
  }
  k_state_from_uv<<<(unsigned)((m->nn_pad + 255) / 256), 256, 0, st>>>(m->n_nodes, m->nn_pad, du, dv, m->d_msqrt,
                                                                       m->d_fixed, w_dst);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && t->has_load) {  // augmented entry of a loaded state
    static const double one = 1.0;
    e = cudaMemcpyAsync(w_dst + 3 * m->nn_pad - 1, &one, sizeof(double), cudaMemcpyHostToDevice, st);
  }
  if (!on_device) {
    cudaStreamSynchronize(st);
    dfree(du);
    dfree(dv);
  }
  if (e != cudaSuccess) return fail(ETP_ERR_CUDA, cudaGetErrorString(e));
  t->hist_count = 0;
  for (bool& v : t->fz_valid) v = false;
  return ETP_OK;
}

}  // extern "C"

namespace etp {

// Device bytes held by a mesh (connectivity, incidence, Dirichlet bits,
// general geometry, element scale, mass factors).
size_t mesh_device_bytes(const etp_mesh* m) {
  size_t b = 4 * (size_t)m->nen * m->n_elems * 2 + 4 * (size_t)(m->n_nodes + 1) + (size_t)m->n_nodes;
  if (m->d_geo64) b += (8 + 4) * 10 * (size_t)m->nq * m->n_elems;
  if (m->d_escale) b += 4 * (size_t)m->n_elems;
  if (m->d_msqrt) b += (8 + 8 + 4) * (size_t)m->nn_pad;
  return b;
}

// Device bytes etp_state_init allocates for one trajectory (the same list of
// buffers, in the same order).
size_t traj_device_bytes(const etp_mesh* m, int precision, int m_cap) {
  const size_t s = precision == ETP_PREC_FP64 ? 8 : 4;
  const size_t L = 6 * (size_t)m->nn_pad;
  const size_t wcand = (size_t)std::min(kMaxCand, m_cap);
  const size_t max_grid = (size_t)std::max(kCgsMaxBlocksPerSm, 4) * m->ctx->num_sms;
  size_t b = 8 * L + 8 * L + s * L * (m_cap + 1) + s * L + s * 3 * m->nen * (size_t)m->n_elems;
  b += 3 * s * 3 * (size_t)m->nn_pad;
  if (m->kind != MAT_LINEAR) b += 3 * frozen_buffer_bytes(m, s);
  b += sizeof(double) * (m_cap + 1) * (size_t)m_cap + sizeof(double) * COEF_NUM * COEF_STRIDE;
  b += std::max(sizeof(double) * max_grid * (kMaxCap + 1), pk_partials_bytes((int64_t)L, m_cap, precision)) +
       sizeof(unsigned int) * 16 + sizeof(KState);
  b += sizeof(double) * (kMaxCap + 1) + sizeof(double) * wcand * EXPM_NMAT * m_cap * (size_t)m_cap + 4096;
  return b;
}

}  // namespace etp

extern "C" {

etp_status etp_traj_footprint(const etp_mesh* m, int precision, int m_cap, size_t* traj_bytes, size_t* mesh_bytes) {
  if (!m) return fail(ETP_ERR_INVALID, "null mesh");
  if (precision != ETP_PREC_FP64 && precision != ETP_PREC_MIXED) return fail(ETP_ERR_INVALID, "unknown precision");
  if (m_cap < 1 || m_cap > kMaxCap) return fail(ETP_ERR_INVALID, "m_cap must be in 1..256");
  if (traj_bytes) *traj_bytes = traj_device_bytes(m, precision, m_cap);
  if (mesh_bytes) *mesh_bytes = mesh_device_bytes(m);
  return ETP_OK;
}

etp_status etp_state_init(etp_mesh* m, const double* u0, const double* v0, int on_device, int precision,
                          int m_cap, etp_traj** out) {
  if (!m || !out || !u0 || !v0) return fail(ETP_ERR_INVALID, "null argument");
  *out = nullptr;
  if (!m->material_ready) return fail(ETP_ERR_INVALID, "etp_material_set must precede etp_state_init");
  if (precision != ETP_PREC_FP64 && precision != ETP_PREC_MIXED) return fail(ETP_ERR_INVALID, "unknown precision");
  if (m_cap < 1 || m_cap > kMaxCap) return fail(ETP_ERR_INVALID, "m_cap must be in 1..256");
  etp_ctx* ctx = m->ctx;
  ETP_CUDA_TRY(cudaSetDevice(ctx->device));
  etp_traj* t = new etp_traj();
  t->mesh = m;
  t->prec = precision;
  t->m_cap = m_cap;
  t->L = 6 * m->nn_pad;
  const size_t s = precision == ETP_PREC_FP64 ? 8 : 4;
  const int64_t L = t->L;
  const int wcand = std::min(kMaxCand, m_cap);
  etp_status st = ETP_OK;
  auto bail = [&](etp_status x) { etp_traj_destroy(t); return x; };
  t->device_bytes = traj_device_bytes(m, precision, m_cap);
  if ((st = dalloc(&t->d_w, 8 * L)) != ETP_OK) return bail(st);
  if ((st = dalloc(&t->d_wtmp, 8 * L)) != ETP_OK) return bail(st);
  if ((st = dalloc((char**)&t->d_V, s * L * (m_cap + 1))) != ETP_OK) return bail(st);
  if ((st = dalloc((char**)&t->d_z, s * L)) != ETP_OK) return bail(st);
  if ((st = dalloc((char**)&t->d_Ye, s * 3 * m->nen * m->n_elems)) != ETP_OK) return bail(st);
  for (int k = 0; k < 3; ++k)
    if ((st = dalloc((char**)&t->d_hist[k], s * 3 * m->nn_pad)) != ETP_OK) return bail(st);
  if (m->kind != MAT_LINEAR) {  // stored frozen coefficients, one set per midpoint-history slot
    const size_t fzb = frozen_buffer_bytes(m, s);
    for (auto& b : t->d_fz)
      if ((st = dalloc((char**)&b, fzb)) != ETP_OK) return bail(st);
    t->fz_bytes = fzb;
    t->fz_version = m->material_version;
  }
  if ((st = dalloc(&t->d_H, sizeof(double) * (m_cap + 1) * m_cap)) != ETP_OK) return bail(st);
  if ((st = dalloc(&t->d_coef, sizeof(double) * COEF_NUM * COEF_STRIDE)) != ETP_OK) return bail(st);
  const int max_grid = std::max(kCgsMaxBlocksPerSm, 4) * ctx->num_sms;
  const size_t part_bytes =
      std::max(sizeof(double) * (size_t)max_grid * (kMaxCap + 1), pk_partials_bytes(L, m_cap, precision));
  if ((st = dalloc(&t->d_partials, part_bytes)) != ETP_OK) return bail(st);
  if ((st = dalloc(&t->d_counter, sizeof(unsigned int) * 16)) != ETP_OK) return bail(st);
  if ((st = dalloc(&t->d_ks, sizeof(KState))) != ETP_OK) return bail(st);
  if ((st = dalloc(&t->d_y, sizeof(double) * (kMaxCap + 1))) != ETP_OK) return bail(st);
  if ((st = dalloc(&t->d_expm_ws, sizeof(double) * (size_t)wcand * EXPM_NMAT * m_cap * m_cap)) != ETP_OK)
    return bail(st);
  t->expm_ws_cand = wcand;
  if ((st = dalloc(&t->d_red, 4096)) != ETP_OK) return bail(st);
  if (cudaMallocHost((void**)&t->h_ks, 4096) != cudaSuccess) {
    t->h_ks = nullptr;
    return bail(fail(ETP_ERR_OOM, "cudaMallocHost failed"));
  }
  cudaStream_t cs = ctx->stream;
  cudaMemsetAsync(t->d_counter, 0, sizeof(unsigned int) * 16, cs);
  cudaMemsetAsync(t->d_ks, 0, sizeof(KState), cs);
  cudaMemsetAsync(t->d_coef, 0, sizeof(double) * COEF_NUM * COEF_STRIDE, cs);
  cudaMemsetAsync(t->d_H, 0, sizeof(double) * (m_cap + 1) * m_cap, cs);
  cudaMemsetAsync(t->d_z, 0, s * L, cs);
  if ((st = upload_uv(t, u0, v0, on_device, t->d_w)) != ETP_OK) return bail(st);
  cudaError_t e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return bail(fail(ETP_ERR_CUDA, cudaGetErrorString(e)));
  *out = t;
  return ETP_OK;
}

void etp_traj_destroy(etp_traj* t) {
  if (!t) return;
  dfree(t->d_w); dfree(t->d_wtmp); dfree(t->d_V); dfree(t->d_z); dfree(t->d_Ye);
  for (auto& h : t->d_hist) dfree(h);
  for (auto& b : t->d_fz) dfree(b);
  dfree(t->d_pbar); dfree(t->d_pbar64);
  dfree(t->d_H); dfree(t->d_coef); dfree(t->d_partials); dfree(t->d_counter); dfree(t->d_ks);
  dfree(t->d_y); dfree(t->d_expm_ws); dfree(t->d_red);
  dfree(t->d_nm);
  if (t->nm_exec) cudaGraphExecDestroy((cudaGraphExec_t)t->nm_exec);
  if (t->h_ks) cudaFreeHost(t->h_ks);
  delete t;
}

}  // extern "C"

namespace etp {

static etp_status extract_u(etp_traj* t, const double* w, void* dst) {
  etp_mesh* m = t->mesh;
  cudaStream_t st = m->ctx->stream;
  const unsigned grid = (unsigned)((3 * m->nn_pad + 255) / 256);
  ProfScope ps(m->ctx, KC_OTHER, 3.0 * m->nn_pad * (8.0 + (t->prec == ETP_PREC_FP64 ? 8 : 4)));
  if (t->prec == ETP_PREC_FP64)
    k_extract_u<double><<<grid, 256, 0, st>>>(m->nn_pad, w, m->d_minvsqrt64, (double*)dst);
  else
    k_extract_u<float><<<grid, 256, 0, st>>>(m->nn_pad, w, m->d_minvsqrt32, (float*)dst);
  ETP_CUDA_TRY(cudaGetLastError());
  return ETP_OK;
}

// Argument checks shared by the step entry points.
etp_status check_step_args(const etp_traj* t, double dt, double tol) {
  (void)t;
  if (!(dt > 0) || !isfinite(dt)) return fail(ETP_ERR_INVALID, "dt must be positive and finite");
  if (!(tol >= 0) || !isfinite(tol)) return fail(ETP_ERR_INVALID, "tol must be non-negative");
  return ETP_OK;
}

// Predictor operator of a nonlinear step (Section 4.2): the extrapolation of
// the midpoint history (u_0 alone at the first step, the newest midpoint at
// the second); *slot_new is the history slot that receives the new midpoint,
// the one that is neither of the two kept states (its stored coefficients, if
// any, become stale as the predictor writes it).
etp_status predictor_setup(etp_traj* t, FrozenSet* fp_out, int* slot_new) {
  FrozenSet fp;
  if (t->hist_count == 0) {
    const int slot_u0 = (t->hist_newest + 2) % 3;  // unused while the history is empty
    t->fz_valid[slot_u0] = false;
    ETP_TRY(extract_u(t, t->d_w, t->d_hist[slot_u0]));
    fp.count = 1;
    fp.u[0] = t->d_hist[slot_u0];
    fp.slot[0] = slot_u0;
  } else if (t->hist_count == 1) {
    fp.count = 1;
    fp.u[0] = t->d_hist[t->hist_newest];
    fp.slot[0] = t->hist_newest;
  } else {
    fp.count = 2;
    fp.u[0] = t->d_hist[t->hist_newest];
    fp.u[1] = t->d_hist[(t->hist_newest + 2) % 3];
    fp.slot[0] = t->hist_newest;
    fp.slot[1] = (t->hist_newest + 2) % 3;
    fp.c[0] = 1.75;
    fp.c[1] = -0.75;
  }
  *slot_new = (t->hist_newest + 1) % 3;
  t->fz_valid[*slot_new] = false;
  *fp_out = fp;
  return ETP_OK;
}

// Corrector operator: the midpoint state the predictor wrote.
FrozenSet corrector_frozen(const etp_traj* t, int slot_new) {
  FrozenSet fc;
  fc.count = 1;
  fc.u[0] = t->d_hist[slot_new];
  fc.slot[0] = slot_new;
  return fc;
}

// Commit a step whose corrector (or linear) solve gave rc: history, state swap.
etp_status step_commit(etp_traj* t, const SolveResult& rc, int slot_new, etp_step_info* loc, etp_step_info* info) {
  if (slot_new >= 0 && rc.converged) {
    t->hist_newest = slot_new;
    t->hist_count = std::min(t->hist_count + 1, 2);
  }
  loc->m_corr = rc.m;
  loc->eps_corr = rc.eps;
  loc->beta = rc.beta;
  loc->converged = rc.converged ? 1 : 0;
  if (info) *info = *loc;
  if (!rc.converged) return fail(ETP_ERR_NOT_CONVERGED, "Krylov solve did not reach tol at m_cap");
  t->nm_valid = false;  // the Newmark path recomputes its acceleration from the new state
  std::swap(t->d_w, t->d_wtmp);
  t->steps++;
  return ETP_OK;
}


}  // namespace etp

extern "C" {

etp_status etp_step_ex(etp_traj* t, double dt, double tol, int m_fixed_pred, int m_fixed_corr,
                       etp_step_info* info) {
  if (!t) return fail(ETP_ERR_INVALID, "null trajectory");
  ETP_TRY(check_step_args(t, dt, tol));
  if (m_fixed_pred < 0 || m_fixed_corr < 0 || m_fixed_pred > t->m_cap || m_fixed_corr > t->m_cap)
    return fail(ETP_ERR_INVALID, "m_fixed must be in 0..m_cap");
  etp_mesh* m = t->mesh;
  ETP_CUDA_TRY(cudaSetDevice(m->ctx->device));
  etp_step_info loc{};
  SolveResult rp, rc;
  int slot_new = -1;
  if (m->kind == MAT_LINEAR) {
    FrozenSet fz;
    ETP_TRY(krylov_solve(t, dt, t->d_w, t->d_wtmp, fz, tol, m_fixed_corr, nullptr, &rc, 0));
  } else {
    FrozenSet fp;
    ETP_TRY(predictor_setup(t, &fp, &slot_new));
    ETP_TRY(krylov_solve(t, 0.5 * dt, t->d_w, t->d_wtmp, fp, tol, m_fixed_pred, t->d_hist[slot_new], &rp, 1));
    if (!rp.converged) {
      loc.m_pred = rp.m; loc.eps_pred = rp.eps; loc.beta = rp.beta;
      if (info) *info = loc;
      return fail(ETP_ERR_NOT_CONVERGED, "predictor Krylov solve did not reach tol at m_cap");
    }
    const FrozenSet fc = corrector_frozen(t, slot_new);
    ETP_TRY(krylov_solve(t, dt, t->d_w, t->d_wtmp, fc, tol, m_fixed_corr, nullptr, &rc, 0));
    loc.m_pred = rp.m;
    loc.eps_pred = rp.eps;
  }
  return step_commit(t, rc, slot_new, &loc, info);
}

etp_status etp_krylov_method(etp_traj* t, int method) {
  if (!t) return fail(ETP_ERR_INVALID, "null trajectory");
  if (method != ETP_KRYLOV_ARNOLDI && method != ETP_KRYLOV_LANCZOS_ENERGY)
    return fail(ETP_ERR_INVALID, "unknown Krylov method");
  if (method == ETP_KRYLOV_LANCZOS_ENERGY && t->mesh->kind != MAT_LINEAR)
    return fail(ETP_ERR_INVALID, "the energy Lanczos process needs a linear material");
  t->krylov = method;
  t->m_hint[0] = t->m_hint[1] = 0;
  return ETP_OK;
}

etp_status etp_step(etp_traj* t, double dt, double tol, int m_fixed, int* m_out, double* err_out) {
  etp_step_info info{};
  etp_status s = etp_step_ex(t, dt, tol, m_fixed, m_fixed, &info);
  if (m_out) *m_out = info.m_corr;
  if (err_out) *err_out = info.eps_corr;
  return s;
}

etp_status etp_energy(etp_traj* t, double* total, double* kinetic, double* potential) {
  if (!t) return fail(ETP_ERR_INVALID, "null trajectory");
  etp_mesh* m = t->mesh;
  etp_ctx* ctx = m->ctx;
  ETP_CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  double* red = t->d_red;
  const int grid = 2 * ctx->num_sms;
  k_sumsq<<<grid, 256, 0, st>>>(3 * m->nn_pad, t->d_w + 3 * m->nn_pad, t->d_partials, t->d_counter, red);
  Prm8 prm;
  for (int i = 0; i < kMaxParams; ++i) prm.v[i] = m->params[i];
  const double hx = m->box_h[0], hy = m->box_h[1], hz = m->box_h[2];
  double* part2 = t->d_partials + 4 * ctx->num_sms;
  if (m->order == 1)
    k_energy_elem<1><<<grid, 128, 0, st>>>(m->n_elems, m->nn_pad, m->d_conn, t->d_w, m->d_minvsqrt64, m->d_geo64,
                                           m->is_box, hx, hy, hz, m->d_escale, m->kind, prm, part2);
  else
    k_energy_elem<2><<<grid, 128, 0, st>>>(m->n_elems, m->nn_pad, m->d_conn, t->d_w, m->d_minvsqrt64, m->d_geo64,
                                           m->is_box, hx, hy, hz, m->d_escale, m->kind, prm, part2);
  k_sum_partials<<<1, 32, 0, st>>>(grid, part2, red + 1);
  if (t->has_load)  // potential of the constant load: -P^T u = -P_bar^T u_bar
    k_dot64<<<grid, 256, 0, st>>>(3 * m->nn_pad, t->d_w, t->d_pbar64, t->d_partials + 8 * ctx->num_sms,
                                  t->d_counter, red + 2);
  ETP_CUDA_TRY(cudaGetLastError());
  double h[3] = {0.0, 0.0, 0.0};
  ETP_CUDA_TRY(cudaMemcpyAsync(h, red, (t->has_load ? 3 : 2) * sizeof(double), cudaMemcpyDeviceToHost, st));
  ETP_CUDA_TRY(cudaStreamSynchronize(st));
  const double ke = 0.5 * h[0], pe = h[1] - h[2];
  if (kinetic) *kinetic = ke;
  if (potential) *potential = pe;
  if (total) *total = ke + pe;
  return ETP_OK;
}

etp_status etp_state_get(etp_traj* t, double* u_out, double* v_out, int on_device) {
  if (!t) return fail(ETP_ERR_INVALID, "null trajectory");
  etp_mesh* m = t->mesh;
  cudaStream_t st = m->ctx->stream;
  ETP_CUDA_TRY(cudaSetDevice(m->ctx->device));
  const size_t nb = sizeof(double) * 3 * m->n_nodes;
  double *du = u_out, *dv = v_out;
  if (!on_device) {
    // reuse the scratch state buffer (2 x 3*nn_pad doubles fit in L doubles)
    du = u_out ? t->d_wtmp : nullptr;
    dv = v_out ? t->d_wtmp + 3 * m->nn_pad : nullptr;
  }
  k_uv_from_state<<<(unsigned)((m->n_nodes + 255) / 256), 256, 0, st>>>(m->n_nodes, m->nn_pad, t->d_w,
                                                                        m->d_minvsqrt64, du, dv);
  ETP_CUDA_TRY(cudaGetLastError());
  if (!on_device) {
    if (u_out) ETP_CUDA_TRY(cudaMemcpyAsync(u_out, du, nb, cudaMemcpyDeviceToHost, st));
    if (v_out) ETP_CUDA_TRY(cudaMemcpyAsync(v_out, dv, nb, cudaMemcpyDeviceToHost, st));
  }
  ETP_CUDA_TRY(cudaStreamSynchronize(st));
  return ETP_OK;
}

etp_status etp_state_set(etp_traj* t, const double* u, const double* v, int on_device) {
  if (!t || !u || !v) return fail(ETP_ERR_INVALID, "null argument");
  t->nm_valid = false;
  ETP_CUDA_TRY(cudaSetDevice(t->mesh->ctx->device));
  if (on_device) return upload_uv(t, u, v, 1, t->d_w);
  // host input: stage in the scratch state buffer (needs 2 x 3*n_nodes doubles <= L)
  etp_mesh* m = t->mesh;
  cudaStream_t st = m->ctx->stream;
  const size_t nb = sizeof(double) * 3 * m->n_nodes;
  double* du = t->d_wtmp;
  double* dv = t->d_wtmp + 3 * m->nn_pad;
  ETP_CUDA_TRY(cudaMemcpyAsync(du, u, nb, cudaMemcpyHostToDevice, st));
  ETP_CUDA_TRY(cudaMemcpyAsync(dv, v, nb, cudaMemcpyHostToDevice, st));
  return upload_uv(t, du, dv, 1, t->d_w);
}

etp_status etp_state_upload(etp_traj* t, const double* u, const double* v, int on_device) {
  if (!t) return fail(ETP_ERR_INVALID, "null trajectory");
  t->nm_valid = false;
  const int hc = t->hist_count;
  bool valid[3];
  for (int k = 0; k < 3; ++k) valid[k] = t->fz_valid[k];
  const etp_status s = etp_state_set(t, u, v, on_device);
  if (s == ETP_OK) {  // same trajectory: the midpoint history (and its coefficients) still apply
    t->hist_count = hc;
    for (int k = 0; k < 3; ++k) t->fz_valid[k] = valid[k];
  }
  return s;
}

int64_t etp_traj_steps(const etp_traj* t) { return t ? t->steps : -1; }

static const uint64_t kMagic = 0x3130505445ull;  // "ETP01"

etp_status etp_load_set(etp_traj* t, const double* P) {
  if (!t) return fail(ETP_ERR_INVALID, "null trajectory");
  t->nm_valid = false;
  etp_mesh* m = t->mesh;
  cudaStream_t st = m->ctx->stream;
  ETP_CUDA_TRY(cudaSetDevice(m->ctx->device));
  const int64_t nn = m->n_nodes, np = m->nn_pad;
  const int64_t xi = 3 * np - 1;
  if (!P) {  // remove the load: plain state again
    ETP_CUDA_TRY(cudaStreamSynchronize(st));
    dfree(t->d_pbar);
    dfree(t->d_pbar64);
    if (t->has_load) t->device_bytes -= (size_t)3 * np * (8 + (t->prec == ETP_PREC_FP64 ? 8 : 4));
    t->has_load = false;
    ETP_CUDA_TRY(cudaMemsetAsync(t->d_w + xi, 0, sizeof(double), st));
    return ETP_OK;
  }
  // P_bar = M^{-1/2} P on the free DOFs, zero on fixed DOFs and padding
  std::vector<double> pb(3 * np, 0.0);
  for (int64_t n = 0; n < nn; ++n)
    for (int c = 0; c < 3; ++c) {
      const double f = P[3 * n + c];
      if (!isfinite(f)) return fail(ETP_ERR_INVALID, "non-finite load");
      if (!(m->h_fixed[n] & (1 << c))) pb[c * np + n] = f / sqrt(m->h_mass[n]);
    }
  const size_t s = t->prec == ETP_PREC_FP64 ? 8 : 4;
  if (!t->has_load) {
    ETP_TRY(dalloc(&t->d_pbar64, sizeof(double) * 3 * np));
    etp_status e = dalloc((char**)&t->d_pbar, s * 3 * np);
    if (e != ETP_OK) { dfree(t->d_pbar64); return e; }
    t->device_bytes += (size_t)3 * np * (8 + s);
  }
  ETP_CUDA_TRY(cudaMemcpyAsync(t->d_pbar64, pb.data(), sizeof(double) * 3 * np, cudaMemcpyHostToDevice, st));
  if (s == 8) {
    ETP_CUDA_TRY(cudaMemcpyAsync(t->d_pbar, pb.data(), sizeof(double) * 3 * np, cudaMemcpyHostToDevice, st));
  } else {
    std::vector<float> pf(pb.begin(), pb.end());
    ETP_CUDA_TRY(cudaMemcpyAsync(t->d_pbar, pf.data(), sizeof(float) * 3 * np, cudaMemcpyHostToDevice, st));
    ETP_CUDA_TRY(cudaStreamSynchronize(st));  // pf leaves scope
  }
  static const double one = 1.0;
  ETP_CUDA_TRY(cudaMemcpyAsync(t->d_w + xi, &one, sizeof(double), cudaMemcpyHostToDevice, st));
  ETP_CUDA_TRY(cudaStreamSynchronize(st));
  t->has_load = true;
  return ETP_OK;
}

etp_status etp_state_save(etp_traj* t, const char* path) {
  if (!t || !path) return fail(ETP_ERR_INVALID, "null argument");
  etp_mesh* m = t->mesh;
  cudaStream_t st = m->ctx->stream;
  const size_t s = t->prec == ETP_PREC_FP64 ? 8 : 4;
  std::vector<double> w(t->L);
  std::vector<char> hist(3 * s * 3 * m->nn_pad);
  ETP_CUDA_TRY(cudaMemcpyAsync(w.data(), t->d_w, 8 * t->L, cudaMemcpyDeviceToHost, st));
  for (int k = 0; k < 3; ++k)
    ETP_CUDA_TRY(cudaMemcpyAsync(hist.data() + k * s * 3 * m->nn_pad, t->d_hist[k], s * 3 * m->nn_pad,
                                 cudaMemcpyDeviceToHost, st));
  ETP_CUDA_TRY(cudaStreamSynchronize(st));
  FILE* f = fopen(path, "wb");
  if (!f) return fail(ETP_ERR_IO, std::string("cannot open ") + path);
  int64_t hdr[6] = {(int64_t)kMagic, t->L, (int64_t)t->prec, t->steps, t->hist_count, t->hist_newest};
  bool ok = fwrite(hdr, sizeof(hdr), 1, f) == 1 && fwrite(w.data(), 8, w.size(), f) == w.size() &&
            fwrite(hist.data(), 1, hist.size(), f) == hist.size();
  ok = (fclose(f) == 0) && ok;
  if (!ok) return fail(ETP_ERR_IO, "checkpoint write failed");
  return ETP_OK;
}

etp_status etp_state_load(etp_traj* t, const char* path) {
  if (!t || !path) return fail(ETP_ERR_INVALID, "null argument");
  t->nm_valid = false;
  etp_mesh* m = t->mesh;
  cudaStream_t st = m->ctx->stream;
  const size_t s = t->prec == ETP_PREC_FP64 ? 8 : 4;
  FILE* f = fopen(path, "rb");
  if (!f) return fail(ETP_ERR_IO, std::string("cannot open ") + path);
  int64_t hdr[6];
  std::vector<double> w(t->L);
  std::vector<char> hist(3 * s * 3 * m->nn_pad);
  bool ok = fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == (int64_t)kMagic && hdr[1] == t->L &&
            hdr[2] == t->prec && fread(w.data(), 8, w.size(), f) == w.size() &&
            fread(hist.data(), 1, hist.size(), f) == hist.size();
  fclose(f);
  if (!ok) return fail(ETP_ERR_IO, "checkpoint does not match this trajectory");
  ETP_CUDA_TRY(cudaMemcpyAsync(t->d_w, w.data(), 8 * t->L, cudaMemcpyHostToDevice, st));
  for (int k = 0; k < 3; ++k)
    ETP_CUDA_TRY(cudaMemcpyAsync(t->d_hist[k], hist.data() + k * s * 3 * m->nn_pad, s * 3 * m->nn_pad,
                                 cudaMemcpyHostToDevice, st));
  ETP_CUDA_TRY(cudaStreamSynchronize(st));
  t->steps = hdr[3];
  t->hist_count = (int)hdr[4];
  t->hist_newest = (int)hdr[5];
  for (bool& v : t->fz_valid) v = false;  // the history slots were rewritten
  return ETP_OK;
}

}  // extern "C"

template <typename T>
static etp_status apply_hbar_impl(etp_mesh* m, const double* x, const double* ustar, double* y,
                                  int kind_override = -1) {
  etp_ctx* ctx = m->ctx;
  cudaStream_t st = ctx->stream;
  const int64_t nn = m->n_nodes, np = m->nn_pad;
  std::vector<T> hx(6 * np, T(0)), hu(3 * np, T(0));
  for (int64_t n = 0; n < nn; ++n)
    for (int c = 0; c < 3; ++c) {
      hx[c * np + n] = (T)x[3 * n + c];
      if (ustar) hu[c * np + n] = (T)ustar[3 * n + c];
    }
  T *dx = nullptr, *du = nullptr, *dYe = nullptr, *dz = nullptr;
  double* dscale = nullptr;
  int* derr = nullptr;
  etp_status s = ETP_OK;
  auto cleanup = [&]() { dfree(dx); dfree(du); dfree(dYe); dfree(dz); dfree(dscale); dfree(derr); };
  if ((s = dalloc(&dx, sizeof(T) * 6 * np)) != ETP_OK || (s = dalloc(&du, sizeof(T) * 3 * np)) != ETP_OK ||
      (s = dalloc(&dYe, sizeof(T) * 3 * m->nen * m->n_elems)) != ETP_OK ||
      (s = dalloc(&dz, sizeof(T) * 6 * np)) != ETP_OK || (s = dalloc(&dscale, sizeof(double))) != ETP_OK ||
      (s = dalloc(&derr, sizeof(int))) != ETP_OK) {
    cleanup();
    return s;
  }
  // the library applies -H_bar to M^{1/2}-scaled vectors; x here is already in that space
  const double one = 1.0;
  cudaMemcpyAsync(dx, hx.data(), sizeof(T) * 6 * np, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(du, hu.data(), sizeof(T) * 3 * np, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dscale, &one, sizeof(double), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(derr, 0, sizeof(int), st);
  FrozenSet fz;
  fz.count = (m->kind == MAT_LINEAR) ? 0 : 1;
  fz.u[0] = du;
  void* dfz[2] = {nullptr, nullptr};
  if (fz.count > 0 && (s = dalloc((char**)&dfz[0], frozen_buffer_bytes(m, sizeof(T)))) != ETP_OK) {
    cleanup();
    return s;
  }
  s = build_frozen<T>(m, fz, dfz, derr);
  if (s == ETP_OK) s = apply_A<T>(m, dx, dscale, fz, dYe, dz, nullptr, nullptr, true, kind_override);
  std::vector<T> hz(6 * np);
  int herr = 0;
  if (s == ETP_OK) {
    cudaMemcpyAsync(hz.data(), dz, sizeof(T) * 6 * np, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = fail(ETP_ERR_CUDA, cudaGetErrorString(e));
  }
  dfree(dfz[0]);
  cleanup();
  if (s != ETP_OK) return s;
  if (herr) return fail(ETP_ERR_INVERTED_ELEMENT, "det F <= 0 at a Gauss point of u*");
  for (int64_t n = 0; n < nn; ++n)
    for (int c = 0; c < 3; ++c) y[3 * n + c] = -(double)hz[(3 + c) * np + n];
  return ETP_OK;
}

extern "C" {

etp_status etp_apply_hbar(etp_mesh* m, int precision, const double* x, const double* ustar, double* y) {
  if (!m || !x || !y) return fail(ETP_ERR_INVALID, "null argument");
  if (!m->material_ready) return fail(ETP_ERR_INVALID, "material not set");
  ETP_CUDA_TRY(cudaSetDevice(m->ctx->device));
  if (precision == ETP_PREC_FP64) return apply_hbar_impl<double>(m, x, ustar, y);
  if (precision == ETP_PREC_MIXED) return apply_hbar_impl<float>(m, x, ustar, y);
  return fail(ETP_ERR_INVALID, "unknown precision");
}

etp_status etp_apply_tangent(etp_mesh* m, const double* x, const double* u, double* y) {
  if (!m || !x || !u || !y) return fail(ETP_ERR_INVALID, "null argument");
  if (!m->material_ready) return fail(ETP_ERR_INVALID, "material not set");
  const int tk = tangent_kind(m->kind);
  if (tk < 0) return fail(ETP_ERR_INVALID, "no consistent tangent for this material");
  ETP_CUDA_TRY(cudaSetDevice(m->ctx->device));
  return apply_hbar_impl<double>(m, x, u, y, tk);
}

etp_status etp_expm_e1(etp_ctx* ctx, int n, const double* H, double tau, double* y) {
  if (!ctx || !H || !y) return fail(ETP_ERR_INVALID, "null argument");
  if (n < 1 || n > kMaxCap) return fail(ETP_ERR_INVALID, "n must be in 1..256");
  ETP_CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const size_t need = sizeof(double) * ((size_t)EXPM_NMAT * n * n + (size_t)n * n + n) + 64;
  if (ctx->expm_ws_bytes < need) {
    dfree(ctx->expm_ws);
    ctx->expm_ws_bytes = 0;
    ETP_TRY(dalloc(&ctx->expm_ws, need));
    ctx->expm_ws_bytes = need;
  }
  double* ws = ctx->expm_ws;
  double* dH = ws + (size_t)EXPM_NMAT * n * n;
  double* dy = dH + (size_t)n * n;
  int* ds = (int*)(dy + n);
  ETP_CUDA_TRY(cudaMemcpyAsync(dH, H, sizeof(double) * n * n, cudaMemcpyHostToDevice, st));
  int hs[4];
  ETP_TRY(run_expm_window(ctx, dH, n, n, n, tau, ws, n, ds, nullptr, hs));
  ExpmParams p{};
  p.H = dH; p.ldH = n; p.j0 = n; p.ncand = 1; p.tau = tau; p.ws = ws; p.ld = n; p.s_arr = ds;
  k_expm_first_column<<<1, 128, 0, st>>>(p, dy);
  ETP_CUDA_TRY(cudaGetLastError());
  ETP_CUDA_TRY(cudaMemcpyAsync(y, dy, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  ETP_CUDA_TRY(cudaStreamSynchronize(st));
  return ETP_OK;
}

etp_status etp_last_hessenberg(etp_traj* t, int* m_out, double* H) {
  if (!t || !m_out) return fail(ETP_ERR_INVALID, "null argument");
  const int m = t->last_m;
  *m_out = m;
  if (!H || m <= 0) return ETP_OK;
  std::vector<double> full((size_t)(t->m_cap + 1) * t->m_cap);
  ETP_CUDA_TRY(cudaMemcpy(full.data(), t->d_H, sizeof(double) * full.size(), cudaMemcpyDeviceToHost));
  for (int c = 0; c < m; ++c)
    for (int r = 0; r <= m; ++r) H[r + (size_t)c * (m + 1)] = full[r + (size_t)c * (t->m_cap + 1)];
  return ETP_OK;
}

etp_status etp_profile_enable(etp_ctx* ctx, int enable) {
  if (!ctx) return fail(ETP_ERR_INVALID, "null context");
  ctx->profiling = enable != 0;
  return ETP_OK;
}

etp_status etp_profile_read(etp_ctx* ctx, int64_t* launches, double* ms, double* bytes, double* flops) {
  if (!ctx) return fail(ETP_ERR_INVALID, "null context");
  ETP_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  for (auto& r : ctx->records) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.start, r.stop) == cudaSuccess) {
      ctx->prof_ms[r.cls] += t;
      ctx->prof_launches[r.cls] += 1;
      ctx->prof_bytes[r.cls] += r.bytes;
      ctx->prof_flops[r.cls] += r.flops;
    }
    ctx->event_pool.push_back(r.start);
    ctx->event_pool.push_back(r.stop);
  }
  ctx->records.clear();
  for (int k = 0; k < ETP_NUM_KERNEL_CLASSES; ++k) {
    if (launches) launches[k] = ctx->prof_launches[k];
    if (ms) ms[k] = ctx->prof_ms[k];
    if (bytes) bytes[k] = ctx->prof_bytes[k];
    if (flops) flops[k] = ctx->prof_flops[k];
  }
  return ETP_OK;
}

etp_status etp_profile_reset(etp_ctx* ctx) {
  if (!ctx) return fail(ETP_ERR_INVALID, "null context");
  int64_t l[ETP_NUM_KERNEL_CLASSES];
  etp_profile_read(ctx, l, nullptr, nullptr, nullptr);
  for (int k = 0; k < ETP_NUM_KERNEL_CLASSES; ++k) {
    ctx->prof_launches[k] = 0;
    ctx->prof_ms[k] = 0;
    ctx->prof_bytes[k] = 0;
    ctx->prof_flops[k] = 0;
  }
  return ETP_OK;
}

int64_t etp_launch_count(const etp_ctx* ctx) { return ctx ? ctx->launches.load() : 0; }

}  // extern "C"
