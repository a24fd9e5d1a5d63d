// Ragged batched time steps: the Krylov solves (Section 4.3) of several
// trajectories -- each its own mesh, size, material, dt and tolerance --
// advance in lockstep, one Arnoldi step per round, and every round issues ONE
// element-pass launch per (order, precision, material, geometry, frozen-state
// count) class and ONE persistent Arnoldi-step launch per precision for all of
// them, instead of one launch pair per trajectory. The a-priori checks of the
// trajectories that reach a check point in a round share two host
// synchronisations. Trajectories leave the lockstep as their solves select m.
//
// Every kernel computes a trajectory's values exactly as its single launch
// does (element terms are per element; the persistent step's sums are per
// tile and summed in tile order; the small exponential is per candidate size),
// so a trajectory gives the same bits stepped alone (etp_step) or in any
// batch.
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "arnoldi_pk.cuh"
#include "etp_host.cuh"
#include "expm_kernels.cuh"
#include "krylov_kernels.cuh"

namespace etp {

template <typename T>
PkParams<T> make_pk_params(etp_traj* t, int j, const T* pbar);

namespace {

// One Krylov solve taking part in a lockstep round.
struct BSolve {
  etp_traj* t = nullptr;
  double tau = 0.0, tol = 0.0;
  const double* w_in = nullptr;
  double* w_out = nullptr;
  FrozenSet fz, fzb;
  void* ustar_out = nullptr;
  int kind = 0;  // 0: corrector or linear, 1: predictor
  int cap = 0, done = 0, win_start = 1, next_check = 0, W = 2;
  bool active = true;
  etp_status st = ETP_OK;
  SolveResult res;
};

// Arnoldi steps between checks after the first one (as the single solve).
int check_window(const etp_traj* t) {
  if (t->L >= (int64_t)4 << 20) return 1;
  return 2;
}

// Persistent step of the items at column count j, all with tile rows TR, in
// cooperative launches of up to kMaxBatch trajectories. Blocks are shared out
// in proportion to each trajectory's tiles within one co-resident wave.
template <typename T, int TR>
etp_status launch_pk_batch_tr(etp_ctx* ctx, const std::vector<BSolve*>& items, int j) {
  const size_t smem = std::max<size_t>(cgs_smem_bytes<T>(j, TR), 1024);
  static std::mutex mu;
  static bool attr_set = false;
  static int bps_cache[kMaxCap + 2] = {};
  int bps = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!attr_set) {
      cudaFuncSetAttribute(k_arnoldi_step_pk_batch<T, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
      attr_set = true;
    }
    int& c = bps_cache[j];
    if (c == 0) {
      int n = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_arnoldi_step_pk_batch<T, TR>, 128, smem) !=
              cudaSuccess ||
          n < 1)
        n = 1;
      c = std::min(n, 2);
    }
    bps = c;
  }
  const int64_t wave = (int64_t)bps * ctx->num_sms;
  for (size_t a = 0; a < items.size(); a += kMaxBatch) {
    const int n = (int)std::min<size_t>(kMaxBatch, items.size() - a);
    PkBatch<T> b{};
    b.n = n;
    int64_t total = 0;
    double bytes = 0.0;
    for (int i = 0; i < n; ++i) {
      etp_traj* t = items[a + i]->t;
      total += t->L / TR;
      bytes += 9.0 * t->mesh->n_nodes * sizeof(T) + (double)(3 * j + 5) * t->L * sizeof(T);
      b.item[i] = make_pk_params<T>(t, j, t->has_load ? (const T*)t->d_pbar : nullptr);
    }
    b.off[0] = 0;
    for (int i = 0; i < n; ++i) {
      const int64_t nt = items[a + i]->t->L / TR;
      const int64_t share = std::min<int64_t>(nt, std::max<int64_t>(1, (wave - n) * nt / std::max<int64_t>(total, 1)));
      b.off[i + 1] = b.off[i] + (int)share;
    }
    ProfScope ps(ctx, KC_FUSED, bytes);
    void* argv[] = {(void*)&b};
    ETP_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_arnoldi_step_pk_batch<T, TR>, dim3(b.off[n]), dim3(128),
                                             argv, smem, ctx->stream));
  }
  return ETP_OK;
}

template <typename T>
etp_status launch_pk_batch(etp_ctx* ctx, const std::vector<BSolve*>& items, int j) {
  if (items.empty()) return ETP_OK;
  switch (pk_tile_rows<T>(j)) {
    case 128: return launch_pk_batch_tr<T, 128>(ctx, items, j);
    case 64: return launch_pk_batch_tr<T, 64>(ctx, items, j);
    default: return launch_pk_batch_tr<T, 32>(ctx, items, j);
  }
}

// Element passes of the items for Arnoldi step j (input column j-1), one
// launch per class of up to kMaxBatch meshes.
template <typename T>
etp_status launch_elem_batch(etp_ctx* ctx, const std::vector<BSolve*>& items, int j) {
  std::map<std::tuple<int, int, int, int>, std::vector<BSolve*>> cls;  // (order, kind, box, ns)
  for (BSolve* it : items) {
    const etp_mesh* m = it->t->mesh;
    const int ns = m->kind == MAT_LINEAR ? 0 : it->fzb.count;
    cls[std::make_tuple(m->order, m->kind, m->is_box ? 1 : 0, ns)].push_back(it);
  }
  for (auto& kv : cls) {
    const int order = std::get<0>(kv.first), kind = std::get<1>(kv.first), ns = std::get<3>(kv.first);
    const bool box = std::get<2>(kv.first) != 0;
    const auto& v = kv.second;
    for (size_t a = 0; a < v.size(); a += kMaxBatch) {
      const int n = (int)std::min<size_t>(kMaxBatch, v.size() - a);
      ElemBatch<T> b{};
      b.n = n;
      double bytes = 0.0, flops = 0.0;
      for (int i = 0; i < n; ++i) {
        etp_traj* t = v[a + i]->t;
        const T* x = (const T*)t->d_V + (int64_t)(j - 1) * t->L;
        const double* xscale = t->d_coef + COEF_SCALE * COEF_STRIDE + (j - 1);
        b.item[i] = make_apply_params<T>(t->mesh, x, xscale, v[a + i]->fzb, (T*)t->d_Ye, &t->d_ks->stop);
        bytes += elem_apply_bytes(t->mesh, ns, sizeof(T));
        flops += elem_apply_flops_of(t->mesh, ns);
      }
      ProfScope ps(ctx, KC_ELEM, bytes, flops);
      const cudaError_t e = order == 1 ? launch_elem_apply_batch<1, T>(b, kind, box, ns, ctx->num_sms, ctx->stream)
                                       : launch_elem_apply_batch<2, T>(b, kind, box, ns, ctx->num_sms, ctx->stream);
      if (e != cudaSuccess) return fail(ETP_ERR_CUDA, std::string("batched element apply: ") + cudaGetErrorString(e));
    }
  }
  return ETP_OK;
}

double taylor_coef(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= i;
  return 1.0 / f;
}

ExpmParams expm_params(etp_traj* t, int j0, int j1, double tau) {
  ExpmParams p{};
  p.H = t->d_H;
  p.ldH = t->m_cap + 1;
  p.j0 = j0;
  p.ncand = j1 - j0 + 1;
  p.tau = tau;
  p.ws = t->d_expm_ws;
  p.ld = t->m_cap;
  p.s_arr = (int*)t->d_red;
  p.ks = t->d_ks;
  for (int k = 0; k <= EXPM_TAYLOR_DEG; ++k) p.coef[k] = taylor_coef(k);
  return p;
}

// A-priori checks (Eq. "subspace error estimate") of the items that reached
// their check point: candidate sizes win_start..done of each, evaluated with
// two host synchronisations for all of them (scaling exponents, then the
// selection); each item's KState lands in its pinned mirror.
etp_status run_checks(etp_ctx* ctx, const std::vector<BSolve*>& chk) {
  if (chk.empty()) return ETP_OK;
  cudaStream_t st = ctx->stream;
  std::vector<ExpmParams> ps(chk.size());
  for (size_t c = 0; c < chk.size(); ++c) {
    BSolve* it = chk[c];
    etp_traj* t = it->t;
    ps[c] = expm_params(t, it->win_start, it->done, it->tau);
    ProfScope pr(ctx, KC_EXPM, 0.0);
    k_expm_prep<<<ps[c].ncand, 256, 0, st>>>(ps[c]);
    ETP_CUDA_TRY(cudaGetLastError());
    ETP_CUDA_TRY(cudaMemcpyAsync((int*)(t->h_ks + 1), ps[c].s_arr, sizeof(int) * ps[c].ncand, cudaMemcpyDeviceToHost,
                                 st));
  }
  ETP_CUDA_TRY(cudaStreamSynchronize(st));
  for (size_t c = 0; c < chk.size(); ++c) {
    BSolve* it = chk[c];
    etp_traj* t = it->t;
    const ExpmParams& p = ps[c];
    const int j1 = it->done;
    const int* h_s = (const int*)(t->h_ks + 1);
    int smax = 0;
    for (int k = 0; k < p.ncand; ++k) smax = std::max(smax, h_s[k]);
    {
      ProfScope pr(ctx, KC_EXPM, 0.0);
      const unsigned gx = (unsigned)((j1 * j1 + 63) / 64);
      k_expm_mm<<<dim3(gx, p.ncand, 1), 64, 0, st>>>(p, 0, 0);
      k_expm_mm<<<dim3(gx, p.ncand, 2), 64, 0, st>>>(p, 1, 0);
      for (int k = 3; k >= 0; --k) k_expm_mm<<<dim3(gx, p.ncand, 1), 64, 0, st>>>(p, 2, k);
      for (int k = 0; k < smax; ++k) k_expm_mm<<<dim3(gx, p.ncand, 1), 64, 0, st>>>(p, 3, k);
      ctx->launches += 6 + smax;
      k_expm_select<<<1, 128, 0, st>>>(p, t->d_ks, it->tol, 0, (j1 >= it->cap) ? 1 : 0, t->d_y);
      ETP_CUDA_TRY(cudaGetLastError());
    }
    ETP_CUDA_TRY(cudaMemcpyAsync(t->h_ks, t->d_ks, sizeof(KState), cudaMemcpyDeviceToHost, st));
  }
  ETP_CUDA_TRY(cudaStreamSynchronize(st));
  return ETP_OK;
}

// Finish a solve whose size is selected (or that failed): the state combine
// and the result, as the single-trajectory solve does.
template <typename T>
etp_status finish_solve(etp_ctx* ctx, BSolve* it) {
  etp_traj* t = it->t;
  etp_mesh* m = t->mesh;
  const KState& ks = *t->h_ks;
  if (ks.err & KERR_TIMEOUT) {
    // a barrier or a copy wait gave up: reset the reduction and barrier words
    cudaMemsetAsync(t->d_counter, 0, 3 * sizeof(unsigned int), ctx->stream);
    return fail(ETP_ERR_CUDA, "a bounded wait of the Arnoldi step timed out");
  }
  if (ks.err & KERR_INVERTED) return fail(ETP_ERR_INVERTED_ELEMENT, "det F <= 0 at a Gauss point of the frozen state");
  if (ks.err) return fail(ETP_ERR_NONFINITE, "non-finite value in the Krylov process");
  if (ks.found_m < 0) return fail(ETP_ERR_INVALID, "Krylov solve ended without a selected size");
  {
    const double s = sizeof(T);
    ProfScope ps(ctx, KC_COMBINE, (double)std::max(ks.found_m - 1, 0) * t->L * s + 2.0 * t->L * 8.0);
    const T* minv = sizeof(T) == 8 ? (const T*)m->d_minvsqrt64 : (const T*)m->d_minvsqrt32;
    k_combine<T><<<4 * ctx->num_sms, 256, 0, ctx->stream>>>(t->L, m->nn_pad, it->w_in, (const T*)t->d_V, t->d_y,
                                                             t->d_coef, t->d_ks, it->w_out, (T*)it->ustar_out, minv);
    ETP_CUDA_TRY(cudaGetLastError());
  }
  it->res.m = ks.found_m;
  it->res.eps = ks.eps;
  it->res.beta = ks.beta;
  it->res.converged = ks.converged != 0;
  t->last_m = ks.found_m;
  if (ks.found_m > 0) t->m_hint[it->kind & 1] = ks.found_m;
  return ETP_OK;
}

template <typename T>
etp_status start_solve(etp_ctx* ctx, BSolve* it) {
  etp_traj* t = it->t;
  {
    ProfScope ps(ctx, KC_OTHER, (double)t->L * (8.0 + sizeof(T)));
    k_init_basis<T><<<2 * ctx->num_sms, 256, 0, ctx->stream>>>(t->L, it->w_in, (T*)t->d_V, t->d_partials,
                                                               t->d_counter, t->d_coef, t->d_ks);
    ETP_CUDA_TRY(cudaGetLastError());
  }
  ETP_TRY(prepare_frozen<T>(t, it->fz, &it->fzb));
  it->cap = t->m_cap;
  const int hint = t->m_hint[it->kind & 1];
  it->W = check_window(t);
  it->next_check = std::min(it->cap, hint >= 2 ? hint - 1 : 8);
  it->next_check = std::min(it->next_check, kMaxCand);  // one launch set per check
  it->done = 0;
  it->win_start = 1;
  return ETP_OK;
}

// Lockstep solves of all items (adaptive m). Every size 1..m of an item is
// checked in ascending order, so each selects the smallest passing m, as the
// single solve does. Per-item failures are recorded in it->st; the return
// value reports a failure of the round itself (a CUDA error).
etp_status solve_lockstep(etp_ctx* ctx, std::vector<BSolve>& items) {
  for (BSolve& it : items) {
    it.active = true;
    const etp_status s = it.t->prec == ETP_PREC_FP64 ? start_solve<double>(ctx, &it) : start_solve<float>(ctx, &it);
    if (s != ETP_OK) { it.st = s; it.active = false; }
  }
  for (int j = 1;; ++j) {
    std::vector<BSolve*> f32, f64;
    for (BSolve& it : items)
      if (it.active) (it.t->prec == ETP_PREC_FP64 ? f64 : f32).push_back(&it);
    if (f32.empty() && f64.empty()) break;
    ETP_TRY(launch_elem_batch<float>(ctx, f32, j));
    ETP_TRY(launch_elem_batch<double>(ctx, f64, j));
    ETP_TRY(launch_pk_batch<float>(ctx, f32, j));
    ETP_TRY(launch_pk_batch<double>(ctx, f64, j));
    std::vector<BSolve*> chk;
    for (BSolve& it : items) {
      if (!it.active) continue;
      it.done = j;
      if (j >= it.next_check) chk.push_back(&it);
    }
    ETP_TRY(run_checks(ctx, chk));
    for (BSolve* it : chk) {
      const KState& ks = *it->t->h_ks;
      if (ks.err || ks.found_m >= 0) {
        const etp_status s =
            it->t->prec == ETP_PREC_FP64 ? finish_solve<double>(ctx, it) : finish_solve<float>(ctx, it);
        if (s != ETP_OK) it->st = s;
        it->active = false;
        continue;
      }
      if (it->done >= it->cap) {  // the last window always selects a size
        it->st = fail(ETP_ERR_INVALID, "Krylov solve ended without a selected size");
        it->active = false;
        continue;
      }
      it->win_start = it->done + 1;
      it->next_check = std::min(it->cap, it->done + it->W);
    }
  }
  return ETP_OK;
}

// Per-trajectory state of one batched step.
struct BStep {
  etp_traj* t = nullptr;
  double dt = 0.0, tol = 0.0;
  int slot_new = -1;
  etp_step_info loc{};
  etp_status st = ETP_OK;
  bool done = false;
};

}  // namespace
}  // namespace etp

using namespace etp;

extern "C" {

etp_status etp_step_batch(etp_traj* const* trajs, int n, const double* dt, const double* tol, etp_step_info* infos,
                          etp_status* statuses) {
  if (n < 0 || n > kMaxBatchStep) return fail(ETP_ERR_INVALID, "n must be in 0..64");
  if (n == 0) return ETP_OK;
  if (!trajs || !dt || !tol) return fail(ETP_ERR_INVALID, "null argument");
  etp_ctx* ctx = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!trajs[i]) return fail(ETP_ERR_INVALID, "null trajectory");
    if (!ctx) ctx = trajs[i]->mesh->ctx;
    if (trajs[i]->mesh->ctx != ctx) return fail(ETP_ERR_INVALID, "all trajectories of a batch must share one context");
    for (int k = 0; k < i; ++k)
      if (trajs[k] == trajs[i]) return fail(ETP_ERR_INVALID, "a trajectory appears twice in the batch");
    ETP_TRY(check_step_args(trajs[i], dt[i], tol[i]));
  }
  ETP_CUDA_TRY(cudaSetDevice(ctx->device));
  std::vector<BStep> S(n);
  for (int i = 0; i < n; ++i) {
    S[i].t = trajs[i];
    S[i].dt = dt[i];
    S[i].tol = tol[i];
  }
  // vectors too long for the persistent step (or no cooperative launch): the
  // single-trajectory path, one after another
  for (BStep& s : S) {
    if (ctx->cooperative && s.t->L <= kPkMaxRows) continue;
    s.st = etp_step_ex(s.t, s.dt, s.tol, 0, 0, &s.loc);
    s.done = true;
  }
  // predictor solves of the nonlinear trajectories (Section 4.2)
  std::vector<BSolve> P;
  std::vector<int> p_of;
  for (int i = 0; i < n; ++i) {
    BStep& s = S[i];
    if (s.done || s.t->mesh->kind == MAT_LINEAR) continue;
    BSolve b;
    const etp_status e = predictor_setup(s.t, &b.fz, &s.slot_new);
    if (e != ETP_OK) { s.st = e; s.done = true; continue; }
    b.t = s.t;
    b.tau = 0.5 * s.dt;
    b.tol = s.tol;
    b.w_in = s.t->d_w;
    b.w_out = s.t->d_wtmp;
    b.ustar_out = s.t->d_hist[s.slot_new];
    b.kind = 1;
    P.push_back(b);
    p_of.push_back(i);
  }
  ETP_TRY(solve_lockstep(ctx, P));
  for (size_t k = 0; k < P.size(); ++k) {
    BStep& s = S[p_of[k]];
    s.loc.m_pred = P[k].res.m;
    s.loc.eps_pred = P[k].res.eps;
    if (P[k].st != ETP_OK) { s.st = P[k].st; s.done = true; continue; }
    if (!P[k].res.converged) {
      s.loc.beta = P[k].res.beta;
      s.st = fail(ETP_ERR_NOT_CONVERGED, "predictor Krylov solve did not reach tol at m_cap");
      s.done = true;
    }
  }
  // corrector solves (the only solve of a linear trajectory)
  std::vector<BSolve> C;
  std::vector<int> c_of;
  for (int i = 0; i < n; ++i) {
    BStep& s = S[i];
    if (s.done) continue;
    BSolve b;
    if (s.t->mesh->kind != MAT_LINEAR) b.fz = corrector_frozen(s.t, s.slot_new);
    b.t = s.t;
    b.tau = s.dt;
    b.tol = s.tol;
    b.w_in = s.t->d_w;
    b.w_out = s.t->d_wtmp;
    b.kind = 0;
    C.push_back(b);
    c_of.push_back(i);
  }
  ETP_TRY(solve_lockstep(ctx, C));
  for (size_t k = 0; k < C.size(); ++k) {
    BStep& s = S[c_of[k]];
    if (C[k].st != ETP_OK) { s.st = C[k].st; s.done = true; continue; }
    s.st = step_commit(s.t, C[k].res, s.slot_new, &s.loc, nullptr);
    s.done = true;
  }
  etp_status first = ETP_OK;
  for (int i = 0; i < n; ++i) {
    if (infos) infos[i] = S[i].loc;
    if (statuses) statuses[i] = S[i].st;
    if (first == ETP_OK && S[i].st != ETP_OK) first = S[i].st;
  }
  return first;
}

}  // extern "C"
