// Ragged batched time steps: the Krylov solves (Section 4.3) of many
// trajectories -- each its own mesh, size, material, precision, dt and
// tolerance -- advance together with iteration-level continuous batching.
// Every tick advances every active solve by one Arnoldi step with ONE
// element-pass launch per (order, precision, material, geometry, frozen-state
// count) class and ONE persistent Arnoldi-step launch per precision and tile
// size for up to 16 trajectories, and evaluates the a-priori checks that are
// due with one batched small-exponential launch set and two host
// synchronisations. A trajectory whose solve selects its size moves on at once
// (predictor -> corrector -> next step), so none waits for another's solve.
//
// Every kernel computes a trajectory's values exactly as its single launch
// does (element terms are per element; the persistent step's sums are per
// tile and summed in tile order; the small exponential is per candidate size),
// so a trajectory gives the same bits stepped alone (etp_step) or in any
// batch.
#include <math.h>

#include <algorithm>
#include <list>
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

// One Krylov solve in the engine.
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

// One trajectory in the engine: its current solve and step phase
// (0 next step to begin, 1 predictor, 2 corrector or linear, 3 leaving).
struct EngineItem {
  etp_traj* t = nullptr;
  double dt = 0.0, tol = 0.0;
  int steps_left = 0;
  int phase = 0;
  bool solo = false;  // vectors too long for the persistent step: etp_step_ex per tick
  int slot_new = -1;
  etp_step_info loc{};
  BSolve solve;
};

namespace {

// Arnoldi steps between checks after the first one (as the single solve).
int check_window(const etp_traj* t) {
  if (t->L >= (int64_t)4 << 20) return 1;
  return 2;
}

// Persistent Arnoldi steps of the items (item i at column count j_i = its
// done + 1), those of one tile size in cooperative launches of up to
// kMaxBatch trajectories (one kernel instance per tile size keeps the code
// each launch fetches small). Blocks are shared out in proportion to each
// trajectory's tiles within one co-resident wave (the results do not depend
// on the share).
template <typename T, int TR>
etp_status launch_pk_batch_tr(etp_ctx* ctx, const std::vector<BSolve*>& items) {
  const void* fn = (const void*)k_arnoldi_step_pk_batch<T, TR>;
  static std::once_flag once;
  std::call_once(once, [fn] { pk_allow_smem(fn); });
  for (size_t a = 0; a < items.size(); a += kMaxBatch) {
    const int n = (int)std::min<size_t>(kMaxBatch, items.size() - a);
    PkBatch<T> b{};
    b.n = n;
    // one tile area for all (the widest); no copy area for the partial sums
    // (read from L2 with all loads in flight; the copy area measured slower
    // in the served batch)
    uint32_t tile = 0;
    for (int i = 0; i < n; ++i) {
      etp_traj* t = items[a + i]->t;
      b.item[i] = make_pk_params<T>(t, items[a + i]->done + 1, t->has_load ? (const T*)t->d_pbar : nullptr);
      pk_step_smem<T>(t->L, b.item[i].c.j, TR, b.item[i]);
      tile = std::max(tile, b.item[i].red_off);
    }
    const size_t smem = std::max<size_t>(tile, 1024);
    for (int i = 0; i < n; ++i) {
      b.item[i].red_off = tile;
      b.item[i].red_bytes = 0;
    }
    const int bps = pk_blocks_per_sm(fn, smem);
    const int64_t wave = (int64_t)bps * ctx->num_sms;
    int64_t total = 0;
    double bytes = 0.0;
    for (int i = 0; i < n; ++i) {
      etp_traj* t = items[a + i]->t;
      total += pk_ntiles(t->L, TR);
      bytes += 9.0 * t->mesh->n_nodes * sizeof(T) + (double)(3 * b.item[i].c.j + 5) * t->L * sizeof(T);
    }
    b.off[0] = 0;
    for (int i = 0; i < n; ++i) {
      const int64_t nt = pk_ntiles(items[a + i]->t->L, TR);
      const int64_t share = std::min<int64_t>(nt, std::max<int64_t>(1, (wave - n) * nt / std::max<int64_t>(total, 1)));
      b.off[i + 1] = b.off[i] + (int)share;
    }
    ProfScope ps(ctx, KC_FUSED, bytes);
    void* argv[] = {(void*)&b};
    ETP_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(b.off[n]), dim3(128), argv, smem, ctx->stream));
  }
  return ETP_OK;
}

template <typename T>
etp_status launch_pk_batch(etp_ctx* ctx, const std::vector<BSolve*>& items) {
  std::vector<BSolve*> by_tr[4];
  for (BSolve* it : items) {
    const int tr = pk_tile_rows<T>(it->done + 1, it->t->L);
    by_tr[tr == 256 ? 0 : tr == 128 ? 1 : tr == 64 ? 2 : 3].push_back(it);
  }
  if (!by_tr[0].empty()) ETP_TRY((launch_pk_batch_tr<T, 256>(ctx, by_tr[0])));
  if (!by_tr[1].empty()) ETP_TRY((launch_pk_batch_tr<T, 128>(ctx, by_tr[1])));
  if (!by_tr[2].empty()) ETP_TRY((launch_pk_batch_tr<T, 64>(ctx, by_tr[2])));
  if (!by_tr[3].empty()) ETP_TRY((launch_pk_batch_tr<T, 32>(ctx, by_tr[3])));
  return ETP_OK;
}

// Element passes of the items for their next Arnoldi step (input column
// done), one launch per class of up to kMaxBatch meshes.
template <typename T>
etp_status launch_elem_batch(etp_ctx* ctx, const std::vector<BSolve*>& items) {
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
        const int j = v[a + i]->done + 1;
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
// their check point: candidate sizes win_start..done of each, evaluated for up
// to kMaxExpmBatch items by one batched launch set and two host
// synchronisations (scaling exponents, then the selection). The exponents of
// all candidates and the states after selection are staged in one array each
// (context-owned), so each synchronisation needs one copy; each item's state
// then lands in its pinned mirror.
etp_status run_checks(etp_ctx* ctx, const std::vector<BSolve*>& all) {
  if (all.empty()) return ETP_OK;
  cudaStream_t st = ctx->stream;
  if (!ctx->d_chk_s) {
    ETP_TRY(dalloc(&ctx->d_chk_s, sizeof(int) * kMaxExpmBatch * kMaxCand));
    ETP_TRY(dalloc((char**)&ctx->d_chk_ks, sizeof(KState) * kMaxExpmBatch));
    if (cudaMallocHost((void**)&ctx->h_chk_s, sizeof(int) * kMaxExpmBatch * kMaxCand) != cudaSuccess ||
        cudaMallocHost(&ctx->h_chk_ks, sizeof(KState) * kMaxExpmBatch) != cudaSuccess)
      return fail(ETP_ERR_OOM, "cudaMallocHost failed");
  }
  KState* d_ks = (KState*)ctx->d_chk_ks;
  const KState* h_ks = (const KState*)ctx->h_chk_ks;
  for (size_t a = 0; a < all.size(); a += kMaxExpmBatch) {
    const int n = (int)std::min<size_t>(kMaxExpmBatch, all.size() - a);
    ExpmBatch b{};
    ExpmSelectBatch sb{};
    b.n = n;
    b.cand_off[0] = 0;
    int jmax = 1;
    for (int i = 0; i < n; ++i) {
      BSolve* it = all[a + i];
      etp_traj* t = it->t;
      b.item[i] = expm_params(t, it->win_start, it->done, it->tau);
      b.item[i].s_arr = ctx->d_chk_s + b.cand_off[i];
      b.cand_off[i + 1] = b.cand_off[i] + b.item[i].ncand;
      sb.sel[i] = ExpmSelect{t->d_ks, it->tol, (it->done >= it->cap) ? 1 : 0, t->d_y, d_ks + i};
      jmax = std::max(jmax, it->done);
    }
    const int ncand = b.cand_off[n];
    {
      ProfScope pr(ctx, KC_EXPM, 0.0);
      k_expm_prep_batch<<<ncand, 256, 0, st>>>(b);
      ETP_CUDA_TRY(cudaGetLastError());
    }
    ETP_CUDA_TRY(cudaMemcpyAsync(ctx->h_chk_s, ctx->d_chk_s, sizeof(int) * ncand, cudaMemcpyDeviceToHost, st));
    ETP_CUDA_TRY(cudaStreamSynchronize(st));
    int smax = 0;
    for (int c = 0; c < ncand; ++c) smax = std::max(smax, ctx->h_chk_s[c]);
    {
      ProfScope pr(ctx, KC_EXPM, 0.0);
      const unsigned gx = (unsigned)((jmax * jmax + 63) / 64);
      k_expm_mm_batch<<<dim3(gx, ncand, 1), 64, 0, st>>>(b, 0, 0);
      k_expm_mm_batch<<<dim3(gx, ncand, 2), 64, 0, st>>>(b, 1, 0);
      for (int k = 3; k >= 0; --k) k_expm_mm_batch<<<dim3(gx, ncand, 1), 64, 0, st>>>(b, 2, k);
      for (int k = 0; k < smax; ++k) k_expm_mm_batch<<<dim3(gx, ncand, 1), 64, 0, st>>>(b, 3, k);
      k_expm_select_batch<<<n, 128, 0, st>>>(b, sb);
      ctx->launches += 6 + smax;
      ETP_CUDA_TRY(cudaGetLastError());
    }
    ETP_CUDA_TRY(cudaMemcpyAsync(ctx->h_chk_ks, d_ks, sizeof(KState) * n, cudaMemcpyDeviceToHost, st));
    ETP_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < n; ++i) *all[a + i]->t->h_ks = h_ks[i];
  }
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
    cudaMemsetAsync(t->d_counter, 0, 16 * sizeof(unsigned int), ctx->stream);
    return fail(ETP_ERR_TIMEOUT, "a bounded wait of the Arnoldi step timed out");
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
  // first check at the previous m of this kind (short vectors: a step costs less than a check round)
  it->next_check = std::min(it->cap, hint >= 2 ? hint : 8);
  it->next_check = std::min(it->next_check, kMaxCand);  // one launch set per check
  it->done = 0;
  it->win_start = 1;
  return ETP_OK;
}


// Start the next step of a trajectory: the predictor solve of a nonlinear
// material (Section 4.2), else the single solve of the linear one.
etp_status begin_step(etp_ctx* ctx, EngineItem* e) {
  etp_traj* t = e->t;
  e->loc = etp_step_info{};
  e->slot_new = -1;
  BSolve& b = e->solve;
  b = BSolve{};
  b.t = t;
  b.tol = e->tol;
  b.w_in = t->d_w;
  b.w_out = t->d_wtmp;
  if (t->mesh->kind == MAT_LINEAR) {
    b.tau = e->dt;
    b.kind = 0;
    e->phase = 2;
  } else {
    ETP_TRY(predictor_setup(t, &b.fz, &e->slot_new));
    b.tau = 0.5 * e->dt;
    b.kind = 1;
    b.ustar_out = t->d_hist[e->slot_new];
    e->phase = 1;
  }
  return t->prec == ETP_PREC_FP64 ? start_solve<double>(ctx, &b) : start_solve<float>(ctx, &b);
}

// The corrector solve of a nonlinear step whose predictor has finished.
etp_status begin_corrector(etp_ctx* ctx, EngineItem* e) {
  etp_traj* t = e->t;
  BSolve& b = e->solve;
  b = BSolve{};
  b.t = t;
  b.tol = e->tol;
  b.tau = e->dt;
  b.kind = 0;
  b.w_in = t->d_w;
  b.w_out = t->d_wtmp;
  b.fz = corrector_frozen(t, e->slot_new);
  e->phase = 2;
  return t->prec == ETP_PREC_FP64 ? start_solve<double>(ctx, &b) : start_solve<float>(ctx, &b);
}

}  // namespace

// Iteration-level continuous batching of Krylov solves: every tick advances
// every active solve by one Arnoldi step (batched launches) and runs the
// checks that are due; a trajectory whose solve selects m moves on at once
// (predictor -> corrector -> next step), so no trajectory waits for another's
// solve to end.
struct RaggedEngine {
  etp_ctx* ctx = nullptr;
  std::list<EngineItem> items;
};

RaggedEngine* ragged_engine_create(etp_ctx* ctx) {
  RaggedEngine* e = new RaggedEngine();
  e->ctx = ctx;
  return e;
}

void ragged_engine_destroy(RaggedEngine* e) { delete e; }

bool ragged_engine_empty(const RaggedEngine* e) { return e->items.empty(); }

// Arnoldi trajectories with vectors the persistent step takes share the
// engine's launches; the rest (long vectors, the energy Lanczos process) are
// stepped by etp_step_ex, one step per tick.
bool ragged_engine_batchable(const RaggedEngine* e, const etp_traj* t) {
  return e->ctx->cooperative && t->L <= kPkMaxRows && t->mesh->ctx == e->ctx && t->krylov == ETP_KRYLOV_ARNOLDI;
}

etp_status ragged_engine_add(RaggedEngine* e, etp_traj* t, double dt, double tol, int n_steps) {
  if (!t || n_steps < 1) return fail(ETP_ERR_INVALID, "bad engine entry");
  if (t->mesh->ctx != e->ctx) return fail(ETP_ERR_INVALID, "trajectory of another context");
  EngineItem it;
  it.t = t;
  it.dt = dt;
  it.tol = tol;
  it.steps_left = n_steps;
  it.solo = !ragged_engine_batchable(e, t);
  e->items.push_back(it);
  return ETP_OK;
}

etp_status ragged_engine_tick(RaggedEngine* e, std::vector<EngineEvent>* events) {
  etp_ctx* ctx = e->ctx;
  ETP_CUDA_TRY(cudaSetDevice(ctx->device));
  auto emit = [&](EngineItem& it, etp_status st) {
    it.steps_left -= 1;
    const bool last = st != ETP_OK || it.steps_left <= 0;
    events->push_back(EngineEvent{it.t, st, it.loc, last});
    if (last) it.phase = 3;
  };
  // trajectories whose vectors are too long for the persistent step: one
  // etp_step_ex each per tick
  for (EngineItem& it : e->items) {
    if (!it.solo || it.phase == 3) continue;
    const etp_status st = etp_step_ex(it.t, it.dt, it.tol, 0, 0, &it.loc);
    emit(it, st);
  }
  // new steps
  for (EngineItem& it : e->items) {
    if (it.solo || it.phase != 0) continue;
    const etp_status st = begin_step(ctx, &it);
    if (st != ETP_OK) emit(it, st);
  }
  std::vector<BSolve*> f32, f64;
  for (EngineItem& it : e->items)
    if ((it.phase == 1 || it.phase == 2) && it.solve.active)
      (it.t->prec == ETP_PREC_FP64 ? f64 : f32).push_back(&it.solve);
  ETP_TRY(launch_elem_batch<float>(ctx, f32));
  ETP_TRY(launch_elem_batch<double>(ctx, f64));
  ETP_TRY(launch_pk_batch<float>(ctx, f32));
  ETP_TRY(launch_pk_batch<double>(ctx, f64));
  std::vector<BSolve*> chk;
  std::vector<EngineItem*> chk_item;
  for (EngineItem& it : e->items) {
    if (!((it.phase == 1 || it.phase == 2) && it.solve.active)) continue;
    BSolve& b = it.solve;
    b.done += 1;
    if (b.done >= b.next_check) {
      chk.push_back(&b);
      chk_item.push_back(&it);
    }
  }
  ETP_TRY(run_checks(ctx, chk));
  for (size_t k = 0; k < chk.size(); ++k) {
    BSolve* b = chk[k];
    EngineItem& it = *chk_item[k];
    const KState& ks = *b->t->h_ks;
    if (!(ks.err || ks.found_m >= 0)) {
      if (b->done >= b->cap) {  // the last window always selects a size
        emit(it, fail(ETP_ERR_INVALID, "Krylov solve ended without a selected size"));
        continue;
      }
      b->win_start = b->done + 1;
      b->next_check = std::min(b->cap, b->done + b->W);
      continue;
    }
    b->active = false;
    const etp_status fs = b->t->prec == ETP_PREC_FP64 ? finish_solve<double>(ctx, b) : finish_solve<float>(ctx, b);
    if (fs != ETP_OK) {
      emit(it, fs);
      continue;
    }
    if (it.phase == 1) {  // predictor done
      it.loc.m_pred = b->res.m;
      it.loc.eps_pred = b->res.eps;
      if (!b->res.converged) {
        it.loc.beta = b->res.beta;
        emit(it, fail(ETP_ERR_NOT_CONVERGED, "predictor Krylov solve did not reach tol at m_cap"));
        continue;
      }
      const etp_status cs = begin_corrector(ctx, &it);
      if (cs != ETP_OK) emit(it, cs);
      continue;
    }
    // corrector (or linear) done: commit the step
    const etp_status st = step_commit(it.t, b->res, it.slot_new, &it.loc, nullptr);
    emit(it, st);
    if (it.phase != 3) it.phase = 0;  // the next step starts at the next tick
  }
  for (auto i = e->items.begin(); i != e->items.end();)
    i = (i->phase == 3) ? e->items.erase(i) : std::next(i);
  return ETP_OK;
}

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
  RaggedEngine eng;
  eng.ctx = ctx;
  for (int i = 0; i < n; ++i) ETP_TRY(ragged_engine_add(&eng, trajs[i], dt[i], tol[i], 1));
  std::vector<EngineEvent> ev;
  while (!ragged_engine_empty(&eng)) ETP_TRY(ragged_engine_tick(&eng, &ev));
  etp_status first = ETP_OK;
  for (int i = 0; i < n; ++i) {
    etp_status st = ETP_ERR_INVALID;
    etp_step_info inf{};
    for (const EngineEvent& x : ev)
      if (x.t == trajs[i]) { st = x.st; inf = x.info; }
    if (infos) infos[i] = inf;
    if (statuses) statuses[i] = st;
    if (first == ETP_OK && st != ETP_OK) first = st;
  }
  return first;
}

}  // extern "C"
