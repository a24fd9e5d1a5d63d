// Continuous batching of propagation requests (served mixed batch).
//
// A batch admits trajectories against a device-memory budget and steps every
// admitted trajectory on a pool of host worker threads. Each trajectory keeps
// its state and Krylov workspace resident; a worker takes the next runnable
// trajectory (round robin), runs one etp_step on it and puts it back, so
// trajectories advance independently (no barrier between them) and their
// kernels overlap on the GPU when they live on different contexts (streams).
// Two trajectories of one context never step at the same time: the context's
// stream and counters belong to one caller at a time.
//
// A ragged batch (etp_batch_create_ragged) has instead one worker per context
// of its trajectories, each running one engine of iteration-level continuous
// batching (batch_solve.cu) on that context's stream: each tick advances every
// active Krylov solve of the context by one Arnoldi step in shared launches,
// and arrivals join at the next tick. Engines of different contexts overlap on
// the GPU (a server puts requests of similar size on one context).
//
// etp_batch_tick blocks until at least one step has finished since the last
// tick (or nothing is left to run), reports how many, and retires the
// trajectories that completed their steps or failed; their device memory
// leaves the budget. Every numerical step is etp_step or the engine's; this
// file only schedules.

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "etp_host.cuh"

namespace etp {

struct BatchEntry {
  etp_traj* t = nullptr;
  etp_ctx* ctx = nullptr;
  int n_steps = 0;
  double dt = 0.0, tol = 0.0;
  size_t bytes = 0;
  bool running = false;
  bool finished = false;
};

struct BatchInfo {
  int steps_done = 0;
  etp_status status = ETP_OK;
  std::vector<float> step_ms;  // host wall time of every step
  bool retired = false;
};

}  // namespace etp

using namespace etp;

struct etp_batch {
  etp_ctx* ctx = nullptr;
  size_t budget = 0;
  size_t reserved = 0;
  std::mutex mu;
  std::condition_variable cv_work;      // a trajectory became runnable, or stop
  std::condition_variable cv_progress;  // a step finished
  std::list<BatchEntry> active;
  std::vector<std::pair<etp_traj*, etp_status>> retired;  // not yet collected
  std::unordered_map<const etp_traj*, BatchInfo> info;
  std::unordered_set<const etp_ctx*> busy;  // contexts with a step in flight
  int64_t steps_since_tick = 0;
  bool stop = false;
  bool ragged = false;  // one engine worker per context of the admitted trajectories
  std::unordered_set<const etp_ctx*> engine_ctxs;  // contexts that have an engine worker
  std::vector<std::thread> workers;
};

namespace {

// First runnable entry in list order (the list is rotated after every step).
std::list<BatchEntry>::iterator next_runnable(etp_batch* b) {
  for (auto it = b->active.begin(); it != b->active.end(); ++it)
    if (!it->running && !it->finished && !b->busy.count(it->ctx)) return it;
  return b->active.end();
}

void worker_loop(etp_batch* b) {
  std::unique_lock<std::mutex> lk(b->mu);
  for (;;) {
    auto it = b->active.end();
    b->cv_work.wait(lk, [&] { return b->stop || (it = next_runnable(b)) != b->active.end(); });
    if (b->stop) return;
    it->running = true;
    b->busy.insert(it->ctx);
    etp_traj* t = it->t;
    const double dt = it->dt, tol = it->tol;
    lk.unlock();
    const auto t0 = std::chrono::steady_clock::now();
    int m = 0;
    double err = 0.0;
    const etp_status st = etp_step(t, dt, tol, 0, &m, &err);
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    lk.lock();
    BatchInfo& inf = b->info[t];
    inf.step_ms.push_back((float)ms);
    if (st == ETP_OK) {
      inf.steps_done += 1;
      b->steps_since_tick += 1;
    } else {
      inf.status = st;
    }
    it->running = false;
    b->busy.erase(it->ctx);
    if (st != ETP_OK || inf.steps_done >= it->n_steps) it->finished = true;
    b->active.splice(b->active.end(), b->active, it);  // round robin
    b->cv_progress.notify_all();
    b->cv_work.notify_all();
  }
}

// Ragged mode: one engine (iteration-level continuous batching) per context
// runs every admitted trajectory of that context, on this worker thread.
// Between ticks, newly admitted trajectories of the context join; each
// finished step is recorded with the wall time since the trajectory's
// previous step finished (or since it joined).
void ragged_loop(etp_batch* b, etp_ctx* ctx) {
  using clock = std::chrono::steady_clock;
  RaggedEngine* eng = ragged_engine_create(ctx);
  std::unordered_map<const etp_traj*, clock::time_point> last;
  std::unique_lock<std::mutex> lk(b->mu);
  auto runnable = [&] {
    for (const auto& e : b->active)
      if (e.ctx == ctx && !e.running && !e.finished) return true;
    return false;
  };
  auto has_entries = [&] {
    for (const auto& e : b->active)
      if (e.ctx == ctx && !e.finished) return true;
    return false;
  };
  for (;;) {
    b->cv_work.wait(lk, [&] { return b->stop || runnable() || !ragged_engine_empty(eng) || !has_entries(); });
    if (b->stop) break;
    if (ragged_engine_empty(eng) && !has_entries()) {
      // nothing of this context is left: the worker ends (a later trajectory of
      // the context starts a new one)
      b->engine_ctxs.erase(ctx);
      break;
    }
    for (auto it = b->active.begin(); it != b->active.end(); ++it) {
      if (it->ctx != ctx || it->running || it->finished) continue;
      const int left = it->n_steps - b->info[it->t].steps_done;
      if (ragged_engine_add(eng, it->t, it->dt, it->tol, std::max(left, 1)) != ETP_OK) {
        b->info[it->t].status = ETP_ERR_INVALID;
        it->finished = true;
        continue;
      }
      it->running = true;
      last[it->t] = clock::now();
    }
    lk.unlock();
    std::vector<EngineEvent> ev;
    const etp_status st_tick = ragged_engine_tick(eng, &ev);
    const auto now = clock::now();
    lk.lock();
    if (st_tick != ETP_OK) {
      // the round itself failed (a CUDA error): every trajectory in the engine fails
      for (auto& e : b->active)
        if (e.running && e.ctx == ctx) {
          b->info[e.t].status = st_tick;
          e.running = false;
          e.finished = true;
        }
      ragged_engine_destroy(eng);
      eng = ragged_engine_create(ctx);
      b->cv_progress.notify_all();
      continue;
    }
    for (const EngineEvent& x : ev) {
      BatchInfo& inf = b->info[x.t];
      inf.step_ms.push_back((float)std::chrono::duration<double, std::milli>(now - last[x.t]).count());
      last[x.t] = now;
      if (x.st == ETP_OK) {
        inf.steps_done += 1;
        b->steps_since_tick += 1;
      } else {
        inf.status = x.st;
      }
      if (x.last) {
        for (auto& e : b->active)
          if (e.t == x.t) {
            e.running = false;
            e.finished = true;
          }
        last.erase(x.t);
      }
    }
    if (!ev.empty()) b->cv_progress.notify_all();
  }
  lk.unlock();
  ragged_engine_destroy(eng);
}

bool anything_to_run(etp_batch* b) {
  for (const auto& e : b->active)
    if (!e.finished) return true;
  return false;
}

}  // namespace

extern "C" {

etp_status etp_batch_create(etp_ctx* ctx, size_t device_budget_bytes, int n_workers, etp_batch** out) {
  if (!ctx || !out) return fail(ETP_ERR_INVALID, "null argument");
  if (n_workers < 1 || n_workers > 256) return fail(ETP_ERR_INVALID, "n_workers must be in 1..256");
  etp_batch* b = new etp_batch();
  b->ctx = ctx;
  b->budget = device_budget_bytes;
  for (int i = 0; i < n_workers; ++i) b->workers.emplace_back(worker_loop, b);
  *out = b;
  return ETP_OK;
}

etp_status etp_batch_create_ragged(etp_ctx* ctx, size_t device_budget_bytes, etp_batch** out) {
  if (!ctx || !out) return fail(ETP_ERR_INVALID, "null argument");
  etp_batch* b = new etp_batch();
  b->ctx = ctx;
  b->budget = device_budget_bytes;
  b->ragged = true;
  *out = b;
  return ETP_OK;
}

void etp_batch_destroy(etp_batch* b) {
  if (!b) return;
  {
    std::lock_guard<std::mutex> lk(b->mu);
    b->stop = true;
  }
  b->cv_work.notify_all();
  for (auto& w : b->workers) w.join();  // a step in flight completes first
  delete b;
}

etp_status etp_batch_admit(etp_batch* b, etp_traj* traj, int n_steps, double dt, double tol) {
  if (!b || !traj) return fail(ETP_ERR_INVALID, "null argument");
  if (n_steps < 1) return fail(ETP_ERR_INVALID, "n_steps must be >= 1");
  if (!(dt > 0) || !(tol >= 0)) return fail(ETP_ERR_INVALID, "dt must be positive and tol non-negative");
  const size_t bytes = traj->device_bytes + mesh_device_bytes(traj->mesh);
  std::lock_guard<std::mutex> lk(b->mu);
  for (const auto& e : b->active)
    if (e.t == traj) return fail(ETP_ERR_INVALID, "trajectory already admitted");
  if (b->reserved + bytes > b->budget) return fail(ETP_ERR_OOM, "device budget of the batch is full (not now)");
  BatchEntry e;
  e.t = traj;
  e.ctx = traj->mesh->ctx;
  e.n_steps = n_steps;
  e.dt = dt;
  e.tol = tol;
  e.bytes = bytes;
  b->active.push_back(e);
  b->reserved += bytes;
  if (b->ragged && !b->engine_ctxs.count(e.ctx)) {  // first trajectory of this context: its engine
    b->engine_ctxs.insert(e.ctx);
    b->workers.emplace_back(ragged_loop, b, e.ctx);
  }
  BatchInfo& inf = b->info[traj];
  inf = BatchInfo();
  b->cv_work.notify_all();
  return ETP_OK;
}

etp_status etp_batch_tick(etp_batch* b, int* n_finished_steps) {
  if (!b) return fail(ETP_ERR_INVALID, "null batch");
  std::unique_lock<std::mutex> lk(b->mu);
  b->cv_progress.wait(lk, [&] { return b->steps_since_tick > 0 || !anything_to_run(b) ||
                                       std::any_of(b->active.begin(), b->active.end(), [](const BatchEntry& e) {
                                         return e.finished && !e.running;
                                       }); });
  if (n_finished_steps) *n_finished_steps = (int)b->steps_since_tick;
  b->steps_since_tick = 0;
  for (auto it = b->active.begin(); it != b->active.end();) {
    if (it->finished && !it->running) {
      BatchInfo& inf = b->info[it->t];
      inf.retired = true;
      b->retired.emplace_back(it->t, inf.status);
      b->reserved -= it->bytes;
      it = b->active.erase(it);
    } else {
      ++it;
    }
  }
  return ETP_OK;
}

etp_status etp_batch_retired(etp_batch* b, etp_traj** trajs, int* statuses, int max, int* n) {
  if (!b || !n || max < 0) return fail(ETP_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(b->mu);
  const int k = std::min<int>(max, (int)b->retired.size());
  for (int i = 0; i < k; ++i) {
    if (trajs) trajs[i] = b->retired[i].first;
    if (statuses) statuses[i] = (int)b->retired[i].second;
  }
  b->retired.erase(b->retired.begin(), b->retired.begin() + k);
  *n = k;
  return ETP_OK;
}

etp_status etp_batch_traj_info(etp_batch* b, const etp_traj* traj, int* steps_done, int* status, int* retired,
                               float* step_ms, int max_ms, int* n_ms) {
  if (!b || !traj) return fail(ETP_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(b->mu);
  auto f = b->info.find(traj);
  if (f == b->info.end()) return fail(ETP_ERR_INVALID, "trajectory was never admitted to this batch");
  const BatchInfo& inf = f->second;
  if (steps_done) *steps_done = inf.steps_done;
  if (status) *status = (int)inf.status;
  if (retired) *retired = inf.retired ? 1 : 0;
  const int k = std::min<int>(std::max(max_ms, 0), (int)inf.step_ms.size());
  if (step_ms)
    for (int i = 0; i < k; ++i) step_ms[i] = inf.step_ms[i];
  if (n_ms) *n_ms = step_ms ? k : (int)inf.step_ms.size();
  return ETP_OK;
}

etp_status etp_batch_forget(etp_batch* b, const etp_traj* traj) {
  if (!b || !traj) return fail(ETP_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(b->mu);
  auto f = b->info.find(traj);
  if (f == b->info.end() || !f->second.retired) return fail(ETP_ERR_INVALID, "trajectory is not retired");
  b->info.erase(f);
  return ETP_OK;
}

etp_status etp_batch_usage(etp_batch* b, size_t* reserved_bytes, int* n_active) {
  if (!b) return fail(ETP_ERR_INVALID, "null batch");
  std::lock_guard<std::mutex> lk(b->mu);
  if (reserved_bytes) *reserved_bytes = b->reserved;
  if (n_active) *n_active = (int)b->active.size();
  return ETP_OK;
}

}  // extern "C"
