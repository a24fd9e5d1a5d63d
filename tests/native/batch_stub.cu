// CPU check of the batch scheduler in csrc/batch.cu (test infrastructure).
//
// Links the real scheduler against a stub etp_step that only sleeps and
// records what it sees, so the host logic runs without a GPU: admission
// against the budget, every trajectory stepped exactly n_steps times, no two
// steps of one context at once, a failing trajectory retired alone with its
// status, tick counts, usage back to zero, clean shutdown. The ragged mode
// runs against a stub engine: one engine per context (never two ticks of one
// engine at once), every trajectory stepped exactly n_steps times, ticks of
// several trajectories, arrivals joining.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../paper_2405_05213_gb300/csrc/etp_host.cuh"

namespace etp {
etp_status fail(etp_status s, const std::string&) { return s; }
size_t mesh_device_bytes(const etp_mesh*) { return 1000; }
}  // namespace etp

static std::mutex g_mu;
static std::map<const etp_ctx*, int> g_in_flight;
static std::map<const etp_traj*, int> g_calls;
static std::atomic<int> g_violations{0};
static std::atomic<int> g_max_concurrent{0};
static std::atomic<int> g_concurrent{0};

extern "C" etp_status etp_step(etp_traj* t, double, double, int, int* m_out, double* err_out) {
  const etp_ctx* c = t->mesh->ctx;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_in_flight[c]++ != 0) g_violations++;
    g_calls[t]++;
  }
  const int now = ++g_concurrent;
  int prev = g_max_concurrent.load();
  while (now > prev && !g_max_concurrent.compare_exchange_weak(prev, now)) {}
  std::this_thread::sleep_for(std::chrono::microseconds(300 + 100 * (t->m_cap % 7)));
  --g_concurrent;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_in_flight[c]--;
  }
  if (m_out) *m_out = 1;
  if (err_out) *err_out = 0.0;
  return t->m_cap == 2 ? ETP_ERR_NOT_CONVERGED : ETP_OK;  // m_cap 2 stands for a solve that fails
}

// Stub of the ragged engine (batch_solve.cu): every tick finishes one step of
// every trajectory in it; m_cap 2 stands for a step that fails.
static std::atomic<int> g_batch_calls{0};   // ticks
static std::atomic<int> g_batch_max{0};     // most trajectories in one tick
static std::atomic<int> g_batch_overlap{0}; // ticks that ran at the same time
static std::atomic<int> g_batch_in_flight{0};

namespace etp {
struct RaggedEngine {
  etp_ctx* ctx;
  std::vector<std::pair<etp_traj*, int>> items;  // trajectory, steps left
};
RaggedEngine* ragged_engine_create(etp_ctx* ctx) { return new RaggedEngine{ctx, {}}; }
void ragged_engine_destroy(RaggedEngine* e) { delete e; }
bool ragged_engine_empty(const RaggedEngine* e) { return e->items.empty(); }
etp_status ragged_engine_add(RaggedEngine* e, etp_traj* t, double, double, int n_steps) {
  if (t->mesh->ctx != e->ctx || n_steps < 1) return ETP_ERR_INVALID;
  e->items.push_back({t, n_steps});
  return ETP_OK;
}
static std::map<const etp_ctx*, int> g_tick_in_flight;  // per context: ticks running now
static std::map<const etp_ctx*, int> g_ticks;           // per context: ticks run

etp_status ragged_engine_tick(RaggedEngine* e, std::vector<EngineEvent>* ev) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_tick_in_flight[e->ctx]++ != 0) g_batch_overlap++;  // two ticks of one engine at once
    g_ticks[e->ctx]++;
  }
  ++g_batch_in_flight;
  g_batch_calls++;
  const int n = (int)e->items.size();
  int prev = g_batch_max.load();
  while (n > prev && !g_batch_max.compare_exchange_weak(prev, n)) {}
  std::vector<std::pair<etp_traj*, int>> keep;
  for (auto& it : e->items) {
    if (it.first->mesh->ctx != e->ctx) g_violations++;
    {
      std::lock_guard<std::mutex> lk(g_mu);
      g_calls[it.first]++;
    }
    const etp_status st = it.first->m_cap == 2 ? ETP_ERR_NOT_CONVERGED : ETP_OK;
    const bool last = st != ETP_OK || it.second <= 1;
    ev->push_back(EngineEvent{it.first, st, etp_step_info{}, last});
    if (!last) keep.push_back({it.first, it.second - 1});
  }
  e->items.swap(keep);
  std::this_thread::sleep_for(std::chrono::microseconds(500));
  --g_batch_in_flight;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_tick_in_flight[e->ctx]--;
  }
  return ETP_OK;
}
}  // namespace etp

#define CHECK(x)                                                   \
  do {                                                             \
    if (!(x)) {                                                    \
      std::printf("FAIL line %d: %s\n", __LINE__, #x);             \
      return 1;                                                    \
    }                                                              \
  } while (0)

int main() {
  const int n_ctx = 3, n_traj = 7;
  std::vector<etp_ctx> ctxs(n_ctx);
  std::vector<etp_mesh> meshes(n_traj);
  std::vector<etp_traj> trajs(n_traj);
  for (int i = 0; i < n_traj; ++i) {
    meshes[i].ctx = &ctxs[i % n_ctx];  // several trajectories share a context
    trajs[i].mesh = &meshes[i];
    trajs[i].m_cap = 10 + i;
    trajs[i].device_bytes = 9000;      // + 1000 of mesh = 10,000 per trajectory
  }
  trajs[5].m_cap = 2;                  // fails at its first step
  etp_batch* b = nullptr;
  CHECK(etp_batch_create(&ctxs[0], 45000, 4, &b) == ETP_OK);
  const int steps[n_traj] = {5, 3, 8, 1, 6, 4, 2};
  int admitted = 0;
  for (int i = 0; i < 4; ++i) {
    CHECK(etp_batch_admit(b, &trajs[i], steps[i], 0.1, 1e-8) == ETP_OK);
    ++admitted;
  }
  CHECK(etp_batch_admit(b, &trajs[4], steps[4], 0.1, 1e-8) == ETP_ERR_OOM);  // 50,000 > 45,000
  CHECK(etp_batch_admit(b, &trajs[0], 1, 0.1, 1e-8) == ETP_ERR_INVALID);     // already admitted
  CHECK(etp_batch_admit(b, &trajs[4], 0, 0.1, 1e-8) == ETP_ERR_INVALID);     // no steps
  size_t reserved = 0;
  int n_active = 0;
  CHECK(etp_batch_usage(b, &reserved, &n_active) == ETP_OK && reserved == 40000 && n_active == 4);
  std::map<etp_traj*, int> retired;
  int total_ticked = 0, guard = 0;
  while ((int)retired.size() < n_traj && guard++ < 100000) {
    int n = 0;
    CHECK(etp_batch_tick(b, &n) == ETP_OK);
    total_ticked += n;
    etp_traj* out[8];
    int st[8], k = 0;
    CHECK(etp_batch_retired(b, out, st, 8, &k) == ETP_OK);
    for (int i = 0; i < k; ++i) retired[out[i]] = st[i];
    while (admitted < n_traj && etp_batch_admit(b, &trajs[admitted], steps[admitted], 0.1, 1e-8) == ETP_OK)
      ++admitted;
    CHECK(etp_batch_usage(b, &reserved, &n_active) == ETP_OK && reserved <= 45000);
  }
  CHECK((int)retired.size() == n_traj);
  int expect_ok_steps = 0;
  for (int i = 0; i < n_traj; ++i) {
    int sd = -1, status = -1, rt = -1, nms = -1;
    float ms[16];
    CHECK(etp_batch_traj_info(b, &trajs[i], &sd, &status, &rt, ms, 16, &nms) == ETP_OK);
    CHECK(rt == 1);
    if (i == 5) {
      CHECK(retired[&trajs[i]] == ETP_ERR_NOT_CONVERGED && status == ETP_ERR_NOT_CONVERGED && sd == 0);
      CHECK(g_calls[&trajs[i]] == 1 && nms == 1);
    } else {
      CHECK(retired[&trajs[i]] == ETP_OK && status == ETP_OK && sd == steps[i]);
      CHECK(g_calls[&trajs[i]] == steps[i] && nms == steps[i]);
      expect_ok_steps += steps[i];
    }
    CHECK(etp_batch_forget(b, &trajs[i]) == ETP_OK);
  }
  CHECK(total_ticked == expect_ok_steps);
  CHECK(etp_batch_usage(b, &reserved, &n_active) == ETP_OK && reserved == 0 && n_active == 0);
  CHECK(g_violations.load() == 0);
  CHECK(g_max_concurrent.load() >= 2 && g_max_concurrent.load() <= n_ctx);
  int n = -1;
  CHECK(etp_batch_tick(b, &n) == ETP_OK && n == 0);  // nothing admitted: returns at once
  etp_batch_destroy(b);

  // ---- ragged mode: all trajectories on one context, stepped in rounds
  g_calls.clear();
  std::vector<etp_mesh> rmeshes(n_traj);
  std::vector<etp_traj> rtrajs(n_traj);
  for (int i = 0; i < n_traj; ++i) {
    rmeshes[i].ctx = &ctxs[i % 2];  // two contexts: two engines
    rtrajs[i].mesh = &rmeshes[i];
    rtrajs[i].m_cap = 10 + i;
    rtrajs[i].device_bytes = 9000;
  }
  rtrajs[5].m_cap = 2;
  etp_batch* rb = nullptr;
  CHECK(etp_batch_create_ragged(&ctxs[0], 45000, &rb) == ETP_OK);
  int radmitted = 0;
  for (int i = 0; i < 4; ++i) {
    CHECK(etp_batch_admit(rb, &rtrajs[i], steps[i], 0.1, 1e-8) == ETP_OK);
    ++radmitted;
  }
  std::map<etp_traj*, int> rretired;
  guard = 0;
  while ((int)rretired.size() < n_traj && guard++ < 100000) {
    int n = 0;
    CHECK(etp_batch_tick(rb, &n) == ETP_OK);
    etp_traj* out[8];
    int st[8], k = 0;
    CHECK(etp_batch_retired(rb, out, st, 8, &k) == ETP_OK);
    for (int i = 0; i < k; ++i) rretired[out[i]] = st[i];
    while (radmitted < n_traj && etp_batch_admit(rb, &rtrajs[radmitted], steps[radmitted], 0.1, 1e-8) == ETP_OK)
      ++radmitted;
  }
  CHECK((int)rretired.size() == n_traj);
  for (int i = 0; i < n_traj; ++i) {
    int sd = -1, status = -1, rt = -1, nms = -1;
    CHECK(etp_batch_traj_info(rb, &rtrajs[i], &sd, &status, &rt, nullptr, 0, &nms) == ETP_OK);
    if (i == 5) {
      CHECK(rretired[&rtrajs[i]] == ETP_ERR_NOT_CONVERGED && sd == 0 && g_calls[&rtrajs[i]] == 1);
    } else {
      CHECK(rretired[&rtrajs[i]] == ETP_OK && sd == steps[i] && g_calls[&rtrajs[i]] == steps[i] && nms == steps[i]);
    }
  }
  CHECK(etp_batch_usage(rb, &reserved, &n_active) == ETP_OK && reserved == 0 && n_active == 0);
  CHECK(g_batch_max.load() >= 2 && g_batch_overlap.load() == 0 && g_violations.load() == 0);
  CHECK(etp::g_ticks[&ctxs[0]] > 0 && etp::g_ticks[&ctxs[1]] > 0);  // each context ran in its own engine
  etp_batch_destroy(rb);
  std::printf("OK max_concurrent=%d ragged_ticks=%d max_tick=%d\n", g_max_concurrent.load(), g_batch_calls.load(),
              g_batch_max.load());
  return 0;
}
