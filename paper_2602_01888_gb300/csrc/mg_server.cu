// Request server: a scheduler thread admits submitted solves while in-flight slots and
// the device-memory budget allow, gives each a resident hierarchy (reusing an idle one of
// the same grid when there is one), enqueues the coefficient build and the captured solve
// graph on a slot stream (so requests that arrive while others are on the GPU overlap with
// them), retires finished requests and records submit-to-result latency.  A request's
// result does not depend on what else is in flight or on which resident hierarchy it got:
// it runs the same kernels and graph as mg_setup_transform + mg_solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <cstdio>
#include <deque>
#include <iterator>
#include <list>
#include <string>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mg.h"
#include "mg_internal_host.h"

namespace mg {

using Clock = std::chrono::steady_clock;

// Completion query of a request.  Tests make it fail on the host (mgk_server_fail_event_queries):
// the next `n` queries report cudaErrorLaunchFailure instead of asking the runtime, so the
// failure path runs without any fault on the device.
static std::atomic<int> g_fail_queries{0};

static cudaError_t event_query(cudaEvent_t ev) {
  int n = g_fail_queries.load();
  while (n > 0)
    if (g_fail_queries.compare_exchange_weak(n, n - 1)) return cudaErrorLaunchFailure;
  return cudaEventQuery(ev);
}

struct Request {
  uint64_t ticket = 0;
  mg_grid_desc grid{};
  mg_map_desc map{};
  mg_solve_opts opts{};
  // page-locked arrays (nullptr when absent), carved from one block of the host pool
  double *xp = nullptr, *yp = nullptr, *eps = nullptr, *rho = nullptr, *bc = nullptr, *phi = nullptr;
  void* block = nullptr;
  Clock::time_point t_submit, t_done;
  mg_problem* prob = nullptr;
  int slot = -1;
  cudaEvent_t done_ev = nullptr;
  mg_status status = MG_OK;
  mg_solve_stats stats{};
  bool finished = false;
};

struct Server {
  mg_ctx* ctx = nullptr;
  mg_server_opts opts{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> pending;
  std::vector<std::shared_ptr<Request>> inflight;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> by_ticket;
  std::vector<cudaStream_t> slots;
  std::vector<int> slot_free;
  std::vector<double> lat_ms;
  Pool host;  // page-locked request buffers
  std::list<std::pair<std::string, mg_problem*>> idle;  // resident, least recently used first
  uint64_t next_ticket = 1, completed = 0, failed = 0, reused = 0, evicted = 0;
  double unknowns_done = 0.0;
  long long batch_sum = 0;
  int ticks = 0;
  size_t ctx_budget = 0;  // the context's device budget before the server lowered it
  bool stopping = false;
  std::thread th;
  Clock::time_point t_start;
  Clock::time_point t_last;
};

static size_t nodes_of(const mg_grid_desc& g) {
  return (size_t)g.nx * (size_t)(g.periodic_y ? g.ny - 1 : g.ny);
}

// Problems whose hierarchy fits a request of the same grid and options are kept resident
// after their request retires and are reused (coefficients rebuilt in place, captured
// solve graph replayed).  Idle ones are freed, least recently used first, only when a new
// hierarchy does not fit the memory budget.
static std::string shape_key(const mg_grid_desc& g, const mg_solve_opts& o) {
  char k[256];
  snprintf(k, sizeof k, "%d:%d:%d:%d:%.17g:%.17g:%.17g:%.17g:%d:%d:%d:%d", g.nx, g.ny, g.periodic_y,
           g.neumann_y, g.x0, g.y0, g.lx, g.ly, (int)o.precision, o.coarse_max, (int)o.outer,
           o.coarse_op);
  return k;
}

static mg_problem* take_idle(Server* S, const std::string& key) {
  for (auto it = S->idle.rbegin(); it != S->idle.rend(); ++it)
    if (it->first == key) {
      mg_problem* P = it->second;
      S->idle.erase(std::next(it).base());
      S->reused++;
      return P;
    }
  return nullptr;
}

static bool evict_idle(Server* S) {
  if (S->idle.empty()) return false;
  mg_problem_free(S->idle.front().second);
  S->idle.pop_front();
  S->evicted++;
  return true;
}

// Resident problem for R: an idle one of the same shape, else a new allocation (evicting
// idle problems while the budget is exhausted).  MG_ERR_OOM: nothing fits right now.
static mg_status acquire_problem(Server* S, Request* R, mg_problem** out) {
  const std::string key = shape_key(R->grid, R->opts);
  *out = take_idle(S, key);
  if (*out) return MG_OK;
  while (true) {
    mg_status st = problem_create(S->ctx, &R->grid, R->opts, out);
    if (st != MG_ERR_OOM || !evict_idle(S)) return st;
  }
}

// Admit, launch, retire; runs on the scheduler thread.
static void server_loop(Server* S) {
  cudaSetDevice(S->ctx->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    // admission: coefficient build and solve go onto the request's slot stream back to
    // back; the scheduler does not wait for either
    bool progressed = false;
    while (!S->pending.empty() && !S->slot_free.empty()) {
      auto R = S->pending.front();
      lk.unlock();
      mg_problem* P = nullptr;
      mg_status st = acquire_problem(S, R.get(), &P);
      lk.lock();
      if (st == MG_ERR_OOM && !S->inflight.empty()) break;  // wait for memory to free up
      S->pending.pop_front();
      progressed = true;
      if (st) {
        R->status = st;
        R->finished = true;
        R->t_done = Clock::now();
        S->failed++;
        S->cv_done.notify_all();
        continue;
      }
      R->prob = P;
      R->slot = S->slot_free.back();
      S->slot_free.pop_back();
      cudaStream_t s = S->slots[R->slot];
      const size_t n = nodes_of(R->grid);
      lk.unlock();
      if (!P->stage) {
        P->stage = (double*)S->ctx->pool.alloc(3 * n * sizeof(double));
        if (P->stage) P->allocs.push_back(P->stage);
      }
      st = P->stage ? MG_OK : set_error(MG_ERR_OOM, "server: no memory for the staging arrays");
      if (!st) {
        mg_map_desc m = R->map;
        m.xp = R->xp;
        m.yp = R->yp;
        st = problem_enqueue_build(P, &m, R->eps, MG_MEM_HOST, s);
      }
      if (!st) {
        cudaMemcpyAsync(P->stage, R->rho, n * sizeof(double), cudaMemcpyHostToDevice, s);
        if (R->bc) cudaMemcpyAsync(P->stage + n, R->bc, n * sizeof(double), cudaMemcpyHostToDevice, s);
        R->opts.warm_start = 0;
        st = enqueue_solve(P, R->opts, P->stage, R->bc ? P->stage + n : nullptr, P->stage + 2 * n,
                           P->stage + 2 * n, s);
      }
      if (!st) {
        cudaError_t e = cudaMemcpyAsync(R->phi, P->stage + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&R->done_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(R->done_ev, s);
        if (e != cudaSuccess) {
          if (R->done_ev) cudaEventDestroy(R->done_ev);
          R->done_ev = nullptr;
          st = set_error(MG_ERR_CUDA, "server: enqueue of request %llu: %s", (unsigned long long)R->ticket,
                         cudaGetErrorString(e));
        }
      }
      lk.lock();
      if (st) {
        R->status = st;
        R->finished = true;
        R->t_done = Clock::now();
        S->failed++;
        S->slot_free.push_back(R->slot);
        lk.unlock();
        cudaStreamSynchronize(s);
        mg_problem_free(R->prob);  // its state is unknown after a failed enqueue
        lk.lock();
        R->prob = nullptr;
        S->cv_done.notify_all();
        continue;
      }
      S->inflight.push_back(R);
    }
    if (!S->inflight.empty()) {
      S->ticks++;
      S->batch_sum += (long long)S->inflight.size();
    }
    // retire finished requests: cudaErrorNotReady keeps a request in flight; any other
    // error fails it (its slot is freed and its problem released, so stop still returns)
    for (size_t k = 0; k < S->inflight.size();) {
      auto R = S->inflight[k];
      const cudaError_t q = event_query(R->done_ev);
      if (q == cudaErrorNotReady) {
        ++k;
        continue;
      }
      mg_problem* P = R->prob;
      lk.unlock();
      mg_status st = MG_OK;
      if (q != cudaSuccess) {
        st = set_error(MG_ERR_CUDA, "server: completion of request %llu: %s",
                       (unsigned long long)R->ticket, cudaGetErrorString(q));
        cudaStreamSynchronize(S->slots[R->slot]);  // nothing of it may still run on its arrays
        mg_problem_free(P);                         // its state is unknown
        P = nullptr;
      } else {
        st = problem_check_build(P);
        if (!st) st = finish_solve(P, &R->stats);
      }
      cudaEventDestroy(R->done_ev);
      lk.lock();
      if (P) S->idle.emplace_back(shape_key(R->grid, R->opts), P);  // stays resident for reuse
      R->prob = nullptr;
      R->status = st;
      R->finished = true;
      R->t_done = Clock::now();
      S->t_last = R->t_done;
      S->lat_ms.push_back(std::chrono::duration<double, std::milli>(R->t_done - R->t_submit).count());
      if (st) S->failed++; else S->completed++;
      S->unknowns_done += (double)(R->grid.nx - 2) *
                          (double)(R->grid.periodic_y ? R->grid.ny - 1 : R->grid.neumann_y ? R->grid.ny : R->grid.ny - 2);
      S->slot_free.push_back(R->slot);
      S->inflight.erase(S->inflight.begin() + k);
      progressed = true;
      S->cv_done.notify_all();
    }
    if (S->stopping && S->pending.empty() && S->inflight.empty()) break;
    if (!progressed) {
      if (S->inflight.empty())
        S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
      else {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(50));
        lk.lock();
      }
    }
  }
  lk.unlock();
  for (auto& kv : S->idle) mg_problem_free(kv.second);
  S->idle.clear();
}

}  // namespace mg

using namespace mg;

struct mg_server {
  Server s;
};

extern "C" mg_status mg_server_start(mg_ctx* ctx, const mg_server_opts* opts, mg_server** out) {
  if (!ctx || !out) return set_error(MG_ERR_ARG, "mg_server_start: NULL argument");
  mg_server* h = new mg_server();
  Server* S = &h->s;
  S->ctx = ctx;
  if (opts) S->opts = *opts;
  if (S->opts.max_inflight <= 0) S->opts.max_inflight = 16;
  S->opts.max_inflight = std::min(S->opts.max_inflight, 64);
  if (S->opts.queue_capacity <= 0) S->opts.queue_capacity = 1 << 16;
  S->ctx_budget = ctx->pool.budget();
  if (S->opts.mem_budget && S->opts.mem_budget < S->ctx_budget) ctx->pool.set_budget(S->opts.mem_budget);
  S->host.pinned_ = true;
  S->host.budget_ = S->opts.host_budget ? S->opts.host_budget : ((size_t)8 << 30);
  cudaSetDevice(ctx->device);
  for (int k = 0; k < S->opts.max_inflight; ++k) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto x : S->slots) cudaStreamDestroy(x);
      delete h;
      return set_error(MG_ERR_CUDA, "mg_server_start: stream creation failed");
    }
    S->slots.push_back(s);
    S->slot_free.push_back(S->opts.max_inflight - 1 - k);
  }
  S->t_start = S->t_last = Clock::now();
  S->th = std::thread(server_loop, S);
  *out = h;
  return MG_OK;
}

extern "C" mg_status mg_serve_submit(mg_server* h, const mg_request* rq, uint64_t* ticket) {
  if (!h || !rq || !ticket || !rq->rho_phys) return set_error(MG_ERR_ARG, "mg_serve_submit: NULL argument");
  Server* S = &h->s;
  const mg_grid_desc& g = rq->grid;
  if (g.nx < 3 || g.ny < 3) return set_error(MG_ERR_SIZE, "mg_serve_submit: grid too small");
  mg_status cm = check_map(&g, &rq->map);
  if (cm) return cm;
  auto R = std::make_shared<Request>();
  R->grid = g;
  R->map = rq->map;
  R->opts = rq->opts;
  const size_t n = nodes_of(g);
  const bool grid_map = rq->map.kind == MG_MAP_GRID;
  const size_t arrays = 2 + (rq->bc ? 1 : 0) + (rq->eps_phys ? 1 : 0) + (grid_map ? 2 : 0);
  R->block = S->host.alloc(arrays * n * sizeof(double));
  if (!R->block)
    return set_error(MG_ERR_BUSY, "mg_serve_submit: host staging budget full (poll finished tickets)");
  double* cur = (double*)R->block;
  auto take = [&](const double* src) {
    double* d = cur;
    cur += n;
    if (src) memcpy(d, src, n * sizeof(double));
    return d;
  };
  R->rho = take(rq->rho_phys);
  R->phi = take(nullptr);
  if (rq->bc) R->bc = take(rq->bc);
  if (rq->eps_phys) R->eps = take(rq->eps_phys);
  if (grid_map) {
    R->xp = take(rq->map.xp);
    R->yp = take(rq->map.yp);
  }
  R->map.xp = R->map.yp = nullptr;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stopping || (int)S->pending.size() >= S->opts.queue_capacity) {
    S->host.release(R->block);
    if (S->stopping) return set_error(MG_ERR_BUSY, "mg_serve_submit: server is stopping");
    return set_error(MG_ERR_BUSY, "mg_serve_submit: queue full (%d pending)", (int)S->pending.size());
  }
  R->ticket = S->next_ticket++;
  R->t_submit = Clock::now();
  S->pending.push_back(R);
  S->by_ticket[R->ticket] = R;
  *ticket = R->ticket;
  S->cv_work.notify_all();
  return MG_OK;
}

extern "C" mg_status mg_serve_poll(mg_server* h, uint64_t ticket, int timeout_ms, double* phi_out,
                                   mg_solve_stats* stats) {
  if (!h) return set_error(MG_ERR_ARG, "mg_serve_poll: NULL server");
  Server* S = &h->s;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->by_ticket.find(ticket);
  if (it == S->by_ticket.end()) return set_error(MG_ERR_NOT_FOUND, "mg_serve_poll: unknown ticket %llu", (unsigned long long)ticket);
  auto R = it->second;
  if (!R->finished) {
    S->cv_done.wait_for(lk, std::chrono::milliseconds(std::max(timeout_ms, 0)), [&] { return R->finished; });
    if (!R->finished) return set_error(MG_ERR_TIMEOUT, "mg_serve_poll: ticket %llu not done", (unsigned long long)ticket);
  }
  S->by_ticket.erase(it);
  lk.unlock();
  if (phi_out && R->status == MG_OK) memcpy(phi_out, R->phi, nodes_of(R->grid) * sizeof(double));
  if (stats) *stats = R->stats;
  mg_status st = R->status;
  S->host.release(R->block);
  R->block = nullptr;
  if (st) return set_error(st, "mg_serve_poll: request %llu failed (status %d)", (unsigned long long)ticket, (int)st);
  return MG_OK;
}

extern "C" mg_status mg_server_stop(mg_server* h, mg_serve_report* rep) {
  if (!h) return set_error(MG_ERR_ARG, "mg_server_stop: NULL server");
  Server* S = &h->s;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
    S->cv_work.notify_all();
  }
  S->th.join();
  if (rep) {
    memset(rep, 0, sizeof(*rep));
    rep->completed = S->completed;
    rep->failed = S->failed;
    rep->wall_s = std::chrono::duration<double>(S->t_last - S->t_start).count();
    rep->unknowns_per_s = rep->wall_s > 0 ? S->unknowns_done / rep->wall_s : 0.0;
    std::vector<double> l = S->lat_ms;
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) {
      if (l.empty()) return 0.0;
      size_t k = (size_t)std::min<double>(l.size() - 1, std::ceil(q * l.size()) - 1);
      return l[k];
    };
    rep->p50_ms = pct(0.50);
    rep->p99_ms = pct(0.99);
    rep->max_ms = l.empty() ? 0.0 : l.back();
    rep->ticks = S->ticks;
    rep->mean_batch = S->ticks ? (double)S->batch_sum / S->ticks : 0.0;
    rep->reused = S->reused;
    rep->evicted = S->evicted;
  }
  for (auto s : S->slots) cudaStreamDestroy(s);
  S->ctx->pool.set_budget(S->ctx_budget);  // the context gets its own budget back
  delete h;
  return MG_OK;
}

extern "C" void mgk_server_fail_event_queries(int count) { g_fail_queries.store(count > 0 ? count : 0); }
