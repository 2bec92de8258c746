// Request server: a scheduler thread admits submitted solves while in-flight slots and
// the device-memory budget allow, builds each request's resident hierarchy, runs its
// captured solve graph on a slot stream (so requests that arrive while others are on
// the GPU overlap with them), retires finished requests and records submit-to-result
// latency.  A request's result does not depend on what else is in flight: it runs the
// same graph as mg_solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mg.h"
#include "mg_internal_host.h"

namespace mg {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  mg_grid_desc grid{};
  mg_map_desc map{};
  mg_solve_opts opts{};
  std::vector<double> xp, yp, eps, rho, bc, phi;
  bool has_eps = false, has_bc = false;
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
  uint64_t next_ticket = 1, completed = 0, failed = 0;
  double unknowns_done = 0.0;
  long long batch_sum = 0;
  int ticks = 0;
  bool stopping = false;
  std::thread th;
  Clock::time_point t_start;
  Clock::time_point t_last;
};

static size_t nodes_of(const mg_grid_desc& g) {
  return (size_t)g.nx * (size_t)(g.periodic_y ? g.ny - 1 : g.ny);
}

// Admit, launch, retire; runs on the scheduler thread.
static void server_loop(Server* S) {
  cudaSetDevice(S->ctx->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    // admission
    bool progressed = false;
    while (!S->pending.empty() && !S->slot_free.empty()) {
      auto R = S->pending.front();
      lk.unlock();
      mg_map_desc m = R->map;
      if (m.kind == MG_MAP_GRID) {
        m.xp = R->xp.data();
        m.yp = R->yp.data();
      }
      mg_problem* P = nullptr;
      mg_status st = mg_setup_transform(S->ctx, &R->grid, &m, R->has_eps ? R->eps.data() : nullptr,
                                        MG_MEM_HOST, &R->opts, &P);
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
      st = P->stage ? MG_OK : MG_ERR_OOM;
      if (!st) {
        cudaMemcpyAsync(P->stage, R->rho.data(), n * sizeof(double), cudaMemcpyHostToDevice, s);
        if (R->has_bc)
          cudaMemcpyAsync(P->stage + n, R->bc.data(), n * sizeof(double), cudaMemcpyHostToDevice, s);
        R->opts.warm_start = 0;
        st = enqueue_solve(P, R->opts, P->stage, R->has_bc ? P->stage + n : nullptr, P->stage + 2 * n,
                           P->stage + 2 * n, s);
      }
      if (!st) {
        cudaEventCreateWithFlags(&R->done_ev, cudaEventDisableTiming);
        cudaEventRecord(R->done_ev, s);
      }
      lk.lock();
      if (st) {
        R->status = st;
        R->finished = true;
        R->t_done = Clock::now();
        S->failed++;
        S->slot_free.push_back(R->slot);
        mg_problem_free(R->prob);
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
    // retire finished requests
    for (size_t k = 0; k < S->inflight.size();) {
      auto R = S->inflight[k];
      if (cudaEventQuery(R->done_ev) != cudaSuccess) {
        ++k;
        continue;
      }
      mg_problem* P = R->prob;
      const size_t n = nodes_of(R->grid);
      lk.unlock();
      R->phi.resize(n);
      cudaStream_t s = S->slots[R->slot];
      cudaMemcpyAsync(R->phi.data(), P->stage + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
      mg_status st = finish_solve(P, &R->stats);
      mg_problem_free(P);
      cudaEventDestroy(R->done_ev);
      lk.lock();
      R->prob = nullptr;
      R->status = st;
      R->finished = true;
      R->t_done = Clock::now();
      S->t_last = R->t_done;
      S->lat_ms.push_back(std::chrono::duration<double, std::milli>(R->t_done - R->t_submit).count());
      if (st) S->failed++; else S->completed++;
      S->unknowns_done += (double)(R->grid.nx - 2) *
                          (double)(R->grid.periodic_y ? R->grid.ny - 1 : R->grid.ny - 2);
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
  if (S->opts.mem_budget && S->opts.mem_budget < ctx->pool.budget_) ctx->pool.budget_ = S->opts.mem_budget;
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
  if (rq->map.kind == MG_MAP_GRID && (!rq->map.xp || !rq->map.yp))
    return set_error(MG_ERR_ARG, "mg_serve_submit: MG_MAP_GRID needs xp and yp");
  auto R = std::make_shared<Request>();
  R->grid = g;
  R->map = rq->map;
  R->opts = rq->opts;
  const size_t n = nodes_of(g);
  R->rho.assign(rq->rho_phys, rq->rho_phys + n);
  if (rq->bc) {
    R->bc.assign(rq->bc, rq->bc + n);
    R->has_bc = true;
  }
  if (rq->eps_phys) {
    R->eps.assign(rq->eps_phys, rq->eps_phys + n);
    R->has_eps = true;
  }
  if (rq->map.kind == MG_MAP_GRID) {
    R->xp.assign(rq->map.xp, rq->map.xp + n);
    R->yp.assign(rq->map.yp, rq->map.yp + n);
  }
  R->map.xp = R->map.yp = nullptr;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stopping) return set_error(MG_ERR_BUSY, "mg_serve_submit: server is stopping");
  if ((int)S->pending.size() >= S->opts.queue_capacity)
    return set_error(MG_ERR_BUSY, "mg_serve_submit: queue full (%d pending)", (int)S->pending.size());
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
  if (phi_out && !R->phi.empty()) memcpy(phi_out, R->phi.data(), R->phi.size() * sizeof(double));
  if (stats) *stats = R->stats;
  mg_status st = R->status;
  S->by_ticket.erase(it);
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
  }
  for (auto s : S->slots) cudaStreamDestroy(s);
  delete h;
  return MG_OK;
}
