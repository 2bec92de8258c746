// Batched solves (mg_batch_solve): independent resident problems of different sizes and
// geometries solved by ONE graph launch.  The batch graph holds, for every problem, its own
// solve chain (initialisation, device-driven WHILE loop of outer iterations, copy-out) as
// an independent branch from a common root, so the instances run concurrently and each
// stops on its own convergence test; a final kernel gathers all solve states for one
// device-to-host copy.  The per-solve arguments of all instances live in one device array
// (one host-to-device copy per batch).  The graph is captured once per (problem list,
// options) and replayed; a problem's result is bitwise the same as with mg_solve, since
// its branch runs the same kernels on the same data in the same order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <set>
#include <mutex>
#include <string>
#include <vector>

#include "mg.h"
#include "mg_internal_host.h"

namespace mg {

static void entry_free(mg_ctx* ctx, BatchEntry* b) {
  if (b->ge.exec) cudaGraphExecDestroy(b->ge.exec);
  if (b->ge.graph) cudaGraphDestroy(b->ge.graph);
  for (void* a : b->allocs) ctx->pool.release(a);
  if (b->h_args) cudaFreeHost(b->h_args);
  if (b->h_states) cudaFreeHost(b->h_states);
  if (b->h_flags) cudaFreeHost(b->h_flags);
  delete b;
}

void batch_cache_clear(mg_ctx* ctx) {
  std::lock_guard<std::mutex> lk(ctx->batches_mu);
  for (auto& kv : ctx->batches) entry_free(ctx, kv.second);
  ctx->batches.clear();
}

void batch_cache_drop(mg_ctx* ctx, const mg_problem* P) {
  std::lock_guard<std::mutex> lk(ctx->batches_mu);
  for (auto it = ctx->batches.begin(); it != ctx->batches.end();) {
    const auto& pr = it->second->probs;
    if (std::find(pr.begin(), pr.end(), P) != pr.end()) {
      entry_free(ctx, it->second);
      it = ctx->batches.erase(it);
    } else {
      ++it;
    }
  }
}

static std::string batch_key(mg_problem* const* probs, int count, const mg_solve_opts& o) {
  std::string k;
  k.reserve((size_t)count * sizeof(void*) + 16);
  const uint64_t g = graph_key(o);
  k.append(reinterpret_cast<const char*>(&g), sizeof g);
  for (int i = 0; i < count; ++i) k.append(reinterpret_cast<const char*>(&probs[i]), sizeof(void*));
  return k;
}

static mg_status make_entry(mg_ctx* ctx, mg_problem* const* probs, int count, const mg_solve_opts& o,
                            BatchEntry** out) {
  BatchEntry* b = new BatchEntry();
  b->probs.assign(probs, probs + count);
  auto alloc = [&](size_t bytes) -> void* {
    void* p = ctx->pool.alloc(bytes);
    if (p) b->allocs.push_back(p);
    return p;
  };
  b->d_args = (SolveArgs*)alloc(sizeof(SolveArgs) * count);
  b->d_states = (SolveState*)alloc(sizeof(SolveState) * count);
  b->d_flags = (int*)alloc(sizeof(int) * 4 * count);
  b->d_src = (SolveState**)alloc(sizeof(SolveState*) * count);
  b->d_srcflags = (int**)alloc(sizeof(int*) * count);
  mg_status st = MG_OK;
  if (!b->d_args || !b->d_states || !b->d_flags || !b->d_src || !b->d_srcflags)
    st = set_error(MG_ERR_OOM, "device memory budget exhausted (batch arrays)");
  if (!st && (cudaMallocHost(&b->h_args, sizeof(SolveArgs) * count) != cudaSuccess ||
              cudaMallocHost(&b->h_states, sizeof(SolveState) * count) != cudaSuccess ||
              cudaMallocHost(&b->h_flags, sizeof(int) * 4 * count) != cudaSuccess))
    st = set_error(MG_ERR_CUDA, "pinned host allocation failed (batch)");
  if (!st) {
    std::vector<SolveState*> src(count);
    std::vector<int*> srcf(count);
    for (int k = 0; k < count; ++k) {
      src[k] = probs[k]->st;
      srcf[k] = probs[k]->flags;
    }
    if (cudaMemcpy(b->d_src, src.data(), sizeof(void*) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_srcflags, srcf.data(), sizeof(void*) * count, cudaMemcpyHostToDevice) !=
            cudaSuccess)
      st = set_error(MG_ERR_CUDA, "batch pointer tables: copy failed");
  }
  if (!st)
    st = build_batch_graph(ctx, probs, count, o, b->d_args, b->d_src, b->d_srcflags, b->d_states,
                           b->d_flags, &b->ge, &b->fixed, &b->body);
  if (st) {
    for (void* a : b->allocs) ctx->pool.release(a);
    if (b->h_args) cudaFreeHost(b->h_args);
    if (b->h_states) cudaFreeHost(b->h_states);
    if (b->h_flags) cudaFreeHost(b->h_flags);
    delete b;
    return st;
  }
  *out = b;
  return MG_OK;
}

mg_status batch_solve_impl(mg_ctx* ctx, int count, mg_problem* const* probs,
                           const double* const* rho, const double* const* bc, double* const* phi,
                           mg_mem_kind mem, const mg_solve_opts& o, mg_solve_stats* stats) {
  if (count == 0) return MG_OK;
  std::set<mg_problem*> seen;
  for (int k = 0; k < count; ++k) {
    if (!probs[k] || !rho[k] || !phi[k]) return set_error(MG_ERR_ARG, "batch entry %d: NULL argument", k);
    if (probs[k]->ctx != ctx) return set_error(MG_ERR_ARG, "batch entry %d: problem of another context", k);
    if (!seen.insert(probs[k]).second)
      return set_error(MG_ERR_ARG, "batch entry %d: the same problem appears twice", k);
    mg_status st = check_opts(probs[k], o);
    if (st) {
      char msg[512];
      snprintf(msg, sizeof msg, "%s", mg_last_error());
      return set_error(st, "batch entry %d: %s", k, msg);
    }
    if (o.smoother == MG_SMOOTH_XLINE && (st = line_prepare(probs[k], ctx->stream)))
      return st;
  }
  const std::string key = batch_key(probs, count, o);
  // held until the batch has run: a problem freed meanwhile on another thread (the server's
  // eviction) cannot destroy an entry in use
  std::lock_guard<std::mutex> batches_lock(ctx->batches_mu);
  BatchEntry* b = nullptr;
  auto it = ctx->batches.find(key);
  if (it != ctx->batches.end()) {
    b = it->second;
  } else {
    mg_status st = make_entry(ctx, probs, count, o, &b);
    if (st) return st;
    ctx->batches[key] = b;
  }
  cudaStream_t s = ctx->stream;
  for (int k = 0; k < count; ++k) {
    mg_problem* P = probs[k];
    const size_t n = (size_t)P->user.nx * rows_stored(P->user.ny, P->user.periodic_y);
    const double *r = rho[k], *bcv = bc ? bc[k] : nullptr, *pin = phi[k];
    double* pout = phi[k];
    if (mem == MG_MEM_HOST) {
      if (!P->stage) {
        P->stage = (double*)ctx->pool.alloc(3 * n * sizeof(double));
        if (!P->stage) return set_error(MG_ERR_OOM, "device memory budget exhausted (staging)");
        P->allocs.push_back(P->stage);
      }
      if (cudaMemcpyAsync(P->stage, r, n * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
          (bcv && cudaMemcpyAsync(P->stage + n, bcv, n * sizeof(double), cudaMemcpyHostToDevice, s) !=
                      cudaSuccess) ||
          (o.warm_start &&
           cudaMemcpyAsync(P->stage + 2 * n, pin, n * sizeof(double), cudaMemcpyHostToDevice, s) !=
               cudaSuccess))
        return set_error(MG_ERR_CUDA, "batch entry %d: input copy failed", k);
      r = P->stage;
      bcv = bcv ? P->stage + n : nullptr;
      pin = pout = P->stage + 2 * n;
    }
    SolveArgs& a = b->h_args[k];
    a.rho = r;
    a.bc = bcv;
    a.phi_in = pin;
    a.phi_out = pout;
    a.user_pitch = P->grid.nx;
    a.mirror = P->mirror;
    a.warm = o.warm_start ? 1 : 0;
    a.max_iters = o.max_iters;
    a.rtol = o.rtol;
    a.n_unknowns = (long long)coarse_unknowns(P->grid.nx, P->grid.ny, P->grid.periodic_y);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  mg_status st = MG_OK;
  if (cudaMemcpyAsync(b->d_args, b->h_args, sizeof(SolveArgs) * count, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaEventRecord(e0, s) != cudaSuccess || cudaGraphLaunch(b->ge.exec, s) != cudaSuccess ||
      cudaEventRecord(e1, s) != cudaSuccess ||
      cudaMemcpyAsync(b->h_states, b->d_states, sizeof(SolveState) * count, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(b->h_flags, b->d_flags, sizeof(int) * 4 * count, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess)
    st = set_error(MG_ERR_CUDA, "batch launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  if (!st && mem == MG_MEM_HOST) {
    for (int k = 0; k < count; ++k) {
      mg_problem* P = probs[k];
      const size_t n = (size_t)P->user.nx * rows_stored(P->user.ny, P->user.periodic_y);
      if (cudaMemcpyAsync(phi[k], P->stage + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess) {
        st = set_error(MG_ERR_CUDA, "batch entry %d: result copy failed", k);
        break;
      }
    }
  }
  if (cudaStreamSynchronize(s) != cudaSuccess && !st)
    st = set_error(MG_ERR_CUDA, "batch: %s", cudaGetErrorString(cudaGetLastError()));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  mg_status worst = MG_OK;
  char msg[512] = "";
  for (int k = 0; k < count; ++k) {
    probs[k]->last_fixed_kernels = b->fixed[k];
    probs[k]->last_body_kernels = b->body[k];
    mg_status s2 = finish_from(probs[k], b->h_states[k], b->h_flags + 4 * k, stats ? &stats[k] : nullptr, ms);
    if (s2 && !worst) {
      worst = s2;
      snprintf(msg, sizeof msg, "batch entry %d: %s", k, mg_last_error());
    }
  }
  if (worst) return set_error(worst, "%s", msg);
  return MG_OK;
}

}  // namespace mg
