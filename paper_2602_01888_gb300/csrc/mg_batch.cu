// Batched solves: every problem keeps its own resident hierarchy, solve state and
// captured solve graph; the graphs of a batch are launched together on the context's
// batch streams so independent problems overlap on the device.  A problem's result does
// not depend on the batch it runs in: it runs the same graph as mg_solve.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <set>
#include <vector>

#include "mg.h"
#include "mg_internal_host.h"

namespace mg {

mg_status batch_solve_impl(mg_ctx* ctx, int count, mg_problem* const* probs,
                           const double* const* rho, const double* const* bc, double* const* phi,
                           mg_mem_kind mem, const mg_solve_opts& o, mg_solve_stats* stats) {
  std::set<mg_problem*> seen;
  for (int k = 0; k < count; ++k) {
    if (!probs[k] || !rho[k] || !phi[k]) return set_error(MG_ERR_ARG, "batch entry %d: NULL argument", k);
    if (probs[k]->ctx != ctx) return set_error(MG_ERR_ARG, "batch entry %d: problem of another context", k);
    if (!seen.insert(probs[k]).second)
      return set_error(MG_ERR_ARG, "batch entry %d: the same problem appears twice", k);
    if (o.precision == MG_PREC_MIXED && !probs[k]->mixed)
      return set_error(MG_ERR_ARG, "batch entry %d: problem not set up for mixed precision", k);
    if (o.coarse_max != probs[k]->coarse_max)
      return set_error(MG_ERR_ARG, "batch entry %d: coarse_max differs from the problem's", k);
  }
  // the work of the context stream (set-up, earlier solves) comes first
  cudaEvent_t ready;
  if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess)
    return set_error(MG_ERR_CUDA, "event creation failed");
  cudaEventRecord(ready, ctx->stream);
  for (int s = 0; s < kBatchStreams; ++s) cudaStreamWaitEvent(ctx->batch[s], ready, 0);
  mg_status first = MG_OK;
  for (int k = 0; k < count && !first; ++k) {
    mg_problem* P = probs[k];
    cudaStream_t s = ctx->batch[k % kBatchStreams];
    const size_t n = (size_t)P->grid.nx * rows_stored(P->grid.ny, P->grid.periodic_y);
    const double *r = rho[k], *b = bc ? bc[k] : nullptr, *pin = phi[k];
    double* pout = phi[k];
    if (mem == MG_MEM_HOST) {
      if (!P->stage) {
        P->stage = (double*)ctx->pool.alloc(3 * n * sizeof(double));
        if (!P->stage) {
          first = set_error(MG_ERR_OOM, "device memory budget exhausted (staging)");
          break;
        }
        P->allocs.push_back(P->stage);
      }
      cudaMemcpyAsync(P->stage, r, n * sizeof(double), cudaMemcpyHostToDevice, s);
      if (b) cudaMemcpyAsync(P->stage + n, b, n * sizeof(double), cudaMemcpyHostToDevice, s);
      if (o.warm_start) cudaMemcpyAsync(P->stage + 2 * n, pin, n * sizeof(double), cudaMemcpyHostToDevice, s);
      r = P->stage;
      b = b ? P->stage + n : nullptr;
      pin = pout = P->stage + 2 * n;
    }
    first = enqueue_solve(P, o, r, b, pin, pout, s);
    if (!first && mem == MG_MEM_HOST)
      cudaMemcpyAsync(phi[k], pout, n * sizeof(double), cudaMemcpyDeviceToHost, s);
  }
  for (int s = 0; s < kBatchStreams; ++s) {
    cudaEventRecord(ready, ctx->batch[s]);
    cudaStreamWaitEvent(ctx->stream, ready, 0);
    cudaStreamSynchronize(ctx->batch[s]);
  }
  cudaEventDestroy(ready);
  if (first) return first;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(MG_ERR_CUDA, "batch: %s", cudaGetErrorString(e));
  mg_status worst = MG_OK;
  char msg[512] = "";
  for (int k = 0; k < count; ++k) {
    mg_status s = finish_solve(probs[k], stats ? &stats[k] : nullptr);
    if (s && !worst) {
      worst = s;
      snprintf(msg, sizeof msg, "batch entry %d: %s", k, mg_last_error());
    }
  }
  if (worst) return set_error(worst, "%s", msg);
  return MG_OK;
}

}  // namespace mg
