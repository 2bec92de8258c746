// Autotuner of the smoother family per level size and precision.
//
// For square levels of a range of sides it builds a sine-warp operator with the library's
// own set-up kernels and times nu = 2 Gauss-Seidel sweeps with every family that can run
// there (per-colour kernels, fused tiles, pipelined tiles, row marching) in every variant
// of it (tile shape and sweeps per launch for the tile kernels, sweeps per pass for row
// marching; mg_tile.h), with CUDA events on the context's stream after a warm-up.  The
// fastest (family, variant) per size becomes the context's policy (SmoothPolicy), used by
// every V-cycle captured afterwards.  All of them perform the same operations per node in
// the same order, so the policy changes timings, not results.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "mg.h"
#include "mg_fused.h"
#include "mg_internal_host.h"
#include "mg_launch.h"
#include "mg_march.h"
#include "mg_pipe.h"
#include "mg_tile.h"
#include "mg_vcycle.h"

namespace mg {

static int pitch32(int n) { return (n + 31) & ~31; }

// Variants of a family for precision T (the per-colour kernels have one).
template <typename T>
static int variants_of(int kind) {
  switch (kind) {
    case SK_FUSED: return fused_variants<T>();
    case SK_PIPE: return pipe_variants<T>();
    case SK_MARCH: return march_variants<T>();
    default: return 1;
  }
}

template <typename T>
static SmoothVariant variant_of(int kind, int v) {
  switch (kind) {
    case SK_FUSED: return fused_variant<T>(v);
    case SK_PIPE: return pipe_variant<T>(v);
    case SK_MARCH: return march_variant<T>(v);
    default: return {0, 0, 1};
  }
}

// Time one family in one variant (ms per 2 sweeps); < 0 when it cannot run at this size.
template <typename T>
static float time_family(mg_ctx* ctx, int kind, int v, const Op<T>& A, T* x, T* x2, const T* b, int* err) {
  cudaStream_t s = ctx->stream;
  const int nyr = A.ny;
  const int ns = variant_of<T>(kind, v).ns;
  auto once = [&]() -> cudaError_t {
    cudaError_t e = cudaSuccess;
    switch (kind) {
      case SK_COLOUR:
        return launch_smooth<T>(A, x, b, 2, 0, nullptr, s);
      case SK_FUSED:
        for (int k = 0; k < 2 / ns && !e; ++k)
          e = launch_smooth_fused<T>(A, k & 1 ? x2 : x, k & 1 ? x : x2, b, 0, nullptr, 0, nullptr, s, v);
        return e;
      case SK_PIPE:
        for (int k = 0; k < 2 / ns && !e; ++k)
          e = launch_smooth_pipe<T>(A, k & 1 ? x2 : x, k & 1 ? x : x2, b, 0, nullptr, 0, nullptr, err, s, v);
        return e;
      case SK_MARCH:
        for (int k = 0; k < 2 / ns && !e; ++k)
          e = launch_smooth_march<T>(A, k & 1 ? x2 : x, k & 1 ? x : x2, b, 0, nullptr, 0, nullptr, s, v);
        return e;
    }
    return cudaErrorInvalidValue;
  };
  // the same applicability rules as the cycle
  if (kind != SK_COLOUR && 2 % ns) return -1.f;
  if (kind == SK_PIPE && (nyr < 64 || A.nx < 160)) return -1.f;
  if (kind == SK_MARCH && nyr < 128) return -1.f;
  for (int w = 0; w < 2; ++w)
    if (once() != cudaSuccess) return -1.f;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int reps = A.nx >= 2049 ? 5 : 20;
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps; ++r) once();
  cudaEventRecord(e1, s);
  float ms = -1.f;
  if (cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess) {
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

template <typename T>
static mg_status tune_size(mg_ctx* ctx, int n, float ms[4], int* best, int* best_var) {
  cudaStream_t s = ctx->stream;
  const int pt = pitch32(n);
  const size_t np = (size_t)pt * n;
  std::vector<void*> held;
  auto get = [&](size_t bytes) -> void* {
    void* q = ctx->pool.alloc(bytes);
    if (q) held.push_back(q);
    return q;
  };
  auto done = [&](mg_status st) {
    cudaStreamSynchronize(s);
    for (void* q : held) ctx->pool.release(q);
    return st;
  };
  double* f64 = (double*)get(10 * np * sizeof(double));
  int* flags = (int*)get(4 * sizeof(int));
  T* t = (T*)get(9 * np * sizeof(T));
  if (!f64 || !flags || !t) return done(set_error(MG_ERR_OOM, "mg_autotune: device memory budget exhausted at side %d", n));
  double *D = f64, *exx = f64 + np, *exy = f64 + 2 * np, *eyy = f64 + 3 * np;
  OpF64 A64{n, n, 0, pt, f64 + 4 * np, f64 + 5 * np, f64 + 6 * np, f64 + 7 * np, f64 + 8 * np, f64 + 9 * np};
  const double prm[4] = {0.1, 0.0, 0.0, 0.0};
  const double h = 1.0 / (n - 1);
  cudaMemsetAsync(f64, 0, 10 * np * sizeof(double), s);
  cudaMemsetAsync(t, 0, 9 * np * sizeof(T), s);
  cudaMemsetAsync(flags, 0, 4 * sizeof(int), s);
  if (launch_eps_analytic(MG_MAP_SINE_WARP, prm, n, n, 0, 0.0, 0.0, h, h, nullptr, pt, D, exx, exy, eyy, flags, s) ||
      launch_assemble(A64, h, h, exx, exy, eyy, s))
    return done(set_error(MG_ERR_CUDA, "mg_autotune: operator build failed"));
  Op<T> A;
  T *x = t + 6 * np, *x2 = t + 7 * np, *b = t + 8 * np;
  if constexpr (sizeof(T) == 4) {
    A = OpF32{n, n, 0, pt, t, t + np, t + 2 * np, t + 3 * np, t + 4 * np, t + 5 * np};
    if (launch_op_to_f32(A64, A, s)) return done(set_error(MG_ERR_CUDA, "mg_autotune: operator build failed"));
  } else {
    A = A64;
  }
  const int kinds[4] = {SK_COLOUR, SK_FUSED, SK_PIPE, SK_MARCH};
  *best = SK_DEFAULT;
  *best_var = -1;
  float bt = 1e30f;
  for (int k = 0; k < 4; ++k) {
    ms[k] = -1.f;  // the family's fastest variant
    for (int v = 0; v < variants_of<T>(kinds[k]); ++v) {
      const float t = time_family<T>(ctx, kinds[k], v, A, x, x2, b, flags + 2);
      if (t > 0.f && (ms[k] < 0.f || t < ms[k])) ms[k] = t;
      if (t > 0.f && t < bt) {
        bt = t;
        *best = kinds[k];
        *best_var = v;
      }
    }
  }
  cudaGetLastError();
  return done(MG_OK);
}

}  // namespace mg

using namespace mg;

extern "C" mg_status mg_autotune(mg_ctx* ctx, int max_side, mg_tune_report* report) {
  if (!ctx) return set_error(MG_ERR_ARG, "mg_autotune: ctx is NULL");
  if (max_side < 33) return set_error(MG_ERR_ARG, "mg_autotune: max_side must be at least 33");
  cudaSetDevice(ctx->device);
  if (report) memset(report, 0, sizeof(*report));
  SmoothPolicy pol[2];
  for (int prec = 0; prec < 2; ++prec) {
    for (int n = 33; n <= max_side && pol[prec].n < 16; n = 2 * n - 1) {
      float ms[4] = {-1.f, -1.f, -1.f, -1.f};
      int best = SK_DEFAULT, var = -1;
      const mg_status st =
          prec ? tune_size<float>(ctx, n, ms, &best, &var) : tune_size<double>(ctx, n, ms, &best, &var);
      if (st) return st;
      pol[prec].side[pol[prec].n] = n;
      pol[prec].kind[pol[prec].n] = best;
      pol[prec].var[pol[prec].n] = var;
      pol[prec].n++;
      if (report && report->count < MG_TUNE_MAX) {
        mg_tune_entry& e = report->entry[report->count++];
        e.precision = prec ? MG_PREC_MIXED : MG_PREC_FP64;
        e.side = n;
        for (int k = 0; k < 4; ++k) e.ms[k] = ms[k];
        e.choice = best;
        const SmoothVariant sv = prec ? variant_of<float>(best, var) : variant_of<double>(best, var);
        e.tile_x = sv.tx;
        e.tile_y = sv.ty;
        e.sweeps_per_launch = sv.ns;
      }
    }
  }
  // the new choice applies to every solve graph captured from now on: drop the captured ones
  cudaStreamSynchronize(ctx->stream);
  batch_cache_clear(ctx);
  {
    std::lock_guard<std::mutex> lk(ctx->problems_mu);
    for (mg_problem* P : ctx->problems) {
      for (auto& kv : P->graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        cudaGraphDestroy(kv.second.graph);
      }
      P->graphs.clear();
    }
  }
  ctx->pol[0] = pol[0];
  ctx->pol[1] = pol[1];
  ctx->tuned = 1;
  return MG_OK;
}
