// Solve-loop kernels on the finest level (FP64): initialisation, residual norms and the
// convergence test (stopping rule ||r|| / ||r_0|| <= rtol, Sec. 3 "repeated until
// convergence"), flexible conjugate-gradient updates around the multigrid
// preconditioner, and the FP32 <-> FP64 hand-over of iterative refinement.
//
// Reductions are deterministic: every block writes one partial sum (fixed-order tree),
// and the last block to finish sums the partials in index order.  Node loops use a grid
// of at most kRedBlocks blocks that strides over the rows.
#include <cuda_runtime.h>

#include "mg_common.cuh"
#include "mg_launch.h"
#include "mg_solve_kernels.h"

namespace mg {

constexpr int kNT = kRedThreads;
// kRedBlocks over the 152 SMs: a loop with at most 32 registers a thread runs in one wave.
constexpr int kRedBlocksPerSM = 8;
constexpr int kMaxVerifyFail = 4;

#define NODE_LOOP(L)                                                            \
  for (int j = blockIdx.y; j < (L).nyr; j += gridDim.y)                         \
    for (int i = blockIdx.x * kNT + threadIdx.x; i < (L).nx; i += gridDim.x * kNT)

// Elementwise loops that move few bytes per node, over the rows of one column (red_grid covers
// every column: grids wider than kRedBlocks x kNT are rejected at set-up), B rows at a time:
// load(u, j) fills slot u from row j (clamped into range, so the loads need no guard and all
// of a batch's loads are in flight together), then use(u, j) consumes the slots of the rows
// that exist, in increasing row order (the order of NODE_LOOP, so sums come out identical).
// With about two hundred rows per thread, one row's loads at a time leave these loops bound
// by load latency.
template <int B, typename Load, typename Use>
__device__ __forceinline__ void rows_batched(int nyr, Load load, Use use) {
  const int g = gridDim.y;
  for (int j0 = blockIdx.y; j0 < nyr; j0 += B * g) {
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int j = j0 + u * g;
      load(u, j < nyr ? j : j0);
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int j = j0 + u * g;
      if (j < nyr) use(u, j);
    }
  }
}

__device__ __forceinline__ unsigned nblocks() { return gridDim.x * gridDim.y; }
__device__ __forceinline__ unsigned bid() { return blockIdx.y * gridDim.x + blockIdx.x; }

// Convergence decision, run by one thread of the last block.
// recursive != 0: rr comes from the recursively updated CG residual; meeting rtol then
// only requests a check of the true residual (residual replacement) in the next pass.
// Scaling between the FP64 residual and the FP32 cycle by a power of two s (the factor
// that brings the residual's rms to [1, 2)).  Multiplying by s in FP32 on the FP32 side of
// the conversion is exact and gives the same value as multiplying in FP64, except for
// entries so far below the rms that they leave the FP32 normal range on one side of the
// conversion (more than 2^60 below it while |log2 s| <= 60), far under FP32 resolution of
// the vector.  It keeps the multiply off the FP64 pipe (GB300 runs FP64 at 1/62 of the
// FP32 rate).
__device__ __forceinline__ bool pow2_fits_f32(double s) { return s >= 0x1p-60 && s <= 0x1p60; }
__device__ __forceinline__ float to_f32_scaled(double v, double s, bool f32ok) {
  return f32ok ? (float)v * (float)s : (float)(v * s);
}
__device__ __forceinline__ double from_f32_scaled(float v, double s, bool f32ok) {
  return f32ok ? (double)(v * (float)s) : s * (double)v;
}

__device__ void decide(SolveState* st, double rr, cudaGraphConditionalHandle h, int has_h,
                       int recursive = 0) {
  const double rel = sqrt(rr) / st->r0;
  st->rr = rr;
  st->rel = rel;
  if (st->hist_n < 256) st->hist[st->hist_n] = rel;
  st->hist_n += 1;
  int done = 0;
  if (!(rel < 1e30)) {  // NaN or Inf
    st->status = 7;
    done = 1;
  } else if (rel <= st->rtol) {
    st->status = 0;
    if (recursive) st->verify = 1; else done = 1;
  } else if (st->it >= st->max_iters) {
    st->status = 6;
    done = 1;
  }
  // power-of-two scaling that brings the rms of r to [1, 2) before the FP32 cycle
  const double rms = sqrt(rr / (double)st->n_unknowns);
  if (rms > 0.0 && rms < 1e300) {
    const int e = ilogb(rms);
    st->scale = ldexp(1.0, -e);
    st->inv_scale = ldexp(1.0, e);
  } else {
    st->scale = st->inv_scale = 1.0;
  }
  st->done = done;
  if (has_h) cudaGraphSetConditional(h, done ? 0u : 1u);
}

// x: Dirichlet ring from bc (or 0), unknowns from the warm start (or 0); b = rho' D (Eq. 11).
__global__ void __launch_bounds__(kNT) k_solve_init(Lvl<double> L, const SolveArgs* __restrict__ a,
                                                    const double* __restrict__ D,
                                                    double* __restrict__ x, double* __restrict__ b,
                                                    SolveState* st) {
  const int up = a->user_pitch, n = a->mirror;
  NODE_LOOP(L) {
    // caller row of this node: itself, or through the even reflection of a Neumann grid
    const int jr = n == 0 ? j : (j >= n ? j - n : n - j);
    const size_t k = (size_t)j * L.pitch + i, u = (size_t)jr * up + i;
    if (is_unknown(L, i, j)) {
      x[k] = a->warm ? a->phi_in[u] : 0.0;
      b[k] = a->rho[u] * D[k];
    } else {
      x[k] = a->bc ? a->bc[u] : 0.0;
      b[k] = 0.0;
    }
  }
  if (bid() == 0 && threadIdx.x == 0) {
    st->it = 0;
    st->done = 0;
    st->status = 0;
    st->hist_n = 0;
    st->verify = 0;
    st->guard = 0;
    st->verify_fail = 0;
    st->x_zero = (!a->warm && a->bc == nullptr) ? 1 : 0;
    st->rtol = a->rtol;
    st->max_iters = a->max_iters;
    st->beta = 0.0;
    st->pq_old = 0.0;
    st->scale = st->inv_scale = 1.0;
    st->n_unknowns = a->n_unknowns;
  }
}

// r = b - A x (written when r != nullptr), ||r||^2 and the reference ||r_0||^2 with the
// unknowns set to zero; the last block sets r0, decides, and sets the graph condition.
__global__ void __launch_bounds__(kNT) k_resid_init(Lvl<double> L, const double* __restrict__ x,
                                                    const double* __restrict__ b,
                                                    double* __restrict__ r, SolveState* st,
                                                    double* part, cudaGraphConditionalHandle h,
                                                    int has_h) {
  __shared__ double sh[kNT / 32];
  __shared__ int flag;
  double s_rr = 0.0, s_r0 = 0.0;
  // a zero iterate (no Dirichlet data, cold start) has r = r_0 = b: every product of the
  // stencil is a zero, so skipping it gives the same values
  const bool xz = st->x_zero != 0;
  NODE_LOOP(L) {
    const size_t k = (size_t)j * L.pitch + i;
    double rv = 0.0;
    if (xz) {
      if (is_unknown(L, i, j)) {
        rv = b[k];
        s_r0 += rv * rv;
        s_rr += rv * rv;
      }
      if (r) r[k] = rv;
      continue;
    }
    if (is_unknown(L, i, j)) {
      rv = b[k] - fma(L.diag[k], x[k], offdiag(L, x, i, j));
      // residual of the same ring with zero unknowns: only Dirichlet neighbours count
      const int jd = row_dn(j, L.nyr), ju = row_up(j, L.nyr);
      const size_t r0 = (size_t)j * L.pitch, rd = (size_t)jd * L.pitch, ru = (size_t)ju * L.pitch;
      double t = 0.0;
      if (!is_unknown(L, i + 1, j)) t += L.cE[r0 + i] * x[r0 + i + 1];
      if (!is_unknown(L, i - 1, j)) t += L.cE[r0 + i - 1] * x[r0 + i - 1];
      if (!is_unknown(L, i, ju)) t += L.cN[r0 + i] * x[ru + i];
      if (!is_unknown(L, i, jd)) t += L.cN[rd + i] * x[rd + i];
      if (!is_unknown(L, i + 1, ju)) t += L.cNE[r0 + i] * x[ru + i + 1];
      if (!is_unknown(L, i - 1, jd)) t += L.cNE[rd + i - 1] * x[rd + i - 1];
      if (!is_unknown(L, i - 1, ju)) t += L.cNW[r0 + i] * x[ru + i - 1];
      if (!is_unknown(L, i + 1, jd)) t += L.cNW[rd + i + 1] * x[rd + i + 1];
      const double z = b[k] - t;
      s_r0 += z * z;
      s_rr += rv * rv;
    }
    if (r) r[k] = rv;
  }
  const double a0 = block_sum<kNT>(s_rr, sh);
  const double a1 = block_sum<kNT>(s_r0, sh);
  if (threadIdx.x == 0) {
    part[bid()] = a0;
    part[nblocks() + bid()] = a1;
  }
  if (last_block_arrival(&st->ticket[0], nblocks(), &flag)) {
    const double rr = reduce_partials<kNT>(part, nblocks(), sh);
    const double q0 = reduce_partials<kNT>(part + nblocks(), nblocks(), sh);
    if (threadIdx.x == 0) {
      st->r0 = (q0 > 0.0) ? sqrt(q0) : 1.0;
      decide(st, rr, h, has_h);
    }
  }
}

// ||b - A x||^2 for the plain-cycle loop; optional r output; the last block decides.
__global__ void __launch_bounds__(kNT) k_resid_check(Lvl<double> L, const double* __restrict__ x,
                                                     const double* __restrict__ b,
                                                     double* __restrict__ r, SolveState* st,
                                                     double* part, cudaGraphConditionalHandle h,
                                                     int has_h) {
  __shared__ double sh[kNT / 32];
  __shared__ int flag;
  double s = 0.0;
  NODE_LOOP(L) {
    const size_t k = (size_t)j * L.pitch + i;
    double rv = 0.0;
    if (is_unknown(L, i, j)) {
      rv = b[k] - fma(L.diag[k], x[k], offdiag(L, x, i, j));
      s += rv * rv;
    }
    if (r) r[k] = rv;
  }
  const double a0 = block_sum<kNT>(s, sh);
  if (threadIdx.x == 0) part[bid()] = a0;
  if (last_block_arrival(&st->ticket[1], nblocks(), &flag)) {
    const double rr = reduce_partials<kNT>(part, nblocks(), sh);
    if (threadIdx.x == 0) decide(st, rr, h, has_h);
  }
}

// b32 = fp32(r * scale) (scale: power of two from the last decision).
__global__ void __launch_bounds__(kNT) k_r_to_f32(Lvl<double> L, const double* __restrict__ r,
                                                  float* __restrict__ b32, int pitch32,
                                                  SolveState* st) {
  if (st->done) return;
  const double sc = st->scale;
  const bool f32ok = pow2_fits_f32(sc);
  NODE_LOOP(L) { b32[(size_t)j * pitch32 + i] = to_f32_scaled(r[(size_t)j * L.pitch + i], sc, f32ok); }
  if (bid() == 0 && threadIdx.x == 0) st->inv_scale_r32 = st->inv_scale;
}

// Plain-cycle refinement step: x += inv_scale * e32 at unknowns; iteration counter.
__global__ void __launch_bounds__(kNT) k_add_f32(Lvl<double> L, double* __restrict__ x,
                                                 const float* __restrict__ e32, int pitch32,
                                                 SolveState* st) {
  if (st->done) return;
  const double is = st->inv_scale_r32;
  const bool f32ok = pow2_fits_f32(is);
  NODE_LOOP(L) {
    if (is_unknown(L, i, j))
      x[(size_t)j * L.pitch + i] += from_f32_scaled(e32[(size_t)j * pitch32 + i], is, f32ok);
  }
}

// Last node of every loop body: counts passes and ends the loop after 2 max_iters + 8
// of them even if no convergence decision was reached (status: not converged).
__global__ void k_loop_guard(SolveState* st, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->guard += 1;
  if (!st->done && st->guard > 2 * st->max_iters + 8) {
    st->done = 1;
    st->status = 6;
    cudaGraphSetConditional(h, 0u);
  }
}

__global__ void k_iter_inc(SolveState* st) {
  if (!st->done && threadIdx.x == 0 && blockIdx.x == 0) st->it += 1;
}

// ---- flexible CG (FCG(1)): p = z + beta p_old, beta = -(z . q_old) / (p_old . q_old);
// alpha = (p . r) / (p . q); x += alpha p; r -= alpha q.
template <typename TZ>
__global__ void __launch_bounds__(kNT, kRedBlocksPerSM) k_fcg_zq(Lvl<double> L, const TZ* __restrict__ z, int zp,
                                                const double* __restrict__ q, SolveState* st,
                                                double* part) {
  if (st->done || st->it == 0) {
    if (!st->done && bid() == 0 && threadIdx.x == 0) st->beta = 0.0;
    return;
  }
  __shared__ double sh[kNT / 32];
  __shared__ int flag;
  const double is = (sizeof(TZ) == 4) ? st->inv_scale_r32 : 1.0;
  const bool f32ok = pow2_fits_f32(is);
  double s = 0.0;
  const int i = blockIdx.x * kNT + threadIdx.x;
  if (i < L.nx) {
    TZ zv[4];
    double qv[4];
    rows_batched<4>(
        L.nyr,
        [&](int u, int j) {
          zv[u] = z[(size_t)j * zp + i];
          qv[u] = q[(size_t)j * L.pitch + i];
        },
        [&](int u, int j) {
          if (is_unknown(L, i, j))
            s += (sizeof(TZ) == 4 ? from_f32_scaled((float)zv[u], is, f32ok) : (double)zv[u]) * qv[u];
        });
  }
  const double a0 = block_sum<kNT>(s, sh);
  if (threadIdx.x == 0) part[bid()] = a0;
  if (last_block_arrival(&st->ticket[2], nblocks(), &flag)) {
    const double zq = reduce_partials<kNT>(part, nblocks(), sh);
    if (threadIdx.x == 0) {
      st->zq = zq;
      st->beta = (st->pq_old != 0.0) ? -zq / st->pq_old : 0.0;
    }
  }
}

// p = z + beta p_old and q = A p computed as q = A z + beta q_old (q_old = A p_old), so
// the stencil only reads z and every other array is updated elementwise in place;
// partial sums of p.q and p.r; the last block sets alpha = (p.r) / (p.q).
template <typename TZ>
__global__ void __launch_bounds__(kNT) k_fcg_pq(Lvl<double> L, const TZ* __restrict__ z, int zp,
                                                double* __restrict__ p, double* __restrict__ q,
                                                const double* __restrict__ r, SolveState* st,
                                                double* part) {
  if (st->done) return;
  __shared__ double sh[kNT / 32];
  __shared__ int flag;
  const double is = (sizeof(TZ) == 4) ? st->inv_scale_r32 : 1.0;
  const double beta = st->beta;
  const bool first = (st->it == 0);
  double spq = 0.0, spr = 0.0;
  NODE_LOOP(L) {
    if (!is_unknown(L, i, j)) continue;
    const size_t k = (size_t)j * L.pitch + i;
    const int jd = row_dn(j, L.nyr), ju = row_up(j, L.nyr);
    const size_t r0 = (size_t)j * zp, rd = (size_t)jd * zp, ru = (size_t)ju * zp;
    const size_t c0 = (size_t)j * L.pitch, cd = (size_t)jd * L.pitch;
    double az = L.cE[c0 + i] * (double)z[r0 + i + 1];
    az = fma(L.cE[c0 + i - 1], (double)z[r0 + i - 1], az);
    az = fma(L.cN[c0 + i], (double)z[ru + i], az);
    az = fma(L.cN[cd + i], (double)z[rd + i], az);
    if (!L.five_point) {
      az = fma(L.cNE[c0 + i], (double)z[ru + i + 1], az);
      az = fma(L.cNE[cd + i - 1], (double)z[rd + i - 1], az);
      az = fma(L.cNW[c0 + i], (double)z[ru + i - 1], az);
      az = fma(L.cNW[cd + i + 1], (double)z[rd + i + 1], az);
    }
    az = fma(L.diag[k], (double)z[r0 + i], az);
    const double zz = is * (double)z[r0 + i];
    const double pn = first ? zz : fma(beta, p[k], zz);
    const double qn = first ? is * az : fma(beta, q[k], is * az);
    p[k] = pn;
    q[k] = qn;
    spq = fma(pn, qn, spq);
    spr = fma(pn, r[k], spr);
  }
  const double a0 = block_sum<kNT>(spq, sh);
  const double a1 = block_sum<kNT>(spr, sh);
  if (threadIdx.x == 0) {
    part[bid()] = a0;
    part[nblocks() + bid()] = a1;
  }
  if (last_block_arrival(&st->ticket[3], nblocks(), &flag)) {
    const double pq = reduce_partials<kNT>(part, nblocks(), sh);
    const double pr = reduce_partials<kNT>(part + nblocks(), nblocks(), sh);
    if (threadIdx.x == 0) {
      st->pq = pq;
      st->pr = pr;
      st->alpha = (pq != 0.0) ? pr / pq : 0.0;
      st->pq_old = pq;
    }
  }
}

// Split form for an FP32 z (the fused form would widen nine FP32 neighbours per node on
// the FP64 pipe): p = inv_scale z + beta p elementwise, then q = A p with the FP64 stencil.
__global__ void __launch_bounds__(kNT, kRedBlocksPerSM) k_fcg_p32(Lvl<double> L, const float* __restrict__ z, int zp,
                                                 double* __restrict__ p, const SolveState* st) {
  if (st->done) return;
  const double is = st->inv_scale_r32;
  const bool f32ok = pow2_fits_f32(is);
  const double beta = st->beta;
  const bool first = (st->it == 0);
  const int i = blockIdx.x * kNT + threadIdx.x;
  if (i < L.nx) {
    float zv[4];
    double pv[4];
    rows_batched<4>(
        L.nyr,
        [&](int u, int j) {
          zv[u] = z[(size_t)j * zp + i];
          pv[u] = p[(size_t)j * L.pitch + i];
        },
        [&](int u, int j) {
          if (!is_unknown(L, i, j)) return;
          const double zz = from_f32_scaled(zv[u], is, f32ok);
          p[(size_t)j * L.pitch + i] = first ? zz : fma(beta, pv[u], zz);
        });
  }
}

__global__ void __launch_bounds__(kNT) k_fcg_q(Lvl<double> L, const double* __restrict__ p,
                                               const double* __restrict__ r,
                                               double* __restrict__ q, SolveState* st,
                                               double* part) {
  if (st->done) return;
  __shared__ double sh[kNT / 32];
  __shared__ int flag;
  double spq = 0.0, spr = 0.0;
  NODE_LOOP(L) {
    if (!is_unknown(L, i, j)) continue;
    const size_t k = (size_t)j * L.pitch + i;
    const double qv = fma(L.diag[k], p[k], offdiag(L, p, i, j));
    q[k] = qv;
    spq = fma(p[k], qv, spq);
    spr = fma(p[k], r[k], spr);
  }
  const double a0 = block_sum<kNT>(spq, sh);
  const double a1 = block_sum<kNT>(spr, sh);
  if (threadIdx.x == 0) {
    part[bid()] = a0;
    part[nblocks() + bid()] = a1;
  }
  if (last_block_arrival(&st->ticket[3], nblocks(), &flag)) {
    const double pq = reduce_partials<kNT>(part, nblocks(), sh);
    const double pr = reduce_partials<kNT>(part + nblocks(), nblocks(), sh);
    if (threadIdx.x == 0) {
      st->pq = pq;
      st->pr = pr;
      st->alpha = (pq != 0.0) ? pr / pq : 0.0;
      st->pq_old = pq;
    }
  }
}

// x += alpha p; r -= alpha q; ||r||^2; and, for the mixed path, the next cycle's
// right-hand side r32 = fp32(r * scale) with the current power-of-two scale.
__global__ void __launch_bounds__(kNT) k_fcg_update(Lvl<double> L, double* __restrict__ x,
                                                    double* __restrict__ r,
                                                    const double* __restrict__ p,
                                                    const double* __restrict__ q,
                                                    float* __restrict__ r32, int p32,
                                                    SolveState* st, double* part,
                                                    cudaGraphConditionalHandle h, int has_h) {
  if (st->done) return;
  __shared__ double sh[kNT / 32];
  __shared__ int flag;
  const double alpha = st->alpha;
  const double sc = st->scale;
  const bool f32ok = pow2_fits_f32(sc);
  double s = 0.0;
  NODE_LOOP(L) {
    if (!is_unknown(L, i, j)) continue;
    const size_t k = (size_t)j * L.pitch + i;
    x[k] = fma(alpha, p[k], x[k]);
    const double rv = fma(-alpha, q[k], r[k]);
    r[k] = rv;
    if (r32) r32[(size_t)j * p32 + i] = to_f32_scaled(rv, sc, f32ok);
    s = fma(rv, rv, s);
  }
  const double a0 = block_sum<kNT>(s, sh);
  if (threadIdx.x == 0) part[bid()] = a0;
  if (last_block_arrival(&st->ticket[4], nblocks(), &flag)) {
    const double rr = reduce_partials<kNT>(part, nblocks(), sh);
    if (threadIdx.x == 0) {
      st->it += 1;
      if (r32) st->inv_scale_r32 = 1.0 / sc;
      decide(st, rr, h, has_h, 1);
    }
  }
}

// Residual replacement: when the recursive residual met rtol, r = b - A x is recomputed;
// the solve stops only if the true residual meets rtol, else CG continues from it.
__global__ void __launch_bounds__(kNT) k_fcg_verify(Lvl<double> L, const double* __restrict__ x,
                                                    const double* __restrict__ b,
                                                    double* __restrict__ r,
                                                    float* __restrict__ r32, int p32,
                                                    SolveState* st, double* part,
                                                    cudaGraphConditionalHandle h, int has_h) {
  if (st->done || !st->verify) return;
  __shared__ double sh[kNT / 32];
  __shared__ int flag;
  const double sc = st->scale;
  const bool f32ok = pow2_fits_f32(sc);
  double s = 0.0;
  NODE_LOOP(L) {
    const size_t k = (size_t)j * L.pitch + i;
    double rv = 0.0;
    if (is_unknown(L, i, j)) {
      rv = b[k] - fma(L.diag[k], x[k], offdiag(L, x, i, j));
      s += rv * rv;
    }
    r[k] = rv;
    if (r32) r32[(size_t)j * p32 + i] = to_f32_scaled(rv, sc, f32ok);
  }
  const double a0 = block_sum<kNT>(s, sh);
  if (threadIdx.x == 0) part[bid()] = a0;
  if (last_block_arrival(&st->ticket[5], nblocks(), &flag)) {
    const double rr = reduce_partials<kNT>(part, nblocks(), sh);
    if (threadIdx.x == 0) {
      st->verify = 0;
      if (r32) st->inv_scale_r32 = 1.0 / sc;
      decide(st, rr, h, has_h, 0);
      // the recursive residual keeps meeting rtol but the true one does not: the true
      // residual has reached its rounding floor above rtol; stop (not converged)
      if (!st->done && ++st->verify_fail >= kMaxVerifyFail) {
        st->done = 1;
        st->status = 6;
        if (has_h) cudaGraphSetConditional(h, 0u);
      }
    }
  }
}

// Batch epilogue: block k copies instance k's solve state and flags into contiguous arrays.
__global__ void k_gather_states(SolveState* const* __restrict__ src, int* const* __restrict__ srcflags,
                                SolveState* dst, int* dflags) {
  const int k = blockIdx.x;
  const unsigned long long* a = reinterpret_cast<const unsigned long long*>(src[k]);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(dst + k);
  for (size_t w = threadIdx.x; w < sizeof(SolveState) / 8; w += blockDim.x) d[w] = a[w];
  if (threadIdx.x < 4) dflags[4 * k + threadIdx.x] = srcflags[k][threadIdx.x];
}

// phi_out (caller layout) = x at every node.
__global__ void __launch_bounds__(kNT) k_copy_out(Lvl<double> L, const double* __restrict__ x,
                                                  const SolveArgs* __restrict__ a) {
  const int up = a->user_pitch, n = a->mirror;
  double* out = a->phi_out;
  NODE_LOOP(L) {
    int jr = j;  // Neumann grid: rows n.. of the doubled system are the caller's rows 0.., row 0 its row n
    if (n) {
      if (j >= n) jr = j - n;
      else if (j == 0) jr = n;
      else continue;
    }
    out[(size_t)jr * up + i] = x[(size_t)j * L.pitch + i];
  }
}

// ------------------------------------------------------------------ launchers
dim3 red_grid(int nx, int nyr) {
  const int gx = (nx + kNT - 1) / kNT;
  int gy = kRedBlocks / gx;
  if (gy < 1) gy = 1;
  if (gy > nyr) gy = nyr;
  return dim3(gx, gy);
}

#define CHK() return cudaGetLastError()

cudaError_t launch_solve_init(const OpF64& A, const SolveArgs* a, const double* D, double* x,
                              double* b, SolveState* st, cudaStream_t s) {
  const Lvl<double> L = lvl_of(A);
  k_solve_init<<<red_grid(L.nx, L.nyr), kNT, 0, s>>>(L, a, D, x, b, st);
  CHK();
}
cudaError_t launch_resid_init(const OpF64& A, const double* x, const double* b, double* r,
                              SolveState* st, double* part, cudaGraphConditionalHandle h,
                              int has_h, cudaStream_t s) {
  const Lvl<double> L = lvl_of(A);
  k_resid_init<<<red_grid(L.nx, L.nyr), kNT, 0, s>>>(L, x, b, r, st, part, h, has_h);
  CHK();
}
cudaError_t launch_resid_check(const OpF64& A, const double* x, const double* b, double* r,
                               SolveState* st, double* part, cudaGraphConditionalHandle h,
                               int has_h, cudaStream_t s) {
  const Lvl<double> L = lvl_of(A);
  k_resid_check<<<red_grid(L.nx, L.nyr), kNT, 0, s>>>(L, x, b, r, st, part, h, has_h);
  CHK();
}
cudaError_t launch_r_to_f32(const OpF64& A, const double* r, float* b32, int pitch32,
                            SolveState* st, cudaStream_t s) {
  const Lvl<double> L = lvl_of(A);
  k_r_to_f32<<<red_grid(L.nx, L.nyr), kNT, 0, s>>>(L, r, b32, pitch32, st);
  CHK();
}
cudaError_t launch_add_f32(const OpF64& A, double* x, const float* e32, int pitch32,
                           SolveState* st, cudaStream_t s) {
  const Lvl<double> L = lvl_of(A);
  k_add_f32<<<red_grid(L.nx, L.nyr), kNT, 0, s>>>(L, x, e32, pitch32, st);
  CHK();
}
cudaError_t launch_loop_guard(SolveState* st, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_loop_guard<<<1, 32, 0, s>>>(st, h);
  CHK();
}
cudaError_t launch_iter_inc(SolveState* st, cudaStream_t s) {
  k_iter_inc<<<1, 32, 0, s>>>(st);
  CHK();
}
template <typename TZ>
cudaError_t launch_fcg_zq(const OpF64& A, const TZ* z, int zp, const double* q, SolveState* st,
                          double* part, cudaStream_t s) {
  const Lvl<double> L = lvl_of(A);
  k_fcg_zq<TZ><<<red_grid(L.nx, L.nyr), kNT, 0, s>>>(L, z, zp, q, st, part);
  CHK();
}
template cudaError_t launch_fcg_zq<double>(const OpF64&, const double*, int, const double*,
                                           SolveState*, double*, cudaStream_t);
template cudaError_t launch_fcg_zq<float>(const OpF64&, const float*, int, const double*,
                                          SolveState*, double*, cudaStream_t);
template <typename TZ>
cudaError_t launch_fcg_pq(const OpF64& A, const TZ* z, int zp, double* p, double* q, const double* r,
                          SolveState* st, double* part, cudaStream_t s) {
  const Lvl<double> L = lvl_of(A);
  k_fcg_pq<TZ><<<red_grid(L.nx, L.nyr), kNT, 0, s>>>(L, z, zp, p, q, r, st, part);
  CHK();
}
template cudaError_t launch_fcg_pq<double>(const OpF64&, const double*, int, double*, double*,
                                           const double*, SolveState*, double*, cudaStream_t);
template <>
cudaError_t launch_fcg_pq<float>(const OpF64& A, const float* z, int zp, double* p, double* q,
                                 const double* r, SolveState* st, double* part, cudaStream_t s) {
  const Lvl<double> L = lvl_of(A);
  k_fcg_p32<<<red_grid(L.nx, L.nyr), kNT, 0, s>>>(L, z, zp, p, st);
  k_fcg_q<<<red_grid(L.nx, L.nyr), kNT, 0, s>>>(L, p, r, q, st, part);
  CHK();
}
cudaError_t launch_fcg_update(const OpF64& A, double* x, double* r, const double* p,
                              const double* q, float* r32, int p32, SolveState* st, double* part,
                              cudaGraphConditionalHandle h, int has_h, cudaStream_t s) {
  const Lvl<double> L = lvl_of(A);
  k_fcg_update<<<red_grid(L.nx, L.nyr), kNT, 0, s>>>(L, x, r, p, q, r32, p32, st, part, h, has_h);
  CHK();
}
cudaError_t launch_fcg_verify(const OpF64& A, const double* x, const double* b, double* r,
                              float* r32, int p32, SolveState* st, double* part,
                              cudaGraphConditionalHandle h, int has_h, cudaStream_t s) {
  const Lvl<double> L = lvl_of(A);
  k_fcg_verify<<<red_grid(L.nx, L.nyr), kNT, 0, s>>>(L, x, b, r, r32, p32, st, part, h, has_h);
  CHK();
}
cudaError_t launch_gather_states(SolveState* const* src, int* const* srcflags, SolveState* dst,
                                 int* dflags, int count, cudaStream_t s) {
  k_gather_states<<<count, 128, 0, s>>>(src, srcflags, dst, dflags);
  CHK();
}
cudaError_t launch_copy_out(const OpF64& A, const double* x, const SolveArgs* a, cudaStream_t s) {
  const Lvl<double> L = lvl_of(A);
  k_copy_out<<<red_grid(L.nx, L.nyr), kNT, 0, s>>>(L, x, a);
  CHK();
}

}  // namespace mg
