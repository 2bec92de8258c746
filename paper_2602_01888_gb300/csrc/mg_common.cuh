// Internal definitions shared by the CUDA translation units of libmg.
//
// Grid/operator layout on the device (every level, both precisions):
//   node (i, j) of a level with nx x ny vertices is stored at i + pitch * j,
//   rows j = 0 .. nyr-1 (nyr = ny - 1 when periodic in y, else ny), pitch a multiple of
//   32 elements so every row starts on a 256-byte (FP64) / 128-byte (FP32) boundary.
//   The operator of a level is the symmetric 9-point matrix A = -L_h of the generalized
//   Poisson equation (Eqs. 16-18 in conservative form) or its Galerkin coarsening; per
//   node we keep its E, N, NE, NW couplings and the diagonal (plus 1/diagonal).  The
//   W, S, SW, SE couplings of node (i, j) are the E, N, NE, NW couplings of its
//   neighbours (i-1, j), (i, j-1), (i-1, j-1), (i+1, j-1): the matrix is symmetric.
//   Dirichlet nodes keep their value in the solution array (boundary data on the finest
//   level, 0 on coarse levels) and are never updated.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mg {

template <typename T>
struct Lvl {
  int nx, ny, nyr, periodic, pitch;
  const T *cE, *cN, *cNE, *cNW, *diag, *dinv;
  // 1: the NE / NW couplings are zero at every node (a map without cross term, Eq. 13 = 0)
  // and are neither read nor multiplied; adding a zero product changes no sum, so the
  // results equal the 9-point form's.
  int five_point;
};

__host__ __device__ inline int rows_stored(int ny, int periodic) { return periodic ? ny - 1 : ny; }

__device__ __forceinline__ int row_dn(int j, int nyr) { return j == 0 ? nyr - 1 : j - 1; }
__device__ __forceinline__ int row_up(int j, int nyr) { return j == nyr - 1 ? 0 : j + 1; }

template <typename T>
__device__ __forceinline__ bool is_unknown(const Lvl<T>& L, int i, int j) {
  if (i < 1 || i > L.nx - 2 || j < 0 || j >= L.nyr) return false;
  return L.periodic || (j >= 1 && j <= L.ny - 2);
}

// Sum of the eight off-diagonal couplings times x at unknown (i, j) (four for a 5-point
// operator: the diagonal terms are zero and skipped).
template <typename T>
__device__ __forceinline__ T offdiag(const Lvl<T>& L, const T* __restrict__ x, int i, int j) {
  const int p = L.pitch;
  const int jd = row_dn(j, L.nyr), ju = row_up(j, L.nyr);
  const size_t r0 = (size_t)j * p, rd = (size_t)jd * p, ru = (size_t)ju * p;
  T s = L.cE[r0 + i] * x[r0 + i + 1];
  s = fma(L.cE[r0 + i - 1], x[r0 + i - 1], s);
  s = fma(L.cN[r0 + i], x[ru + i], s);
  s = fma(L.cN[rd + i], x[rd + i], s);
  if (L.five_point) return s;
  s = fma(L.cNE[r0 + i], x[ru + i + 1], s);
  s = fma(L.cNE[rd + i - 1], x[rd + i - 1], s);
  s = fma(L.cNW[r0 + i], x[ru + i - 1], s);
  s = fma(L.cNW[rd + i + 1], x[rd + i + 1], s);
  return s;
}

// Forward colour order (i mod 2, j mod 2): (0,0), (1,1), (1,0), (0,1).
__host__ __device__ inline int colour_ci(int c) { return (c == 1 || c == 2) ? 1 : 0; }
__host__ __device__ inline int colour_cj(int c) { return (c == 0 || c == 2) ? 0 : 1; }

// Device-side solve state (one per solve in flight).  Scalars are produced by the
// "last block" of a reducing kernel from per-block partial sums in a fixed order, so
// every result is bitwise reproducible run to run.
struct SolveState {
  double r0;          // reference norm ||r_0||_2
  double rr;          // ||r||_2^2 of the current iterate
  double rel;         // sqrt(rr) / r0
  double rz;          // previous-direction quantities of flexible CG
  double pq, pr, zq, pq_old;
  double alpha, beta;
  double scale;       // power-of-two scaling of r before the FP32 cycle (mixed)
  double inv_scale;
  double inv_scale_r32;  // 1/scale of the r32 the current FP32 cycle started from
  double rtol;
  int it;             // iterations done
  int max_iters;
  int done;           // 1 once converged / exhausted / diverged: later kernels exit at once
  int status;         // 0 running/converged, 6 not converged, 7 diverged
  int hist_n;
  int verify;         // recursive residual met rtol: recompute the true one next
  int guard;          // body passes; bounds the device-driven loop whatever happens
  int verify_fail;    // true-residual checks that did not meet rtol
  int x_zero;         // the initial iterate is zero everywhere (cold start, no Dirichlet data)
  int pad_;
  long long n_unknowns;  // for the rms used by the FP32 scaling
  unsigned int ticket[8];  // arrival counters of the last-block reductions
  double hist[256];
};

static_assert(sizeof(SolveState) % 8 == 0, "SolveState is copied as 8-byte words");

// ---- deterministic block reduction -------------------------------------------------
// Sums v over the block in a fixed order (warp shuffle tree, then warps in order).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh /* >= NT/32 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < NT / 32; ++w) t += sh[w];
  }
  __syncthreads();
  return t;  // valid in thread 0
}

// After each block has written partial[blockLinear], the block that arrives last
// (counted with an atomic ticket) returns true in all its threads; it then owns the
// final fixed-order reduction.  The ticket is reset for the next use.
__device__ __forceinline__ bool last_block_arrival(unsigned int* ticket, unsigned int nblocks,
                                                   int* sh_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = atomicAdd(ticket, 1u);
    *sh_flag = (t == nblocks - 1);
  }
  __syncthreads();
  bool last = *sh_flag;
  if (last && threadIdx.x == 0) *ticket = 0u;
  if (last) __threadfence();
  return last;
}

// Fixed-order sum of n partials by one block (tree over a strided split; the order
// depends only on n and the block size).
template <int NT>
__device__ double reduce_partials(const double* __restrict__ part, int n, double* sh) {
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += NT) v += ((volatile const double*)part)[k];
  return block_sum<NT>(v, sh);
}

}  // namespace mg
