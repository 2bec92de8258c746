// Zebra x-line Gauss-Seidel: the unknowns of every row j of one parity are solved together,
// with the row's own W/E couplings kept in a tridiagonal system and the couplings to the
// rows above and below (N, S and the diagonals) and to the row's Dirichlet ends moved to the
// right-hand side (the rows of one parity share no coupling).  A line smoother keeps the
// multigrid cycle's convergence when the coupling along x dominates, as on the annulus of
// Eq. 29, where the per-node (point) smoother leaves smooth-in-x, oscillatory-in-y error.
//
// The tridiagonal systems are solved by cyclic reduction, which is parallel within a row.
// A row's matrix does not change between sweeps, so its reduction multipliers are computed
// once per operator (k_line_factor) and a sweep only reduces the right-hand side and
// substitutes back (k_line_zebra), with the row staged in shared memory.  The row length
// N = nx - 2 is padded to a power of two Np with identity equations.
//
// Layout of the factors (per row, row stride Np elements, in five arrays):
//   alpha, gamma: the multipliers of reduction level k (stride s = 2^k) for the combining
//     equations i = 2s(m + 1) - 1, stored at offset Np - Np/2^k + m;
//   afin, cfin, binv: for every equation i, its sub/super-diagonal entries and reciprocal
//     pivot at the level where it is eliminated (back substitution).
#include <cuda_runtime.h>

#include "mg_common.cuh"
#include "mg_kernels.h"
#include "mg_launch.h"
#include "mg_line.h"

namespace mg {

static constexpr int kLT = 256;

__host__ __device__ inline int line_np(int nx) {
  int np = 1;
  while (np < nx - 2) np <<= 1;
  return np < 2 ? 2 : np;
}

__host__ __device__ inline int line_levels(int np) {
  int k = 0;
  while ((1 << k) < np) ++k;
  return k;
}

template <typename T>
__device__ __forceinline__ bool row_active(const Lvl<T>& L, int j) {
  return L.periodic || (j >= 1 && j <= L.ny - 2);
}

// Reduction multipliers of row blockIdx.x.  Shared memory: a, b, c of Np entries each.
template <typename T>
__global__ void __launch_bounds__(kLT) k_line_factor(Lvl<T> L, LineFactors<T> F) {
  const int j = blockIdx.x;
  if (j >= L.nyr || !row_active(L, j)) return;
  const int N = L.nx - 2, Np = F.np, K = line_levels(Np);
  extern __shared__ __align__(16) unsigned char line_smem[];
  T* a = reinterpret_cast<T*>(line_smem);
  T* bb = a + Np;
  T* c = bb + Np;
  const size_t r0 = (size_t)j * L.pitch, f0 = (size_t)j * Np;
  for (int t = threadIdx.x; t < Np; t += blockDim.x) {
    if (t < N) {
      const int i = t + 1;
      a[t] = t >= 1 ? L.cE[r0 + i - 1] : T(0);
      bb[t] = L.diag[r0 + i];
      c[t] = t <= N - 2 ? L.cE[r0 + i] : T(0);
    } else {  // padding: identity equations
      a[t] = T(0);
      bb[t] = T(1);
      c[t] = T(0);
    }
  }
  __syncthreads();
  for (int k = 0; k < K; ++k) {
    const int s = 1 << k;
    // equations eliminated at this level (i = 2s m + s - 1) are final now
    for (int m = threadIdx.x; m < Np / (2 * s); m += blockDim.x) {
      const int i = 2 * s * m + s - 1;
      F.afin[f0 + i] = a[i];
      F.cfin[f0 + i] = c[i];
      F.binv[f0 + i] = T(1) / bb[i];
    }
    // combining equations i = 2s(m + 1) - 1 absorb their neighbours at distance s; the
    // neighbours are not combining at this level, so reading and writing do not overlap
    const int off = Np - Np / s;
    for (int m = threadIdx.x; m < Np / (2 * s); m += blockDim.x) {
      const int i = 2 * s * (m + 1) - 1;
      const bool up = i + s < Np;
      const T al = -a[i] / bb[i - s];
      const T ga = up ? -c[i] / bb[i + s] : T(0);
      F.alpha[f0 + off + m] = al;
      F.gamma[f0 + off + m] = ga;
      const T na = al * a[i - s];
      const T nc = up ? ga * c[i + s] : T(0);
      const T nb = bb[i] + al * c[i - s] + (up ? ga * a[i + s] : T(0));
      a[i] = na;
      c[i] = nc;
      bb[i] = nb;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {  // the last combining equation has no neighbour left
    F.afin[f0 + Np - 1] = T(0);
    F.cfin[f0 + Np - 1] = T(0);
    F.binv[f0 + Np - 1] = T(1) / bb[Np - 1];
  }
}

// One half-sweep: rows j = par, par + 2, ... (grid: one CTA per such row).  Shared memory:
// the row's right-hand side, overwritten by its solution, Np entries.
template <typename T>
__global__ void __launch_bounds__(kLT) k_line_zebra(Lvl<T> L, LineFactors<T> F, T* __restrict__ x,
                                                    const T* __restrict__ b, int par,
                                                    const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int j = par + 2 * blockIdx.x;
  if (j >= L.nyr || !row_active(L, j)) return;
  const int N = L.nx - 2, Np = F.np, K = line_levels(Np);
  extern __shared__ __align__(16) unsigned char line_smem[];
  T* d = reinterpret_cast<T*>(line_smem);
  const int p = L.pitch;
  const int jd = row_dn(j, L.nyr), ju = row_up(j, L.nyr);
  const size_t r0 = (size_t)j * p, rd = (size_t)jd * p, ru = (size_t)ju * p, f0 = (size_t)j * Np;
  for (int t = threadIdx.x; t < Np; t += blockDim.x) {
    T v = T(0);
    if (t < N) {
      const int i = t + 1;
      // couplings leaving the row, in the order of the point smoother's sum minus E/W
      T off = L.cN[r0 + i] * x[ru + i];
      off = fma(L.cN[rd + i], x[rd + i], off);
      off = fma(L.cNE[r0 + i], x[ru + i + 1], off);
      off = fma(L.cNE[rd + i - 1], x[rd + i - 1], off);
      off = fma(L.cNW[r0 + i], x[ru + i - 1], off);
      off = fma(L.cNW[rd + i + 1], x[rd + i + 1], off);
      if (i == 1) off = fma(L.cE[r0], x[r0], off);
      if (i == N) off = fma(L.cE[r0 + i], x[r0 + i + 1], off);
      v = b[r0 + i] - off;
    }
    d[t] = v;
  }
  __syncthreads();
  // forward reduction of the right-hand side
  for (int k = 0; k < K; ++k) {
    const int s = 1 << k, off = Np - Np / s;
    for (int m = threadIdx.x; m < Np / (2 * s); m += blockDim.x) {
      const int i = 2 * s * (m + 1) - 1;
      T v = fma(F.alpha[f0 + off + m], d[i - s], d[i]);
      if (i + s < Np) v = fma(F.gamma[f0 + off + m], d[i + s], v);
      d[i] = v;
    }
    __syncthreads();
  }
  // back substitution, from the last equation down; solutions overwrite d
  if (threadIdx.x == 0) d[Np - 1] *= F.binv[f0 + Np - 1];
  __syncthreads();
  for (int k = K - 1; k >= 0; --k) {
    const int s = 1 << k;
    for (int m = threadIdx.x; m < Np / (2 * s); m += blockDim.x) {
      const int i = 2 * s * m + s - 1;
      T v = d[i];
      if (i - s >= 0) v -= F.afin[f0 + i] * d[i - s];
      v -= F.cfin[f0 + i] * d[i + s];
      d[i] = v * F.binv[f0 + i];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < N; t += blockDim.x) x[r0 + t + 1] = d[t];
}

// ------------------------------------------------------------------ launchers
template <typename T>
size_t line_factor_elems(int nx, int ny, int periodic) {
  return (size_t)5 * line_np(nx) * rows_stored(ny, periodic);
}

template <typename T>
bool line_supported(int nx) {
  return nx >= 3 && (size_t)3 * line_np(nx) * sizeof(T) <= kLineSmemMax;
}

template <typename T>
LineFactors<T> line_factors_at(T* base, int nx, int ny, int periodic) {
  LineFactors<T> F;
  F.np = line_np(nx);
  const size_t n = (size_t)F.np * rows_stored(ny, periodic);
  F.alpha = base;
  F.gamma = base + n;
  F.afin = base + 2 * n;
  F.cfin = base + 3 * n;
  F.binv = base + 4 * n;
  return F;
}

template <typename T>
cudaError_t launch_line_factor(const Op<T>& A, const LineFactors<T>& F, cudaStream_t s) {
  if (!line_supported<T>(A.nx) || F.np != line_np(A.nx)) return cudaErrorInvalidValue;
  const Lvl<T> L = lvl_of(A);
  const size_t sm = (size_t)3 * F.np * sizeof(T);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_line_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kLineSmemMax);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_line_factor<T><<<L.nyr, kLT, sm, s>>>(L, F);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_line_rows(const Op<T>& A, const LineFactors<T>& F, T* x, const T* b, int par,
                             const int* skip, cudaStream_t s) {
  if (!line_supported<T>(A.nx) || F.np != line_np(A.nx)) return cudaErrorInvalidValue;
  const Lvl<T> L = lvl_of(A);
  const size_t sm = (size_t)F.np * sizeof(T);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_line_zebra<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kLineSmemMax / 3));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int rows = (L.nyr - par + 1) / 2;
  if (rows <= 0) return cudaSuccess;
  k_line_zebra<T><<<rows, kLT, sm, s>>>(L, F, x, b, par, skip);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_line_smooth(const Op<T>& A, const LineFactors<T>& F, T* x, const T* b, int sweeps,
                               int rev, const int* skip, cudaStream_t s) {
  for (int sw = 0; sw < sweeps; ++sw)
    for (int h = 0; h < 2; ++h) {
      const cudaError_t e = launch_line_rows<T>(A, F, x, b, rev ? 1 - h : h, skip, s);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

#define MG_LINE_INST(T)                                                                          \
  template size_t line_factor_elems<T>(int, int, int);                                          \
  template bool line_supported<T>(int);                                                          \
  template LineFactors<T> line_factors_at<T>(T*, int, int, int);                                \
  template cudaError_t launch_line_factor<T>(const Op<T>&, const LineFactors<T>&, cudaStream_t); \
  template cudaError_t launch_line_rows<T>(const Op<T>&, const LineFactors<T>&, T*, const T*, int, \
                                           const int*, cudaStream_t);                           \
  template cudaError_t launch_line_smooth<T>(const Op<T>&, const LineFactors<T>&, T*, const T*, int, \
                                             int, const int*, cudaStream_t);
MG_LINE_INST(float)
MG_LINE_INST(double)

}  // namespace mg

// ------------------------------------------------------------------ C ABI
using namespace mg;

extern "C" size_t mgk_line_factor_elems(int nx, int ny, int periodic) {
  if (nx < 3 || ny < 3) return 0;
  return line_factor_elems<double>(nx, ny, periodic);
}

template <typename T, typename OPK>
static int line_factor_abi(const OPK* A, T* f, void* stream) {
  if (!A || A->nx < 3 || A->ny < 3 || A->pitch < A->nx || !f || !line_supported<T>(A->nx)) return 1;
  const cudaError_t e = launch_line_factor<T>(op_from(*A), line_factors_at<T>(f, A->nx, A->ny, A->periodic),
                                              (cudaStream_t)stream);
  return e == cudaSuccess ? 0 : 4;
}

// sweeps < 0: one half-sweep of parity par; else `sweeps` sweeps in the order given by rev.
template <typename T, typename OPK>
static int line_rows_abi(const OPK* A, const T* f, T* phi, const T* b, int par, int sweeps, int rev,
                         void* stream) {
  if (!A || A->nx < 3 || A->ny < 3 || A->pitch < A->nx || !f || !phi || !b || !line_supported<T>(A->nx))
    return 1;
  if (A->periodic && (A->ny - 1) % 2) return 1;  // zebra order needs an even row count
  const LineFactors<T> F = line_factors_at<T>(const_cast<T*>(f), A->nx, A->ny, A->periodic);
  const cudaError_t e =
      sweeps < 0 ? launch_line_rows<T>(op_from(*A), F, phi, b, par, nullptr, (cudaStream_t)stream)
                 : launch_line_smooth<T>(op_from(*A), F, phi, b, sweeps, rev, nullptr, (cudaStream_t)stream);
  return e == cudaSuccess ? 0 : 4;
}

extern "C" int mgk_line_factor_f64(const mgk_op_f64* A, double* factors, void* stream) {
  return line_factor_abi<double>(A, factors, stream);
}
extern "C" int mgk_line_factor_f32(const mgk_op_f32* A, float* factors, void* stream) {
  return line_factor_abi<float>(A, factors, stream);
}
extern "C" int mgk_line_rows_f64(const mgk_op_f64* A, const double* factors, double* phi, const double* b,
                                 int parity, void* stream) {
  if (parity != 0 && parity != 1) return 1;
  return line_rows_abi<double>(A, factors, phi, b, parity, -1, 0, stream);
}
extern "C" int mgk_line_rows_f32(const mgk_op_f32* A, const float* factors, float* phi, const float* b,
                                 int parity, void* stream) {
  if (parity != 0 && parity != 1) return 1;
  return line_rows_abi<float>(A, factors, phi, b, parity, -1, 0, stream);
}
extern "C" int mgk_line_smooth_f64(const mgk_op_f64* A, const double* factors, double* phi, const double* b,
                                   int sweeps, int reverse, void* stream) {
  if (sweeps < 0) return 1;
  return line_rows_abi<double>(A, factors, phi, b, 0, sweeps, reverse ? 1 : 0, stream);
}
extern "C" int mgk_line_smooth_f32(const mgk_op_f32* A, const float* factors, float* phi, const float* b,
                                   int sweeps, int reverse, void* stream) {
  if (sweeps < 0) return 1;
  return line_rows_abi<float>(A, factors, phi, b, 0, sweeps, reverse ? 1 : 0, stream);
}
