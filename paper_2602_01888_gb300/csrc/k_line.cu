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
//   afin, cfin, binv: the sub/super-diagonal entries and reciprocal pivot of the equations
//     eliminated at level k (i = 2s m + s - 1), at the same offset Np - Np/2^k + m; the
//     last equation (the root of the reduction) at Np - 1.
// Every phase of both kernels thus reads its factors as one contiguous run.  In shared
// memory, element i sits at i + i / (128 / sizeof(T)): one pad word per 128 bytes, so the
// strided accesses of the reduction levels (stride 2^(k+1)) hit distinct banks.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>
#include <vector>

#include "mg_common.cuh"
#include "mg_kernels.h"
#include "mg_launch.h"
#include "mg_line.h"

namespace mg {

static constexpr int kLT = 256;  // threads of a line CTA

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

// Padded shared-memory index and the padded length of a row of Np elements.
template <typename T>
__host__ __device__ __forceinline__ int sx(int i) {
  return i + i / (128 / (int)sizeof(T));
}
template <typename T>
__host__ __device__ inline size_t line_row_smem(int np) {
  return (size_t)(sx<T>(np - 1) + 1) * sizeof(T);
}

// Asynchronous copy of one element from global to shared memory (4 or 8 bytes, naturally
// aligned).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}

// Bilinear prolongation (Eq. 24) at a node of an even fine row jn (a coarse row): the coarse
// value at even columns, the mean of its two coarse neighbours at odd ones.
template <typename T>
__device__ __forceinline__ T prolong_even_row(const T* __restrict__ eH, int pitch_c, int jn, int c) {
  const size_t a = (size_t)(jn >> 1) * pitch_c + (c >> 1);
  return (c & 1) ? T(0.5) * (__ldg(eH + a) + __ldg(eH + a + 1)) : __ldg(eH + a);
}

template <typename T>
__device__ __forceinline__ bool row_active(const Lvl<T>& L, int j) {
  return L.periodic || (j >= 1 && j <= L.ny - 2);
}

// Coarse-grid correction of the even rows (the rows that coincide with coarse rows): x += P eH
// at their unknowns, before the first post-smoothing half-sweep solves the odd rows from them.
// That half-sweep and the next one never read the old values of the rows they solve, so the
// result equals adding P eH to every row and smoothing, with one pass over half the rows.
// VEC: each thread takes one 16-byte chunk of a row and corrects the chunk's unknowns (the
// launcher chooses it when every row starts 16-byte aligned); otherwise one element each.
// Grid: (chunks or columns / kLT, even rows).
template <typename T, bool VEC>
__global__ void __launch_bounds__(256) k_line_prolong_even(Lvl<T> L, T* __restrict__ x,
                                                           const T* __restrict__ eH, int pitch_c,
                                                           const int* __restrict__ skip) {
  if (skip && *skip) return;
  constexpr int V = VEC ? 16 / (int)sizeof(T) : 1;
  const int jn = 2 * blockIdx.y;
  const int c0 = (blockIdx.x * blockDim.x + threadIdx.x) * V;
  if (jn >= L.nyr || !row_active(L, jn) || c0 > L.nx - 2) return;
  T* const r = x + (size_t)jn * L.pitch + c0;
  if constexpr (VEC) {
    using V16 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    V16 w = *reinterpret_cast<V16*>(r);
    T* const e = reinterpret_cast<T*>(&w);
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int c = c0 + u;
      if (c >= 1 && c <= L.nx - 2) e[u] = e[u] + prolong_even_row(eH, pitch_c, jn, c);
    }
    *reinterpret_cast<V16*>(r) = w;
  } else if (c0 >= 1) {
    r[0] = r[0] + prolong_even_row(eH, pitch_c, jn, c0);
  }
}

// Reduction multipliers of row blockIdx.x.  The first level reads the row's three diagonals
// from global memory (each entry once) and keeps only the Np / 2 equations it leaves
// (the odd ones), compacted, in shared memory: a, b, c of Np / 2 entries each, half of what
// the whole row would take, so that twice as many rows are factored at once (the kernel is
// bound by its dependent chain of levels, not by its few bytes).  Equation i' of the compacted
// system is equation 2 i' + 1 of the row, and level k of the row is level k - 1 of the
// compacted system, with the same arithmetic in the same order.
template <typename T>
__device__ __forceinline__ void row_diags(const Lvl<T>& L, size_t r0, int N, int t, T& a, T& b, T& c) {
  if (t < N) {
    const int i = t + 1;
    a = t >= 1 ? L.cE[r0 + i - 1] : T(0);
    b = L.diag[r0 + i];
    c = t <= N - 2 ? L.cE[r0 + i] : T(0);
  } else {  // padding: identity equations
    a = T(0);
    b = T(1);
    c = T(0);
  }
}

template <typename T>
__global__ void __launch_bounds__(kLT) k_line_factor(Lvl<T> L, LineFactors<T> F) {
  const int j = blockIdx.x;
  if (j >= L.nyr || !row_active(L, j)) return;
  const int N = L.nx - 2, Np = F.np, K = line_levels(Np), Nh = Np / 2;
  extern __shared__ __align__(16) unsigned char line_smem[];
  const int rs = (int)(line_row_smem<T>(Nh) / sizeof(T));
  T* a = reinterpret_cast<T*>(line_smem);
  T* bb = a + rs;
  T* c = bb + rs;
  const size_t r0 = (size_t)j * L.pitch, f0 = (size_t)j * Np;
  // level 0: equations 2m are final; equations 2m + 1 absorb their two neighbours
  for (int m = threadIdx.x; m < Nh; m += blockDim.x) {
    T ae, be, ce, ad, bd, cd, au = T(0), bu = T(1), cu = T(0);
    row_diags(L, r0, N, 2 * m, ad, bd, cd);  // the eliminated equation below
    row_diags(L, r0, N, 2 * m + 1, ae, be, ce);
    const bool up = 2 * m + 2 < Np;
    if (up) row_diags(L, r0, N, 2 * m + 2, au, bu, cu);
    F.afin[f0 + m] = ad;
    F.cfin[f0 + m] = cd;
    F.binv[f0 + m] = T(1) / bd;
    const T al = -ae / bd;
    const T ga = up ? -ce / bu : T(0);
    F.alpha[f0 + m] = al;
    F.gamma[f0 + m] = ga;
    const int q = sx<T>(m);
    a[q] = al * ad;
    c[q] = up ? ga * cu : T(0);
    bb[q] = be + al * cd + (up ? ga * au : T(0));
  }
  __syncthreads();
  for (int k = 1; k < K; ++k) {
    const int s = 1 << (k - 1), off = Np - Np / (1 << k);  // s: distance in the compacted system
    // equations eliminated at this level (i = 2s m + s - 1) are final now
    for (int m = threadIdx.x; m < Nh / (2 * s); m += blockDim.x) {
      const int q = sx<T>(2 * s * m + s - 1);
      F.afin[f0 + off + m] = a[q];
      F.cfin[f0 + off + m] = c[q];
      F.binv[f0 + off + m] = T(1) / bb[q];
    }
    // combining equations i = 2s(m + 1) - 1 absorb their neighbours at distance s; the
    // neighbours are not combining at this level, so reading and writing do not overlap
    for (int m = threadIdx.x; m < Nh / (2 * s); m += blockDim.x) {
      const int i = 2 * s * (m + 1) - 1;
      const bool up = i + s < Nh;
      const int q = sx<T>(i), qd = sx<T>(i - s), qu = up ? sx<T>(i + s) : q;
      const T al = -a[q] / bb[qd];
      const T ga = up ? -c[q] / bb[qu] : T(0);
      F.alpha[f0 + off + m] = al;
      F.gamma[f0 + off + m] = ga;
      const T na = al * a[qd];
      const T nc = up ? ga * c[qu] : T(0);
      const T nb = bb[q] + al * c[qd] + (up ? ga * a[qu] : T(0));
      a[q] = na;
      c[q] = nc;
      bb[q] = nb;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {  // the root: no neighbour left
    F.afin[f0 + Np - 1] = T(0);
    F.cfin[f0 + Np - 1] = T(0);
    F.binv[f0 + Np - 1] = T(1) / bb[sx<T>(Nh - 1)];
  }
}

// Factors of the deepest reduction levels (those with at most kLineDeep / 2 equations),
// the last kLineDeep entries of each factor row, are staged in shared memory when a CTA
// starts: their levels then cost no global round trip (the reduction is a chain of
// dependent levels, and each global round trip is one DRAM latency).
constexpr int kLineDeep = 128;

template <typename T>
__host__ __device__ inline size_t zebra_smem(int np) {
  return line_row_smem<T>(np) + (size_t)5 * (np < kLineDeep ? np : kLineDeep) * sizeof(T);
}

// One half-sweep: rows j = par, par + 2, ... (grid: one CTA per such row).  Shared memory:
// the row's right-hand side, overwritten by its solution (padded row), then the deep-level
// factors.  A half-sweep reads rows of the other parity only (and the Dirichlet row ends),
// which no CTA of the launch writes, so x is read through the read-only path.  LU: loop
// iterations whose global loads a thread issues together (the kernel is bound by load
// latency); resident CTAs per SM at the longest rows: 6 (FP32; 5 for the 9-point form with
// four iterations' loads, whose registers do not fit six) / 3 (FP64), which is also what
// shared memory allows there.
// Right-hand-side variants of a half-sweep (compile-time, so the common one carries no extra
// code): the iterate as stored; a zero iterate (nothing read).  FIVE: a 5-point operator
// (L.five_point), whose zero NE / NW couplings are neither loaded nor multiplied.
enum LineMode : int { LM_PLAIN = 0, LM_ZERO = 1 };

template <typename T, int LU, int MODE, bool FIVE = false>
__global__ void __launch_bounds__(kLT, sizeof(T) == 8 ? 3 : (LU <= 2 || FIVE ? 6 : 5))
    k_line_zebra(Lvl<T> L, LineFactors<T> F, T* __restrict__ x, const T* __restrict__ b, int par,
                 const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int j = par + 2 * blockIdx.x;
  if (j >= L.nyr || !row_active(L, j)) return;
  const int N = L.nx - 2, Np = F.np, K = line_levels(Np);
  const int deep = Np < kLineDeep ? Np : kLineDeep, d0 = Np - deep;
  const size_t f0 = (size_t)j * Np;
  extern __shared__ __align__(16) unsigned char line_smem[];
  T* d = reinterpret_cast<T*>(line_smem);
  T* dfac = reinterpret_cast<T*>(line_smem + line_row_smem<T>(Np));  // 5 x deep: alpha gamma afin cfin binv
  // deep-level factors: asynchronous copies now, waited for before the first reduction level
  for (int e = threadIdx.x; e < 5 * deep; e += kLT) {
    const int a = e / deep, m = e - a * deep;
    const T* src = a == 0 ? F.alpha : a == 1 ? F.gamma : a == 2 ? F.afin : a == 3 ? F.cfin : F.binv;
    cp_async_elem(dfac + e, src + f0 + d0 + m);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  const int p = L.pitch;
  const int jd = row_dn(j, L.nyr), ju = row_up(j, L.nyr);
  const size_t r0 = (size_t)j * p, rd = (size_t)jd * p, ru = (size_t)ju * p;
  for (int t0 = threadIdx.x; t0 < Np; t0 += LU * kLT) {
    T v[LU];
#pragma unroll
    for (int u = 0; u < LU; ++u) {
      const int t = t0 + u * kLT;
      v[u] = T(0);
      if (t < N) {
        const int i = t + 1;
        if constexpr (MODE == LM_ZERO) {  // the iterate is zero: every coupling term vanishes
          v[u] = __ldg(b + r0 + i);
        } else {
          auto nb = [&](size_t row0, int, int c) -> T { return __ldg(x + row0 + c); };
          // couplings leaving the row, in the order of the point smoother's sum minus E/W
          T off = __ldg(L.cN + r0 + i) * nb(ru, ju, i);
          off = fma(__ldg(L.cN + rd + i), nb(rd, jd, i), off);
          if constexpr (!FIVE) {
            off = fma(__ldg(L.cNE + r0 + i), nb(ru, ju, i + 1), off);
            off = fma(__ldg(L.cNE + rd + i - 1), nb(rd, jd, i - 1), off);
            off = fma(__ldg(L.cNW + r0 + i), nb(ru, ju, i - 1), off);
            off = fma(__ldg(L.cNW + rd + i + 1), nb(rd, jd, i + 1), off);
          }
          if (i == 1) off = fma(L.cE[r0], __ldg(x + r0), off);
          if (i == N) off = fma(L.cE[r0 + i], __ldg(x + r0 + i + 1), off);
          v[u] = __ldg(b + r0 + i) - off;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < LU; ++u)
      if (t0 + u * kLT < Np) d[sx<T>(t0 + u * kLT)] = v[u];
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  // forward reduction of the right-hand side
  for (int k = 0; k < K; ++k) {
    const int s = 1 << k, off = Np - Np / s, cnt = Np / (2 * s);
    const bool staged = off >= d0;
    for (int m0 = threadIdx.x; m0 < cnt; m0 += LU * kLT) {
      T al[LU], ga[LU];
#pragma unroll
      for (int u = 0; u < LU; ++u) {
        const int m = m0 + u * kLT;
        if (staged) {
          al[u] = m < cnt ? dfac[off - d0 + m] : T(0);
          ga[u] = m < cnt ? dfac[deep + off - d0 + m] : T(0);
        } else {
          al[u] = m < cnt ? __ldg(F.alpha + f0 + off + m) : T(0);
          ga[u] = m < cnt ? __ldg(F.gamma + f0 + off + m) : T(0);
        }
      }
#pragma unroll
      for (int u = 0; u < LU; ++u) {
        const int m = m0 + u * kLT;
        if (m < cnt) {
          const int i = 2 * s * (m + 1) - 1, q = sx<T>(i);
          T v = fma(al[u], d[sx<T>(i - s)], d[q]);
          if (i + s < Np) v = fma(ga[u], d[sx<T>(i + s)], v);
          d[q] = v;
        }
      }
    }
    __syncthreads();
  }
  // back substitution, from the root down; solutions overwrite d
  if (threadIdx.x == 0) d[sx<T>(Np - 1)] *= dfac[4 * deep + deep - 1];
  __syncthreads();
  for (int k = K - 1; k >= 0; --k) {
    const int s = 1 << k, off = Np - Np / s, cnt = Np / (2 * s);
    const bool staged = off >= d0;
    for (int m0 = threadIdx.x; m0 < cnt; m0 += LU * kLT) {
      T af[LU], cf[LU], bi[LU];
#pragma unroll
      for (int u = 0; u < LU; ++u) {
        const int m = m0 + u * kLT;
        if (staged) {
          af[u] = m < cnt ? dfac[2 * deep + off - d0 + m] : T(0);
          cf[u] = m < cnt ? dfac[3 * deep + off - d0 + m] : T(0);
          bi[u] = m < cnt ? dfac[4 * deep + off - d0 + m] : T(0);
        } else {
          af[u] = m < cnt ? __ldg(F.afin + f0 + off + m) : T(0);
          cf[u] = m < cnt ? __ldg(F.cfin + f0 + off + m) : T(0);
          bi[u] = m < cnt ? __ldg(F.binv + f0 + off + m) : T(0);
        }
      }
#pragma unroll
      for (int u = 0; u < LU; ++u) {
        const int m = m0 + u * kLT;
        if (m < cnt) {
          const int i = 2 * s * m + s - 1, q = sx<T>(i);
          T v = d[q];
          if (i - s >= 0) v -= af[u] * d[sx<T>(i - s)];
          v -= cf[u] * d[sx<T>(i + s)];
          d[q] = v * bi[u];
        }
      }
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < N; t += kLT) x[r0 + t + 1] = d[sx<T>(t)];
}

// ------------------------------------------------------------------ partition solver
// Rows of kPartMinNp to kPartMaxNp (padded) unknowns are solved by a partition method instead
// of cyclic reduction over the whole row: the row is cut into kPP segments of S = Np / kPP
// unknowns; the last unknown of each segment is a separator, the other S - 1 form the
// segment's interior, coupled to the rest of the row only through the two separators around
// it.  Eliminating the interiors (one sequential tridiagonal solve per segment, one thread
// each) leaves a tridiagonal system of kPP separator unknowns (the Schur complement), solved
// by cyclic reduction in shared memory; the interiors then follow from the two spike vectors
// of each segment.  The result is the exact solution of the row system, as with cyclic
// reduction over the whole row, up to rounding order.  A sweep's dependent chain of global
// loads is thus a few coalesced batches per thread (interior factors stored segment-minor:
// entry k of every segment contiguous), instead of one round trip per reduction level.
//
// Factor layout per row (the same five arrays of Np entries as cyclic reduction):
//   interior entry k (0 <= k < S - 1) of segment t at k * kPP + t:
//     alpha: sub-diagonal a_k of the interior system (0 for k = 0),
//     gamma: 1 / m_k, the reciprocal Thomas pivot,
//     afin:  c'_k, the eliminated super-diagonal (0 for k = S - 2),
//     cfin:  w_k, the left spike (interior response to the separator before the segment),
//     binv:  v_k, the right spike (response to the separator ending the segment);
//   entries (S - 1) kPP .. Np - 1: the cyclic-reduction factors of the separator system, in
//   the layout described at the top of this file for a row of kPP unknowns.
constexpr int kPP = 256;            // segments per row = threads of a partition CTA

// Padded row lengths solved by the partition method: measured faster than cyclic reduction
// over the whole row on GB300 for 2048 and 4096 (FP32 half-sweeps of 2049^2: 0.078 ms against
// 0.108; 4097^2: 0.256 against 0.276; FP64 0.147 / 0.516 against 0.205 / 0.579), slower for
// 8192 (FP32 0.92 against 0.90 ms: segments of 32 make each thread's sequential chain three
// times 31 dependent steps, and its loads ahead need registers that cost resident rows).
constexpr int kPartMinNp = 2048, kPartMaxNp = 4096;
constexpr int kPartCtas = 4;  // resident CTAs per SM (the kernel's register budget)

__host__ __device__ inline bool line_partitioned(int np) { return np >= kPartMinNp && np <= kPartMaxNp; }

// Coefficients (sub, diagonal, super) of unknown ii of a row system; padding rows (ii >= N)
// are identity equations.
template <typename T>
__device__ __forceinline__ void row_coef(const Lvl<T>& L, size_t r0, int N, int ii, T& a, T& bb, T& c) {
  if (ii < N) {
    a = ii >= 1 ? L.cE[r0 + ii] : T(0);
    bb = L.diag[r0 + ii + 1];
    c = ii <= N - 2 ? L.cE[r0 + ii + 1] : T(0);
  } else {
    a = T(0);
    bb = T(1);
    c = T(0);
  }
}

// Cyclic-reduction factors of a tridiagonal system of n (a power of two) equations held in
// shared memory (padded index sx), written at offset base of the five factor arrays.  The
// same recurrences as k_line_factor; a, bb, c are overwritten.
template <typename T>
__device__ void cr_factor(T* a, T* bb, T* c, int n, const LineFactors<T>& F, size_t base) {
  const int K = line_levels(n);
  for (int k = 0; k < K; ++k) {
    const int s = 1 << k, off = n - n / s;
    for (int m = threadIdx.x; m < n / (2 * s); m += blockDim.x) {
      const int q = sx<T>(2 * s * m + s - 1);
      F.afin[base + off + m] = a[q];
      F.cfin[base + off + m] = c[q];
      F.binv[base + off + m] = T(1) / bb[q];
    }
    for (int m = threadIdx.x; m < n / (2 * s); m += blockDim.x) {
      const int i = 2 * s * (m + 1) - 1;
      const bool up = i + s < n;
      const int q = sx<T>(i), qd = sx<T>(i - s), qu = up ? sx<T>(i + s) : q;
      const T al = -a[q] / bb[qd];
      const T ga = up ? -c[q] / bb[qu] : T(0);
      F.alpha[base + off + m] = al;
      F.gamma[base + off + m] = ga;
      const T na = al * a[qd];
      const T nc = up ? ga * c[qu] : T(0);
      const T nb = bb[q] + al * c[qd] + (up ? ga * a[qu] : T(0));
      a[q] = na;
      c[q] = nc;
      bb[q] = nb;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    F.afin[base + n - 1] = T(0);
    F.cfin[base + n - 1] = T(0);
    F.binv[base + n - 1] = T(1) / bb[sx<T>(n - 1)];
  }
}

// Partition factors of row blockIdx.x (thread t: segment t).  Shared memory: the separator
// system's a, b, c (padded rows of kPP) and the spikes' first entries.
template <typename T>
__global__ void __launch_bounds__(kPP) k_line_pfactor(Lvl<T> L, LineFactors<T> F) {
  const int j = blockIdx.x;
  if (j >= L.nyr || !row_active(L, j)) return;
  const int N = L.nx - 2, Np = F.np, S = Np / kPP, t = threadIdx.x;
  extern __shared__ __align__(16) unsigned char line_smem[];
  const int rs = (int)(line_row_smem<T>(kPP) / sizeof(T));
  T* sa = reinterpret_cast<T*>(line_smem);
  T* sb = sa + rs;
  T* sc = sb + rs;
  T* w0 = sc + rs;  // w_t[0], v_t[0] of every segment
  T* v0 = w0 + kPP;
  const size_t r0 = (size_t)j * L.pitch, f0 = (size_t)j * Np;
  const int i0 = t * S;  // first unknown of the segment
  // interior Thomas factorization, k = 0 .. S - 2
  T cprev = T(0);
  for (int k = 0; k <= S - 2; ++k) {
    T a, bb, c;
    row_coef(L, r0, N, i0 + k, a, bb, c);
    const T ai = k == 0 ? T(0) : a;      // coupling to the separator before the segment: a spike
    const T ci = k == S - 2 ? T(0) : c;  // coupling to the separator ending it: a spike
    const T im = T(1) / (bb - ai * cprev);
    const T cp = ci * im;
    const size_t e = f0 + (size_t)k * kPP + t;
    F.alpha[e] = ai;
    F.gamma[e] = im;
    F.afin[e] = cp;
    cprev = cp;
  }
  // spikes: w = T^-1 (a_first e_0), v = T^-1 (c_last e_{S-2}); forward then backward
  {
    T a0, b0, c0, al, bl, cl;
    row_coef(L, r0, N, i0, a0, b0, c0);
    row_coef(L, r0, N, i0 + S - 2, al, bl, cl);
    T wp = T(0), vp = T(0);
    for (int k = 0; k <= S - 2; ++k) {
      const size_t e = f0 + (size_t)k * kPP + t;
      const T ai = F.alpha[e], im = F.gamma[e];
      wp = ((k == 0 ? a0 : T(0)) - ai * wp) * im;
      vp = ((k == S - 2 ? cl : T(0)) - ai * vp) * im;
      F.cfin[e] = wp;
      F.binv[e] = vp;
    }
    T wn = T(0), vn = T(0);
    for (int k = S - 2; k >= 0; --k) {
      const size_t e = f0 + (size_t)k * kPP + t;
      const T cp = F.afin[e];
      const T w = F.cfin[e] - cp * wn, v = F.binv[e] - cp * vn;
      F.cfin[e] = w;
      F.binv[e] = v;
      wn = w;
      vn = v;
    }
    w0[t] = wn;
    v0[t] = vn;
  }
  __syncthreads();
  // separator system (Schur complement): equation of the separator ending segment t
  {
    T as, bs, cs;
    row_coef(L, r0, N, i0 + S - 1, as, bs, cs);
    const size_t el = f0 + (size_t)(S - 2) * kPP + t;  // last interior entry of the segment
    const T wl = F.cfin[el], vl = F.binv[el];
    const bool nx_ = t + 1 < kPP;
    const T wn = nx_ ? w0[t + 1] : T(0), vn = nx_ ? v0[t + 1] : T(0);
    const int q = sx<T>(t);
    sa[q] = -as * wl;
    sb[q] = bs - as * vl - cs * wn;
    sc[q] = -cs * vn;
  }
  __syncthreads();
  cr_factor<T>(sa, sb, sc, kPP, F, f0 + (size_t)(S - 1) * kPP);
}

// Shared memory of a partition half-sweep: the interior values (segment-minor, rows of
// kPP + 1 to keep the row-order accesses on distinct banks), the separators, the separator
// system's right-hand side / solution (padded) and its factors.
template <typename T>
__host__ __device__ inline size_t part_smem(int np) {
  const int S = np / kPP;
  return ((size_t)(S - 1) * (kPP + 1) + kPP + (line_row_smem<T>(kPP) / sizeof(T)) + 5 * kPP) * sizeof(T);
}

// One half-sweep with the partition solver: rows j = par, par + 2, ... (one CTA per row).
// SS = segment length (template, so the per-segment loops unroll and their coalesced global
// loads are issued ahead of the dependent arithmetic).
template <typename T, int SS, int LU, int MODE>
__global__ void __launch_bounds__(kPP, kPartCtas)
    k_line_part(Lvl<T> L, LineFactors<T> F, T* __restrict__ x, const T* __restrict__ b, int par,
                const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int j = par + 2 * blockIdx.x;
  if (j >= L.nyr || !row_active(L, j)) return;
  constexpr int NI = SS - 1;       // interior unknowns per segment
  constexpr int RS = kPP + 1;      // row stride of the interior block in shared memory
  const int N = L.nx - 2, Np = F.np;
  const int t = threadIdx.x;
  const size_t f0 = (size_t)j * Np;
  extern __shared__ __align__(16) unsigned char line_smem[];
  T* dI = reinterpret_cast<T*>(line_smem);  // interior: entry k of segment t at k * RS + t
  T* dS = dI + (size_t)NI * RS;             // separators
  T* dR = dS + kPP;                         // separator system, padded (sx)
  T* fR = dR + line_row_smem<T>(kPP) / sizeof(T);  // its factors: 5 x kPP
  // separator-system factors: asynchronous copies now, waited for before its reduction
  {
    const size_t base = f0 + (size_t)NI * kPP;
    for (int e = t; e < 5 * kPP; e += kPP) {
      const int a = e / kPP, m = e - a * kPP;
      const T* src = a == 0 ? F.alpha : a == 1 ? F.gamma : a == 2 ? F.afin : a == 3 ? F.cfin : F.binv;
      cp_async_elem(fR + e, src + base + m);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  const int p = L.pitch;
  const int jd = row_dn(j, L.nyr), ju = row_up(j, L.nyr);
  const size_t r0 = (size_t)j * p, rd = (size_t)jd * p, ru = (size_t)ju * p;
  // right-hand side of every unknown, in row order, stored by segment
  for (int t0 = t; t0 < Np; t0 += LU * kPP) {
    T v[LU];
#pragma unroll
    for (int u = 0; u < LU; ++u) {
      const int tt = t0 + u * kPP;
      v[u] = T(0);
      if (tt < N) {
        const int i = tt + 1;
        if constexpr (MODE == LM_ZERO) {
          v[u] = __ldg(b + r0 + i);
        } else {
          auto nb = [&](size_t row0, int, int c) -> T { return __ldg(x + row0 + c); };
          T off = __ldg(L.cN + r0 + i) * nb(ru, ju, i);
          off = fma(__ldg(L.cN + rd + i), nb(rd, jd, i), off);
          if (!L.five_point) {
            off = fma(__ldg(L.cNE + r0 + i), nb(ru, ju, i + 1), off);
            off = fma(__ldg(L.cNE + rd + i - 1), nb(rd, jd, i - 1), off);
            off = fma(__ldg(L.cNW + r0 + i), nb(ru, ju, i - 1), off);
            off = fma(__ldg(L.cNW + rd + i + 1), nb(rd, jd, i + 1), off);
          }
          if (i == 1) off = fma(L.cE[r0], __ldg(x + r0), off);
          if (i == N) off = fma(L.cE[r0 + i], __ldg(x + r0 + i + 1), off);
          v[u] = __ldg(b + r0 + i) - off;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < LU; ++u) {
      const int tt = t0 + u * kPP;
      if (tt < Np) {
        const int sg = tt / SS, k = tt - sg * SS;
        if (k < NI)
          dI[k * RS + sg] = v[u];
        else
          dS[sg] = v[u];
      }
    }
  }
  __syncthreads();
  // interior of segment t: forward and backward Thomas substitution in place in shared
  // memory; the loops unroll, so the coalesced factor loads are issued ahead of the dependent
  // arithmetic as far as registers allow
  {
    const T* fa = F.alpha + f0 + t;
    const T* fg = F.gamma + f0 + t;
    const T* fc = F.afin + f0 + t;
    T dp = T(0);
#pragma unroll
    for (int k = 0; k < NI; ++k) {
      dp = (dI[k * RS + t] - __ldg(fa + (size_t)k * kPP) * dp) * __ldg(fg + (size_t)k * kPP);
      dI[k * RS + t] = dp;
    }
    T yn = T(0);
#pragma unroll
    for (int k = NI - 1; k >= 0; --k) {
      yn = dI[k * RS + t] - __ldg(fc + (size_t)k * kPP) * yn;
      dI[k * RS + t] = yn;
    }
  }
  __syncthreads();
  // right-hand side of the separator system: the separator's equation with its neighbouring
  // interior unknowns replaced by their values for zero separators (y)
  {
    const int is = t * SS + SS - 1;  // the separator's unknown index
    T as = T(0), cs = T(0);
    if (is < N) {
      as = is >= 1 ? L.cE[r0 + is] : T(0);
      cs = is <= N - 2 ? L.cE[r0 + is + 1] : T(0);
    }
    const T yl = dI[(NI - 1) * RS + t];
    const T yr = t + 1 < kPP ? dI[t + 1] : T(0);
    dR[sx<T>(t)] = dS[t] - as * yl - cs * yr;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  // separator system by cyclic reduction, factors in shared memory
  {
    constexpr int n = kPP;
    const int K = line_levels(n);
    for (int k = 0; k < K; ++k) {
      const int s = 1 << k, off = n - n / s, cnt = n / (2 * s);
      for (int m = t; m < cnt; m += kPP) {
        const int i = 2 * s * (m + 1) - 1, q = sx<T>(i);
        T v = fma(fR[off + m], dR[sx<T>(i - s)], dR[q]);
        if (i + s < n) v = fma(fR[n + off + m], dR[sx<T>(i + s)], v);
        dR[q] = v;
      }
      __syncthreads();
    }
    if (t == 0) dR[sx<T>(n - 1)] *= fR[4 * n + n - 1];
    __syncthreads();
    for (int k = K - 1; k >= 0; --k) {
      const int s = 1 << k, off = n - n / s, cnt = n / (2 * s);
      for (int m = t; m < cnt; m += kPP) {
        const int i = 2 * s * m + s - 1, q = sx<T>(i);
        T v = dR[q];
        if (i - s >= 0) v -= fR[2 * n + off + m] * dR[sx<T>(i - s)];
        v -= fR[3 * n + off + m] * dR[sx<T>(i + s)];
        dR[q] = v * fR[4 * n + off + m];
      }
      __syncthreads();
    }
  }
  // interiors from their separators: x = y - x_left w - x_right v
  {
    const T xl = t > 0 ? dR[sx<T>(t - 1)] : T(0);
    const T xr = dR[sx<T>(t)];
    const T* fw = F.cfin + f0 + t;
    const T* fv = F.binv + f0 + t;
#pragma unroll
    for (int k = 0; k < NI; ++k)
      dI[k * RS + t] = dI[k * RS + t] - xl * __ldg(fw + (size_t)k * kPP) - xr * __ldg(fv + (size_t)k * kPP);
    dS[t] = xr;
  }
  __syncthreads();
  for (int tt = t; tt < N; tt += kPP) {
    const int sg = tt / SS, k = tt - sg * SS;
    x[r0 + tt + 1] = k < NI ? dI[k * RS + sg] : dS[sg];
  }
}

// ------------------------------------------------------------------ launchers
template <typename T>
size_t line_factor_elems(int nx, int ny, int periodic) {
  return (size_t)5 * line_np(nx) * rows_stored(ny, periodic);
}

template <typename T>
bool line_supported(int nx) {
  const int np = line_np(nx);
  return nx >= 3 && 3 * line_row_smem<T>(np) <= kLineSmemMax && 3 * zebra_smem<T>(np) <= kLineSmemMax &&
         (!line_partitioned(np) || kPartCtas * part_smem<T>(np) <= kLineSmemMax);
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
  if (line_partitioned(F.np)) {
    const size_t sm = 3 * line_row_smem<T>(kPP) + 2 * kPP * sizeof(T);
    k_line_pfactor<T><<<L.nyr, kPP, sm, s>>>(L, F);
    return cudaGetLastError();
  }
  const size_t sm = 3 * line_row_smem<T>(F.np / 2);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_line_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kLineSmemMax);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_line_factor<T>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_line_factor<T><<<L.nyr, kLT, sm, s>>>(L, F);
  return cudaGetLastError();
}

// Raise the dynamic shared-memory limit of every half-sweep variant of precision T, once
// (thread-safe static initialisation).  All variants share one function type, so the limit
// is set for each explicitly.
template <typename T>
static cudaError_t zebra_attributes() {
  static const cudaError_t st = [] {
    std::vector<const void*> ks;
    auto add = [&](auto lu_c, auto five_c) {
      constexpr int U = decltype(lu_c)::value;
      constexpr bool F5 = decltype(five_c)::value;
      ks.push_back((const void*)k_line_zebra<T, U, LM_PLAIN, F5>);
      ks.push_back((const void*)k_line_zebra<T, U, LM_ZERO, F5>);
    };
    auto add_lu = [&](auto lu_c) {
      add(lu_c, std::false_type());
      add(lu_c, std::true_type());
    };
    add_lu(std::integral_constant<int, 1>());
    add_lu(std::integral_constant<int, 2>());
    add_lu(std::integral_constant<int, 4>());
    for (const void* k : ks) {
      const cudaError_t e =
          cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kLineSmemMax / 3));
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }();
  return st;
}

// Raise the dynamic shared-memory limit of every partition half-sweep variant of precision
// T, once, and let kPartCtas CTAs share an SM.
template <typename T>
static cudaError_t part_attributes() {
  static const cudaError_t st = [] {
    std::vector<const void*> ks;
    auto add = [&](auto ss) {
      constexpr int SS = decltype(ss)::value;
      ks.push_back((const void*)k_line_part<T, SS, 2, LM_PLAIN>);
      ks.push_back((const void*)k_line_part<T, SS, 2, LM_ZERO>);
    };
    add(std::integral_constant<int, kPartMinNp / kPP>());
    add(std::integral_constant<int, kPartMaxNp / kPP>());
    for (const void* k : ks) {
      cudaError_t e =
          cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kLineSmemMax / kPartCtas));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }();
  return st;
}

template <typename T>
static cudaError_t launch_part_rows(const Lvl<T>& L, const LineFactors<T>& F, T* x, const T* b, int par,
                                    int rows, const int* skip, cudaStream_t s, int zero_start) {
  const cudaError_t ea = part_attributes<T>();
  if (ea != cudaSuccess) return ea;
  const size_t sm = part_smem<T>(F.np);
  auto go = [&](auto ss) -> cudaError_t {
    constexpr int SS = decltype(ss)::value;
    if (zero_start)
      k_line_part<T, SS, 2, LM_ZERO><<<rows, kPP, sm, s>>>(L, F, x, b, par, skip);
    else
      k_line_part<T, SS, 2, LM_PLAIN><<<rows, kPP, sm, s>>>(L, F, x, b, par, skip);
    return cudaGetLastError();
  };
  if (F.np == kPartMinNp) return go(std::integral_constant<int, kPartMinNp / kPP>());
  if (F.np == kPartMaxNp) return go(std::integral_constant<int, kPartMaxNp / kPP>());
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_line_rows(const Op<T>& A, const LineFactors<T>& F, T* x, const T* b, int par,
                             const int* skip, cudaStream_t s, const T* eH, int pitch_c, int zero_start) {
  if (!line_supported<T>(A.nx) || F.np != line_np(A.nx)) return cudaErrorInvalidValue;
  if (eH && (par != 1 || (A.nx - 1) % 2 || (A.ny - 1) % 2)) return cudaErrorInvalidValue;
  const Lvl<T> L = lvl_of(A);
  if (eH) {  // the coarse correction enters through the even rows the odd ones are solved from
    constexpr int V = 16 / (int)sizeof(T);
    const bool vec = A.pitch % V == 0 && reinterpret_cast<uintptr_t>(x) % 16 == 0;
    const int erows = (L.nyr + 1) / 2, cols = vec ? (A.nx - 1 + V - 1) / V : A.nx - 1;
    const dim3 g((unsigned)((cols + kLT - 1) / kLT), (unsigned)erows);
    if (vec) k_line_prolong_even<T, true><<<g, kLT, 0, s>>>(L, x, eH, pitch_c, skip);
    else k_line_prolong_even<T, false><<<g, kLT, 0, s>>>(L, x, eH, pitch_c, skip);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (line_partitioned(F.np)) {
    const int rows = (L.nyr - par + 1) / 2;
    if (rows <= 0) return cudaSuccess;
    return launch_part_rows<T>(L, F, x, b, par, rows, skip, s, zero_start);
  }
  const size_t sm = zebra_smem<T>(F.np);
  const int rows = (L.nyr - par + 1) / 2;
  if (rows <= 0) return cudaSuccess;
  // loads batched per thread: measured best on GB300 per precision and row length (FP32 8193^2:
  // 0.90 ms per sweep at 4, 0.97 at 2, 1.02 at 1; 4097^2: 2 best; FP64: 2)
  const int lu = sizeof(T) == 8 ? 2 : (F.np >= 8192 ? 4 : 2);
  const cudaError_t ea = zebra_attributes<T>();
  if (ea != cudaSuccess) return ea;
  auto go = [&](auto kern) -> cudaError_t {
    kern<<<rows, kLT, sm, s>>>(L, F, x, b, par, skip);
    return cudaGetLastError();
  };
  auto mode5 = [&](auto lu_c, auto five_c) -> cudaError_t {
    constexpr int U = decltype(lu_c)::value;
    constexpr bool F5 = decltype(five_c)::value;
    if (zero_start) return go(k_line_zebra<T, U, LM_ZERO, F5>);
    return go(k_line_zebra<T, U, LM_PLAIN, F5>);
  };
  auto mode = [&](auto lu_c) -> cudaError_t {
    return L.five_point ? mode5(lu_c, std::true_type()) : mode5(lu_c, std::false_type());
  };
  if (lu == 4) return mode(std::integral_constant<int, 4>());
  if (lu == 2) return mode(std::integral_constant<int, 2>());
  return mode(std::integral_constant<int, 1>());
}

template <typename T>
cudaError_t launch_line_smooth(const Op<T>& A, const LineFactors<T>& F, T* x, const T* b, int sweeps,
                               int rev, const int* skip, cudaStream_t s, const T* eH, int pitch_c,
                               int zero_start) {
  if (eH && (!rev || sweeps < 1)) return cudaErrorInvalidValue;
  for (int sw = 0; sw < sweeps; ++sw)
    for (int h = 0; h < 2; ++h) {
      const bool first = sw == 0 && h == 0;
      const cudaError_t e = launch_line_rows<T>(A, F, x, b, rev ? 1 - h : h, skip, s, first ? eH : nullptr,
                                                pitch_c, first ? zero_start : 0);
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
                                           const int*, cudaStream_t, const T*, int, int);       \
  template cudaError_t launch_line_smooth<T>(const Op<T>&, const LineFactors<T>&, T*, const T*, int, \
                                             int, const int*, cudaStream_t, const T*, int, int);
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
