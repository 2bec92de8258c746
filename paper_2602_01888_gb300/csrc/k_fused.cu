// Fused multigrid kernels (Sec. 3 cycle, Sec. 2.1 Gauss-Seidel with omega = 1):
//
//  k_smooth_fused  one launch = NS four-colour Gauss-Seidel sweeps on a TX x TY tile,
//                  optionally preceded by the prolongation-correction x += P e_H (Eq. 24).
//                  The tile and a halo of 4 NS nodes (each colour phase shrinks the region
//                  whose values are exact by one node) are staged in shared memory; the
//                  halo work is recomputed by neighbouring tiles instead of synchronising
//                  across the grid.  Input and output iterates are different arrays, so a
//                  tile never sees a neighbour's updated values.
//  k_tail          one CTA runs the whole V-cycle below a small level (smoothing,
//                  residual + full weighting, coarsest dense inverse, prolongation), with
//                  __syncthreads between the phases instead of kernel launches.
#include <mutex>

#include "mg_common.cuh"
#include "mg_fused.h"
#include "mg_launch.h"
#include "mg_tile.h"

namespace mg {

// Row index modulo the period (a staged region may span the period more than once on
// very small periodic levels).
template <typename T>
__device__ __forceinline__ int lwrap(int j, int nyr) {
  j %= nyr;
  return j < 0 ? j + nyr : j;
}

// Bilinear interpolation of the coarse correction at fine node (i, j) (j wrapped).
template <typename T>
__device__ __forceinline__ T interp(const T* eH, int pitchc, int nyrc, int i, int j) {
  const int I = i >> 1, J = j >> 1;
  const int Jp = (J + 1 == nyrc) ? 0 : J + 1;
  const size_t a = (size_t)J * pitchc + I, c = (size_t)Jp * pitchc + I;
  if (!(i & 1) && !(j & 1)) return eH[a];
  if ((i & 1) && !(j & 1)) return T(0.5) * (eH[a] + eH[a + 1]);
  if (!(i & 1)) return T(0.5) * (eH[a] + eH[c]);
  return T(0.25) * ((eH[a] + eH[a + 1]) + (eH[c] + eH[c + 1]));
}

template <typename T, int TX, int TY, int NS>
__global__ void __launch_bounds__(kFusedThreads)
    k_smooth_fused(Lvl<T> L, const T* __restrict__ xin, T* __restrict__ xout,
                   const T* __restrict__ b, int rev, const T* __restrict__ eH, int pitchc,
                   int nyrc, const int* __restrict__ skip) {
  if (skip && *skip) return;
  constexpr int H = 4 * NS, RX = TX + 2 * H, RY = TY + 2 * H, RN = RX * RY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sx = reinterpret_cast<T*>(smem_raw);
  T* sb = sx + RN;
  T* sE = sb + RN;
  T* sN = sE + RN;
  T* sNE = sN + RN;
  T* sNW = sNE + RN;
  T* sD = sNW + RN;
  const int i0 = blockIdx.x * TX - H, j0 = blockIdx.y * TY - H;
  const int p = L.pitch;
  for (int t = threadIdx.x; t < RN; t += blockDim.x) {
    const int lx = t % RX, ly = t / RX;
    const int i = i0 + lx;
    int j = j0 + ly;
    bool in = (i >= 0 && i < L.nx);
    if (L.periodic) j = lwrap<T>(j, L.nyr);
    else in = in && (j >= 0 && j < L.nyr);
    T vx = T(0), vb = T(0), ve = T(0), vn = T(0), vne = T(0), vnw = T(0), vd = T(0);
    if (in) {
      const size_t k = (size_t)j * p + i;
      vx = xin[k];
      vb = b[k];
      ve = L.cE[k];
      vn = L.cN[k];
      vne = L.cNE[k];
      vnw = L.cNW[k];
      vd = L.dinv[k];
      if (eH && is_unknown(L, i, j)) vx += interp<T>(eH, pitchc, nyrc, i, j);
    }
    sx[t] = vx;
    sb[t] = vb;
    sE[t] = ve;
    sN[t] = vn;
    sNE[t] = vne;
    sNW[t] = vnw;
    sD[t] = vd;
  }
  __syncthreads();
#pragma unroll 1
  for (int ph = 0; ph < 4 * NS; ++ph) {
    const int c = rev ? 3 - (ph & 3) : (ph & 3);
    const int ci = colour_ci(c), cj = colour_cj(c);
    const int lo = ph + 1, hx = RX - 2 - ph, hy = RY - 2 - ph;
    const int sx0 = lo + ((ci - i0 - lo) & 1), sy0 = lo + ((cj - j0 - lo) & 1);
    const int ncx = hx >= sx0 ? (hx - sx0) / 2 + 1 : 0;
    const int ncy = hy >= sy0 ? (hy - sy0) / 2 + 1 : 0;
    for (int t = threadIdx.x; t < ncx * ncy; t += blockDim.x) {
      const int lx = sx0 + 2 * (t % ncx), ly = sy0 + 2 * (t / ncx);
      const int i = i0 + lx;
      int j = j0 + ly;
      if (L.periodic) j = lwrap<T>(j, L.nyr);
      else if (j < 0 || j >= L.nyr) continue;
      if (!is_unknown(L, i, j)) continue;
      const int k = ly * RX + lx;
      T s = sE[k] * sx[k + 1];
      s = fma(sE[k - 1], sx[k - 1], s);
      s = fma(sN[k], sx[k + RX], s);
      s = fma(sN[k - RX], sx[k - RX], s);
      s = fma(sNE[k], sx[k + RX + 1], s);
      s = fma(sNE[k - RX - 1], sx[k - RX - 1], s);
      s = fma(sNW[k], sx[k + RX - 1], s);
      s = fma(sNW[k - RX + 1], sx[k - RX + 1], s);
      sx[k] = (sb[k] - s) * sD[k];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < TX * TY; t += blockDim.x) {
    const int lx = H + t % TX, ly = H + t / TX;
    const int i = i0 + lx, j = j0 + ly;  // unwrapped: each node is written by one tile only
    if (i >= L.nx || j >= L.nyr) continue;
    xout[(size_t)j * p + i] = sx[ly * RX + lx];
  }
}

// ------------------------------------------------------------------ tail (one CTA)
// Off-diagonal row sum without restrict qualifiers: in the tail kernel the iterate is
// written by other threads of the block between phases, so its loads must stay coherent.
template <typename T>
__device__ __forceinline__ T offdiag_nr(const Lvl<T>& L, const T* x, int i, int j) {
  const int p = L.pitch;
  const int jd = row_dn(j, L.nyr), ju = row_up(j, L.nyr);
  const size_t r0 = (size_t)j * p, rd = (size_t)jd * p, ru = (size_t)ju * p;
  T s = L.cE[r0 + i] * x[r0 + i + 1];
  s = fma(L.cE[r0 + i - 1], x[r0 + i - 1], s);
  s = fma(L.cN[r0 + i], x[ru + i], s);
  s = fma(L.cN[rd + i], x[rd + i], s);
  s = fma(L.cNE[r0 + i], x[ru + i + 1], s);
  s = fma(L.cNE[rd + i - 1], x[rd + i - 1], s);
  s = fma(L.cNW[r0 + i], x[ru + i - 1], s);
  s = fma(L.cNW[rd + i + 1], x[rd + i + 1], s);
  return s;
}

template <typename T>
__device__ void tail_smooth(const TailLevel<T>& v, int sweeps, int rev) {
  const Lvl<T>& L = v.L;
  for (int s = 0; s < sweeps; ++s)
    for (int c4 = 0; c4 < 4; ++c4) {
      const int c = rev ? 3 - c4 : c4;
      const int ci = colour_ci(c), cj = colour_cj(c);
      const int ncx = (L.nx - ci + 1) / 2, ncy = (L.nyr - cj + 1) / 2;
      for (int t = threadIdx.x; t < ncx * ncy; t += blockDim.x) {
        const int i = ci + 2 * (t % ncx), j = cj + 2 * (t / ncx);
        if (!is_unknown(L, i, j)) continue;
        const size_t k = (size_t)j * L.pitch + i;
        v.x[k] = (v.b[k] - offdiag_nr(L, v.x, i, j)) * L.dinv[k];
      }
      __syncthreads();
    }
}

// Zebra x-line Gauss-Seidel on a tail level (shared memory, pitch = nx): the rows of one
// parity, then the other (reverse order when rev), one thread per row solving its
// tridiagonal system (diagonal and E couplings) by the Thomas algorithm: the rows of the tail
// levels have at most a few dozen unknowns, fewer sequential steps than cyclic reduction's
// barriers.  Right-hand side: b minus the couplings to the rows above and below and to the
// row's two Dirichlet ends, as in k_line_zebra.  The eliminated super-diagonal goes to the
// level's scratch array t and the eliminated right-hand side into x itself (a row's old
// values are never read), then the back substitution runs in place.
template <typename T>
__device__ void tail_line(const TailLevel<T>& v, int sweeps, int rev) {
  const Lvl<T>& L = v.L;
  const int N = L.nx - 2, p = L.pitch;
  T* x = v.x;
  T* cp = v.t;
  for (int s = 0; s < sweeps; ++s)
    for (int h = 0; h < 2; ++h) {
      const int par = rev ? 1 - h : h;
      const int nrows = (L.nyr - par + 1) / 2;
      for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
        const int j = par + 2 * r;
        if (!(L.periodic || (j >= 1 && j <= L.ny - 2))) continue;
        const int jd = row_dn(j, L.nyr), ju = row_up(j, L.nyr);
        const int r0 = j * p, rd = jd * p, ru = ju * p;
        T cprev = T(0), dprev = T(0);
        for (int i = 1; i <= N; ++i) {
          T off = L.cN[r0 + i] * x[ru + i];
          off = fma(L.cN[rd + i], x[rd + i], off);
          if (!L.five_point) {
            off = fma(L.cNE[r0 + i], x[ru + i + 1], off);
            off = fma(L.cNE[rd + i - 1], x[rd + i - 1], off);
            off = fma(L.cNW[r0 + i], x[ru + i - 1], off);
            off = fma(L.cNW[rd + i + 1], x[rd + i + 1], off);
          }
          if (i == 1) off = fma(L.cE[r0], x[r0], off);
          if (i == N) off = fma(L.cE[r0 + i], x[r0 + i + 1], off);
          const T rhs = v.b[r0 + i] - off;
          const T a = i > 1 ? L.cE[r0 + i - 1] : T(0);  // coupling to the left unknown
          const T c = i < N ? L.cE[r0 + i] : T(0);      // and to the right one
          const T rm = T(1) / (L.diag[r0 + i] - a * cprev);
          cprev = c * rm;
          dprev = (rhs - a * dprev) * rm;
          cp[r0 + i] = cprev;
          x[r0 + i] = dprev;
        }
        for (int i = N - 1; i >= 1; --i) x[r0 + i] = x[r0 + i] - cp[r0 + i] * x[r0 + i + 1];
      }
      __syncthreads();
    }
}

// Bytes of shared memory that hold every array of the tail levels.
template <typename T>
size_t tail_smem_bytes(const TailArgs<T>& a) {
  size_t n = 0;
  for (int l = 0; l < a.nlev; ++l) n += (size_t)a.lv[l].L.nx * a.lv[l].L.nyr;
  return n * 9 * sizeof(T);
}

// The tail levels are copied into shared memory (compact rows, pitch = nx), the cycle
// runs there, and only the top level's iterate is written back.
template <typename T>
__global__ void __launch_bounds__(kTailThreads) k_tail(TailArgs<T> a, const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double bs[kCoarseMax];
  __shared__ TailLevel<T> S[kMaxTail];
  const int nl = a.nlev;
  {
    T* p = reinterpret_cast<T*>(smem_raw);
    for (int l = 0; l < nl; ++l) {
      const Lvl<T>& G = a.lv[l].L;
      const int n = G.nx * G.nyr;
      Lvl<T> L = G;
      L.pitch = G.nx;
      T* cE = p; T* cN = p + n; T* cNE = p + 2 * n; T* cNW = p + 3 * n;
      T* dg = p + 4 * n; T* di = p + 5 * n;
      L.cE = cE; L.cN = cN; L.cNE = cNE; L.cNW = cNW; L.diag = dg; L.dinv = di;
      T* xs = p + 6 * n;
      T* bsm = p + 7 * n;
      if (threadIdx.x == 0) {
        S[l].L = L;
        S[l].x = xs;
        S[l].b = bsm;
        S[l].t = p + 8 * n;
      }
      p += 9 * n;
      for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int i = q % G.nx, j = q / G.nx;
        const size_t k = (size_t)j * G.pitch + i;
        cE[q] = G.cE[k];
        cN[q] = G.cN[k];
        cNE[q] = G.cNE[k];
        cNW[q] = G.cNW[k];
        dg[q] = G.diag[k];
        di[q] = G.dinv[k];
        xs[q] = (l == 0) ? a.lv[0].x[k] : T(0);
        bsm[q] = (l == 0) ? a.lv[0].b[k] : T(0);
      }
    }
  }
  __syncthreads();
  for (int l = 0; l < nl - 1; ++l) {
    const TailLevel<T>& f = S[l];
    const TailLevel<T>& g = S[l + 1];
    if (a.line) tail_line(f, a.nu1, 0);
    else tail_smooth(f, a.nu1, 0);
    for (int t = threadIdx.x; t < f.L.nx * f.L.nyr; t += blockDim.x) {
      const int i = t % f.L.nx, j = t / f.L.nx;
      f.t[t] = is_unknown(f.L, i, j) ? f.b[t] - fma(f.L.diag[t], f.x[t], offdiag_nr(f.L, f.x, i, j)) : T(0);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < g.L.nx * g.L.nyr; t += blockDim.x) {
      const int I = t % g.L.nx, J = t / g.L.nx;
      T v = T(0);
      if (is_unknown(g.L, I, J)) {
        const int fi = 2 * I, fj = 2 * J;
        const int jd = row_dn(fj, f.L.nyr), ju = row_up(fj, f.L.nyr);
        const T* r = f.t;
        const int p = f.L.nx, r0 = fj * p, rd = jd * p, ru = ju * p;
        const T edge = r[r0 + fi - 1] + r[r0 + fi + 1] + r[rd + fi] + r[ru + fi];
        const T corner = r[rd + fi - 1] + r[rd + fi + 1] + r[ru + fi - 1] + r[ru + fi + 1];
        v = (T(4) * r[r0 + fi] + T(2) * edge + corner) * T(0.0625);
      }
      g.b[t] = v;
      g.x[t] = T(0);
    }
    __syncthreads();
  }
  {
    const TailLevel<T>& c = S[nl - 1];
    const int ux = c.L.nx - 2, uy = c.L.periodic ? c.L.nyr : c.L.ny - 2;
    const int m = ux * uy, j0 = c.L.periodic ? 0 : 1;
    for (int q = threadIdx.x; q < m; q += blockDim.x) bs[q] = (double)c.b[(j0 + q / ux) * c.L.nx + 1 + q % ux];
    __syncthreads();
    for (int q = threadIdx.x; q < m; q += blockDim.x) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) s = fma(a.inv[(size_t)k * m + q], bs[k], s);
      c.x[(j0 + q / ux) * c.L.nx + 1 + q % ux] = (T)s;
    }
    __syncthreads();
  }
  for (int l = nl - 2; l >= 0; --l) {
    const TailLevel<T>& f = S[l];
    const TailLevel<T>& g = S[l + 1];
    for (int t = threadIdx.x; t < f.L.nx * f.L.nyr; t += blockDim.x) {
      const int i = t % f.L.nx, j = t / f.L.nx;
      if (is_unknown(f.L, i, j)) f.x[t] += interp<T>(g.x, g.L.nx, g.L.nyr, i, j);
    }
    __syncthreads();
    if (a.line) tail_line(f, a.nu2, 1);
    else tail_smooth(f, a.nu2, 1);
  }
  {
    const Lvl<T>& G = a.lv[0].L;
    for (int q = threadIdx.x; q < G.nx * G.nyr; q += blockDim.x)
      a.lv[0].x[(size_t)(q / G.nx) * G.pitch + q % G.nx] = S[0].x[q];
  }
}

// ------------------------------------------------------------------ launchers
// Variants (owned tile, sweeps per launch); the staged region of a variant is
// (tx + 8 ns) x (ty + 8 ns) nodes of seven arrays, at most 179 KB (FP64 64 x 24, two sweeps).
constexpr SmoothVariant kFusedTable[] = {{32, 32, 1}, {64, 16, 1}, {64, 24, 1},
                                         {32, 32, 2}, {64, 16, 2}, {64, 24, 2}};
constexpr int kFusedCount = (int)(sizeof(kFusedTable) / sizeof(kFusedTable[0]));

template <typename T>
static int fused_default() {
  return sizeof(T) == 8 ? 0 : 5;  // FP64 32 x 32, one sweep; FP32 64 x 24, two sweeps
}

template <typename T>
int fused_variants() {
  return kFusedCount;
}

template <typename T>
SmoothVariant fused_variant(int v) {
  return kFusedTable[(v < 0 || v >= kFusedCount) ? fused_default<T>() : v];
}

template <typename T>
int fused_sweeps(int v) {
  return fused_variant<T>(v).ns;
}

template <typename T, int TX, int TY, int NS>
static cudaError_t fused_impl(const Op<T>& A, const T* xin, T* xout, const T* b, int rev, const T* eH,
                              int pitch_c, const int* skip, cudaStream_t s) {
  constexpr int H = 4 * NS;
  constexpr size_t sm = (size_t)7 * (TX + 2 * H) * (TY + 2 * H) * sizeof(T);
  static_assert(sm <= 227 * 1024, "staged region must fit in shared memory");
  auto kern = k_smooth_fused<T, TX, TY, NS>;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [&] {
    attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  });
  if (attr != cudaSuccess) return attr;
  const Lvl<T> L = lvl_of(A);
  const int nyc = (A.ny - 1) / 2 + 1;
  dim3 grid((L.nx + TX - 1) / TX, (L.nyr + TY - 1) / TY);
  kern<<<grid, kFusedThreads, sm, s>>>(L, xin, xout, b, rev, eH, pitch_c,
                                      eH ? rows_stored(nyc, A.periodic) : 0, skip);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_smooth_fused(const Op<T>& A, const T* xin, T* xout, const T* b, int rev,
                                const T* eH, int pitch_c, const int* skip, cudaStream_t s, int v) {
  if (v < 0 || v >= kFusedCount) v = fused_default<T>();
  switch (v) {
    case 0: return fused_impl<T, 32, 32, 1>(A, xin, xout, b, rev, eH, pitch_c, skip, s);
    case 1: return fused_impl<T, 64, 16, 1>(A, xin, xout, b, rev, eH, pitch_c, skip, s);
    case 2: return fused_impl<T, 64, 24, 1>(A, xin, xout, b, rev, eH, pitch_c, skip, s);
    case 3: return fused_impl<T, 32, 32, 2>(A, xin, xout, b, rev, eH, pitch_c, skip, s);
    case 4: return fused_impl<T, 64, 16, 2>(A, xin, xout, b, rev, eH, pitch_c, skip, s);
    default: return fused_impl<T, 64, 24, 2>(A, xin, xout, b, rev, eH, pitch_c, skip, s);
  }
}

template <typename T>
cudaError_t launch_tail(const TailArgs<T>& a, const int* skip, cudaStream_t s) {
  const size_t sm = tail_smem_bytes(a);
  if (sm > kTailSmemMax) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTailSmemMax);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_tail<T><<<1, kTailThreads, sm, s>>>(a, skip);
  return cudaGetLastError();
}

template <typename T>
size_t tail_bytes(const TailArgs<T>& a) {
  return tail_smem_bytes(a);
}
template size_t tail_bytes<double>(const TailArgs<double>&);
template size_t tail_bytes<float>(const TailArgs<float>&);

template int fused_sweeps<double>(int);
template int fused_sweeps<float>(int);
template int fused_variants<double>();
template int fused_variants<float>();
template SmoothVariant fused_variant<double>(int);
template SmoothVariant fused_variant<float>(int);
template cudaError_t launch_smooth_fused<double>(const Op<double>&, const double*, double*,
                                                 const double*, int, const double*, int, const int*,
                                                 cudaStream_t, int);
template cudaError_t launch_smooth_fused<float>(const Op<float>&, const float*, float*, const float*,
                                                int, const float*, int, const int*, cudaStream_t, int);
template cudaError_t launch_tail<double>(const TailArgs<double>&, const int*, cudaStream_t);
template cudaError_t launch_tail<float>(const TailArgs<float>&, const int*, cudaStream_t);

}  // namespace mg
