// Setup kernels: coefficient build (Eqs. 1, 10-15, 39-42), fine-level operator,
// right-hand side (Eq. 11), Galerkin coarse operators (Sec. 3) and the coarsest-level
// inverse.  They run once per problem (or per geometry update); everything is FP64
// except the Galerkin products of the mixed-precision hierarchy, which are FP32.
#include "mg_common.cuh"
#include "mg_kernels.h"
#include "mg_launch.h"

namespace mg {

static const double kPi = 3.14159265358979323846;

// eps = det(J) J^-1 (s I) J^-T for J = [[a, b], [c, d]] (Eqs. 10, 12-15).  cross = 0: a map
// whose Eq. 13 vanishes identically (J^T J diagonal); eps_xy is then written as the exact
// zero instead of the rounding residue of the general formula.
__device__ __forceinline__ void store_eps(double a, double b, double c, double d, double s,
                                          size_t k, double* D, double* exx, double* exy,
                                          double* eyy, int* folded, int cross = 1) {
  const double det = a * d - b * c;
  if (!(det > 0.0)) atomicOr(folded, 1);
  D[k] = det;
  const double sd = s / det;            // one division per node
  exx[k] = sd * (d * d + b * b);        // Eq. 12
  exy[k] = cross ? sd * (-d * c - b * a) : 0.0;  // Eq. 13 = Eq. 14
  eyy[k] = sd * (c * c + a * a);        // Eq. 15
}

// One CTA per 32 x 32 tile of nodes (32 x 8 threads, four rows each).  Every analytic map's
// Jacobian is built from transcendental factors of x alone and of y alone, so they are
// evaluated once per column and once per row of the tile, in shared memory, rather than once
// per node: FP64 transcendentals, not memory traffic, bound this kernel otherwise.  The
// factors are the same calls on the same arguments as a per-node evaluation, so the results
// do not change.
constexpr int kEpsTile = 32;

__global__ void __launch_bounds__(256) k_eps_analytic(int kind, double p0, double p1, double p2,
                                                      double p3, int nx, int nyr, double x0, double y0,
                                                      double hx, double hy,
                                                      const double* __restrict__ eps, int pitch,
                                                      double* D, double* exx, double* exy, double* eyy,
                                                      int* folded, int cross) {
  __shared__ double colv[4][kEpsTile], rowv[2][kEpsTile];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i0 = blockIdx.x * kEpsTile, j0 = blockIdx.y * kEpsTile;
  if (ty == 0) {  // factors of x
    const double x = x0 + (i0 + tx) * hx;
    if (kind == 1) {
      sincos(kPi * x, &colv[0][tx], &colv[1][tx]);
      sincos(2.0 * kPi * x, &colv[2][tx], &colv[3][tx]);
    } else if (kind == 3) {
      colv[0][tx] = cosh(p1 * x);
    }
  } else if (ty == 1) {  // factors of y
    const double y = y0 + (j0 + tx) * hy;
    if (kind == 1) sincos(kPi * y, &rowv[0][tx], &rowv[1][tx]);
    else if (kind == 2) sincos(y, &rowv[0][tx], &rowv[1][tx]);
    else if (kind == 3) rowv[0][tx] = cosh(p1 * y);
  }
  __syncthreads();
  const int i = i0 + tx;
  if (i >= nx) return;
  const double x = x0 + i * hx;
#pragma unroll
  for (int r = 0; r < kEpsTile / 8; ++r) {
    const int ly = ty + 8 * r, j = j0 + ly;
    if (j >= nyr) break;
    double a = 1.0, b = 0.0, c = 0.0, d = 1.0;  // Jxx Jxy Jyx Jyy
    switch (kind) {
      case 1: {  // sine warp
        const double sx = colv[0][tx], cx = colv[1][tx], s2x = colv[2][tx], c2x = colv[3][tx];
        const double sy = rowv[0][ly], cy = rowv[1][ly];
        a = 1.0 + p0 * kPi * cx * sy;
        b = p0 * kPi * sx * cy;
        c = p0 * 2.0 * kPi * c2x * sy;
        d = 1.0 + p0 * kPi * s2x * cy;
        break;
      }
      case 2: {  // polar, Eq. 29
        const double sy = rowv[0][ly], cy = rowv[1][ly];
        a = cy;
        b = -x * sy;
        c = sy;
        d = x * cy;
        break;
      }
      case 3:  // sinh stretching, Eq. 52
        a = p0 * p1 * colv[0][tx];
        d = p0 * p1 * rowv[0][ly];
        break;
      case 4:  // affine
        a = p0;
        b = p1;
        c = p2;
        d = p3;
        break;
      default:
        break;
    }
    const size_t k = (size_t)j * pitch + i;
    store_eps(a, b, c, d, eps ? eps[k] : 1.0, k, D, exx, exy, eyy, folded, cross);
  }
}

// Even reflection of a grid with Neumann y sides into the periodic grid of twice the height
// (2n rows, n = ny - 1): row j' of the doubled grid copies row j' - n (j' >= n) or n - j'
// (j' < n) of the source, with eps_xy negated in the mirrored half and zero on the two
// Neumann rows (j' = 0, n), where an odd function vanishes.
__global__ void k_mirror_eps(int nx, int n, int ps, const double* __restrict__ D0,
                             const double* __restrict__ exx0, const double* __restrict__ exy0,
                             const double* __restrict__ eyy0, int pd, double* D, double* exx,
                             double* exy, double* eyy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int jd = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || jd >= 2 * n) return;
  const int js = jd >= n ? jd - n : n - jd;
  const double sg = (jd == 0 || jd == n) ? 0.0 : (jd > n ? 1.0 : -1.0);
  const size_t s = (size_t)js * ps + i, d = (size_t)jd * pd + i;
  D[d] = D0[s];
  exx[d] = exx0[s];
  exy[d] = sg * exy0[s];
  eyy[d] = eyy0[s];
}

// d/dx: central difference (Eqs. 39, 41), one-sided second order at the line ends;
// i2h = 1 / (2 hx).
__device__ __forceinline__ double ddx(const double* __restrict__ f, size_t r, int i, int nx,
                                      double i2h) {
  if (i == 0) return (-3.0 * f[r] + 4.0 * f[r + 1] - f[r + 2]) * i2h;
  if (i == nx - 1) return (3.0 * f[r + nx - 1] - 4.0 * f[r + nx - 2] + f[r + nx - 3]) * i2h;
  return (f[r + i + 1] - f[r + i - 1]) * i2h;
}

// d/dy (Eqs. 40, 42); a periodic line wraps and adds `jump` across the seam; i2h = 1 / (2 hy).
__device__ __forceinline__ double ddy(const double* __restrict__ f, int i, int j, int ny, int nyr,
                                      int periodic, int pitch, double i2h, double jump) {
  if (periodic) {
    const double fp = (j + 1 >= nyr) ? f[(size_t)(j + 1 - nyr) * pitch + i] + jump
                                     : f[(size_t)(j + 1) * pitch + i];
    const double fm = (j - 1 < 0) ? f[(size_t)(j - 1 + nyr) * pitch + i] - jump
                                  : f[(size_t)(j - 1) * pitch + i];
    return (fp - fm) * i2h;
  }
  if (j == 0)
    return (-3.0 * f[i] + 4.0 * f[(size_t)pitch + i] - f[2 * (size_t)pitch + i]) * i2h;
  if (j == ny - 1)
    return (3.0 * f[(size_t)(ny - 1) * pitch + i] - 4.0 * f[(size_t)(ny - 2) * pitch + i] +
            f[(size_t)(ny - 3) * pitch + i]) * i2h;
  return (f[(size_t)(j + 1) * pitch + i] - f[(size_t)(j - 1) * pitch + i]) * i2h;
}

__global__ void k_eps_grid(int nx, int ny, int nyr, int periodic, double i2hx, double i2hy,
                           const double* __restrict__ xp, const double* __restrict__ yp,
                           double jump_x, double jump_y, const double* __restrict__ eps,
                           int pitch, double* D, double* exx, double* exy, double* eyy,
                           int* folded) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= nyr) return;
  const size_t r = (size_t)j * pitch, k = r + i;
  const double a = ddx(xp, r, i, nx, i2hx);                                  // Eq. 39
  const double b = ddy(xp, i, j, ny, nyr, periodic, pitch, i2hy, jump_x);    // Eq. 40
  const double c = ddx(yp, r, i, nx, i2hx);                                  // Eq. 41
  const double d = ddy(yp, i, j, ny, nyr, periodic, pitch, i2hy, jump_y);    // Eq. 42
  store_eps(a, b, c, d, eps ? eps[k] : 1.0, k, D, exx, exy, eyy, folded);
}

// Couplings of the symmetric conservative 9-point operator A = -L_h.  five: eps_xy is zero
// everywhere, so the NE / NW couplings are zero and written without reading it.
template <typename T>
__global__ void k_assemble_couplings(int nx, int ny, int nyr, int periodic, int pitch, T ihx2,
                                     T ihy2, T ixy4, const T* __restrict__ exx,
                                     const T* __restrict__ exy,
                                     const T* __restrict__ eyy, T* cE, T* cN,
                                     T* cNE, T* cNW, int five) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= nyr) return;
  const size_t k = (size_t)j * pitch + i;
  const bool has_up = periodic || (j + 1 <= ny - 1);
  const int ju = (j + 1 == nyr) ? 0 : j + 1;
  const size_t ku = (size_t)ju * pitch + i;
  T e = T(0), n = T(0), ne = T(0), nw = T(0);
  if (i + 1 <= nx - 1) e = T(-0.5) * (exx[k] + exx[k + 1]) * ihx2;
  if (has_up) {
    n = T(-0.5) * (eyy[k] + eyy[ku]) * ihy2;
    if (!five) {
      if (i + 1 <= nx - 1) ne = -(exy[k + 1] + exy[ku]) * ixy4;  // to (i+1, j+1)
      if (i >= 1) nw = (exy[k - 1] + exy[ku]) * ixy4;             // to (i-1, j+1)
    }
  }
  cE[k] = e;
  cN[k] = n;
  cNE[k] = ne;
  cNW[k] = nw;
}

// diag = -(sum of the 8 couplings) at unknowns (zero row sums), 1 at Dirichlet nodes; the
// zero NE / NW terms of a 5-point operator are left out of the sum (which they do not change).
// dinv = 1 / diag unless dinv is null (a mixed-precision hierarchy takes its FP32 reciprocal
// from the FP32 diagonal instead and never reads an FP64 one).
template <typename T>
__global__ void k_assemble_diag(int nx, int ny, int nyr, int periodic, int pitch,
                                const T* __restrict__ cE, const T* __restrict__ cN,
                                const T* __restrict__ cNE, const T* __restrict__ cNW,
                                T* diag, T* dinv, int five) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= nyr) return;
  const size_t k = (size_t)j * pitch + i;
  const bool unk = (i >= 1 && i <= nx - 2) && (periodic || (j >= 1 && j <= ny - 2));
  if (!unk) {
    diag[k] = T(1);
    if (dinv) dinv[k] = T(1);
    return;
  }
  const int jd = (j == 0) ? nyr - 1 : j - 1;
  const size_t ks = (size_t)jd * pitch + i;
  T s = cE[k] + cE[k - 1] + cN[k] + cN[ks];
  if (!five) s = s + cNE[k] + cNE[ks - 1] + cNW[k] + cNW[ks + 1];
  diag[k] = -s;
  if (dinv) dinv[k] = T(1) / (-s);
}

// One pass for an operator without cross term (5-point, eps_xy = 0): the E and N couplings
// of k_assemble_couplings, the diagonal (and its reciprocal when dinv is given) of
// k_assemble_diag and, when fE is given, the FP32 copy of k_op_to_f32 with the reciprocal of
// the FP32 diagonal (pitch pf).  A warp covers 32 columns of a row and each thread marches
// down kAsmRows rows: the coupling to the W neighbour is the left lane's E coupling (shuffle),
// the one to the S neighbour the thread's N coupling of the row before; the first lane and the
// first row of a strip compute theirs again.  A coupling is rounded like the separate
// kernel's: -(1/2)(a + b) / h^2 is the sum times the exact constant -(1/2) / h^2 (halving is
// exact), one rounding per operation (__dadd_rn, __dmul_rn: no contracted multiply-add), so
// the values are bitwise those of the separate kernels.  NE / NW get zeros, as from
// k_assemble_couplings, for the kernels that have no 5-point form.  GB300 issues FP64 at a
// low rate: ten FP64 operations per node here, as many as the three separate kernels take.
constexpr int kAsmRows = 8;

__global__ void __launch_bounds__(256) k_assemble_five(int nx, int ny, int nyr, int periodic, int pitch, double mx,
                                                       double my, const double* __restrict__ exx,
                                                       const double* __restrict__ eyy, double* cE, double* cN,
                                                       double* cNE, double* cNW, double* diag, double* dinv, int pf,
                                                       float* fE, float* fN, float* fNE, float* fNW, float* fdiag,
                                                       float* fdinv) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int jb = (blockIdx.y * blockDim.y + threadIdx.y) * kAsmRows;
  const bool col = i < nx;
  const bool has_e = i + 1 <= nx - 1;
  double n_prev = 0.0;
  for (int r = 0; r < kAsmRows; ++r) {
    const int j = jb + r;
    if (j >= nyr) break;  // the same for the whole warp (one row per warp)
    const size_t k = (size_t)j * pitch + i;
    const int ju = (j + 1 == nyr) ? 0 : j + 1;
    const double e = (col && has_e) ? __dmul_rn(__dadd_rn(exx[k], exx[k + 1]), mx) : 0.0;
    const double n = (col && (periodic || j + 1 <= ny - 1))
                         ? __dmul_rn(__dadd_rn(eyy[k], eyy[(size_t)ju * pitch + i]), my) : 0.0;
    double ew = __shfl_up_sync(0xffffffffu, e, 1);
    double ns = n_prev;
    n_prev = n;
    if (!col) continue;
    const bool unk = (i >= 1 && i <= nx - 2) && (periodic || (j >= 1 && j <= ny - 2));
    double d = 1.0;
    if (unk) {
      if (threadIdx.x == 0) ew = __dmul_rn(__dadd_rn(exx[k - 1], exx[k]), mx);
      if (r == 0) ns = __dmul_rn(__dadd_rn(eyy[(size_t)((j == 0) ? nyr - 1 : j - 1) * pitch + i], eyy[k]), my);
      d = -__dadd_rn(__dadd_rn(__dadd_rn(e, ew), n), ns);
    }
    cE[k] = e;
    cN[k] = n;
    cNE[k] = 0.0;
    cNW[k] = 0.0;
    diag[k] = d;
    if (dinv) dinv[k] = unk ? 1.0 / d : 1.0;
    if (fE) {
      const size_t kf = (size_t)j * pf + i;
      fE[kf] = (float)e;
      fN[kf] = (float)n;
      fNE[kf] = 0.0f;
      fNW[kf] = 0.0f;
      const float dg = (float)d;
      fdiag[kf] = dg;
      fdinv[kf] = 1.0f / dg;
    }
  }
}

__global__ void k_rhs(int nx, int ny, int nyr, int periodic, int pitch,
                      const double* __restrict__ rho, int rho_pitch, const double* __restrict__ D,
                      double* b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= nyr) return;
  const bool unk = (i >= 1 && i <= nx - 2) && (periodic || (j >= 1 && j <= ny - 2));
  const size_t k = (size_t)j * pitch + i;
  b[k] = unk ? rho[(size_t)j * rho_pitch + i] * D[k] : 0.0;  // Eq. 11
}

// Tensor of the next coarser level of a rediscretized hierarchy: each of the three nodal
// fields at coarse node (I, J), full weighting (1/16)[1 2 1; 2 4 2; 1 2 1] about fine node
// (2I, 2J) where all eight fine neighbours exist (rows wrap when periodic), the coincident
// fine value on the coarse boundary ring.
// TS / TD: precision of the fine and of the coarse fields (the mixed path coarsens in FP32).
// five: the cross term is zero on the fine level, so on the coarse one (written, not computed).
template <typename TS, typename TD>
__global__ void k_coarsen_eps(int nxf, int nyrf, int pf, int nxc, int nyc, int nyrc, int pc, int periodic,
                              const TS* __restrict__ f0, const TS* __restrict__ f1,
                              const TS* __restrict__ f2, TD* c0, TD* c1, TD* c2, int five) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= nxc || J >= nyrc) return;
  const int fi = 2 * I, fj = 2 * J;
  const bool inner = (I >= 1 && I <= nxc - 2) && (periodic || (J >= 1 && J <= nyc - 2));
  const int jd = fj == 0 ? nyrf - 1 : fj - 1, ju = fj + 1 == nyrf ? 0 : fj + 1;
  const size_t r0 = (size_t)fj * pf, rd = (size_t)jd * pf, ru = (size_t)ju * pf, K = (size_t)J * pc + I;
  const TS* const f[3] = {f0, f1, f2};
  TD* const c[3] = {c0, c1, c2};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a == 1 && five) {
      c[a][K] = TD(0);
      continue;
    }
    const TS* g = f[a];
    TD v;
    if (inner)
      v = (TD(4) * TD(g[r0 + fi]) +
           TD(2) * (TD(g[r0 + fi - 1]) + TD(g[r0 + fi + 1]) + TD(g[rd + fi]) + TD(g[ru + fi])) +
           (TD(g[rd + fi - 1]) + TD(g[rd + fi + 1]) + TD(g[ru + fi - 1]) + TD(g[ru + fi + 1]))) / TD(16);
    else
      v = TD(g[r0 + fi]);
    c[a][K] = v;
  }
}

// Bilinear weight of a fine offset d from a coarse node (in fine units).
__host__ __device__ constexpr double pw(int d) { return d == 0 ? 1.0 : ((d == 1 || d == -1) ? 0.5 : 0.0); }

// A[(fi,fj),(fi+di,fj+dj)] through the symmetric storage of a level.
template <typename T>
__device__ __forceinline__ T fine_entry(const Lvl<T>& F, int fi, int fj, int di, int dj) {
  const size_t r0 = (size_t)fj * F.pitch, rd = (size_t)row_dn(fj, F.nyr) * F.pitch;
  if (dj == 0) {
    if (di == 0) return F.diag[r0 + fi];
    return di > 0 ? F.cE[r0 + fi] : F.cE[r0 + fi - 1];
  }
  if (dj > 0) {
    if (di == 0) return F.cN[r0 + fi];
    return di > 0 ? F.cNE[r0 + fi] : F.cNW[r0 + fi];
  }
  if (di == 0) return F.cN[rd + fi];
  return di < 0 ? F.cNE[rd + fi - 1] : F.cNW[rd + fi + 1];
}

// A_H = (1/4) P^T A_h P: for each coarse unknown I, row(I, I+o) = (1/4) sum_k sum_l
// P(k, I) A(k, l) P(l, I+o) over fine k in the 3x3 support of I and the 9 stencil
// neighbours l of k, for the five entries stored (o = centre, E, N, NE, NW; the others are
// the symmetric partners' entries).  Every loop is unrolled so the bilinear weights are
// constants and only the (k, l, o) triples with non-zero weight remain (109 multiply-adds).
// FIVE: the fine operator is 5-point (F.five_point): its diagonal entries are zero and their
// products, which would add zeros, are skipped (69 multiply-adds, the same sums).
template <typename T, bool FIVE>
__global__ void k_galerkin(Lvl<T> F, int nxc, int nyc, int nyrc, int pitchc, T* cE, T* cN, T* cNE,
                           T* cNW, T* diag, T* dinv) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= nxc || J >= nyrc) return;
  const size_t K = (size_t)J * pitchc + I;
  const bool unk = (I >= 1 && I <= nxc - 2) && (F.periodic || (J >= 1 && J <= nyc - 2));
  if (!unk) {
    cE[K] = cN[K] = cNE[K] = cNW[K] = T(0);
    diag[K] = dinv[K] = T(1);
    return;
  }
  T row[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) row[a][b] = T(0);
#pragma unroll
  for (int kj = -1; kj <= 1; ++kj) {
    int fj = 2 * J + kj;
    if (fj < 0) fj += F.nyr;
    if (fj >= F.nyr) fj -= F.nyr;
#pragma unroll
    for (int ki = -1; ki <= 1; ++ki) {
      const int fi = 2 * I + ki;
#pragma unroll
      for (int lj = -1; lj <= 1; ++lj)
#pragma unroll
        for (int li = -1; li <= 1; ++li) {
          if (FIVE && li != 0 && lj != 0) continue;
          const T a = fine_entry(F, fi, fj, li, lj);
#pragma unroll
          for (int oj = 0; oj <= 1; ++oj)
#pragma unroll
            for (int oi = -1; oi <= 1; ++oi) {
              if (oj == 0 && oi < 0) continue;  // W: not stored
              const double w = 0.25 * pw(ki) * pw(kj) * pw(ki + li - 2 * oi) * pw(kj + lj - 2 * oj);
              if (w != 0.0) row[oi + 1][oj + 1] = fma((T)w, a, row[oi + 1][oj + 1]);
            }
        }
    }
  }
  diag[K] = row[1][1];
  dinv[K] = T(1) / row[1][1];
  cE[K] = row[2][1];
  cN[K] = row[1][2];
  cNE[K] = row[2][2];
  cNW[K] = row[0][2];
}

__global__ void k_op_to_f32(int nx, int nyr, int ps, int pd, const double* __restrict__ a0,
                            const double* __restrict__ a1, const double* __restrict__ a2,
                            const double* __restrict__ a3, const double* __restrict__ a4,
                            const double* __restrict__ a5, float* b0, float* b1, float* b2,
                            float* b3, float* b4, float* b5, int five, int dinv_f32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= nyr) return;
  const size_t s = (size_t)j * ps + i, d = (size_t)j * pd + i;
  b0[d] = (float)a0[s];
  b1[d] = (float)a1[s];
  b2[d] = five ? 0.0f : (float)a2[s];  // a 5-point operator's NE / NW are zero: not read
  b3[d] = five ? 0.0f : (float)a3[s];
  const float dg = (float)a4[s];
  b4[d] = dg;
  b5[d] = dinv_f32 ? 1.0f / dg : (float)a5[s];  // dinv_f32: reciprocal of the FP32 diagonal
}

// Dense matrix of the coarsest level's unknowns, inverted by Gauss-Jordan elimination
// (SPD: no pivoting) in one CTA.  The matrix lives in shared memory when it fits
// (m <= kCoarseSmemM), else in the output array.
__global__ void __launch_bounds__(kCoarseThreads) k_coarse_factor(Lvl<double> L, double* out,
                                                                        int* status) {
  extern __shared__ __align__(16) double smat[];
  __shared__ double rowk[kCoarseMax];
  const int ux = L.nx - 2;
  const int uy = L.periodic ? L.nyr : L.ny - 2;
  const int m = ux * uy;
  const int j0 = L.periodic ? 0 : 1;
  double* M = (m <= kCoarseSmemM) ? smat : out;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) M[e] = 0.0;
  __syncthreads();
  for (int p = threadIdx.x; p < m; p += blockDim.x) {
    const int i = 1 + p % ux, j = j0 + p / ux;
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        const int ni = i + di;
        int nj = j + dj;
        if (L.periodic) nj = (nj + L.nyr) % L.nyr;
        const bool unk = (ni >= 1 && ni <= L.nx - 2) &&
                         (L.periodic || (nj >= 1 && nj <= L.ny - 2));
        if (!unk) continue;
        const int q = (ni - 1) + ux * (nj - j0);
        M[(size_t)p * m + q] += fine_entry(L, i, j, di, dj);
      }
  }
  __syncthreads();
  // Gauss-Jordan: at step k every thread owns whole rows and updates them against the
  // scaled pivot row, which all threads read from shared memory.
  for (int k = 0; k < m; ++k) {
    const double piv = M[(size_t)k * m + k];
    if (!(piv > 0.0)) {
      if (threadIdx.x == 0) *status = 11;
      return;  // uniform: every thread read the same pivot
    }
    const double ip = 1.0 / piv;
    for (int jj = threadIdx.x; jj < m; jj += blockDim.x) rowk[jj] = (jj == k) ? ip : M[(size_t)k * m + jj] * ip;
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      double* Mi = M + (size_t)i * m;
      if (i == k) {
        for (int jj = 0; jj < m; ++jj) Mi[jj] = rowk[jj];
        continue;
      }
      const double f = Mi[k];
      for (int jj = 0; jj < m; ++jj) Mi[jj] = (jj == k) ? -f * ip : fma(-f, rowk[jj], Mi[jj]);
    }
    __syncthreads();
  }
  if (M != out)
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) out[e] = M[e];
  if (threadIdx.x == 0) *status = 0;
}

// ------------------------------------------------------------------ host launchers
static dim3 grid2(int nx, int ny, dim3 b) { return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y); }

cudaError_t launch_eps_analytic(int kind, const double* prm, int nx, int ny, int periodic,
                                double x0, double y0, double hx, double hy, const double* eps,
                                int pitch, double* D, double* exx, double* exy, double* eyy,
                                int* folded, cudaStream_t s) {
  const int nyr = rows_stored(ny, periodic);
  dim3 b(32, 8), g((nx + kEpsTile - 1) / kEpsTile, (nyr + kEpsTile - 1) / kEpsTile);
  k_eps_analytic<<<g, b, 0, s>>>(kind, prm[0], prm[1], prm[2], prm[3], nx, nyr, x0, y0, hx, hy, eps, pitch,
                                 D, exx, exy, eyy, folded, map_kind_five_point(kind, prm) ? 0 : 1);
  return cudaGetLastError();
}

cudaError_t launch_mirror_eps(int nx, int n, int ps, const double* D0, const double* exx0,
                              const double* exy0, const double* eyy0, int pd, double* D, double* exx,
                              double* exy, double* eyy, cudaStream_t s) {
  dim3 b(32, 8);
  k_mirror_eps<<<grid2(nx, 2 * n, b), b, 0, s>>>(nx, n, ps, D0, exx0, exy0, eyy0, pd, D, exx, exy, eyy);
  return cudaGetLastError();
}

cudaError_t launch_eps_grid(int nx, int ny, int periodic, double hx, double hy, const double* xp,
                            const double* yp, double jx, double jy, const double* eps, int pitch,
                            double* D, double* exx, double* exy, double* eyy, int* folded,
                            cudaStream_t s) {
  const int nyr = rows_stored(ny, periodic);
  dim3 b(32, 8);
  k_eps_grid<<<grid2(nx, nyr, b), b, 0, s>>>(nx, ny, nyr, periodic, 0.5 / hx, 0.5 / hy, xp, yp, jx, jy, eps,
                                             pitch, D, exx, exy, eyy, folded);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_assemble(const Op<T>& A, double hx, double hy, const T* exx, const T* exy, const T* eyy,
                            cudaStream_t s, bool dinv) {
  const int nyr = rows_stored(A.ny, A.periodic);
  dim3 b(32, 8);
  k_assemble_couplings<T><<<grid2(A.nx, nyr, b), b, 0, s>>>(
      A.nx, A.ny, nyr, A.periodic, A.pitch, T(1.0 / (hx * hx)), T(1.0 / (hy * hy)), T(1.0 / (4.0 * hx * hy)),
      exx, exy, eyy, A.cE, A.cN, A.cNE, A.cNW, A.five_point);
  k_assemble_diag<T><<<grid2(A.nx, nyr, b), b, 0, s>>>(A.nx, A.ny, nyr, A.periodic, A.pitch, A.cE,
                                                       A.cN, A.cNE, A.cNW, A.diag, dinv ? A.dinv : nullptr,
                                                       A.five_point);
  return cudaGetLastError();
}
template cudaError_t launch_assemble<double>(const OpF64&, double, double, const double*, const double*,
                                             const double*, cudaStream_t, bool);
template cudaError_t launch_assemble<float>(const OpF32&, double, double, const float*, const float*,
                                            const float*, cudaStream_t, bool);

cudaError_t launch_assemble_five(const OpF64& A, const OpF32* B, double hx, double hy, const double* exx,
                                 const double* eyy, cudaStream_t s, bool dinv) {
  const int nyr = rows_stored(A.ny, A.periodic);
  dim3 b(32, 8), g((A.nx + 31) / 32, (nyr + 8 * kAsmRows - 1) / (8 * kAsmRows));
  // -(1/2) / h^2 exactly (halving is exact), as k_assemble_couplings rounds its couplings
  k_assemble_five<<<g, b, 0, s>>>(
      A.nx, A.ny, nyr, A.periodic, A.pitch, -0.5 * (1.0 / (hx * hx)), -0.5 * (1.0 / (hy * hy)), exx, eyy, A.cE, A.cN, A.cNE,
      A.cNW, A.diag, dinv ? A.dinv : nullptr, B ? B->pitch : 0, B ? B->cE : nullptr, B ? B->cN : nullptr,
      B ? B->cNE : nullptr, B ? B->cNW : nullptr, B ? B->diag : nullptr, B ? B->dinv : nullptr);
  return cudaGetLastError();
}

cudaError_t launch_rhs(const OpF64& A, const double* rho, int rho_pitch, const double* D, double* b,
                       cudaStream_t s) {
  const int nyr = rows_stored(A.ny, A.periodic);
  dim3 bl(32, 8);
  k_rhs<<<grid2(A.nx, nyr, bl), bl, 0, s>>>(A.nx, A.ny, nyr, A.periodic, A.pitch, rho, rho_pitch, D,
                                            b);
  return cudaGetLastError();
}

template <typename TS, typename TD>
cudaError_t launch_coarsen_eps(const Op<TS>& F, const Op<TD>& C, const TS* const* e, TD* const* c,
                               cudaStream_t s) {
  const int nyrc = rows_stored(C.ny, C.periodic);
  dim3 b(32, 8);
  k_coarsen_eps<TS, TD><<<grid2(C.nx, nyrc, b), b, 0, s>>>(F.nx, rows_stored(F.ny, F.periodic), F.pitch, C.nx,
                                                            C.ny, nyrc, C.pitch, C.periodic, e[0], e[1], e[2],
                                                            c[0], c[1], c[2], C.five_point);
  return cudaGetLastError();
}
template cudaError_t launch_coarsen_eps<double, double>(const OpF64&, const OpF64&, const double* const*,
                                                        double* const*, cudaStream_t);
template cudaError_t launch_coarsen_eps<double, float>(const OpF64&, const OpF32&, const double* const*,
                                                       float* const*, cudaStream_t);
template cudaError_t launch_coarsen_eps<float, float>(const OpF32&, const OpF32&, const float* const*,
                                                      float* const*, cudaStream_t);

template <typename T>
cudaError_t launch_galerkin(const Op<T>& F, const Op<T>& C, cudaStream_t s) {
  const int nyrc = rows_stored(C.ny, C.periodic);
  dim3 b(32, 4);
  if (F.five_point)
    k_galerkin<T, true><<<grid2(C.nx, nyrc, b), b, 0, s>>>(lvl_of(F), C.nx, C.ny, nyrc, C.pitch, C.cE,
                                                           C.cN, C.cNE, C.cNW, C.diag, C.dinv);
  else
    k_galerkin<T, false><<<grid2(C.nx, nyrc, b), b, 0, s>>>(lvl_of(F), C.nx, C.ny, nyrc, C.pitch, C.cE,
                                                            C.cN, C.cNE, C.cNW, C.diag, C.dinv);
  return cudaGetLastError();
}
template cudaError_t launch_galerkin<double>(const OpF64&, const OpF64&, cudaStream_t);
template cudaError_t launch_galerkin<float>(const OpF32&, const OpF32&, cudaStream_t);

// Coarsest operator in FP64 from an FP32 level (mixed path: its hierarchy is FP32).
__global__ void k_op_to_f64(int nx, int nyr, int ps, int pd, const float* __restrict__ a0,
                            const float* __restrict__ a1, const float* __restrict__ a2,
                            const float* __restrict__ a3, const float* __restrict__ a4, double* b0,
                            double* b1, double* b2, double* b3, double* b4, double* b5) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= nyr) return;
  const size_t s = (size_t)j * ps + i, d = (size_t)j * pd + i;
  b0[d] = a0[s];
  b1[d] = a1[s];
  b2[d] = a2[s];
  b3[d] = a3[s];
  b4[d] = a4[s];
  b5[d] = 1.0 / (double)a4[s];
}

cudaError_t launch_op_to_f64(const OpF32& A, const OpF64& B, cudaStream_t s) {
  const int nyr = rows_stored(A.ny, A.periodic);
  dim3 b(32, 8);
  k_op_to_f64<<<grid2(A.nx, nyr, b), b, 0, s>>>(A.nx, nyr, A.pitch, B.pitch, A.cE, A.cN, A.cNE, A.cNW,
                                                A.diag, B.cE, B.cN, B.cNE, B.cNW, B.diag, B.dinv);
  return cudaGetLastError();
}

cudaError_t launch_op_to_f32(const OpF64& A, const OpF32& B, cudaStream_t s, bool dinv_f32) {
  const int nyr = rows_stored(A.ny, A.periodic);
  dim3 b(32, 8);
  k_op_to_f32<<<grid2(A.nx, nyr, b), b, 0, s>>>(A.nx, nyr, A.pitch, B.pitch, A.cE, A.cN, A.cNE,
                                                A.cNW, A.diag, A.dinv, B.cE, B.cN, B.cNE, B.cNW,
                                                B.diag, B.dinv, A.five_point, dinv_f32 ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_coarse_factor(const OpF64& A, double* inv, int* status, cudaStream_t s) {
  const int m = coarse_unknowns(A.nx, A.ny, A.periodic);
  const size_t sm = (m <= kCoarseSmemM) ? (size_t)m * m * sizeof(double) : 0;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_coarse_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kCoarseSmemM * kCoarseSmemM * sizeof(double)));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_coarse_factor<<<1, kCoarseThreads, sm, s>>>(lvl_of(A), inv, status);
  return cudaGetLastError();
}

}  // namespace mg

// ------------------------------------------------------------------ C ABI (mg_kernels.h)
using namespace mg;

static bool op_ok(const mgk_op_f64* A) {
  return A && A->nx >= 3 && A->ny >= 3 && A->pitch >= A->nx && A->cE && A->cN && A->cNE && A->cNW &&
         A->diag && A->dinv && (!A->periodic || A->ny >= 3);
}

extern "C" int mgk_eps_analytic(int kind, const double* params4, int nx, int ny, int periodic,
                                double x0, double y0, double hx, double hy, const double* eps_phys,
                                int pitch, double* D, double* exx, double* exy, double* eyy,
                                int* folded, void* stream) {
  if (kind < 0 || kind > 4 || !params4 || nx < 3 || ny < 3 || pitch < nx || !D || !exx || !exy ||
      !eyy || !folded)
    return 1;
  return launch_eps_analytic(kind, params4, nx, ny, periodic, x0, y0, hx, hy, eps_phys, pitch, D,
                             exx, exy, eyy, folded, (cudaStream_t)stream) == cudaSuccess ? 0 : 4;
}

extern "C" int mgk_eps_grid(int nx, int ny, int periodic, double hx, double hy, const double* xp,
                            const double* yp, double jump_x, double jump_y, const double* eps_phys,
                            int pitch, double* D, double* exx, double* exy, double* eyy,
                            int* folded, void* stream) {
  if (nx < 3 || ny < 3 || (periodic ? ny - 1 : ny) < 3 || pitch < nx || !xp || !yp || !D || !exx ||
      !exy || !eyy || !folded)
    return 1;
  return launch_eps_grid(nx, ny, periodic, hx, hy, xp, yp, jump_x, jump_y, eps_phys, pitch, D, exx,
                         exy, eyy, folded, (cudaStream_t)stream) == cudaSuccess ? 0 : 4;
}

extern "C" int mgk_assemble(const mgk_op_f64* A, double hx, double hy, const double* exx,
                            const double* exy, const double* eyy, void* stream) {
  if (!op_ok(A) || !exx || !exy || !eyy || !(hx > 0) || !(hy > 0)) return 1;
  return launch_assemble(op_from(*A), hx, hy, exx, exy, eyy, (cudaStream_t)stream) == cudaSuccess
             ? 0 : 4;
}

extern "C" int mgk_assemble_five(const mgk_op_f64* A, const mgk_op_f32* B, double hx, double hy,
                                 const double* exx, const double* eyy, void* stream) {
  if (!op_ok(A) || !A->five_point || !exx || !eyy || !(hx > 0) || !(hy > 0)) return 1;
  if (B && (B->nx != A->nx || B->ny != A->ny || B->periodic != A->periodic || B->pitch < B->nx || !B->cE ||
            !B->cN || !B->cNE || !B->cNW || !B->diag || !B->dinv))
    return 1;
  const OpF32 b = B ? op_from(*B) : OpF32();
  return launch_assemble_five(op_from(*A), B ? &b : nullptr, hx, hy, exx, eyy, (cudaStream_t)stream, true) ==
                 cudaSuccess
             ? 0 : 4;
}

extern "C" int mgk_rhs(const mgk_op_f64* A, const double* rho_phys, const double* D, double* b,
                       void* stream) {
  if (!A || A->nx < 3 || A->ny < 3 || A->pitch < A->nx || !rho_phys || !D || !b) return 1;
  return launch_rhs(op_from(*A), rho_phys, A->pitch, D, b, (cudaStream_t)stream) == cudaSuccess
             ? 0 : 4;
}

extern "C" int mgk_coarsen_eps(const mgk_op_f64* fine, const mgk_op_f64* coarse, const double* e0,
                               const double* e1, const double* e2, double* c0, double* c1, double* c2,
                               void* stream) {
  if (!fine || !coarse || !e0 || !e1 || !e2 || !c0 || !c1 || !c2 || fine->nx < 3 || fine->ny < 3 ||
      fine->pitch < fine->nx || coarse->pitch < coarse->nx || (fine->nx - 1) % 2 || (fine->ny - 1) % 2 ||
      coarse->nx != (fine->nx - 1) / 2 + 1 || coarse->ny != (fine->ny - 1) / 2 + 1 ||
      coarse->periodic != fine->periodic)
    return 1;
  const double* e[3] = {e0, e1, e2};
  double* c[3] = {c0, c1, c2};
  return launch_coarsen_eps(op_from(*fine), op_from(*coarse), e, c, (cudaStream_t)stream) == cudaSuccess ? 0
                                                                                                        : 4;
}

extern "C" int mgk_galerkin(const mgk_op_f64* fine, const mgk_op_f64* coarse, void* stream) {
  if (!op_ok(fine) || !op_ok(coarse) || (fine->nx - 1) % 2 || (fine->ny - 1) % 2 ||
      coarse->nx != (fine->nx - 1) / 2 + 1 || coarse->ny != (fine->ny - 1) / 2 + 1 ||
      coarse->periodic != fine->periodic)
    return 1;
  return launch_galerkin<double>(op_from(*fine), op_from(*coarse), (cudaStream_t)stream) ==
                 cudaSuccess ? 0 : 4;
}

extern "C" int mgk_op_to_f32(const mgk_op_f64* src, const mgk_op_f32* dst, void* stream) {
  if (!op_ok(src) || !dst || dst->nx != src->nx || dst->ny != src->ny || dst->pitch < dst->nx ||
      !dst->cE || !dst->cN || !dst->cNE || !dst->cNW || !dst->diag || !dst->dinv)
    return 1;
  return launch_op_to_f32(op_from(*src), op_from(*dst), (cudaStream_t)stream) == cudaSuccess ? 0
                                                                                                : 4;
}

extern "C" int mgk_coarse_factor(const mgk_op_f64* A, double* inv, int* status, void* stream) {
  if (!op_ok(A) || !inv || !status) return 1;
  const int uy = A->periodic ? A->ny - 1 : A->ny - 2;
  if ((A->nx - 2) * uy > kCoarseMax || uy < 1) return 1;
  return launch_coarse_factor(op_from(*A), inv, status, (cudaStream_t)stream) == cudaSuccess ? 0
                                                                                               : 4;
}
