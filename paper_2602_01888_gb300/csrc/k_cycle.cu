// Multigrid cycle kernels (Sec. 3, Eqs. 19-24) for FP64 and FP32 levels:
// four-colour Gauss-Seidel smoothing (Sec. 2.1 with omega = 1), weighted Jacobi,
// residual (Eq. 20) fused with full-weighting restriction, bilinear prolongation with
// correction (Eq. 24) and the single-CTA coarsest solve.
#include "mg_common.cuh"
#include "mg_kernels.h"
#include "mg_launch.h"

namespace mg {

// One colour phase: x = (b - offdiag x) / diag at the unknowns of colour (ci, cj).
// Unknowns of one colour are not coupled by the 9-point stencil, so they update in
// parallel exactly as in a sequential sweep.
template <typename T>
__global__ void __launch_bounds__(256) k_gs_colour(Lvl<T> L, T* __restrict__ x,
                                                   const T* __restrict__ b, int ci, int cj,
                                                   const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int i = ci + 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int j = cj + 2 * (blockIdx.y * blockDim.y + threadIdx.y);
  if (!is_unknown(L, i, j)) return;
  const size_t k = (size_t)j * L.pitch + i;
  x[k] = (b[k] - offdiag(L, x, i, j)) * L.dinv[k];
}

// One colour phase of successive over-relaxation: x += omega (gs - x) at the unknowns of
// the colour, gs the Gauss-Seidel value (the comparison iteration of Sec. 4).
template <typename T>
__global__ void __launch_bounds__(256) k_sor_colour(Lvl<T> L, T* __restrict__ x, const T* __restrict__ b,
                                                    int ci, int cj, T omega, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int i = ci + 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int j = cj + 2 * (blockIdx.y * blockDim.y + threadIdx.y);
  if (!is_unknown(L, i, j)) return;
  const size_t k = (size_t)j * L.pitch + i;
  const T gs = (b[k] - offdiag(L, x, i, j)) * L.dinv[k];
  x[k] = fma(omega, gs - x[k], x[k]);
}

template <typename T>
__global__ void __launch_bounds__(256) k_residual(Lvl<T> L, const T* __restrict__ x,
                                                  const T* __restrict__ b, T* __restrict__ r,
                                                  const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= L.nx || j >= L.nyr) return;
  const size_t k = (size_t)j * L.pitch + i;
  r[k] = is_unknown(L, i, j) ? b[k] - fma(L.diag[k], x[k], offdiag(L, x, i, j)) : T(0);
}

template <typename T>
__global__ void __launch_bounds__(256) k_jacobi_update(Lvl<T> L, T* __restrict__ x,
                                                       const T* __restrict__ r, T omega,
                                                       const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (!is_unknown(L, i, j)) return;
  const size_t k = (size_t)j * L.pitch + i;
  x[k] = fma(omega * r[k], L.dinv[k], x[k]);
}

// r = b - A x on a (2 kRRX + 1) x (2 kRRY + 1) fine window staged in shared memory,
// then bH = full weighting of r at the kRRX x kRRY coarse nodes of the block; the
// coarse solution array is zeroed alongside (zero initial guess of the correction).
template <typename T>
__global__ void __launch_bounds__(kRRX* kRRY)
    k_resid_restrict(Lvl<T> L, const T* __restrict__ x, const T* __restrict__ b,
                     T* __restrict__ bH, T* __restrict__ xH, int nxc, int nyc, int nyrc,
                     int pitchc, const int* __restrict__ skip) {
  if (skip && *skip) return;
  constexpr int WX = 2 * kRRX + 1, WY = 2 * kRRY + 1;
  __shared__ T rs[WY][WX + 1];
  const int I0 = blockIdx.x * kRRX, J0 = blockIdx.y * kRRY;
  const int fi0 = 2 * I0 - 1, fj0 = 2 * J0 - 1;
  for (int t = threadIdx.x; t < WX * WY; t += blockDim.x) {
    const int li = t % WX, lj = t / WX;
    const int i = fi0 + li;
    int j = fj0 + lj;
    if (L.periodic) j = (j < 0) ? j + L.nyr : (j >= L.nyr ? j - L.nyr : j);
    T r = T(0);
    if (is_unknown(L, i, j)) {
      const size_t k = (size_t)j * L.pitch + i;
      r = b[k] - fma(L.diag[k], x[k], offdiag(L, x, i, j));
    }
    rs[lj][li] = r;
  }
  __syncthreads();
  const int I = I0 + threadIdx.x % kRRX, J = J0 + threadIdx.x / kRRX;
  if (I < nxc && J < nyrc) {
    const bool unk = (I >= 1 && I <= nxc - 2) && (L.periodic || (J >= 1 && J <= nyc - 2));
    T v = T(0);
    if (unk) {
      const int ci = 2 * (I - I0) + 1, cj = 2 * (J - J0) + 1;
      const T edge = rs[cj][ci - 1] + rs[cj][ci + 1] + rs[cj - 1][ci] + rs[cj + 1][ci];
      const T corner = rs[cj - 1][ci - 1] + rs[cj - 1][ci + 1] + rs[cj + 1][ci - 1] + rs[cj + 1][ci + 1];
      v = (T(4) * rs[cj][ci] + T(2) * edge + corner) * T(0.0625);
    }
    const size_t K = (size_t)J * pitchc + I;
    bH[K] = v;
    if (xH) xH[K] = T(0);
  }
}

// Residual and full weighting after zebra x-line pre-smoothing, whose last half-sweep solved
// every odd row exactly from its even neighbours: b - A x is then zero on the odd rows up to
// the rounding of the row solves, and full weighting at coarse node (I, J) keeps only the
// fine row 2J, bH = (4 r(2I) + 2 (r(2I-1) + r(2I+1))) / 16 (the stencil's odd-row and corner
// terms vanish).  Half of the fine residuals are computed, from even rows of b, diag and the
// couplings and from all rows of x.  One thread per coarse node computes r(2I) and r(2I+1)
// of row 2J; r(2I-1) is its left neighbour's r(2I+1), handed over in shared memory (the
// block's first thread computes the one left of the block).  Summation order as in
// k_resid_restrict with the odd-row terms zero.
template <typename T>
__global__ void __launch_bounds__(kREven) k_resid_restrict_even(Lvl<T> L, const T* __restrict__ x,
                                                                const T* __restrict__ b, T* __restrict__ bH,
                                                                T* __restrict__ xH, int nxc, int nyc,
                                                                int pitchc, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ T rodd[kREven + 1];
  const int J = blockIdx.y, j = 2 * J;
  const int I = blockIdx.x * kREven + threadIdx.x;
  const auto res = [&](int i) -> T {
    if (!is_unknown(L, i, j)) return T(0);
    const size_t k = (size_t)j * L.pitch + i;
    return b[k] - fma(L.diag[k], x[k], offdiag(L, x, i, j));
  };
  T r0 = T(0), r1 = T(0);
  if (I < nxc) {
    r0 = res(2 * I);
    r1 = res(2 * I + 1);
  }
  if (threadIdx.x == 0) rodd[0] = res(2 * I - 1);
  rodd[threadIdx.x + 1] = r1;
  __syncthreads();
  if (I >= nxc) return;
  const bool unk = (I >= 1 && I <= nxc - 2) && (L.periodic || (J >= 1 && J <= nyc - 2));
  const size_t K = (size_t)J * pitchc + I;
  bH[K] = unk ? (T(4) * r0 + T(2) * (rodd[threadIdx.x] + r1)) * T(0.0625) : T(0);
  if (xH) xH[K] = T(0);
}

// x += P eH (bilinear: injection at coincident nodes, 1/2 on edges, 1/4 at centres).
template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add(Lvl<T> L, T* __restrict__ x,
                                                     const T* __restrict__ eH, int nyrc,
                                                     int pitchc, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (!is_unknown(L, i, j)) return;
  const int I = i >> 1, J = j >> 1;
  const int Jp = (J + 1 == nyrc) ? 0 : J + 1;
  const size_t a = (size_t)J * pitchc + I, c = (size_t)Jp * pitchc + I;
  T v;
  if (!(i & 1) && !(j & 1)) v = eH[a];
  else if ((i & 1) && !(j & 1)) v = T(0.5) * (eH[a] + eH[a + 1]);
  else if (!(i & 1)) v = T(0.5) * (eH[a] + eH[c]);
  else v = T(0.25) * ((eH[a] + eH[a + 1]) + (eH[c] + eH[c + 1]));
  x[(size_t)j * L.pitch + i] += v;
}

// x = inv * b at the coarsest unknowns (lexicographic, i fastest), one CTA.
template <typename T>
__global__ void __launch_bounds__(kCoarseThreads) k_coarse_solve(Lvl<T> L,
                                                                 const double* __restrict__ inv,
                                                                 const T* __restrict__ b,
                                                                 T* __restrict__ x,
                                                                 const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double bs[kCoarseMax];
  const int ux = L.nx - 2;
  const int uy = L.periodic ? L.nyr : L.ny - 2;
  const int m = ux * uy, j0 = L.periodic ? 0 : 1;
  for (int p = threadIdx.x; p < m; p += blockDim.x) {
    const int i = 1 + p % ux, j = j0 + p / ux;
    bs[p] = (double)b[(size_t)j * L.pitch + i];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < m; t += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < m; ++k) s = fma(inv[(size_t)k * m + t], bs[k], s);
    const int i = 1 + t % ux, j = j0 + t / ux;
    x[(size_t)j * L.pitch + i] = (T)s;
  }
}

// ------------------------------------------------------------------ launchers
static inline dim3 g2(int nx, int ny, dim3 b) { return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y); }

template <typename T>
cudaError_t launch_gs_colour(const Op<T>& A, T* phi, const T* b, int colour, const int* skip,
                             cudaStream_t s) {
  const Lvl<T> L = lvl_of(A);
  const int ci = colour_ci(colour), cj = colour_cj(colour);
  const int ncx = (L.nx - ci + 1) / 2, ncy = (L.nyr - cj + 1) / 2;
  dim3 bl(32, 8);
  k_gs_colour<T><<<g2(ncx, ncy, bl), bl, 0, s>>>(L, phi, b, ci, cj, skip);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_smooth(const Op<T>& A, T* phi, const T* b, int sweeps, int reverse,
                          const int* skip, cudaStream_t s) {
  for (int sw = 0; sw < sweeps; ++sw)
    for (int c = 0; c < 4; ++c) {
      cudaError_t e = launch_gs_colour(A, phi, b, reverse ? 3 - c : c, skip, s);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_sor(const Op<T>& A, T* phi, const T* b, int sweeps, double omega, const int* skip,
                       cudaStream_t s) {
  const Lvl<T> L = lvl_of(A);
  dim3 bl(32, 8);
  for (int sw = 0; sw < sweeps; ++sw)
    for (int c = 0; c < 4; ++c) {
      const int ci = colour_ci(c), cj = colour_cj(c);
      const int ncx = (L.nx - ci + 1) / 2, ncy = (L.nyr - cj + 1) / 2;
      k_sor_colour<T><<<g2(ncx, ncy, bl), bl, 0, s>>>(L, phi, b, ci, cj, (T)omega, skip);
    }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual(const Op<T>& A, const T* phi, const T* b, T* r, const int* skip,
                            cudaStream_t s) {
  const Lvl<T> L = lvl_of(A);
  dim3 bl(32, 8);
  k_residual<T><<<g2(L.nx, L.nyr, bl), bl, 0, s>>>(L, phi, b, r, skip);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_jacobi(const Op<T>& A, T* phi, const T* b, T* tmp, int sweeps, double omega,
                          const int* skip, cudaStream_t s) {
  const Lvl<T> L = lvl_of(A);
  dim3 bl(32, 8);
  for (int sw = 0; sw < sweeps; ++sw) {
    k_residual<T><<<g2(L.nx, L.nyr, bl), bl, 0, s>>>(L, phi, b, tmp, skip);
    k_jacobi_update<T><<<g2(L.nx, L.nyr, bl), bl, 0, s>>>(L, phi, tmp, (T)omega, skip);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_resid_restrict(const Op<T>& A, const T* phi, const T* b, T* bH, T* phiH,
                                  int pitch_c, const int* skip, cudaStream_t s) {
  const Lvl<T> L = lvl_of(A);
  const int nxc = (A.nx - 1) / 2 + 1, nyc = (A.ny - 1) / 2 + 1;
  const int nyrc = rows_stored(nyc, A.periodic);
  dim3 grid((nxc + kRRX - 1) / kRRX, (nyrc + kRRY - 1) / kRRY);
  k_resid_restrict<T><<<grid, kRRX * kRRY, 0, s>>>(L, phi, b, bH, phiH, nxc, nyc, nyrc, pitch_c,
                                                   skip);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_resid_restrict_even(const Op<T>& A, const T* phi, const T* b, T* bH, T* phiH,
                                       int pitch_c, const int* skip, cudaStream_t s) {
  const Lvl<T> L = lvl_of(A);
  const int nxc = (A.nx - 1) / 2 + 1, nyc = (A.ny - 1) / 2 + 1;
  const int nyrc = rows_stored(nyc, A.periodic);
  dim3 grid((nxc + kREven - 1) / kREven, nyrc);
  k_resid_restrict_even<T><<<grid, kREven, 0, s>>>(L, phi, b, bH, phiH, nxc, nyc, pitch_c, skip);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_add(const Op<T>& A, T* phi, const T* eH, int pitch_c, const int* skip,
                               cudaStream_t s) {
  const Lvl<T> L = lvl_of(A);
  const int nyc = (A.ny - 1) / 2 + 1;
  dim3 bl(32, 8);
  k_prolong_add<T><<<g2(L.nx, L.nyr, bl), bl, 0, s>>>(L, phi, eH, rows_stored(nyc, A.periodic),
                                                      pitch_c, skip);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_solve(const Op<T>& A, const double* inv, const T* b, T* x,
                                const int* skip, cudaStream_t s) {
  k_coarse_solve<T><<<1, kCoarseThreads, 0, s>>>(lvl_of(A), inv, b, x, skip);
  return cudaGetLastError();
}

#define MG_INST(T)                                                                               \
  template cudaError_t launch_gs_colour<T>(const Op<T>&, T*, const T*, int, const int*,        \
                                           cudaStream_t);                                        \
  template cudaError_t launch_smooth<T>(const Op<T>&, T*, const T*, int, int, const int*,      \
                                        cudaStream_t);                                           \
  template cudaError_t launch_sor<T>(const Op<T>&, T*, const T*, int, double, const int*,       \
                                     cudaStream_t);                                              \
  template cudaError_t launch_residual<T>(const Op<T>&, const T*, const T*, T*, const int*,    \
                                          cudaStream_t);                                         \
  template cudaError_t launch_jacobi<T>(const Op<T>&, T*, const T*, T*, int, double,           \
                                        const int*, cudaStream_t);                               \
  template cudaError_t launch_resid_restrict<T>(const Op<T>&, const T*, const T*, T*, T*, int, \
                                                const int*, cudaStream_t);                       \
  template cudaError_t launch_resid_restrict_even<T>(const Op<T>&, const T*, const T*, T*, T*,  \
                                                     int, const int*, cudaStream_t);             \
  template cudaError_t launch_prolong_add<T>(const Op<T>&, T*, const T*, int, const int*,      \
                                             cudaStream_t);                                      \
  template cudaError_t launch_coarse_solve<T>(const Op<T>&, const double*, const T*, T*,       \
                                              const int*, cudaStream_t);
MG_INST(double)
MG_INST(float)
#undef MG_INST

}  // namespace mg

// ------------------------------------------------------------------ C ABI (mg_kernels.h)
using namespace mg;

template <typename OP>
static bool opk(const OP* A) {
  return A && A->nx >= 3 && A->ny >= 3 && A->pitch >= A->nx && A->cE && A->cN && A->cNE &&
         A->cNW && A->diag && A->dinv && (A->periodic ? A->ny - 1 : A->ny) >= 2;
}

static int rc(cudaError_t e) { return e == cudaSuccess ? 0 : 4; }

extern "C" int mgk_smooth_f64(const mgk_op_f64* A, double* phi, const double* b, int sweeps,
                              int reverse, void* stream) {
  if (!opk(A) || !phi || !b || sweeps < 0) return 1;
  return rc(launch_smooth(op_from(*A), phi, b, sweeps, reverse, nullptr, (cudaStream_t)stream));
}
extern "C" int mgk_smooth_f32(const mgk_op_f32* A, float* phi, const float* b, int sweeps,
                              int reverse, void* stream) {
  if (!opk(A) || !phi || !b || sweeps < 0) return 1;
  return rc(launch_smooth(op_from(*A), phi, b, sweeps, reverse, nullptr, (cudaStream_t)stream));
}
extern "C" int mgk_sor_f64(const mgk_op_f64* A, double* phi, const double* b, int sweeps, double omega,
                           void* stream) {
  if (!opk(A) || !phi || !b || sweeps < 0 || !(omega > 0.0 && omega < 2.0)) return 1;
  return rc(launch_sor(op_from(*A), phi, b, sweeps, omega, nullptr, (cudaStream_t)stream));
}
extern "C" int mgk_sor_f32(const mgk_op_f32* A, float* phi, const float* b, int sweeps, double omega,
                           void* stream) {
  if (!opk(A) || !phi || !b || sweeps < 0 || !(omega > 0.0 && omega < 2.0)) return 1;
  return rc(launch_sor(op_from(*A), phi, b, sweeps, omega, nullptr, (cudaStream_t)stream));
}
extern "C" int mgk_jacobi_f64(const mgk_op_f64* A, double* phi, const double* b, double* tmp,
                              int sweeps, double omega, void* stream) {
  if (!opk(A) || !phi || !b || !tmp || sweeps < 0) return 1;
  return rc(launch_jacobi(op_from(*A), phi, b, tmp, sweeps, omega, nullptr, (cudaStream_t)stream));
}
extern "C" int mgk_residual_f64(const mgk_op_f64* A, const double* phi, const double* b,
                                double* r, void* stream) {
  if (!opk(A) || !phi || !b || !r) return 1;
  return rc(launch_residual(op_from(*A), phi, b, r, nullptr, (cudaStream_t)stream));
}
extern "C" int mgk_resid_restrict_f64(const mgk_op_f64* A, const double* phi, const double* b,
                                      double* bH, int pitch_c, void* stream) {
  if (!opk(A) || !phi || !b || !bH || (A->nx - 1) % 2 || (A->ny - 1) % 2 ||
      pitch_c < (A->nx - 1) / 2 + 1)
    return 1;
  return rc(launch_resid_restrict(op_from(*A), phi, b, bH, (double*)nullptr, pitch_c, nullptr,
                                  (cudaStream_t)stream));
}
extern "C" int mgk_resid_restrict_f32(const mgk_op_f32* A, const float* phi, const float* b,
                                      float* bH, int pitch_c, void* stream) {
  if (!opk(A) || !phi || !b || !bH || (A->nx - 1) % 2 || (A->ny - 1) % 2 ||
      pitch_c < (A->nx - 1) / 2 + 1)
    return 1;
  return rc(launch_resid_restrict(op_from(*A), phi, b, bH, (float*)nullptr, pitch_c, nullptr,
                                  (cudaStream_t)stream));
}
extern "C" int mgk_resid_restrict_even_f64(const mgk_op_f64* A, const double* phi, const double* b,
                                           double* bH, int pitch_c, void* stream) {
  if (!opk(A) || !phi || !b || !bH || (A->nx - 1) % 2 || (A->ny - 1) % 2 ||
      pitch_c < (A->nx - 1) / 2 + 1)
    return 1;
  return rc(launch_resid_restrict_even(op_from(*A), phi, b, bH, (double*)nullptr, pitch_c, nullptr,
                                       (cudaStream_t)stream));
}
extern "C" int mgk_resid_restrict_even_f32(const mgk_op_f32* A, const float* phi, const float* b,
                                           float* bH, int pitch_c, void* stream) {
  if (!opk(A) || !phi || !b || !bH || (A->nx - 1) % 2 || (A->ny - 1) % 2 ||
      pitch_c < (A->nx - 1) / 2 + 1)
    return 1;
  return rc(launch_resid_restrict_even(op_from(*A), phi, b, bH, (float*)nullptr, pitch_c, nullptr,
                                       (cudaStream_t)stream));
}
extern "C" int mgk_prolong_add_f64(const mgk_op_f64* A, double* phi, const double* eH,
                                   int pitch_c, void* stream) {
  if (!A || A->nx < 3 || A->ny < 3 || A->pitch < A->nx || !phi || !eH || (A->nx - 1) % 2 ||
      (A->ny - 1) % 2 || pitch_c < (A->nx - 1) / 2 + 1)
    return 1;
  return rc(launch_prolong_add(op_from(*A), phi, eH, pitch_c, nullptr, (cudaStream_t)stream));
}
extern "C" int mgk_prolong_add_f32(const mgk_op_f32* A, float* phi, const float* eH, int pitch_c,
                                   void* stream) {
  if (!A || A->nx < 3 || A->ny < 3 || A->pitch < A->nx || !phi || !eH || (A->nx - 1) % 2 ||
      (A->ny - 1) % 2 || pitch_c < (A->nx - 1) / 2 + 1)
    return 1;
  return rc(launch_prolong_add(op_from(*A), phi, eH, pitch_c, nullptr, (cudaStream_t)stream));
}
extern "C" int mgk_coarse_solve_f64(const mgk_op_f64* A, const double* inv, const double* b,
                                    double* x, void* stream) {
  if (!opk(A) || !inv || !b || !x ||
      coarse_unknowns(A->nx, A->ny, A->periodic) > kCoarseMax)
    return 1;
  return rc(launch_coarse_solve(op_from(*A), inv, b, x, nullptr, (cudaStream_t)stream));
}
extern "C" int mgk_coarse_solve_f32(const mgk_op_f32* A, const double* inv, const float* b,
                                    float* x, void* stream) {
  if (!opk(A) || !inv || !b || !x ||
      coarse_unknowns(A->nx, A->ny, A->periodic) > kCoarseMax)
    return 1;
  return rc(launch_coarse_solve(op_from(*A), inv, b, x, nullptr, (cudaStream_t)stream));
}
