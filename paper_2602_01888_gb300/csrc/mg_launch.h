// Host-side views and kernel launchers shared by the translation units of libmg.
#pragma once
#include <cuda_runtime.h>

#include "mg_common.cuh"
#include "mg_kernels.h"

namespace mg {

constexpr int kCoarseMax = 256;      // unknowns of the coarsest level (dense inverse)
constexpr int kCoarseThreads = 256;  // threads of the single-CTA coarsest solve
constexpr int kCoarseFactorThreads = 1024;
constexpr int kCoarseSmemM = 128;    // coarsest inverses up to this order are formed in shared memory
constexpr int kRRX = 16, kRRY = 16;  // coarse tile of the residual + restriction kernel
constexpr int kREven = 128;          // coarse nodes (threads) per block of the even-row form

template <typename T>
struct Op {
  int nx, ny, periodic, pitch;
  T *cE, *cN, *cNE, *cNW, *diag, *dinv;
  int five_point = 0;  // cNE, cNW are zero everywhere and are not read (see Lvl)
};
using OpF64 = Op<double>;
using OpF32 = Op<float>;

template <typename T>
inline Lvl<T> lvl_of(const Op<T>& A) {
  Lvl<T> L;
  L.nx = A.nx;
  L.ny = A.ny;
  L.nyr = rows_stored(A.ny, A.periodic);
  L.periodic = A.periodic;
  L.pitch = A.pitch;
  L.cE = A.cE;
  L.cN = A.cN;
  L.cNE = A.cNE;
  L.cNW = A.cNW;
  L.diag = A.diag;
  L.dinv = A.dinv;
  L.five_point = A.five_point;
  return L;
}

inline OpF64 op_from(const mgk_op_f64& a) {
  return OpF64{a.nx, a.ny, a.periodic, a.pitch, a.cE, a.cN, a.cNE, a.cNW, a.diag, a.dinv,
               a.five_point ? 1 : 0};
}
inline OpF32 op_from(const mgk_op_f32& a) {
  return OpF32{a.nx, a.ny, a.periodic, a.pitch, a.cE, a.cN, a.cNE, a.cNW, a.diag, a.dinv,
               a.five_point ? 1 : 0};
}

// Whether an analytic map (kind and params as MG_MAP_* of mg.h: 0 identity, 1 sine warp,
// 2 polar, 3 sinh, 4 affine) has no cross term: J^T J is diagonal, so Eq. 13 vanishes
// identically and the finest operator is a 5-point stencil.  Identity, polar (Eq. 29) and
// sinh stretching (Eq. 52) always; an affine map when its shear terms are zero.
inline int map_kind_five_point(int kind, const double* prm) {
  if (kind == 0 || kind == 2 || kind == 3) return 1;
  if (kind == 4) return prm[1] == 0.0 && prm[2] == 0.0;
  return 0;
}

inline int coarse_unknowns(int nx, int ny, int periodic) {
  return (nx - 2) * (periodic ? ny - 1 : ny - 2);
}

// ---- setup (k_setup.cu)
cudaError_t launch_eps_analytic(int kind, const double* prm, int nx, int ny, int periodic,
                                double x0, double y0, double hx, double hy, const double* eps,
                                int pitch, double* D, double* exx, double* exy, double* eyy,
                                int* folded, cudaStream_t s);
cudaError_t launch_eps_grid(int nx, int ny, int periodic, double hx, double hy, const double* xp,
                            const double* yp, double jx, double jy, const double* eps, int pitch,
                            double* D, double* exx, double* exy, double* eyy, int* folded,
                            cudaStream_t s);
// Reflect coefficients built on a grid with Neumann y sides (ny = n + 1 rows, pitch ps) into
// the periodic grid of twice the height (2n rows, pitch pd).
cudaError_t launch_mirror_eps(int nx, int n, int ps, const double* D0, const double* exx0,
                              const double* exy0, const double* eyy0, int pd, double* D, double* exx,
                              double* exy, double* eyy, cudaStream_t s);
// Nodal tensor (e[0..2]: eps_xx, eps_xy, eps_yy of level F) coarsened to level C (c[0..2]):
// full weighting inside, injection on the boundary ring (rediscretized hierarchies).
template <typename TS, typename TD>
cudaError_t launch_coarsen_eps(const Op<TS>& F, const Op<TD>& C, const TS* const* e, TD* const* c,
                               cudaStream_t s);
// dinv = false: A.dinv is not written (a mixed-precision hierarchy's FP64 level 0, whose
// reciprocal diagonal is taken in FP32 by launch_op_to_f32 with dinv_f32).
// In FP32 for the coarse levels of a mixed rediscretized hierarchy.
template <typename T>
cudaError_t launch_assemble(const Op<T>& A, double hx, double hy, const T* exx, const T* exy, const T* eyy,
                            cudaStream_t s, bool dinv = true);
// The same for an operator without cross term (A.five_point) in one pass, with the FP32 copy of
// op_to_f32 (reciprocal of the FP32 diagonal) when B is given; bitwise the separate kernels'
// values.  dinv: write A's FP64 reciprocal diagonal.
cudaError_t launch_assemble_five(const OpF64& A, const OpF32* B, double hx, double hy, const double* exx,
                                 const double* eyy, cudaStream_t s, bool dinv);
cudaError_t launch_rhs(const OpF64& A, const double* rho, int rho_pitch, const double* D, double* b,
                       cudaStream_t s);
template <typename T>
cudaError_t launch_galerkin(const Op<T>& F, const Op<T>& C, cudaStream_t s);
cudaError_t launch_op_to_f64(const OpF32& A, const OpF64& B, cudaStream_t s);
// dinv_f32: B.dinv = 1 / B.diag in FP32 instead of the rounded A.dinv (A.dinv is not read).
cudaError_t launch_op_to_f32(const OpF64& A, const OpF32& B, cudaStream_t s, bool dinv_f32 = false);
cudaError_t launch_coarse_factor(const OpF64& A, double* inv, int* status, cudaStream_t s);

// ---- cycle (k_cycle.cu).  `skip` (nullable device int): when *skip != 0 the kernel
// returns at once (used inside the solve graph after convergence).
template <typename T>
cudaError_t launch_gs_colour(const Op<T>& A, T* phi, const T* b, int colour, const int* skip,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_smooth(const Op<T>& A, T* phi, const T* b, int sweeps, int reverse,
                          const int* skip, cudaStream_t s);
// `sweeps` sweeps of four-colour SOR with factor omega (forward colour order).
template <typename T>
cudaError_t launch_sor(const Op<T>& A, T* phi, const T* b, int sweeps, double omega, const int* skip,
                       cudaStream_t s);
template <typename T>
cudaError_t launch_residual(const Op<T>& A, const T* phi, const T* b, T* r, const int* skip,
                            cudaStream_t s);
template <typename T>
cudaError_t launch_jacobi(const Op<T>& A, T* phi, const T* b, T* tmp, int sweeps, double omega,
                          const int* skip, cudaStream_t s);
// phiH (nullable) is zeroed on the coarse grid at the same time.
template <typename T>
cudaError_t launch_resid_restrict(const Op<T>& A, const T* phi, const T* b, T* bH, T* phiH,
                                  int pitch_c, const int* skip, cudaStream_t s);
// The same after a pre-smoothing whose last half-sweep solved every odd row exactly (zebra
// x-line): the odd rows' residual is taken as zero and only the even rows' is computed.
template <typename T>
cudaError_t launch_resid_restrict_even(const Op<T>& A, const T* phi, const T* b, T* bH, T* phiH,
                                       int pitch_c, const int* skip, cudaStream_t s);
template <typename T>
cudaError_t launch_prolong_add(const Op<T>& A, T* phi, const T* eH, int pitch_c, const int* skip,
                               cudaStream_t s);
template <typename T>
cudaError_t launch_coarse_solve(const Op<T>& A, const double* inv, const T* b, T* x,
                                const int* skip, cudaStream_t s);

}  // namespace mg
