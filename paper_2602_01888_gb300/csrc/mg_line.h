// Zebra x-line Gauss-Seidel smoother (k_line.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

#include "mg_launch.h"

namespace mg {

// Largest dynamic shared memory a line kernel may use (one CTA per SM).
constexpr size_t kLineSmemMax = 227 * 1024;

// Cyclic-reduction factors of the tridiagonal row systems of one level (row stride np).
template <typename T>
struct LineFactors {
  int np = 0;  // padded row length: nx - 2 rounded up to a power of two (at least 2)
  T *alpha = nullptr, *gamma = nullptr;                 // reduction multipliers, by level
  T *afin = nullptr, *cfin = nullptr, *binv = nullptr;  // back-substitution coefficients
};

// Elements of type T that the factors of an nx x ny level take.
template <typename T>
size_t line_factor_elems(int nx, int ny, int periodic);

// Whether a level of width nx fits the line kernels' shared memory.
template <typename T>
bool line_supported(int nx);

// View of the factors of an nx x ny level stored from `base`.
template <typename T>
LineFactors<T> line_factors_at(T* base, int nx, int ny, int periodic);

// Factor every row of A (call again whenever A changes).
template <typename T>
cudaError_t launch_line_factor(const Op<T>& A, const LineFactors<T>& F, cudaStream_t s);

// One half-sweep: solve every row j with j mod 2 == par for its unknowns, in place in x.
// eH (nullable, par == 1 only): coarse correction (row pitch pitch_c), added by bilinear
// prolongation to the even rows first (the rows the half-sweep reads); the odd rows' old
// values are never read, so they need not be corrected, and the even rows are solved again
// by the next half-sweep.  zero_start: x is zero at every unknown.
template <typename T>
cudaError_t launch_line_rows(const Op<T>& A, const LineFactors<T>& F, T* x, const T* b, int par,
                             const int* skip, cudaStream_t s, const T* eH = nullptr, int pitch_c = 0,
                             int zero_start = 0);

// `sweeps` zebra sweeps: parity 0 then 1 per sweep (rev: 1 then 0).  eH (rev only) and
// zero_start apply to the first half-sweep, as above.
template <typename T>
cudaError_t launch_line_smooth(const Op<T>& A, const LineFactors<T>& F, T* x, const T* b, int sweeps,
                               int rev, const int* skip, cudaStream_t s, const T* eH = nullptr,
                               int pitch_c = 0, int zero_start = 0);

}  // namespace mg
