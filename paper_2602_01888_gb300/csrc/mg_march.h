// Row-marching temporally blocked smoother (k_march.cu).
#pragma once
#include <cuda_runtime.h>

#include "mg_launch.h"

namespace mg {

// Sweeps one launch performs, and the strip width (owned columns) of one CTA.
template <typename T>
int march_sweeps();
template <typename T>
int march_strip_width();

// xout = march_sweeps<T>() Gauss-Seidel sweeps of (xin [+ P eH]) in forward (rev = 0) or
// reversed colour order; xin != xout; every array 16-byte aligned, pitch a multiple of
// 16 bytes.  eH (nullable): coarse correction with row pitch pitch_c.
template <typename T>
cudaError_t launch_smooth_march(const Op<T>& A, const T* xin, T* xout, const T* b, int rev,
                                const T* eH, int pitch_c, const int* skip, cudaStream_t s);

}  // namespace mg
