// Row-marching temporally blocked smoother (k_march.cu).
#pragma once
#include <cuda_runtime.h>

#include "mg_launch.h"

namespace mg {

// Sweeps one launch performs, and the strip width (owned columns) of one CTA, for variant v
// (mg_tile.h; v < 0: the precision's default).
template <typename T>
int march_sweeps(int v = -1);
template <typename T>
int march_strip_width(int v = -1);

// xout = march_sweeps<T>(v) Gauss-Seidel sweeps of (xin [+ P eH]) in forward (rev = 0) or
// reversed colour order; xin != xout; every array 16-byte aligned, pitch a multiple of
// 16 bytes.  eH (nullable): coarse correction with row pitch pitch_c.
template <typename T>
cudaError_t launch_smooth_march(const Op<T>& A, const T* xin, T* xout, const T* b, int rev,
                                const T* eH, int pitch_c, const int* skip, cudaStream_t s, int v = -1);

}  // namespace mg
