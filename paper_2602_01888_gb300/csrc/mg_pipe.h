// Persistent pipelined fused smoother (k_pipe.cu).
#pragma once
#include <cuda_runtime.h>

#include "mg_launch.h"

namespace mg {

constexpr int kPipeThreads = 512;
constexpr long long kPipeSpinLimit = 1ll << 26;  // mbarrier polls before a wait gives up

// Sweeps one launch performs for this precision and variant (mg_tile.h; v < 0: default).
template <typename T>
int pipe_sweeps(int v = -1);

// xout = pipe_sweeps<T>(v) Gauss-Seidel sweeps of (xin [+ P eH]); xin != xout; every array
// 16-byte aligned with a pitch that keeps rows 16-byte aligned.  *err (nullable device
// int) is set when a copy wait times out.  v: tile variant (mg_tile.h).
template <typename T>
cudaError_t launch_smooth_pipe(const Op<T>& A, const T* xin, T* xout, const T* b, int rev,
                               const T* eH, int pitch_c, const int* skip, int* err,
                               cudaStream_t s, int v = -1);

}  // namespace mg
