// Fused smoothing and single-CTA tail kernels (k_fused.cu).
#pragma once
#include <cuda_runtime.h>

#include "mg_common.cuh"
#include "mg_launch.h"

namespace mg {

constexpr int kFusedThreads = 256;
constexpr int kTailThreads = 1024;
constexpr int kMaxTail = 10;
// Shared memory the tail kernel may use (its levels are staged there); the static
// coarse right-hand side (2 KB) comes on top.
constexpr size_t kTailSmemMax = 220 * 1024;

template <typename T>
struct TailLevel {
  Lvl<T> L;
  T* x;  // current iterate (in place)
  T* b;  // right-hand side
  T* t;  // residual scratch
};

// Levels lv[0] (finest handled by the tail) .. lv[nlev-1] (coarsest, dense inverse inv).
template <typename T>
struct TailArgs {
  int nlev, nu1, nu2;
  int line;  // 1: zebra x-line Gauss-Seidel on the tail levels, 0: four-colour Gauss-Seidel
  const double* inv;
  TailLevel<T> lv[kMaxTail];
};

// Sweeps fused per launch of k_smooth_fused for this precision and variant (mg_tile.h;
// v < 0: the default variant).
template <typename T>
int fused_sweeps(int v = -1);

// xout = NS Gauss-Seidel sweeps applied to (xin + P eH when eH != nullptr); rev = colour
// order reversed.  xin and xout must be different arrays.  v: tile variant (mg_tile.h).
template <typename T>
cudaError_t launch_smooth_fused(const Op<T>& A, const T* xin, T* xout, const T* b, int rev,
                                const T* eH, int pitch_c, const int* skip, cudaStream_t s, int v = -1);

template <typename T>
cudaError_t launch_tail(const TailArgs<T>& a, const int* skip, cudaStream_t s);

// Shared-memory bytes the tail kernel needs for these levels.
template <typename T>
size_t tail_bytes(const TailArgs<T>& a);

}  // namespace mg
