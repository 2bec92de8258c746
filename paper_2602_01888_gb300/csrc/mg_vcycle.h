// Host-side emission of one V-cycle (mg_vcycle.cu).
#pragma once
#include <cuda_runtime.h>

#include "mg_launch.h"

namespace mg {

constexpr int kMaxVLevels = 24;

// A hierarchy as seen by one cycle: level l operator, iterate x, right-hand side b and a
// second iterate array t (ping-pong partner / residual scratch); inv = coarsest inverse.
template <typename T>
struct VLevels {
  int L = 0;
  Op<T> A[kMaxVLevels];
  T* x[kMaxVLevels];
  T* b[kMaxVLevels];
  T* t[kMaxVLevels];
  const double* inv = nullptr;
  int* err = nullptr;  // device flag set when a bounded wait of a kernel gives up
};

// Enqueue one V(nu1, nu2) cycle starting from the iterate in V.x[0]; *result receives the
// array (V.x[0] or V.t[0]) that holds the level-0 result.
template <typename T>
cudaError_t emit_vcycle(const VLevels<T>& V, int smoother, int nu1, int nu2, double omega,
                        const int* skip, cudaStream_t s, T** result);

template <typename T>
int tail_nodes();

}  // namespace mg
