// Host-side emission of one V-cycle (mg_vcycle.cu).
#pragma once
#include <cuda_runtime.h>

#include "mg_launch.h"
#include "mg_line.h"

namespace mg {

constexpr int kMaxVLevels = 24;

// Smoother family for a level: the per-colour kernels (four launches a sweep), the fused
// tile kernel, the pipelined tile kernel, the row-marching kernel.
enum SmoothKind : int { SK_DEFAULT = 0, SK_COLOUR = 1, SK_FUSED = 2, SK_PIPE = 3, SK_MARCH = 4 };

// Measured choice of smoother family and variant by level size (filled by mg_autotune):
// entry k says that square levels of side[k] smooth fastest with kind[k], variant var[k] (tile
// shape or sweeps per pass, mg_tile.h).  A level takes the choice of the entry nearest to it
// in node count (log scale); kinds that cannot run on a level fall back to the size-threshold
// rule.
struct SmoothPolicy {
  int n = 0;
  int side[16] = {};
  int kind[16] = {};
  int var[16] = {};
  int lookup(long long nodes, int* var_out = nullptr) const;
};

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
  const SmoothPolicy* pol = nullptr;  // measured smoother choice (nullable)
  LineFactors<T> lf[kMaxVLevels];     // line-smoother factors of levels 0 .. L-2 (line smoother)
};

// Enqueue one V(nu1, nu2) cycle starting from the iterate in V.x[0]; *result receives the
// array (V.x[0] or V.t[0]) that holds the level-0 result.  x0_zero: the caller's iterate is
// zero at every unknown (the preconditioner's start) and its Dirichlet nodes are zero, so a
// smoother that can use it need not read it (the caller may skip clearing it when
// vcycle_reads_x0() says so).
template <typename T>
cudaError_t emit_vcycle(const VLevels<T>& V, int smoother, int nu1, int nu2, double omega,
                        const int* skip, cudaStream_t s, T** result, bool x0_zero = false);

// Whether emit_vcycle with x0_zero reads the unknowns of V.x[0]: false for the line
// smoother with pre-smoothing, whose first half-sweep starts from zero without reading.
inline bool vcycle_reads_x0(int smoother, int nu1) { return !(smoother == 2 && nu1 > 0); }

template <typename T>
int tail_nodes();

}  // namespace mg
