// Launchers of the solve-loop kernels (k_solve.cu) used by the host orchestration.
#pragma once
#include <cuda_runtime.h>

#include "mg_common.cuh"
#include "mg_launch.h"

namespace mg {

constexpr int kRedBlocks = 1216;  // upper bound of blocks (and partial sums) per reduction
constexpr int kRedThreads = 256;  // threads per block of the finest-level loops (one column each)

// Per-solve arguments read by the kernels through device memory, so one captured graph
// serves every call: the caller's arrays (contiguous rows of user_pitch elements).
struct SolveArgs {
  const double* rho;
  const double* bc;      // nullable
  const double* phi_in;  // warm start
  double* phi_out;
  int user_pitch;
  int warm;
  int max_iters;
  int mirror;  // Neumann y sides: n = ny - 1 of the caller's grid (its row r is row r + n of the
               // doubled system, r < n; row n is row 0; row j' < n mirrors row n - j'); else 0
  double rtol;
  long long n_unknowns;
};

dim3 red_grid(int nx, int nyr);
cudaError_t launch_solve_init(const OpF64& A, const SolveArgs* a, const double* D, double* x,
                              double* b, SolveState* st, cudaStream_t s);
cudaError_t launch_resid_init(const OpF64& A, const double* x, const double* b, double* r,
                              SolveState* st, double* part, cudaGraphConditionalHandle h,
                              int has_h, cudaStream_t s);
cudaError_t launch_resid_check(const OpF64& A, const double* x, const double* b, double* r,
                               SolveState* st, double* part, cudaGraphConditionalHandle h,
                               int has_h, cudaStream_t s);
cudaError_t launch_r_to_f32(const OpF64& A, const double* r, float* b32, int pitch32,
                            SolveState* st, cudaStream_t s);
cudaError_t launch_add_f32(const OpF64& A, double* x, const float* e32, int pitch32,
                           SolveState* st, cudaStream_t s);
cudaError_t launch_iter_inc(SolveState* st, cudaStream_t s);
cudaError_t launch_loop_guard(SolveState* st, cudaGraphConditionalHandle h, cudaStream_t s);
template <typename TZ>
cudaError_t launch_fcg_zq(const OpF64& A, const TZ* z, int zp, const double* q, SolveState* st,
                          double* part, cudaStream_t s);
template <typename TZ>
cudaError_t launch_fcg_pq(const OpF64& A, const TZ* z, int zp, double* p, double* q, const double* r,
                          SolveState* st, double* part, cudaStream_t s);
cudaError_t launch_fcg_update(const OpF64& A, double* x, double* r, const double* p,
                              const double* q, float* r32, int p32, SolveState* st, double* part,
                              cudaGraphConditionalHandle h, int has_h, cudaStream_t s);
cudaError_t launch_fcg_verify(const OpF64& A, const double* x, const double* b, double* r,
                              float* r32, int p32, SolveState* st, double* part,
                              cudaGraphConditionalHandle h, int has_h, cudaStream_t s);
cudaError_t launch_gather_states(SolveState* const* src, int* const* srcflags, SolveState* dst,
                                 int* dflags, int count, cudaStream_t s);
cudaError_t launch_copy_out(const OpF64& A, const double* x, const SolveArgs* a, cudaStream_t s);

}  // namespace mg
