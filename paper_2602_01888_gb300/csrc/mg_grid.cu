// Numerical grid generation (Sec. 4.2, Eqs. 36-37): the physical coordinates x'(x, y),
// y'(x, y) of a boundary-fitted grid are discrete-harmonic functions of the computational
// coordinates, with Dirichlet data on the outer boundary and on internal nodes (the ring of
// an immersed body, whose nodes carry a boundary map such as Eq. 44).
//
// The solve runs through the library's own multigrid: the operator is the 5-point
// Laplacian that the identity map assembles (eps = I); every coupling between a free node
// and a fixed interior node is moved to the right-hand side and zeroed on both sides, and
// the fixed rows become identity rows (x = value).  The operator stays symmetric positive
// definite, its Galerkin hierarchy is built as usual, and flexible CG preconditioned by
// V(2,2) solves for x' and for y' from the caller's initial guess.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

#include "mg.h"
#include "mg_common.cuh"
#include "mg_internal_host.h"
#include "mg_launch.h"

namespace mg {

static constexpr int kGT = 256;

// rho at every unknown: the fixed value at fixed nodes (identity rows, det J = 1), minus the
// sum of coupling x fixed value over fixed interior neighbours elsewhere.  fixed, v and rho
// are node arrays with row stride nx.
__global__ void __launch_bounds__(kGT) k_mask_rhs(Lvl<double> L, const unsigned char* __restrict__ fixed,
                                                  const double* __restrict__ v, double* __restrict__ rho) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= L.nx || j >= L.nyr) return;
  const size_t u = (size_t)j * L.nx + i;
  if (!is_unknown(L, i, j)) {
    rho[u] = 0.0;
    return;
  }
  if (fixed[u]) {
    rho[u] = v[u];
    return;
  }
  const int p = L.pitch;
  const int jd = row_dn(j, L.nyr), ju = row_up(j, L.nyr);
  const size_t r0 = (size_t)j * p, rd = (size_t)jd * p;
  const size_t q0 = (size_t)j * L.nx, qd = (size_t)jd * L.nx, qu = (size_t)ju * L.nx;
  // neighbour (ii, jj) contributes coupling * value when it is a fixed unknown
  auto term = [&](double c, int ii, int jj, size_t qrow) -> double {
    return (is_unknown(L, ii, jj) && fixed[qrow + ii]) ? c * v[qrow + ii] : 0.0;
  };
  double s = term(L.cE[r0 + i], i + 1, j, q0);
  s += term(L.cE[r0 + i - 1], i - 1, j, q0);
  s += term(L.cN[r0 + i], i, ju, qu);
  s += term(L.cN[rd + i], i, jd, qd);
  s += term(L.cNE[r0 + i], i + 1, ju, qu);
  s += term(L.cNE[rd + i - 1], i - 1, jd, qd);
  s += term(L.cNW[r0 + i], i - 1, ju, qu);
  s += term(L.cNW[rd + i + 1], i + 1, jd, qd);
  rho[u] = -s;
}

// Decouple the fixed interior nodes: identity rows at fixed nodes, and every stored coupling
// that touches a fixed interior node set to zero, whichever node stores it (boundary nodes
// included, so that a fixed node next to the boundary keeps no coupling either).  Run after
// k_mask_rhs read the couplings.
__global__ void __launch_bounds__(kGT) k_mask_apply(Op<double> A, Lvl<double> L, const unsigned char* __restrict__ fixed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  const int nyr = L.nyr;
  if (i >= A.nx || j >= nyr) return;
  const size_t k = (size_t)j * A.pitch + i;
  const size_t u = (size_t)j * A.nx + i;
  if (is_unknown(L, i, j) && fixed[u]) {
    A.cE[k] = A.cN[k] = A.cNE[k] = A.cNW[k] = 0.0;
    A.diag[k] = A.dinv[k] = 1.0;
    return;
  }
  if (!L.periodic && j == nyr - 1) {  // no north neighbours: only the east coupling exists
    if (i + 1 < A.nx && is_unknown(L, i + 1, j) && fixed[u + 1]) A.cE[k] = 0.0;
    return;
  }
  const int ju = row_up(j, nyr);
  const size_t qu = (size_t)ju * A.nx;
  auto fixed_unknown = [&](int ii, int jj, size_t qrow) {
    return ii >= 0 && ii < A.nx && is_unknown(L, ii, jj) && fixed[qrow + ii];
  };
  if (fixed_unknown(i + 1, j, (size_t)j * A.nx)) A.cE[k] = 0.0;
  if (fixed_unknown(i, ju, qu)) A.cN[k] = 0.0;
  if (fixed_unknown(i + 1, ju, qu)) A.cNE[k] = 0.0;
  if (fixed_unknown(i - 1, ju, qu)) A.cNW[k] = 0.0;
}

}  // namespace mg

using namespace mg;

extern "C" mg_status mg_harmonic_grid(mg_ctx* ctx, const mg_grid_desc* grid, const unsigned char* fixed,
                                      const double* xp, const double* yp, double* xp_out,
                                      double* yp_out, mg_mem_kind mem, double rtol,
                                      mg_solve_stats* stats) {
  if (!ctx || !grid || !fixed || !xp || !yp || !xp_out || !yp_out)
    return set_error(MG_ERR_ARG, "mg_harmonic_grid: NULL argument");
  if (mem != MG_MEM_HOST && mem != MG_MEM_DEVICE) return set_error(MG_ERR_ARG, "mg_harmonic_grid: bad memory kind");
  if (!(rtol > 0.0)) return set_error(MG_ERR_ARG, "mg_harmonic_grid: rtol must be positive");
  if (grid->neumann_y) return set_error(MG_ERR_ARG, "mg_harmonic_grid: Neumann sides are not supported");
  mg_solve_opts o;
  mg_default_opts(&o);
  o.precision = MG_PREC_FP64;
  o.outer = MG_OUTER_FCG;
  o.rtol = rtol;
  o.max_iters = 400;
  o.warm_start = 1;
  mg_problem* P = nullptr;
  mg_status st = problem_create(ctx, grid, o, &P);
  if (st) return st;
  cudaStream_t s = ctx->stream;
  const int nx = grid->nx, nyr = grid->periodic_y ? grid->ny - 1 : grid->ny;
  const size_t n = (size_t)nx * nyr;
  // device staging: mask, the two coordinate arrays (initial guess and Dirichlet data),
  // the two right-hand sides and, for host memory, the two results
  std::vector<void*> tmp;
  auto dalloc = [&](size_t bytes) -> void* {
    void* q = ctx->pool.alloc(bytes);
    if (q) tmp.push_back(q);
    return q;
  };
  auto cleanup = [&](mg_status code) {
    char keep[512];
    snprintf(keep, sizeof keep, "%s", mg_last_error());
    cudaStreamSynchronize(s);
    for (void* q : tmp) ctx->pool.release(q);
    mg_problem_free(P);
    return code ? set_error(code, "%s", keep) : MG_OK;
  };
  const bool host = mem == MG_MEM_HOST;
  const unsigned char* mask_d = fixed;
  const double *xin = xp, *yin = yp;
  double *xo = xp_out, *yo = yp_out;
  if (host) {
    unsigned char* m = (unsigned char*)dalloc(n);
    double* a = (double*)dalloc(4 * n * sizeof(double));
    if (!m || !a) return cleanup(set_error(MG_ERR_OOM, "mg_harmonic_grid: device memory budget exhausted"));
    cudaMemcpyAsync(m, fixed, n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(a, xp, n * sizeof(double), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(a + n, yp, n * sizeof(double), cudaMemcpyHostToDevice, s);
    mask_d = m;
    xin = a;
    yin = a + n;
    xo = a + 2 * n;
    yo = a + 3 * n;
  }
  double* rho = (double*)dalloc(2 * n * sizeof(double));
  if (!rho) return cleanup(set_error(MG_ERR_OOM, "mg_harmonic_grid: device memory budget exhausted"));
  // identity map: eps = I, det J = 1, the 5-point Laplacian; then the mask
  mg_map_desc id{};
  id.kind = MG_MAP_IDENTITY;
  FineHook hook = [&](mg_problem* Q, cudaStream_t ss) -> mg_status {
    const Lvl<double> L = lvl_of(Q->lev[0].A);
    const dim3 g((nx + kGT - 1) / kGT, nyr);
    k_mask_rhs<<<g, kGT, 0, ss>>>(L, mask_d, xin, rho);
    k_mask_rhs<<<g, kGT, 0, ss>>>(L, mask_d, yin, rho + n);
    k_mask_apply<<<g, kGT, 0, ss>>>(Q->lev[0].A, L, mask_d);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MG_OK : set_error(MG_ERR_CUDA, "mg_harmonic_grid: %s", cudaGetErrorString(e));
  };
  st = problem_enqueue_build(P, &id, nullptr, MG_MEM_DEVICE, s, &hook);
  if (!st && cudaStreamSynchronize(s) != cudaSuccess) st = set_error(MG_ERR_CUDA, "mg_harmonic_grid: build failed");
  if (!st) st = problem_check_build(P);
  if (st) return cleanup(st);
  // x' then y': warm start from the caller's arrays (which also carry the boundary data)
  const double* in[2] = {xin, yin};
  double* out[2] = {xo, yo};
  for (int c = 0; c < 2 && !st; ++c) {
    st = enqueue_solve(P, o, rho + c * n, in[c], in[c], out[c], s);
    if (!st && cudaStreamSynchronize(s) != cudaSuccess) st = set_error(MG_ERR_CUDA, "mg_harmonic_grid: solve failed");
    if (!st) st = finish_solve(P, stats ? &stats[c] : nullptr);
  }
  if (!st && host) {
    if (cudaMemcpyAsync(xp_out, xo, n * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(yp_out, yo, n * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      st = set_error(MG_ERR_CUDA, "mg_harmonic_grid: copy-out failed");
  }
  return cleanup(st);
}
