// Host orchestration of libmg: contexts with a device memory pool, resident problems
// (coefficient build + multigrid hierarchy), solves captured as CUDA graphs whose
// iteration loop is a device-driven WHILE node, and batched solves.  C ABI of mg.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "mg.h"
#include "mg_launch.h"
#include "mg_solve_kernels.h"
#include "mg_internal_host.h"
#include "mg_line.h"
#include "mg_vcycle.h"

namespace mg {

// ------------------------------------------------------------------ errors
static thread_local char g_err[512] = "";

mg_status set_error(mg_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return s;
}

#define CU(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return set_error(MG_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
  } while (0)

// ------------------------------------------------------------------ memory pool
// Slabs of device memory obtained with cudaMalloc (or page-locked host memory from
// cudaMallocHost); best-fit ranges inside them, coalesced on release; total slab bytes
// capped by the budget.
void* Pool::alloc(size_t n) {
  std::lock_guard<std::mutex> lk(mu_);
  n = (n + 255) & ~size_t(255);
  if (n == 0) n = 256;
  for (int pass = 0; pass < 2; ++pass) {
    int best_s = -1;
    size_t best_off = 0, best_len = SIZE_MAX;
    for (size_t s = 0; s < slabs_.size(); ++s)
      for (auto& fr : slabs_[s].free_)
        if (fr.second >= n && fr.second < best_len) {
          best_s = (int)s;
          best_off = fr.first;
          best_len = fr.second;
        }
    if (best_s >= 0) {
      Slab& sl = slabs_[best_s];
      sl.free_.erase(best_off);
      if (best_len > n) sl.free_[best_off + n] = best_len - n;
      char* p = sl.base + best_off;
      live_[p] = {best_s, n};
      used_ += n;
      return p;
    }
    if (pass == 1) break;
    size_t want = std::max(n, slab_min_);
    if (reserved_ + want > budget_) want = n;
    if (reserved_ + want > budget_) return nullptr;
    void* base = nullptr;
    if ((pinned_ ? cudaMallocHost(&base, want) : cudaMalloc(&base, want)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    Slab sl;
    sl.base = (char*)base;
    sl.size = want;
    sl.free_[0] = want;
    slabs_.push_back(sl);
    reserved_ += want;
  }
  return nullptr;
}

void Pool::release(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(mu_);
  auto it = live_.find(p);
  if (it == live_.end()) return;
  Slab& sl = slabs_[it->second.first];
  size_t off = (char*)p - sl.base, len = it->second.second;
  used_ -= len;
  live_.erase(it);
  auto nx = sl.free_.lower_bound(off);
  if (nx != sl.free_.end() && off + len == nx->first) {
    len += nx->second;
    nx = sl.free_.erase(nx);
  }
  if (nx != sl.free_.begin()) {
    auto pv = std::prev(nx);
    if (pv->first + pv->second == off) {
      pv->second += len;
      return;
    }
  }
  sl.free_[off] = len;
}

Pool::~Pool() {
  for (auto& s : slabs_) {
    if (pinned_) cudaFreeHost(s.base);
    else cudaFree(s.base);
  }
}

// ------------------------------------------------------------------ hierarchy sizes
// Same rule as the oracle: coarsen while both n-1 are even, the coarse grid keeps
// unknowns in both directions and the current level has more than coarse_max unknowns.
int count_levels(int nx, int ny, int periodic, int coarse_max, int* nxs, int* nys) {
  int L = 1;
  nxs[0] = nx;
  nys[0] = ny;
  while (L < kMaxLevels) {
    if (coarse_unknowns(nx, ny, periodic) <= coarse_max) break;
    if ((nx - 1) % 2 || (ny - 1) % 2) break;
    const int nxc = (nx - 1) / 2 + 1, nyc = (ny - 1) / 2 + 1;
    if (nxc < 3 || nyc < 3) break;
    if (periodic && nyc - 1 < 2) break;
    nx = nxc;
    ny = nyc;
    nxs[L] = nx;
    nys[L] = ny;
    ++L;
  }
  return L;
}

static int pitch_for(int nx) { return (nx + 31) & ~31; }

}  // namespace mg

using namespace mg;

// ------------------------------------------------------------------ context
extern "C" const char* mg_last_error(void) { return g_err; }

extern "C" void mg_default_opts(mg_solve_opts* o) {
  if (!o) return;
  o->precision = MG_PREC_FP64;
  o->outer = MG_OUTER_FCG;
  o->smoother = MG_SMOOTH_GS4;
  o->nu1 = 2;
  o->nu2 = 2;
  o->omega_j = 0.8;
  o->rtol = 1e-10;
  o->max_iters = 200;
  o->coarse_max = 64;
  o->warm_start = 0;
  o->coarse_op = MG_COARSE_GALERKIN;
}

extern "C" mg_status mg_create(int device, size_t mem_budget, mg_ctx** out) {
  if (!out) return set_error(MG_ERR_ARG, "mg_create: out is NULL");
  *out = nullptr;
  int n = 0;
  CU(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return set_error(MG_ERR_ARG, "mg_create: no CUDA device %d", device);
  CU(cudaSetDevice(device));
  size_t fr = 0, tot = 0;
  CU(cudaMemGetInfo(&fr, &tot));
  mg_ctx* c = new mg_ctx();
  c->device = device;
  c->pool.budget_ = mem_budget ? mem_budget : (size_t)(0.9 * (double)fr);
  if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->cap_stream2, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return set_error(MG_ERR_CUDA, "mg_create: stream creation failed");
  }
  c->stream = c->own_stream;
  for (int k = 0; k < kBatchStreams; ++k) cudaStreamCreateWithFlags(&c->batch[k], cudaStreamNonBlocking);
  *out = c;
  return MG_OK;
}

extern "C" void mg_destroy(mg_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  batch_cache_clear(c);
  // problems the caller did not free: their memory belongs to this context's pool
  std::vector<mg_problem*> left;
  {
    std::lock_guard<std::mutex> lk(c->problems_mu);
    left.assign(c->problems.begin(), c->problems.end());
  }
  for (mg_problem* P : left) mg_problem_free(P);
  for (int k = 0; k < kBatchStreams; ++k) cudaStreamDestroy(c->batch[k]);
  cudaStreamDestroy(c->own_stream);
  cudaStreamDestroy(c->cap_stream);
  cudaStreamDestroy(c->cap_stream2);
  delete c;
}

extern "C" mg_status mg_set_stream(mg_ctx* c, void* stream) {
  if (!c) return set_error(MG_ERR_ARG, "mg_set_stream: ctx is NULL");
  c->stream = stream ? (cudaStream_t)stream : c->own_stream;
  return MG_OK;
}

extern "C" mg_status mg_mem_info(mg_ctx* c, size_t* used, size_t* budget) {
  if (!c) return set_error(MG_ERR_ARG, "mg_mem_info: ctx is NULL");
  if (used) *used = c->pool.used();
  if (budget) *budget = c->pool.budget_;
  return MG_OK;
}

// ------------------------------------------------------------------ problems
namespace mg {

template <typename T>
static T* palloc(mg_problem* P, size_t count) {
  void* p = P->ctx->pool.alloc(count * sizeof(T));
  if (p) P->allocs.push_back(p);
  return (T*)p;
}

static void problem_release(mg_problem* P) {
  for (auto& kv : P->graphs) {
    cudaGraphExecDestroy(kv.second.exec);
    cudaGraphDestroy(kv.second.graph);
  }
  P->graphs.clear();
  for (void* a : P->allocs) P->ctx->pool.release(a);
  P->allocs.clear();
  if (P->h_args) cudaFreeHost(P->h_args);
  if (P->h_state) cudaFreeHost(P->h_state);
  if (P->h_flags) cudaFreeHost(P->h_flags);
  if (P->ev0) cudaEventDestroy(P->ev0);
  if (P->ev1) cudaEventDestroy(P->ev1);
  if (P->evb0) cudaEventDestroy(P->evb0);
  if (P->evb1) cudaEventDestroy(P->evb1);
}

// Allocate every array of the hierarchy (FP64 levels, FP32 mirrors when mixed, the
// finest-level solve vectors and the coarsest inverse).
static mg_status problem_alloc(mg_problem* P, bool mixed) {
  for (int l = 0; l < P->nlev; ++l) {
    LevelMem& M = P->lev[l];
    const int nx = P->nxs[l], ny = P->nys[l], nyr = rows_stored(ny, P->grid.periodic_y);
    const int pt = pitch_for(nx);
    const size_t n = (size_t)pt * nyr;
    double* blk = palloc<double>(P, 9 * n);
    if (!blk) return set_error(MG_ERR_OOM, "device memory budget exhausted (level %d)", l);
    M.A = OpF64{nx, ny, P->grid.periodic_y, pt, blk, blk + n, blk + 2 * n, blk + 3 * n,
                blk + 4 * n, blk + 5 * n};
    M.x = blk + 6 * n;
    M.b = blk + 7 * n;
    M.t = blk + 8 * n;
    if (mixed) {
      float* f = palloc<float>(P, 9 * n);
      if (!f) return set_error(MG_ERR_OOM, "device memory budget exhausted (FP32 level %d)", l);
      M.A32 = OpF32{nx, ny, P->grid.periodic_y, pt, f, f + n, f + 2 * n, f + 3 * n, f + 4 * n,
                    f + 5 * n};
      M.x32 = f + 6 * n;
      M.b32 = f + 7 * n;
      M.t32 = f + 8 * n;
    }
    CU(cudaMemsetAsync(blk, 0, 9 * n * sizeof(double), P->ctx->stream));
    if (mixed) CU(cudaMemsetAsync(M.A32.cE, 0, 9 * n * sizeof(float), P->ctx->stream));
  }
  const size_t n0 = (size_t)P->lev[0].A.pitch * rows_stored(P->grid.ny, P->grid.periodic_y);
  double* v = palloc<double>(P, 5 * n0);
  if (!v) return set_error(MG_ERR_OOM, "device memory budget exhausted (solve vectors)");
  P->D = v;
  P->r = v + n0;
  P->z = v + 2 * n0;
  P->p = v + 3 * n0;
  P->q = v + 4 * n0;
  CU(cudaMemsetAsync(v, 0, 5 * n0 * sizeof(double), P->ctx->stream));
  const OpF64& C = P->lev[P->nlev - 1].A;
  P->m = coarse_unknowns(C.nx, C.ny, C.periodic);
  P->inv = palloc<double>(P, (size_t)P->m * P->m);
  P->part = palloc<double>(P, 4 * kRedBlocks);
  P->st = palloc<SolveState>(P, 1);
  P->args = palloc<SolveArgs>(P, 1);
  P->flags = palloc<int>(P, 4);
  if (!P->inv || !P->part || !P->st || !P->args || !P->flags)
    return set_error(MG_ERR_OOM, "device memory budget exhausted (solver state)");
  CU(cudaMemsetAsync(P->st, 0, sizeof(SolveState), P->ctx->stream));
  CU(cudaMallocHost(&P->h_args, sizeof(SolveArgs)));
  CU(cudaMallocHost(&P->h_state, sizeof(SolveState)));
  CU(cudaMallocHost(&P->h_flags, 4 * sizeof(int)));
  CU(cudaEventCreate(&P->ev0));
  CU(cudaEventCreate(&P->ev1));
  CU(cudaEventCreate(&P->evb0));
  CU(cudaEventCreate(&P->evb1));
  return MG_OK;
}

// Line-smoother factors: levels 0 .. nlev-2 back to back, in the precision of the cycle
// (FP32 for the mixed path).
template <typename T>
static T* line_base(const mg_problem* P, int l) {
  T* p = (T*)P->line;
  for (int q = 0; q < l; ++q) p += line_factor_elems<T>(P->nxs[q], P->nys[q], P->grid.periodic_y);
  return p;
}

template <typename T>
static LineFactors<T> line_level(const mg_problem* P, int l) {
  return line_factors_at<T>(line_base<T>(P, l), P->nxs[l], P->nys[l], P->grid.periodic_y);
}

static mg_status line_enqueue_factor(mg_problem* P, cudaStream_t s) {
  for (int l = 0; l < P->nlev - 1; ++l) {
    if (P->mixed) CU(launch_line_factor<float>(P->lev[l].A32, line_level<float>(P, l), s));
    else CU(launch_line_factor<double>(P->lev[l].A, line_level<double>(P, l), s));
  }
  return MG_OK;
}

mg_status line_prepare(mg_problem* P, cudaStream_t s) {
  if (P->line || P->nlev < 2) return MG_OK;
  const size_t esz = P->mixed ? sizeof(float) : sizeof(double);
  size_t elems = 0;
  for (int l = 0; l < P->nlev - 1; ++l) elems += line_factor_elems<double>(P->nxs[l], P->nys[l], P->grid.periodic_y);
  void* p = P->ctx->pool.alloc(elems * esz);
  if (!p) return set_error(MG_ERR_OOM, "device memory budget exhausted (line-smoother factors)");
  P->allocs.push_back(p);
  P->line = p;
  return line_enqueue_factor(P, s);
}

// Whether a map's transformed tensor has no cross term (Eq. 13 vanishes identically; the
// coefficient build then writes eps_xy = 0 exactly): its finest operator is a 5-point stencil.
static int map_five_point(const mg_map_desc* map) {
  return map->kind == MG_MAP_GRID ? 0 : map_kind_five_point(map->kind, map->params);
}

// A change of the finest operator's 5-point property changes which kernels a solve runs, so
// graphs captured with the old one (the problem's own, and captured batches holding it) are
// dropped once the work queued before the build has finished.
static void set_five_point(mg_problem* P, int five, cudaStream_t s) {
  if (P->lev[0].A.five_point == five) return;
  if (!P->graphs.empty()) {
    cudaStreamSynchronize(s);
    cudaStreamSynchronize(P->ctx->stream);
    for (auto& kv : P->graphs) {
      cudaGraphExecDestroy(kv.second.exec);
      cudaGraphDestroy(kv.second.graph);
    }
    P->graphs.clear();
  }
  batch_cache_drop(P->ctx, P);
  // a rediscretized hierarchy keeps the property on every level (the coarsened cross term of a
  // zero one is zero); Galerkin coarse levels are 9-point
  for (int l = 0; l < P->nlev; ++l) {
    const int f = (l == 0 || P->coarse_op == MG_COARSE_REDISCRETIZE) ? five : 0;
    P->lev[l].A.five_point = f;
    P->lev[l].A32.five_point = f;
  }
}

// Coefficients of the finest level from the map, then the Galerkin hierarchy and the
// coarsest inverse, enqueued on stream s.  Reads host or device inputs.  The map and SPD
// flags land in P->h_flags; problem_check_build reads them once s has been synchronised.
mg_status problem_enqueue_build(mg_problem* P, const mg_map_desc* map, const double* eps_phys,
                                mg_mem_kind mem, cudaStream_t s, const FineHook* hook) {
  // coefficients are computed on the caller's grid (for Neumann sides, then reflected into
  // the doubled periodic grid the hierarchy lives on)
  const mg_grid_desc& g = P->user;
  const int nx = g.nx, ny = g.ny, nyr = rows_stored(ny, g.periodic_y);
  const double hx = g.lx / (nx - 1), hy = g.ly / (ny - 1);
  const size_t nn = (size_t)nx * nyr;
  LevelMem& F = P->lev[0];
  const int pt = F.A.pitch;
  const size_t np = (size_t)pt * rows_stored(P->grid.ny, P->grid.periodic_y);
  CU(cudaEventRecord(P->evb0, s));
  // temporaries: eps components in the fine level's scratch arrays (x, b, t), inputs
  // staged in pitched layout in q / z / p; a Neumann grid's own D and eps go to x, b, t, r
  // and their reflection to D, q, z, p (the staged inputs are consumed by then)
  double *Dk = P->D, *exx = F.x, *exy = F.b, *eyy = F.t;
  if (P->mirror) {
    Dk = F.x;
    exx = F.b;
    exy = F.t;
    eyy = P->r;
  }
  const double* eps_d = nullptr;
  const double *xp_d = nullptr, *yp_d = nullptr;
  auto stage = [&](const double* src, double* dst) -> cudaError_t {
    return cudaMemcpy2DAsync(dst, pt * sizeof(double), src, nx * sizeof(double), nx * sizeof(double),
                             nyr, mem == MG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                             s);
  };
  if (eps_phys) {
    CU(stage(eps_phys, P->q));
    eps_d = P->q;
  }
  if (map->kind == MG_MAP_GRID) {
    CU(stage(map->xp, P->z));
    CU(stage(map->yp, P->p));
    xp_d = P->z;
    yp_d = P->p;
  }
  (void)nn;
  set_five_point(P, map_five_point(map), s);
  CU(cudaMemsetAsync(P->flags, 0, 4 * sizeof(int), s));
  if (map->kind == MG_MAP_GRID) {
    CU(launch_eps_grid(nx, ny, g.periodic_y, hx, hy, xp_d, yp_d, map->jump_x, map->jump_y, eps_d, pt,
                       Dk, exx, exy, eyy, P->flags, s));
  } else {
    CU(launch_eps_analytic(map->kind, map->params, nx, ny, g.periodic_y, g.x0, g.y0, hx, hy, eps_d,
                           pt, Dk, exx, exy, eyy, P->flags, s));
  }
  if (P->mirror) {
    CU(launch_mirror_eps(nx, P->mirror, pt, Dk, exx, exy, eyy, pt, P->D, P->q, P->z, P->p, s));
    exx = P->q;
    exy = P->z;
    eyy = P->p;
  }
  // a mixed hierarchy never runs an FP64 smoother: its level-0 reciprocal diagonal is the FP32
  // one, taken from the FP32 diagonal, so the FP64 division per node is skipped.  Without a
  // cross term (and without a caller's change of the finest operator, which the FP32 copy
  // must follow) couplings, diagonal and the FP32 copy come from one pass.
  const bool five_pass = F.A.five_point && !(hook && *hook);
  const bool f32_done = five_pass && P->mixed;
  if (five_pass) CU(launch_assemble_five(F.A, P->mixed ? &F.A32 : nullptr, hx, hy, exx, eyy, s, !P->mixed));
  else CU(launch_assemble(F.A, hx, hy, exx, exy, eyy, s, !P->mixed));
  if (hook && *hook) {  // a caller's change of the finest operator before coarsening
    mg_status hs = (*hook)(P, s);
    if (hs) return hs;
  }
  if (P->coarse_op == MG_COARSE_REDISCRETIZE) {
    // each coarse level: the tensor of the level above coarsened (into the level's scratch
    // arrays x, b, t), then assembled on the coarse grid like the finest level; a mixed
    // hierarchy does it in FP32 (its cycle runs on FP32 operators; the coarsest is widened to
    // FP64 for its dense inverse, as with Galerkin products)
    double hxl = hx, hyl = hy;
    if (!P->mixed) {
      const double* e[3] = {exx, exy, eyy};
      for (int l = 1; l < P->nlev; ++l) {
        LevelMem& C = P->lev[l];
        double* c[3] = {C.x, C.b, C.t};
        CU((launch_coarsen_eps<double, double>(P->lev[l - 1].A, C.A, e, c, s)));
        hxl *= 2.0;
        hyl *= 2.0;
        CU(launch_assemble<double>(C.A, hxl, hyl, c[0], c[1], c[2], s));
        for (int k = 0; k < 3; ++k) e[k] = c[k];
      }
    } else {
      if (!f32_done) CU(launch_op_to_f32(F.A, F.A32, s, true));
      const double* e64[3] = {exx, exy, eyy};
      const float* e[3] = {nullptr, nullptr, nullptr};
      for (int l = 1; l < P->nlev; ++l) {
        LevelMem& C = P->lev[l];
        float* c[3] = {C.x32, C.b32, C.t32};
        if (l == 1) CU((launch_coarsen_eps<double, float>(F.A, C.A32, e64, c, s)));
        else CU((launch_coarsen_eps<float, float>(P->lev[l - 1].A32, C.A32, e, c, s)));
        hxl *= 2.0;
        hyl *= 2.0;
        CU(launch_assemble<float>(C.A32, hxl, hyl, c[0], c[1], c[2], s));
        for (int k = 0; k < 3; ++k) e[k] = c[k];
      }
      if (P->nlev > 1) CU(launch_op_to_f64(P->lev[P->nlev - 1].A32, P->lev[P->nlev - 1].A, s));
    }
    // the coarse levels' iterates, right-hand sides and scratch held the tensors: zero them
    // again (the cycles rely on zero Dirichlet rings on coarse levels)
    for (int l = 1; l < P->nlev; ++l) {
      const LevelMem& C = P->lev[l];
      const size_t n = (size_t)C.A.pitch * rows_stored(C.A.ny, C.A.periodic);
      if (P->mixed) CU(cudaMemsetAsync(C.x32, 0, 3 * n * sizeof(float), s));  // x32, b32, t32 contiguous
      else CU(cudaMemsetAsync(C.x, 0, 3 * n * sizeof(double), s));            // x, b, t contiguous
    }
  } else if (!P->mixed) {
    for (int l = 1; l < P->nlev; ++l) CU(launch_galerkin<double>(P->lev[l - 1].A, P->lev[l].A, s));
  } else {
    // the FP32 cycle only needs FP32 coarse operators: Galerkin products in FP32, and the
    // coarsest one widened to FP64 for its dense inverse
    if (!f32_done) CU(launch_op_to_f32(F.A, F.A32, s, true));
    for (int l = 1; l < P->nlev; ++l) CU(launch_galerkin<float>(P->lev[l - 1].A32, P->lev[l].A32, s));
    if (P->nlev > 1) CU(launch_op_to_f64(P->lev[P->nlev - 1].A32, P->lev[P->nlev - 1].A, s));
  }
  CU(launch_coarse_factor(P->lev[P->nlev - 1].A, P->inv, P->flags + 1, s));
  P->setup_kernels =
      P->coarse_op == MG_COARSE_REDISCRETIZE
          ? 1 + 2 + 3 * (P->nlev - 1) + (P->mixed ? 1 + (P->nlev > 1 ? 1 : 0) : 0) + 1 + (P->mirror ? 1 : 0)
          : 1 + 2 + (P->mixed ? 1 + (P->nlev - 1) + (P->nlev > 1 ? 1 : 0) : P->nlev - 1) + 1 +
                (P->mirror ? 1 : 0);
  if (five_pass) P->setup_kernels -= f32_done ? 2 : 1;  // one kernel for two (three with the FP32 copy)
  if (P->line) {  // the line smoother's row factors follow the new operators
    mg_status ls = line_enqueue_factor(P, s);
    if (ls) return ls;
    P->setup_kernels += P->nlev - 1;
  }
  // restore the scratch vectors used as staging (solves rely on their zero Dirichlet entries)
  if (eps_phys || map->kind == MG_MAP_GRID || P->mirror)
    CU(cudaMemsetAsync(P->z, 0, 3 * np * sizeof(double), s));
  CU(cudaEventRecord(P->evb1, s));
  CU(cudaMemcpyAsync(P->h_flags, P->flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
  return MG_OK;
}

// Outcome of an enqueued build; the build's stream must have been synchronised.  The
// flags stay valid after a solve on the same stream (solves do not touch them).
mg_status problem_check_build(mg_problem* P) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, P->evb0, P->evb1);
  P->setup_ms = ms;
  if (P->h_flags[0]) return set_error(MG_ERR_MAP_FOLDED, "det J <= 0 at some node: the map folds");
  if (P->h_flags[1]) return set_error(MG_ERR_NOT_SPD, "coarsest operator is not SPD (non-positive pivot)");
  return MG_OK;
}

static mg_status problem_build(mg_problem* P, const mg_map_desc* map, const double* eps_phys,
                               mg_mem_kind mem) {
  cudaStream_t s = P->ctx->stream;
  mg_status st = problem_enqueue_build(P, map, eps_phys, mem, s);
  if (st) return st;
  CU(cudaStreamSynchronize(s));
  return problem_check_build(P);
}

static mg_status check_grid(const mg_grid_desc* g, int coarse_max, int* nlev, int* nxs, int* nys) {
  if (g->nx < 3 || g->ny < 3 || !(g->lx > 0) || !(g->ly > 0))
    return set_error(MG_ERR_SIZE, "grid too small or empty domain (nx=%d ny=%d)", g->nx, g->ny);
  if (g->periodic_y && (g->ny - 1) % 2)
    return set_error(MG_ERR_SIZE, "periodic y needs an even number of rows (ny-1=%d)", g->ny - 1);
  if ((size_t)g->nx * g->ny > ((size_t)1 << 31))
    return set_error(MG_ERR_SIZE, "grid larger than 2^31 nodes");
  if (g->nx > kRedBlocks * kRedThreads)  // the finest-level loops give each thread one column
    return set_error(MG_ERR_SIZE, "grid wider than %d nodes", kRedBlocks * kRedThreads);
  if (coarse_max < 1 || coarse_max > kCoarseMax)
    return set_error(MG_ERR_ARG, "coarse_max must be in [1, %d]", kCoarseMax);
  *nlev = count_levels(g->nx, g->ny, g->periodic_y, coarse_max, nxs, nys);
  const int L = *nlev - 1;
  if (coarse_unknowns(nxs[L], nys[L], g->periodic_y) > kCoarseMax)
    return set_error(MG_ERR_SIZE,
                     "grid %dx%d: coarsest level %dx%d has more than %d unknowns; sides must be "
                     "m*2^k+1 with a small m",
                     g->nx, g->ny, nxs[L], nys[L], kCoarseMax);
  return MG_OK;
}

mg_status check_map(const mg_grid_desc* g, const mg_map_desc* m) {
  if (!m) return set_error(MG_ERR_ARG, "map is NULL");
  if (m->kind < MG_MAP_IDENTITY || m->kind > MG_MAP_GRID)
    return set_error(MG_ERR_ARG, "unknown map kind %d", m->kind);
  if (m->kind == MG_MAP_GRID && (!m->xp || !m->yp))
    return set_error(MG_ERR_ARG, "MG_MAP_GRID needs xp and yp");
  (void)g;
  return MG_OK;
}

}  // namespace mg

namespace mg {
// A problem with its hierarchy allocated (zeroed) but no coefficients yet.
mg_status problem_create(mg_ctx* ctx, const mg_grid_desc* grid, const mg_solve_opts& o,
                         mg_problem** out) {
  *out = nullptr;
  if (o.coarse_op != MG_COARSE_GALERKIN && o.coarse_op != MG_COARSE_REDISCRETIZE)
    return set_error(MG_ERR_ARG, "bad coarse_op %d", o.coarse_op);
  cudaSetDevice(ctx->device);
  mg_problem* P = new mg_problem();
  P->ctx = ctx;
  P->grid = *grid;
  P->user = *grid;
  if (grid->neumann_y) {  // solved on the periodic grid of twice the height (even reflection)
    if (grid->periodic_y || grid->neumann_y != 1 || grid->ny < 3) {
      delete P;
      return set_error(MG_ERR_ARG, "neumann_y must be 0 or 1 and excludes periodic_y");
    }
    P->mirror = grid->ny - 1;
    P->grid.ny = 2 * (grid->ny - 1) + 1;
    P->grid.y0 = grid->y0 - grid->ly;
    P->grid.ly = 2.0 * grid->ly;
    P->grid.periodic_y = 1;
    P->grid.neumann_y = 0;
  }
  P->coarse_max = o.coarse_max;
  P->coarse_op = o.coarse_op;
  P->mixed = (o.precision == MG_PREC_MIXED);
  mg_status st = check_grid(&P->grid, o.coarse_max, &P->nlev, P->nxs, P->nys);
  if (!st) st = problem_alloc(P, P->mixed);
  if (!st && cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    st = set_error(MG_ERR_CUDA, "problem_create: %s", cudaGetErrorString(cudaGetLastError()));
  if (st) {
    char keep[512];
    snprintf(keep, sizeof keep, "%s", g_err);
    cudaStreamSynchronize(ctx->stream);
    problem_release(P);
    delete P;
    return set_error(st, "%s", keep);
  }
  {
    std::lock_guard<std::mutex> lk(ctx->problems_mu);
    ctx->problems.insert(P);
  }
  *out = P;
  return MG_OK;
}
}  // namespace mg

extern "C" mg_status mg_setup_transform(mg_ctx* ctx, const mg_grid_desc* grid,
                                        const mg_map_desc* map, const double* eps_phys,
                                        mg_mem_kind mem, const mg_solve_opts* opts,
                                        mg_problem** out) {
  if (!ctx || !grid || !out) return set_error(MG_ERR_ARG, "mg_setup_transform: NULL argument");
  *out = nullptr;
  mg_solve_opts o;
  if (opts) o = *opts; else mg_default_opts(&o);
  mg_status st = check_map(grid, map);
  if (st) return st;
  mg_problem* P = nullptr;
  st = problem_create(ctx, grid, o, &P);
  if (st) return st;
  st = problem_build(P, map, eps_phys, mem);
  if (st) {
    char keep[512];
    snprintf(keep, sizeof keep, "%s", g_err);
    cudaStreamSynchronize(ctx->stream);
    problem_release(P);
    delete P;
    return set_error(st, "%s", keep);
  }
  *out = P;
  return MG_OK;
}

extern "C" int mg_map_five_point(const mg_map_desc* map) { return map ? map_five_point(map) : 0; }

extern "C" int mg_problem_five_point(const mg_problem* P) { return P ? P->lev[0].A.five_point : -1; }

extern "C" mg_status mg_update_transform(mg_problem* P, const mg_map_desc* map,
                                         const double* eps_phys, mg_mem_kind mem) {
  if (!P) return set_error(MG_ERR_ARG, "mg_update_transform: problem is NULL");
  mg_status st = check_map(&P->user, map);
  if (st) return st;
  cudaSetDevice(P->ctx->device);
  return problem_build(P, map, eps_phys, mem);
}

extern "C" mg_status mg_batch_update_transform(mg_ctx* ctx, int count, mg_problem* const* probs,
                                               const mg_map_desc* maps, const double* const* eps_phys,
                                               mg_mem_kind mem, mg_status* statuses) {
  if (!ctx || count < 0 || (count > 0 && (!probs || !maps)))
    return set_error(MG_ERR_ARG, "mg_batch_update_transform: NULL argument");
  for (int k = 0; k < count; ++k) {
    if (!probs[k] || probs[k]->ctx != ctx)
      return set_error(MG_ERR_ARG, "mg_batch_update_transform: problem %d is NULL or from another context", k);
    mg_status st = check_map(&probs[k]->user, &maps[k]);
    if (st) return st;
  }
  if (count == 0) return MG_OK;
  cudaSetDevice(ctx->device);
  // fork: instance k builds on batch stream k mod kBatchStreams, after the work already
  // queued on the context stream; join back onto the context stream
  cudaEvent_t fork = nullptr, join[kBatchStreams] = {};
  mg_status st = MG_OK;
  auto cleanup = [&]() {
    if (fork) cudaEventDestroy(fork);
    for (auto& e : join)
      if (e) cudaEventDestroy(e);
  };
  if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(fork, ctx->stream) != cudaSuccess) {
    cleanup();
    return set_error(MG_ERR_CUDA, "mg_batch_update_transform: event setup failed");
  }
  const int ns = std::min(count, kBatchStreams);
  for (int b = 0; b < ns; ++b) {
    if (cudaEventCreateWithFlags(&join[b], cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamWaitEvent(ctx->batch[b], fork, 0) != cudaSuccess) {
      cleanup();
      return set_error(MG_ERR_CUDA, "mg_batch_update_transform: event setup failed");
    }
  }
  std::vector<mg_status> enq(count, MG_OK);
  for (int k = 0; k < count; ++k)
    enq[k] = problem_enqueue_build(probs[k], &maps[k], eps_phys ? eps_phys[k] : nullptr, mem,
                                   ctx->batch[k % kBatchStreams]);
  for (int b = 0; b < ns; ++b) {
    cudaEventRecord(join[b], ctx->batch[b]);
    cudaStreamWaitEvent(ctx->stream, join[b], 0);
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  cleanup();
  if (e != cudaSuccess) return set_error(MG_ERR_CUDA, "mg_batch_update_transform: %s", cudaGetErrorString(e));
  for (int k = 0; k < count; ++k) {
    mg_status sk = enq[k] ? enq[k] : problem_check_build(probs[k]);
    if (statuses) statuses[k] = sk;
    if (sk && !st) st = sk;
  }
  if (st) return set_error(st, "mg_batch_update_transform: at least one instance failed (first status %d)", (int)st);
  return MG_OK;
}

extern "C" void mg_problem_free(mg_problem* P) {
  if (!P) return;
  cudaSetDevice(P->ctx->device);
  cudaStreamSynchronize(P->ctx->stream);
  batch_cache_drop(P->ctx, P);  // captured batches that reference the problem's arrays
  {
    std::lock_guard<std::mutex> lk(P->ctx->problems_mu);
    P->ctx->problems.erase(P);
  }
  problem_release(P);
  delete P;
}

extern "C" mg_status mg_problem_info(const mg_problem* P, int* levels, int* nx_out, int* ny_out) {
  if (!P) return set_error(MG_ERR_ARG, "mg_problem_info: problem is NULL");
  if (levels) *levels = P->nlev;
  for (int l = 0; l < P->nlev; ++l) {
    if (nx_out) nx_out[l] = P->nxs[l];
    if (ny_out) ny_out[l] = P->nys[l];
  }
  return MG_OK;
}

// ------------------------------------------------------------------ solve graphs
namespace mg {

// Level table of the problem for one cycle in precision T; level 0 uses (x0, b0) and the
// level's scratch array as its ping-pong partner.
template <typename T>
static void level_table(mg_problem* P, T* x0, T* b0, VLevels<T>* V) {
  V->L = P->nlev;
  V->inv = P->inv;
  for (int l = 0; l < P->nlev; ++l) {
    LevelMem& M = P->lev[l];
    if constexpr (sizeof(T) == 4) {
      V->A[l] = M.A32;
      V->x[l] = M.x32;
      V->b[l] = M.b32;
      V->t[l] = M.t32;
    } else {
      V->A[l] = M.A;
      V->x[l] = M.x;
      V->b[l] = M.b;
      V->t[l] = M.t;
    }
  }
  V->x[0] = x0;
  V->b[0] = b0;
  V->err = P->flags + 2;
  V->pol = P->ctx->tuned ? &P->ctx->pol[sizeof(T) == 4 ? 1 : 0] : nullptr;
  if (P->line && (sizeof(T) == 4) == (P->mixed != 0))
    for (int l = 0; l < P->nlev - 1; ++l) V->lf[l] = line_level<T>(P, l);
}

template <typename T>
static mg_status emit_vcycle_on(mg_problem* P, T* x0, T* b0, const mg_solve_opts& o,
                                const int* skip, cudaStream_t s, T** result, bool x0_zero = false) {
  VLevels<T> V;
  level_table<T>(P, x0, b0, &V);
  CU(emit_vcycle<T>(V, o.smoother, o.nu1, o.nu2, o.omega_j, skip, s, result, x0_zero));
  return MG_OK;
}

// Body of one outer iteration.
static mg_status emit_body(mg_problem* P, const mg_solve_opts& o, cudaGraphConditionalHandle h,
                           int has_h, cudaStream_t s) {
  LevelMem& F = P->lev[0];
  const int* skip = &P->st->done;
  const size_t n0 = (size_t)F.A.pitch * rows_stored(F.A.ny, F.A.periodic);
  const bool mixed = (o.precision == MG_PREC_MIXED);
  mg_status st;
  if (o.outer == MG_OUTER_SOR) {  // single-level baseline: nu1 SOR sweeps per tested iteration
    CU(launch_resid_check(F.A, F.x, F.b, nullptr, P->st, P->part, h, has_h, s));
    CU(launch_sor<double>(F.A, F.x, F.b, o.nu1, o.omega_j, skip, s));
    CU(launch_iter_inc(P->st, s));
    return MG_OK;
  }
  if (o.outer == MG_OUTER_VCYCLE) {
    if (!mixed) {
      CU(launch_resid_check(F.A, F.x, F.b, nullptr, P->st, P->part, h, has_h, s));
      double* res = nullptr;
      if ((st = emit_vcycle_on<double>(P, F.x, F.b, o, skip, s, &res))) return st;
      if (res != F.x) CU(cudaMemcpyAsync(F.x, res, n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
      CU(launch_resid_check(F.A, F.x, F.b, P->r, P->st, P->part, h, has_h, s));
      CU(launch_r_to_f32(F.A, P->r, F.b32, F.A32.pitch, P->st, s));
      if (vcycle_reads_x0(o.smoother, o.nu1)) CU(cudaMemsetAsync(F.x32, 0, n0 * sizeof(float), s));
      float* res = nullptr;
      if ((st = emit_vcycle_on<float>(P, F.x32, F.b32, o, skip, s, &res, true))) return st;
      CU(launch_add_f32(F.A, F.x, res, F.A32.pitch, P->st, s));
    }
    CU(launch_iter_inc(P->st, s));
    return MG_OK;
  }
  // flexible CG preconditioned by one V-cycle; for the mixed path the cycle's right-hand
  // side r32 was written by the previous update (or the initialisation / verification)
  CU(launch_fcg_verify(F.A, F.x, F.b, P->r, mixed ? F.b32 : nullptr, F.A32.pitch, P->st, P->part, h,
                       has_h, s));
  if (!mixed) {
    if (vcycle_reads_x0(o.smoother, o.nu1)) CU(cudaMemsetAsync(P->z, 0, n0 * sizeof(double), s));
    double* res = nullptr;
    if ((st = emit_vcycle_on<double>(P, P->z, P->r, o, skip, s, &res, true))) return st;
    CU(launch_fcg_zq<double>(F.A, res, F.A.pitch, P->q, P->st, P->part, s));
    CU(launch_fcg_pq<double>(F.A, res, F.A.pitch, P->p, P->q, P->r, P->st, P->part, s));
  } else {
    if (vcycle_reads_x0(o.smoother, o.nu1)) CU(cudaMemsetAsync(F.x32, 0, n0 * sizeof(float), s));
    float* res = nullptr;
    if ((st = emit_vcycle_on<float>(P, F.x32, F.b32, o, skip, s, &res, true))) return st;
    CU(launch_fcg_zq<float>(F.A, res, F.A32.pitch, P->q, P->st, P->part, s));
    CU(launch_fcg_pq<float>(F.A, res, F.A32.pitch, P->p, P->q, P->r, P->st, P->part, s));
  }
  CU(launch_fcg_update(F.A, F.x, P->r, P->p, P->q, mixed ? F.b32 : nullptr, F.A32.pitch, P->st,
                       P->part, h, has_h, s));
  return MG_OK;
}

uint64_t graph_key(const mg_solve_opts& o) {
  uint64_t k = (uint64_t)o.precision | ((uint64_t)o.outer << 2) | ((uint64_t)o.smoother << 4) |
               ((uint64_t)(o.nu1 & 255) << 8) | ((uint64_t)(o.nu2 & 255) << 16);
  uint64_t w;
  float om = (float)o.omega_j;
  uint32_t ob;
  memcpy(&ob, &om, 4);
  w = ob;
  return k ^ (w << 24);
}

// One solve captured into the graph g that stream cs is capturing: init -> initial
// residual (sets the condition) -> WHILE(condition){ one outer iteration; the last kernel
// re-sets the condition } -> copy out.  `args` is the device argument block the kernels
// read; the loop body is captured on cs2.  Counts the kernel nodes it adds.
static mg_status capture_solve_chain(mg_problem* P, const mg_solve_opts& o, SolveArgs* args,
                                     cudaStream_t cs, cudaStream_t cs2, cudaGraph_t g,
                                     int* fixed_kernels, int* body_kernels) {
  LevelMem& F = P->lev[0];
  const bool fcg = (o.outer == MG_OUTER_FCG);
  const bool r32 = fcg && o.precision == MG_PREC_MIXED;
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaGraphConditionalHandle h = 0;
  if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess)
    return set_error(MG_ERR_CUDA, "conditional handle creation failed");
  if (launch_solve_init(F.A, args, P->D, F.x, F.b, P->st, cs) != cudaSuccess ||
      launch_resid_init(F.A, F.x, F.b, fcg ? P->r : nullptr, P->st, P->part, h, 1, cs) !=
          cudaSuccess ||
      (r32 && launch_r_to_f32(F.A, P->r, F.b32, F.A32.pitch, P->st, cs) != cudaSuccess))
    return set_error(MG_ERR_CUDA, "capture of solve init failed");
  *fixed_kernels = 3 + (r32 ? 1 : 0);
  if (cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps) != cudaSuccess)
    return set_error(MG_ERR_CUDA, "capture info failed");
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  if (cudaGraphAddNode(&cnode, g, deps, nullptr, ndeps, &cp) != cudaSuccess)
    return set_error(MG_ERR_CUDA, "adding the WHILE node failed");
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies) !=
      cudaSuccess)
    return set_error(MG_ERR_CUDA, "capture dependency update failed");
  if (cudaStreamBeginCaptureToGraph(cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
      cudaSuccess)
    return set_error(MG_ERR_CUDA, "body capture failed to start");
  mg_status st = emit_body(P, o, h, 1, cs2);
  if (!st && launch_loop_guard(P->st, h, cs2) != cudaSuccess)
    st = set_error(MG_ERR_CUDA, "capture of the loop guard failed");
  cudaGraph_t body_out = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs2, &body_out);
  if (!st && e2 != cudaSuccess)
    st = set_error(MG_ERR_CUDA, "body capture failed: %s", cudaGetErrorString(e2));
  if (st) return st;
  *body_kernels = 0;
  {
    size_t n = 0;
    cudaGraphGetNodes(body, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (n) cudaGraphGetNodes(body, nodes.data(), &n);
    for (size_t q = 0; q < n; ++q) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[q], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
        ++*body_kernels;
    }
  }
  if (launch_copy_out(F.A, F.x, args, cs) != cudaSuccess)
    return set_error(MG_ERR_CUDA, "capture of copy-out failed");
  *fixed_kernels += 1;
  return MG_OK;
}

static mg_status build_graph(mg_problem* P, const mg_solve_opts& o, GraphEntry* ge) {
  cudaStream_t cs = P->ctx->cap_stream, cs2 = P->ctx->cap_stream2;
  CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaGraph_t g = nullptr;
  cudaStreamCaptureStatus cst;
  mg_status st = MG_OK;
  int fixed = 0, body = 0;
  if (cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, nullptr, nullptr, nullptr) != cudaSuccess)
    st = set_error(MG_ERR_CUDA, "capture info failed");
  if (!st) st = capture_solve_chain(P, o, P->args, cs, cs2, g, &fixed, &body);
  cudaGraph_t gout = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &gout);
  if (st) {
    if (gout) cudaGraphDestroy(gout);
    cudaGetLastError();
    return st;
  }
  if (e != cudaSuccess) return set_error(MG_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
  ge->fixed_kernels = fixed;
  ge->body_kernels = body;
  cudaGraphExec_t ex;
  e = cudaGraphInstantiate(&ex, gout, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(gout);
    return set_error(MG_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  }
  ge->graph = gout;
  ge->exec = ex;
  return MG_OK;
}

// The whole batch as one graph: an empty root node, then for every instance its own
// solve chain as an independent branch (they run concurrently), then one kernel that
// gathers every instance's solve state and flags into contiguous arrays.
mg_status build_batch_graph(mg_ctx* ctx, mg_problem* const* probs, int count, const mg_solve_opts& o,
                            SolveArgs* d_args, SolveState* const* d_src, int* const* d_srcflags,
                            SolveState* d_states, int* d_flags, GraphEntry* ge,
                            std::vector<int>* fixed, std::vector<int>* body) {
  cudaStream_t cs = ctx->cap_stream, cs2 = ctx->cap_stream2;
  CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaGraph_t g = nullptr;
  cudaStreamCaptureStatus cst;
  mg_status st = MG_OK;
  std::vector<cudaGraphNode_t> leaves;
  fixed->assign(count, 0);
  body->assign(count, 0);
  do {
    if (cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, nullptr, nullptr, nullptr) != cudaSuccess) {
      st = set_error(MG_ERR_CUDA, "capture info failed");
      break;
    }
    cudaGraphNode_t root;
    cudaGraphNodeParams ep = {};
    ep.type = cudaGraphNodeTypeEmpty;
    if (cudaGraphAddNode(&root, g, nullptr, nullptr, 0, &ep) != cudaSuccess) {
      st = set_error(MG_ERR_CUDA, "adding the batch root node failed");
      break;
    }
    for (int k = 0; k < count && !st; ++k) {
      if (cudaStreamUpdateCaptureDependencies(cs, &root, nullptr, 1, cudaStreamSetCaptureDependencies) !=
          cudaSuccess) {
        st = set_error(MG_ERR_CUDA, "capture dependency update failed");
        break;
      }
      st = capture_solve_chain(probs[k], o, d_args + k, cs, cs2, g, &(*fixed)[k], &(*body)[k]);
      if (st) break;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      if (cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &nd) != cudaSuccess) {
        st = set_error(MG_ERR_CUDA, "capture info failed");
        break;
      }
      for (size_t q = 0; q < nd; ++q) leaves.push_back(deps[q]);
    }
    if (st) break;
    if (cudaStreamUpdateCaptureDependencies(cs, leaves.data(), nullptr, leaves.size(),
                                            cudaStreamSetCaptureDependencies) != cudaSuccess) {
      st = set_error(MG_ERR_CUDA, "capture join failed");
      break;
    }
    if (launch_gather_states(d_src, d_srcflags, d_states, d_flags, count, cs) != cudaSuccess) {
      st = set_error(MG_ERR_CUDA, "capture of the state gather failed");
      break;
    }
  } while (0);
  cudaGraph_t gout = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &gout);
  if (st) {
    if (gout) cudaGraphDestroy(gout);
    cudaGetLastError();
    return st;
  }
  if (e != cudaSuccess) return set_error(MG_ERR_CUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
  cudaGraphExec_t ex;
  e = cudaGraphInstantiate(&ex, gout, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(gout);
    return set_error(MG_ERR_CUDA, "batch graph instantiation failed: %s", cudaGetErrorString(e));
  }
  ge->graph = gout;
  ge->exec = ex;
  return MG_OK;
}

mg_status check_opts(const mg_problem* P, const mg_solve_opts& o) {
  if (o.precision != MG_PREC_FP64 && o.precision != MG_PREC_MIXED)
    return set_error(MG_ERR_ARG, "bad precision %d", o.precision);
  if ((o.precision == MG_PREC_MIXED) != (P->mixed != 0))
    return set_error(MG_ERR_ARG, "solve precision differs from the precision the problem was set up with");
  if (o.outer != MG_OUTER_VCYCLE && o.outer != MG_OUTER_FCG && o.outer != MG_OUTER_SOR)
    return set_error(MG_ERR_ARG, "bad outer iteration %d", o.outer);
  if (o.outer == MG_OUTER_SOR) {
    if (o.precision != MG_PREC_FP64) return set_error(MG_ERR_ARG, "the SOR iteration runs in FP64 only");
    if (o.nu1 < 1 || o.nu1 > 16) return set_error(MG_ERR_ARG, "SOR: nu1 (sweeps per iteration) must be 1..16");
    if (!(o.omega_j > 0.0 && o.omega_j < 2.0)) return set_error(MG_ERR_ARG, "SOR: omega_j must lie in (0, 2)");
    if (o.max_iters < 1 || !(o.rtol >= 0)) return set_error(MG_ERR_ARG, "bad rtol / max_iters");
    return MG_OK;
  }
  if (o.smoother != MG_SMOOTH_GS4 && o.smoother != MG_SMOOTH_JACOBI && o.smoother != MG_SMOOTH_XLINE)
    return set_error(MG_ERR_ARG, "bad smoother %d", o.smoother);
  if (o.smoother == MG_SMOOTH_XLINE &&
      !(P->mixed ? line_supported<float>(P->grid.nx) : line_supported<double>(P->grid.nx)))
    return set_error(MG_ERR_SIZE, "line smoother: rows of %d nodes exceed the line kernels' shared memory",
                     P->grid.nx);
  if (o.nu1 < 0 || o.nu2 < 0 || o.nu1 + o.nu2 == 0 || o.nu1 > 16 || o.nu2 > 16)
    return set_error(MG_ERR_ARG, "bad smoothing counts %d, %d", o.nu1, o.nu2);
  if (o.max_iters < 1 || !(o.rtol >= 0)) return set_error(MG_ERR_ARG, "bad rtol / max_iters");
  if (o.coarse_max != P->coarse_max)
    return set_error(MG_ERR_ARG, "coarse_max differs from the one the problem was set up with");
  if (o.coarse_op != P->coarse_op)
    return set_error(MG_ERR_ARG, "coarse_op differs from the one the problem was set up with");
  return MG_OK;
}

// Host-driven loop (MG_SOLVE_LOOP=host, read at every solve): the same kernels in the same
// order launched directly on the stream, with one stream synchronisation per outer
// iteration to read the convergence flag.  Used by per-kernel profilers, which do not
// support kernels inside graphs with conditional nodes.
static bool host_loop_mode() {
  const char* e = getenv("MG_SOLVE_LOOP");
  return e && strcmp(e, "host") == 0;
}

static mg_status run_host_loop(mg_problem* P, const mg_solve_opts& o, cudaStream_t s, int* passes) {
  LevelMem& F = P->lev[0];
  const bool fcg = (o.outer == MG_OUTER_FCG);
  CU(launch_solve_init(F.A, P->args, P->D, F.x, F.b, P->st, s));
  CU(launch_resid_init(F.A, F.x, F.b, fcg ? P->r : nullptr, P->st, P->part, 0, 0, s));
  if (fcg && o.precision == MG_PREC_MIXED)
    CU(launch_r_to_f32(F.A, P->r, F.b32, F.A32.pitch, P->st, s));
  *passes = 0;
  for (int pass = 0; pass < 2 * o.max_iters + 8; ++pass) {
    int done = 0;
    CU(cudaMemcpyAsync(&done, &P->st->done, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (done) break;
    mg_status st = emit_body(P, o, 0, 0, s);
    if (st) return st;
    ++*passes;
  }
  CU(launch_copy_out(F.A, F.x, P->args, s));
  return MG_OK;
}

// Enqueue one solve on stream s (inputs already device-resident at the given pointers).
mg_status enqueue_solve(mg_problem* P, const mg_solve_opts& o, const double* rho, const double* bc,
                        const double* phi_in, double* phi_out, cudaStream_t s) {
  const bool host_loop = host_loop_mode();
  if (o.smoother == MG_SMOOTH_XLINE) {
    mg_status lst = line_prepare(P, s);
    if (lst) return lst;
  }
  const uint64_t key = graph_key(o);
  auto it = P->graphs.find(key);
  if (it == P->graphs.end()) {  // also built in host-loop mode, for its kernel counts
    GraphEntry ge;
    mg_status st = build_graph(P, o, &ge);
    if (st) return st;
    it = P->graphs.emplace(key, ge).first;
  }
  SolveArgs* a = P->h_args;
  a->rho = rho;
  a->bc = bc;
  a->phi_in = phi_in;
  a->phi_out = phi_out;
  a->user_pitch = P->grid.nx;
  a->mirror = P->mirror;
  a->warm = o.warm_start ? 1 : 0;
  a->max_iters = o.max_iters;
  a->rtol = o.rtol;
  a->n_unknowns = (long long)coarse_unknowns(P->grid.nx, P->grid.ny, P->grid.periodic_y);
  CU(cudaMemcpyAsync(P->args, a, sizeof(SolveArgs), cudaMemcpyHostToDevice, s));
  CU(cudaEventRecord(P->ev0, s));
  if (host_loop) {
    int passes = 0;
    mg_status st = run_host_loop(P, o, s, &passes);
    if (st) return st;
    // the graph's loop body also holds the loop guard, which the host loop replaces
    P->last_fixed_kernels = it->second.fixed_kernels + passes * (it->second.body_kernels - 1);
    P->last_body_kernels = 0;
  } else {
    CU(cudaGraphLaunch(it->second.exec, s));
    P->last_fixed_kernels = it->second.fixed_kernels;
    P->last_body_kernels = it->second.body_kernels;
  }
  CU(cudaEventRecord(P->ev1, s));
  CU(cudaMemcpyAsync(P->h_state, P->st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(P->h_flags, P->flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
  return MG_OK;
}

mg_status finish_solve(mg_problem* P, mg_solve_stats* stats) {
  return finish_from(P, *P->h_state, P->h_flags, stats, -1.0);
}

// Stats and status of a finished solve from its copied-back state; solve_ms < 0: time it
// from the problem's own events.
mg_status finish_from(mg_problem* P, const SolveState& S, const int* flags, mg_solve_stats* stats,
                      double solve_ms) {
  if (flags[2]) return set_error(MG_ERR_TIMEOUT, "a bounded wait inside a smoothing kernel gave up");
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->iters = S.it;
    stats->levels = P->nlev;
    stats->rel_residual = S.rel;
    stats->setup_ms = P->setup_ms;
    if (solve_ms < 0) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, P->ev0, P->ev1);
      stats->solve_ms = ms;
    } else {
      stats->solve_ms = solve_ms;
    }
    const int n = std::min(S.hist_n, MG_HIST_MAX);
    for (int k = 0; k < n; ++k) stats->hist[k] = S.hist[k];
    stats->kernel_launches = P->last_fixed_kernels + S.guard * P->last_body_kernels;
    stats->setup_kernel_launches = P->setup_kernels;
  }
  if (S.status == 7) return set_error(MG_ERR_DIVERGED, "solve diverged (NaN/Inf residual)");
  if (S.status == 6)
    return set_error(MG_ERR_NOT_CONVERGED, "not converged after %d iterations (rel %.3e)", S.it, S.rel);
  return MG_OK;
}

}  // namespace mg

extern "C" mg_status mg_cycle_time(mg_problem* P, const mg_solve_opts* opts, int reps, double* ms_per_cycle) {
  if (!P || !ms_per_cycle || reps < 1) return set_error(MG_ERR_ARG, "mg_cycle_time: bad argument");
  mg_solve_opts o;
  if (opts) o = *opts; else mg_default_opts(&o);
  mg_status st = check_opts(P, o);
  if (st) return st;
  if (o.outer == MG_OUTER_SOR) return set_error(MG_ERR_ARG, "mg_cycle_time: the SOR iteration has no cycle");
  cudaSetDevice(P->ctx->device);
  cudaStream_t s = P->ctx->stream, cs = P->ctx->cap_stream;
  if (o.smoother == MG_SMOOTH_XLINE && (st = line_prepare(P, s))) return st;
  CU(cudaStreamSynchronize(s));
  // one cycle as the solves run it (same levels, kernels and smoother policy), captured once;
  // it reads the level-0 right-hand side and writes only cycle scratch arrays
  LevelMem& F = P->lev[0];
  CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  if (P->mixed) {
    float* res = nullptr;
    st = emit_vcycle_on<float>(P, F.x32, F.b32, o, nullptr, cs, &res, true);
  } else {
    double* res = nullptr;
    st = emit_vcycle_on<double>(P, P->z, P->r, o, nullptr, cs, &res, true);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  if (st || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st ? st : set_error(MG_ERR_CUDA, "mg_cycle_time: capture failed: %s", cudaGetErrorString(e));
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return set_error(MG_ERR_CUDA, "mg_cycle_time: %s", cudaGetErrorString(e));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = cudaGraphLaunch(ex, s);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(ex, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGraphExecDestroy(ex);
  if (e != cudaSuccess) return set_error(MG_ERR_CUDA, "mg_cycle_time: %s", cudaGetErrorString(e));
  *ms_per_cycle = ms / reps;
  return MG_OK;
}

// Device address of a page-locked (cudaHostAlloc / cudaHostRegister) host array, through
// which kernels read and write it over the host link; nullptr for pageable memory.
static double* pinned_view(const double* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // an unknown pointer leaves a (non-sticky) error: clear it
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? static_cast<double*>(a.devicePointer) : nullptr;
}

extern "C" mg_status mg_solve(mg_problem* P, const double* rho_phys, const double* bc, double* phi,
                              mg_mem_kind mem, const mg_solve_opts* opts, mg_solve_stats* stats) {
  if (!P || !rho_phys || !phi) return set_error(MG_ERR_ARG, "mg_solve: NULL argument");
  mg_solve_opts o;
  if (opts) o = *opts; else mg_default_opts(&o);
  mg_status st = check_opts(P, o);
  if (st) return st;
  cudaSetDevice(P->ctx->device);
  cudaStream_t s = P->ctx->stream;
  const size_t n = (size_t)P->user.nx * rows_stored(P->user.ny, P->user.periodic_y);
  const double *rho = rho_phys, *bcd = bc, *pin = phi;
  double* pout = phi;
  bool staged = false;
  if (mem == MG_MEM_HOST) {
    // page-locked arrays: the solve's first kernel reads rho, bc (and a warm start) and its
    // last kernel writes phi in place over the host link, each once, instead of a copy to and
    // from staging arrays around the solve
    double* rv = pinned_view(rho_phys);
    double* bv = bc ? pinned_view(bc) : nullptr;
    double* pv = pinned_view(phi);
    if (rv && (!bc || bv) && pv) {
      rho = rv;
      bcd = bv;
      pin = pout = pv;
      mem = MG_MEM_DEVICE;
    }
  }
  if (mem == MG_MEM_HOST) {
    staged = true;
    if (!P->stage) {
      P->stage = palloc<double>(P, 3 * n);
      if (!P->stage) return set_error(MG_ERR_OOM, "device memory budget exhausted (staging)");
    }
    CU(cudaMemcpyAsync(P->stage, rho_phys, n * sizeof(double), cudaMemcpyHostToDevice, s));
    if (bc) CU(cudaMemcpyAsync(P->stage + n, bc, n * sizeof(double), cudaMemcpyHostToDevice, s));
    if (o.warm_start)
      CU(cudaMemcpyAsync(P->stage + 2 * n, phi, n * sizeof(double), cudaMemcpyHostToDevice, s));
    rho = P->stage;
    bcd = bc ? P->stage + n : nullptr;
    pin = P->stage + 2 * n;
    pout = P->stage + 2 * n;
  } else if (mem != MG_MEM_DEVICE) {
    return set_error(MG_ERR_ARG, "bad memory kind");
  }
  st = enqueue_solve(P, o, rho, bcd, pin, pout, s);
  if (st) return st;
  if (staged) CU(cudaMemcpyAsync(phi, pout, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return finish_solve(P, stats);
}

extern "C" mg_status mg_batch_solve(mg_ctx* ctx, int count, mg_problem* const* probs,
                                    const double* const* rho, const double* const* bc,
                                    double* const* phi, mg_mem_kind mem, const mg_solve_opts* opts,
                                    mg_solve_stats* stats) {
  if (!ctx || count < 0 || (count && (!probs || !rho || !phi)))
    return set_error(MG_ERR_ARG, "mg_batch_solve: NULL argument");
  mg_solve_opts o;
  if (opts) o = *opts; else mg_default_opts(&o);
  if (mem != MG_MEM_DEVICE && mem != MG_MEM_HOST) return set_error(MG_ERR_ARG, "bad memory kind");
  cudaSetDevice(ctx->device);
  return batch_solve_impl(ctx, count, probs, rho, bc, phi, mem, o, stats);
}
