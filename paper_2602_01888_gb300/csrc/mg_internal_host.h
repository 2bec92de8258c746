// Host-side structures of libmg (context, pool, problem) shared by its C++ sources.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <map>
#include <set>
#include <string>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "mg.h"
#include "mg_launch.h"
#include "mg_solve_kernels.h"
#include "mg_vcycle.h"

namespace mg {

constexpr int kMaxLevels = 24;
constexpr int kBatchStreams = 8;

mg_status set_error(mg_status s, const char* fmt, ...);

// Device memory pool: slabs from cudaMalloc, best-fit sub-allocation with coalescing.
class Pool {
 public:
  void* alloc(size_t n);
  void release(void* p);
  size_t used() const { return used_; }
  size_t budget() {
    std::lock_guard<std::mutex> lk(mu_);
    return budget_;
  }
  void set_budget(size_t b) {
    std::lock_guard<std::mutex> lk(mu_);
    budget_ = b;
  }
  ~Pool();
  size_t budget_ = 0;
  bool pinned_ = false;  // slabs of page-locked host memory instead of device memory

 private:
  struct Slab {
    char* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> length
  };
  std::vector<Slab> slabs_;
  std::unordered_map<void*, std::pair<int, size_t>> live_;
  size_t reserved_ = 0, used_ = 0;
  size_t slab_min_ = (size_t)64 << 20;
  std::mutex mu_;
};

struct LevelMem {
  OpF64 A{};
  double *x = nullptr, *b = nullptr, *t = nullptr;
  OpF32 A32{};
  float *x32 = nullptr, *b32 = nullptr, *t32 = nullptr;
};

struct GraphEntry {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int fixed_kernels = 0;  // kernel nodes outside the loop
  int body_kernels = 0;   // kernel nodes of one loop pass
};

}  // namespace mg

namespace mg {
// A captured batch: the graph over a fixed list of problems and its argument / state arrays.
struct BatchEntry {
  std::vector<mg_problem*> probs;
  GraphEntry ge;
  std::vector<int> fixed, body;  // kernel nodes per instance outside / inside its loop
  SolveArgs* d_args = nullptr;
  SolveArgs* h_args = nullptr;
  SolveState* d_states = nullptr;
  SolveState* h_states = nullptr;
  int* d_flags = nullptr;
  int* h_flags = nullptr;
  SolveState** d_src = nullptr;
  int** d_srcflags = nullptr;
  std::vector<void*> allocs;
};
}  // namespace mg

struct mg_ctx {
  int device = 0;
  mg::Pool pool;
  std::set<mg_problem*> problems;  // live problems, freed by mg_destroy if still there
  std::mutex problems_mu;          // the server's scheduler thread creates problems too
  std::map<std::string, mg::BatchEntry*> batches;
  std::mutex batches_mu;  // batches: the server's scheduler thread frees problems too
  cudaStream_t stream = nullptr, own_stream = nullptr, cap_stream = nullptr, cap_stream2 = nullptr;
  cudaStream_t batch[mg::kBatchStreams] = {};
  mg::SmoothPolicy pol[2];  // measured smoother choice: [0] FP64, [1] FP32 (mg_autotune)
  int tuned = 0;
};

struct mg_problem {
  mg_ctx* ctx = nullptr;
  mg_grid_desc grid{};  // the grid the hierarchy is built on (the doubled periodic grid for Neumann sides)
  mg_grid_desc user{};  // the caller's grid (its arrays' layout)
  int mirror = 0;       // Neumann sides: ny - 1 of the caller's grid, else 0
  int nlev = 0, coarse_max = 64, mixed = 0;
  int coarse_op = 0;  // mg_coarse_op of the set-up
  int nxs[mg::kMaxLevels] = {}, nys[mg::kMaxLevels] = {};
  mg::LevelMem lev[mg::kMaxLevels];
  double *D = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  double* inv = nullptr;
  int m = 0;
  double* part = nullptr;
  mg::SolveState* st = nullptr;
  mg::SolveArgs* args = nullptr;
  int* flags = nullptr;
  double* stage = nullptr;  // device copies of host inputs/outputs (3 node arrays)
  void* line = nullptr;     // line-smoother factors of levels 0 .. nlev-2 (cycle precision)
  mg::SolveArgs* h_args = nullptr;
  mg::SolveState* h_state = nullptr;
  int* h_flags = nullptr;  // folded, coarse status, kernel wait timeout
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;    // around the last solve
  cudaEvent_t evb0 = nullptr, evb1 = nullptr;  // around the last coefficient build
  double setup_ms = 0.0;
  int setup_kernels = 0;
  int last_fixed_kernels = 0, last_body_kernels = 0;
  std::map<uint64_t, mg::GraphEntry> graphs;
  std::vector<void*> allocs;
};

namespace mg {
mg_status problem_create(mg_ctx* ctx, const mg_grid_desc* grid, const mg_solve_opts& o,
                         mg_problem** out);
mg_status check_map(const mg_grid_desc* g, const mg_map_desc* m);
// Work enqueued between the assembly of the finest operator and its coarsening.  It may zero
// couplings; if it makes a NE / NW coupling nonzero it must clear lev[0]'s five_point.
using FineHook = std::function<mg_status(mg_problem*, cudaStream_t)>;
mg_status problem_enqueue_build(mg_problem* P, const mg_map_desc* map, const double* eps_phys,
                                mg_mem_kind mem, cudaStream_t s, const FineHook* hook = nullptr);
mg_status problem_check_build(mg_problem* P);
mg_status enqueue_solve(mg_problem* P, const mg_solve_opts& o, const double* rho, const double* bc,
                        const double* phi_in, double* phi_out, cudaStream_t s);
mg_status finish_solve(mg_problem* P, mg_solve_stats* stats);
mg_status finish_from(mg_problem* P, const SolveState& S, const int* flags, mg_solve_stats* stats,
                      double solve_ms);
mg_status build_batch_graph(mg_ctx* ctx, mg_problem* const* probs, int count, const mg_solve_opts& o,
                            SolveArgs* d_args, SolveState* const* d_src, int* const* d_srcflags,
                            SolveState* d_states, int* d_flags, GraphEntry* ge,
                            std::vector<int>* fixed, std::vector<int>* body);
void batch_cache_clear(mg_ctx* ctx);
// Drop the captured batches that contain problem P (its arrays are about to be freed).
void batch_cache_drop(mg_ctx* ctx, const mg_problem* P);
uint64_t graph_key(const mg_solve_opts& o);
mg_status check_opts(const mg_problem* P, const mg_solve_opts& o);
// Allocate and compute the line-smoother factors on stream s if the problem has none yet.
mg_status line_prepare(mg_problem* P, cudaStream_t s);
mg_status batch_solve_impl(mg_ctx* ctx, int count, mg_problem* const* probs,
                           const double* const* rho, const double* const* bc, double* const* phi,
                           mg_mem_kind mem, const mg_solve_opts& o, mg_solve_stats* stats);
}  // namespace mg
