/*
 * mg.h - C ABI of the GB300 transformed-coefficient geometric multigrid library.
 *
 * The library solves the generalized Poisson equation of Gautam & Paradkar,
 * "Multigrid Poisson Solver for Complex Geometries Using Finite Difference Method":
 * a coordinate map x -> x' (Eq. 1) turns Poisson's equation on a complex physical
 * domain into
 *
 *     -div( eps(x, y) grad phi ) = rho          (Eq. 7 with E = -grad phi, Eqs. 16-17)
 *
 * on a uniform computational grid, with the symmetric 2x2 tensor
 * eps = det(J) J^-1 eps' J^-T (Eq. 10, components Eqs. 12-15) and rho = rho' det(J)
 * (Eq. 11).  The discrete operator is the symmetric conservative 9-point form of
 * the paper's Eq. 18 stencil; it is solved by geometric multigrid V-cycles
 * (Sec. 3, Eqs. 19-24), optionally accelerated by flexible conjugate gradients and
 * optionally with an FP32 cycle inside FP64 iterative refinement.  phi on the
 * computational nodes is phi' on the mapped nodes (Eq. 6).
 *
 * Conventions for every entry point:
 *  - Node (i, j): i = 0..nx-1 along x, j along y.  Caller arrays are row-major and
 *    contiguous, a[i + nx * j], with nyr rows: nyr = ny - 1 for a grid periodic in y
 *    (row ny-1 coincides with row 0), nyr = ny otherwise.
 *  - The caller owns every array it passes; the library copies inputs in and writes
 *    outputs into the caller's buffers before the call returns (solver entry points)
 *    or in stream order (mgk_* kernel entry points).
 *  - Opaque handles are owned by the library and released by their _free / _destroy
 *    / _stop call.
 *  - Every call returns an mg_status and never aborts; mg_last_error() gives a
 *    thread-local message for the last failing call on the calling thread.
 *  - A context is used by one host thread at a time (or under external locking);
 *    the server is internally synchronized.  While a server runs on a context, use the
 *    context only through the mg_serve_* calls: the scheduler thread creates, runs and
 *    frees problems on it.
 *  - Sizes: nx, ny >= 3 and each of nx-1, ny-1 must be m * 2^k with m <= 32 so the
 *    multigrid hierarchy is exact; anything else is MG_ERR_SIZE.
 */
#ifndef MG_H_
#define MG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MG_OK = 0,
  MG_ERR_ARG = 1,            /* null pointer, bad enum, inconsistent descriptor */
  MG_ERR_SIZE = 2,           /* grid not of the form m * 2^k + 1, too small or too large */
  MG_ERR_OOM = 3,            /* device memory budget of the context exhausted */
  MG_ERR_CUDA = 4,           /* a CUDA runtime call failed (message has the CUDA error) */
  MG_ERR_MAP_FOLDED = 5,     /* det J <= 0 at some node (Eq. 10 needs det J > 0) */
  MG_ERR_NOT_CONVERGED = 6,  /* max iterations reached; best iterate and stats written */
  MG_ERR_DIVERGED = 7,       /* NaN/Inf or growth of the residual */
  MG_ERR_TIMEOUT = 8,        /* a bounded wait expired (device task wait or serve poll) */
  MG_ERR_BUSY = 9,           /* server queue full */
  MG_ERR_NOT_FOUND = 10,     /* unknown ticket */
  MG_ERR_NOT_SPD = 11        /* coarsest-level factorization met a non-positive pivot */
} mg_status;

typedef enum { MG_MEM_HOST = 0, MG_MEM_DEVICE = 1 } mg_mem_kind;

typedef enum {
  MG_MAP_IDENTITY = 0,  /* x' = x, y' = y */
  MG_MAP_SINE_WARP = 1, /* x' = x + a sin(pi x) sin(pi y), y' = y + a sin(2 pi x) sin(pi y); params {a} */
  MG_MAP_POLAR = 2,     /* x' = x cos y, y' = x sin y (Eq. 29) */
  MG_MAP_SINH = 3,      /* x' = s sinh(alpha x), y' = s sinh(alpha y) (Eq. 52); params {s, alpha} */
  MG_MAP_AFFINE = 4,    /* x' = a11 x + a12 y, y' = a21 x + a22 y; params {a11, a12, a21, a22} */
  MG_MAP_GRID = 5       /* mapped node coordinates given (xp, yp); Jacobian by Eqs. 39-42 */
} mg_map_kind;

typedef enum { MG_PREC_FP64 = 0, MG_PREC_MIXED = 1 } mg_precision;
/* Outer iteration: plain V-cycles, flexible CG preconditioned by one V-cycle, or - as the
 * single-level baseline the paper compares multigrid against (Sec. 4) - four-colour SOR on the
 * finest operator: each iteration is nu1 sweeps (1..16) with factor omega_j (0 < omega_j < 2;
 * the paper uses 1.875), the residual tested before each iteration; FP64 only, no cycle. */
typedef enum { MG_OUTER_VCYCLE = 0, MG_OUTER_FCG = 1, MG_OUTER_SOR = 2 } mg_outer;
/* Smoother: four-colour point Gauss-Seidel (the paper's smoother in parallel order),
 * weighted Jacobi, or zebra x-line Gauss-Seidel (rows of one parity solved as tridiagonal
 * systems; for operators dominated by the x coupling, e.g. the annulus of Eq. 29).  The line
 * smoother runs on every level but the coarsest; it needs nx <= 8194 in FP64 and 16386 in the
 * mixed precision, and factors the row systems once per coefficient build. */
typedef enum { MG_SMOOTH_GS4 = 0, MG_SMOOTH_JACOBI = 1, MG_SMOOTH_XLINE = 2 } mg_smoother;

/* Uniform computational grid: nx x ny vertices on [x0, x0+lx] x [y0, y0+ly]; hx = lx/(nx-1),
 * hy = ly/(ny-1).  x sides are Dirichlet; y sides Dirichlet or periodic. */
typedef struct {
  int nx, ny;
  double x0, y0, lx, ly;
  int periodic_y;
  /* 1: homogeneous Neumann condition on the two y sides (zero normal derivative, Eq. 28); their
   * nodes are unknowns, the x sides stay Dirichlet, periodic_y must be 0.  Caller arrays keep
   * the nx x ny layout.  Solved as the periodic problem of twice the height whose coefficients,
   * charge and data are the even reflection of these (eps_xy odd, so set to 0 on the two
   * Neumann rows): exact for grids that meet the Neumann sides orthogonally, twice the
   * unknowns and memory of the grid.  Not for mg_harmonic_grid. */
  int neumann_y;
} mg_grid_desc;

/* Coordinate map (Eq. 1).  For MG_MAP_GRID, xp and yp hold the mapped coordinates of
 * every stored node (caller layout, memory kind of the call); for a periodic-y grid,
 * (jump_x, jump_y) is added to (x', y') when row nyr-1 wraps to row 0 (0 for a closed map). */
typedef struct {
  int kind;
  double params[4];
  const double *xp, *yp;
  double jump_x, jump_y;
} mg_map_desc;

/* Coarse operators (Sec. 3 names A_H only): the Galerkin product R A P (default, 9-point
 * on every coarse level), or the fine assembly (Eqs. 12-18 in the conservative form) applied
 * on each coarse grid to the tensor coarsened from the level above: full weighting at coarse
 * unknowns, injection on the boundary ring.  A rediscretized hierarchy of a map without cross
 * term stays 5-point on every level. */
typedef enum { MG_COARSE_GALERKIN = 0, MG_COARSE_REDISCRETIZE = 1 } mg_coarse_op;

typedef struct {
  int precision;      /* mg_precision */
  int outer;          /* mg_outer: plain V-cycles, or flexible CG preconditioned by one V-cycle */
  int smoother;       /* mg_smoother */
  int nu1, nu2;       /* pre / post smoothing sweeps */
  double omega_j;     /* weighted-Jacobi factor; the SOR factor for MG_OUTER_SOR */
  double rtol;        /* stop when ||r||_2 / ||r_0||_2 <= rtol (r_0: residual of zero unknowns) */
  int max_iters;      /* cycles (VCYCLE), CG iterations (FCG) or SOR iterations of nu1 sweeps (SOR) */
  int coarse_max;     /* coarsest level: first level with at most this many unknowns (<= 256) */
  int warm_start;     /* 1: phi holds the initial guess of the unknowns */
  int coarse_op;      /* mg_coarse_op: how the coarse operators are built (fixed at set-up) */
} mg_solve_opts;

#define MG_HIST_MAX 256

typedef struct {
  int iters;              /* cycles or CG iterations run */
  int levels;             /* multigrid levels */
  double rel_residual;    /* final ||r|| / ||r_0|| (FP64) */
  double setup_ms;        /* coefficient build + coarsening of the problem */
  double solve_ms;        /* device time of the solve */
  double hist[MG_HIST_MAX]; /* relative residual before each iteration (iters + 1 entries) */
  int kernel_launches;    /* kernels the solve launched on the device */
  int setup_kernel_launches; /* kernels of the last coefficient build / coarsening */
} mg_solve_stats;

typedef struct mg_ctx mg_ctx;
typedef struct mg_problem mg_problem;

/* Thread-local message of the last failing call ("" if none). */
const char *mg_last_error(void);

/* Default options: FP64, flexible CG, four-colour Gauss-Seidel V(2,2), omega_j 0.8,
 * rtol 1e-10, 200 iterations, coarse_max 64, cold start. */
void mg_default_opts(mg_solve_opts *opts);

/* Create a context on CUDA device `device` with a device-memory budget (bytes, 0 = 90% of
 * free memory).  The context owns a memory pool and a stream (replace with mg_set_stream). */
mg_status mg_create(int device, size_t mem_budget_bytes, mg_ctx **out);
/* Waits for the device, then frees every problem of the context that is still alive and
 * the context itself; handles of those problems must not be used afterwards. */
void mg_destroy(mg_ctx *ctx);
/* Run all later work of the context on `stream` (a cudaStream_t; NULL = the context's own). */
mg_status mg_set_stream(mg_ctx *ctx, void *stream);
/* Bytes of the pool currently in use / the budget. */
mg_status mg_mem_info(mg_ctx *ctx, size_t *used, size_t *budget);

/*
 * Build a resident problem: Jacobian of the map (analytic, or Eqs. 39-42 on the mapped
 * grid), tensor eps (Eqs. 10, 12-15) times the scalar eps' (eps_phys, NULL = 1, Eq. 10
 * with eps' = s I), fine-level 9-point operator, Galerkin coarse operators on every level
 * and the coarsest-level inverse.  opts->precision fixes the precision of the hierarchy:
 * MG_PREC_FP64 builds FP64 Galerkin operators; MG_PREC_MIXED keeps the finest operator in
 * FP64 (for the outer residual) and builds the cycle's hierarchy in FP32 (Galerkin
 * products in FP32, coarsest inverse in FP64).  Later solves must use the same precision.
 * opts may be NULL for the defaults.
 * Errors: MG_ERR_SIZE, MG_ERR_ARG, MG_ERR_OOM, MG_ERR_MAP_FOLDED, MG_ERR_NOT_SPD, MG_ERR_CUDA.
 */
mg_status mg_setup_transform(mg_ctx *ctx, const mg_grid_desc *grid, const mg_map_desc *map,
                             const double *eps_phys, mg_mem_kind mem, const mg_solve_opts *opts,
                             mg_problem **out);
/* Recompute the coefficients of an existing problem in place for a new map / eps' on the
 * same grid (no allocation).  Same errors as mg_setup_transform. */
mg_status mg_update_transform(mg_problem *prob, const mg_map_desc *map, const double *eps_phys,
                              mg_mem_kind mem);
/*
 * mg_update_transform for `count` problems of one context with a single synchronisation:
 * the coefficient builds of different problems run concurrently on the context's batch
 * streams.  maps / eps_phys (nullable array; its entries nullable) are indexed like probs;
 * every array has the memory kind `mem`.  statuses (nullable, count entries) receives each
 * instance's outcome (MG_OK, MG_ERR_MAP_FOLDED, MG_ERR_NOT_SPD, ...); the return value is
 * MG_OK or the first failing instance's status.  Argument errors (NULL problem, a problem of
 * another context, a map that does not fit its grid) are detected before any work starts.
 * This entry point has no counterpart in the paper: it batches the per-problem setup.
 */
mg_status mg_batch_update_transform(mg_ctx *ctx, int count, mg_problem *const *probs,
                                    const mg_map_desc *maps, const double *const *eps_phys,
                                    mg_mem_kind mem, mg_status *statuses);
void mg_problem_free(mg_problem *prob);
/* Levels and per-level sizes (nx_out/ny_out: arrays of at least 24 ints, nullable). */
mg_status mg_problem_info(const mg_problem *prob, int *levels, int *nx_out, int *ny_out);
/*
 * 1 if the map's transformed tensor has no cross term, exactly: eps_xy (Eq. 13) is zero at
 * every node as computed, because J^T J is diagonal with a zero product in Eq. 13 (the
 * identity, the polar map of Eq. 29, the sinh stretching of Eq. 52, an affine map with
 * params[1] = params[2] = 0).  The finest operator of such a map is a 5-point stencil, and
 * the solver runs the 5-point forms of its finest-level kernels (which skip the zero NE / NW
 * couplings; results identical to the 9-point forms).  0 otherwise or for NULL.
 */
int mg_map_five_point(const mg_map_desc *map);
/* Whether the problem's current finest operator is handled as a 5-point stencil (the map of
 * its last coefficient build passed mg_map_five_point): 1 / 0, -1 for NULL. */
int mg_problem_five_point(const mg_problem *prob);

/*
 * Solve for phi.  rho_phys: rho' at every node (only unknowns are used; rho = rho' det J,
 * Eq. 11).  bc: node array whose Dirichlet-side values are the boundary data (NULL = 0).
 * phi: out = solution at every node (Dirichlet sides = bc); in = initial guess of the
 * unknowns when opts->warm_start.  All three arrays have the memory kind `mem`.  Host arrays
 * that are all page-locked (cudaHostAlloc, cudaHostRegister) are read and written in place by
 * the solve's first and last kernels over the host link; otherwise they are copied through
 * device staging arrays.  Either way the call returns once phi is written.
 * Errors: MG_ERR_NOT_CONVERGED (phi and stats still written), MG_ERR_DIVERGED, MG_ERR_ARG,
 * MG_ERR_CUDA.
 */
/* Device time of one multigrid cycle of a resident problem as its solves with `opts` run it
 * (the same levels, kernels and smoother choice; FP32 cycle for a mixed problem), captured once
 * and replayed `reps` times after two warm-up replays on the context's stream; *ms_per_cycle
 * receives the mean.  Benchmarking aid (project addition): the cycle reads the level-0
 * right-hand side left by the last solve and writes only the cycle's scratch arrays. */
mg_status mg_cycle_time(mg_problem *prob, const mg_solve_opts *opts, int reps, double *ms_per_cycle);

mg_status mg_solve(mg_problem *prob, const double *rho_phys, const double *bc, double *phi,
                   mg_mem_kind mem, const mg_solve_opts *opts, mg_solve_stats *stats);

/*
 * Solve `count` independent problems (different sizes and geometries allowed) in one
 * batched execution.  Arrays are indexed like probs; stats has count entries (nullable).
 * Each result equals that of mg_solve on the same problem and options (bitwise).
 */
mg_status mg_batch_solve(mg_ctx *ctx, int count, mg_problem *const *probs,
                         const double *const *rho_phys, const double *const *bc,
                         double *const *phi, mg_mem_kind mem, const mg_solve_opts *opts,
                         mg_solve_stats *stats);

/*
 * Numerical grid generation (Sec. 4.2, Eqs. 36-37): discrete-harmonic physical coordinates
 * x'(x, y), y'(x, y) on the computational grid `grid`, with Dirichlet data on the outer
 * boundary ring and at the interior nodes where fixed[] != 0 (for instance the ring of an
 * immersed body carrying the Eq. 44 boundary map).  fixed (1 byte per node), xp, yp (node
 * arrays, row-major, i fastest) have the memory kind `mem`; xp/yp hold the Dirichlet data at
 * the outer ring and at fixed nodes and the initial guess elsewhere.  xp_out / yp_out
 * (caller-owned, same kind) receive the solution at every node.  The 5-point Laplacian is
 * solved to the relative residual rtol by the library's FP64 multigrid-preconditioned CG,
 * with every coupling to a fixed interior node moved to the right-hand side.  stats
 * (nullable) receives 2 entries (x', y').  Errors: MG_ERR_ARG, MG_ERR_SIZE, MG_ERR_OOM,
 * MG_ERR_NOT_CONVERGED, MG_ERR_CUDA.
 */
mg_status mg_harmonic_grid(mg_ctx *ctx, const mg_grid_desc *grid, const unsigned char *fixed,
                           const double *xp, const double *yp, double *xp_out, double *yp_out,
                           mg_mem_kind mem, double rtol, mg_solve_stats *stats);

/*
 * Autotuner of the smoother per level size (project addition; the paper has a single
 * sequential smoother).  For square levels of sides 33, 65, ..., up to max_side, in FP64 and
 * FP32, it times two Gauss-Seidel sweeps (Sec. 2.1) with each kernel family that can run at
 * that size -- per-colour kernels, fused shared-memory tiles, pipelined tiles, row marching
 * -- in each of the family's variants (tile shapes 32x32, 64x16, 64x24 and one or two
 * sweeps per launch for the tile kernels, where shared memory allows; one or two sweeps per
 * pass for row marching), on a sine-warp operator built by the library, and records the
 * fastest.  Every solve graph captured on the context afterwards takes, at each level, the
 * choice of the tuned size nearest in node count (all variants compute the same values, so
 * results do not change); graphs captured before are dropped.  Call it when no solve or
 * server is running on the context.  report (nullable) receives per (precision, side) the
 * best time in ms of each family in the order colour, fused, pipelined, marching (-1: cannot
 * run), the choice (1-4 in that order) and the chosen variant's tile (tile_x x tile_y owned
 * nodes; marching: tile_x owned columns of a strip, tile_y 0; per-colour: 0 x 0) and sweeps
 * per launch.
 */
#define MG_TUNE_MAX 32
typedef struct {
  int precision; /* MG_PREC_FP64 or MG_PREC_MIXED (the FP32 cycle) */
  int side;
  float ms[4];
  int choice;
  int tile_x, tile_y, sweeps_per_launch;
} mg_tune_entry;
typedef struct {
  int count;
  mg_tune_entry entry[MG_TUNE_MAX];
} mg_tune_report;
mg_status mg_autotune(mg_ctx *ctx, int max_side, mg_tune_report *report);

/* ------------------------------------------------------------------ serving */
typedef struct mg_server mg_server;

typedef struct {
  int max_inflight;       /* requests resident on the device at once */
  int queue_capacity;     /* pending requests; beyond it mg_serve_submit returns MG_ERR_BUSY */
  size_t mem_budget;      /* device bytes for resident hierarchies (0 = the context's budget) */
  size_t host_budget;     /* page-locked host bytes for the arrays of submitted, not yet polled
                             requests (0 = 8 GiB); when full, mg_serve_submit returns MG_ERR_BUSY */
} mg_server_opts;

/* A request: everything is copied in at submit time (host memory), into page-locked
 * buffers owned by the server until the ticket is polled. */
typedef struct {
  mg_grid_desc grid;
  mg_map_desc map;          /* xp/yp host arrays for MG_MAP_GRID */
  const double *eps_phys;   /* nullable */
  const double *rho_phys;
  const double *bc;         /* nullable */
  mg_solve_opts opts;
} mg_request;

typedef struct {
  uint64_t completed, failed;
  double wall_s, unknowns_per_s;
  double p50_ms, p99_ms, max_ms;  /* submit -> result latency */
  double mean_batch;              /* mean requests in flight per scheduler tick */
  int ticks;
  uint64_t reused;                /* requests served by an already resident hierarchy */
  uint64_t evicted;               /* idle hierarchies freed to make room */
} mg_serve_report;

mg_status mg_server_start(mg_ctx *ctx, const mg_server_opts *opts, mg_server **out);
mg_status mg_serve_submit(mg_server *srv, const mg_request *req, uint64_t *ticket);
/* Wait up to timeout_ms for the ticket; on success copies phi (host, caller layout) and
 * stats and forgets the ticket.  MG_ERR_TIMEOUT if not done yet, MG_ERR_NOT_FOUND if unknown. */
mg_status mg_serve_poll(mg_server *srv, uint64_t ticket, int timeout_ms, double *phi_out,
                        mg_solve_stats *stats);
mg_status mg_server_stop(mg_server *srv, mg_serve_report *report);

#ifdef __cplusplus
}
#endif
#endif /* MG_H_ */
