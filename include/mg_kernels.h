/*
 * mg_kernels.h - single-kernel entry points of libmg on caller-owned device memory.
 *
 * Each call enqueues one step of the solver on `stream` (a cudaStream_t; NULL = the
 * legacy default stream) and returns at once; results appear in stream order.  All
 * pointers are device pointers owned by the caller.  Arrays use the pitched layout:
 * node (i, j) at a[i + pitch * j], rows j = 0 .. nyr-1 with nyr = ny - 1 if periodic in
 * y, else ny; pitch >= nx.  Return values: 0 = enqueued, 1 = bad argument (null pointer,
 * size, pitch), 4 = CUDA launch error.  Nothing is allocated.
 *
 * Operator storage (see mg.h): cE, cN, cNE, cNW hold the couplings of node (i, j) to
 * (i+1, j), (i, j+1), (i+1, j+1), (i-1, j+1); diag and dinv = 1/diag the diagonal.
 * five_point != 0 declares that cNE and cNW are zero at every node (the operator of a map
 * whose transformed tensor has no cross term: eps_xy of Eq. 13 vanishes identically, as for
 * the polar map of Eq. 29 and the sinh stretching of Eq. 52); the kernels then neither read
 * nor multiply them, with results identical to the 9-point form on those zeros.  The two
 * arrays must still hold zeros (the Galerkin coarsening and the point smoothers read them).
 * 0 = a general 9-point operator.
 */
#ifndef MG_KERNELS_H_
#define MG_KERNELS_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx, ny, periodic, pitch;
  double *cE, *cN, *cNE, *cNW, *diag, *dinv;
  int five_point;
} mgk_op_f64;

typedef struct {
  int nx, ny, periodic, pitch;
  float *cE, *cN, *cNE, *cNW, *diag, *dinv;
  int five_point;
} mgk_op_f32;

/*
 * Coefficient build, analytic map (kind: MG_MAP_* of mg.h, params as there): Jacobian
 * J_ab = dx'_a/dx_b (Eq. 1) at node x = x0 + i hx, y = y0 + j hy; D = det J; eps from
 * Eqs. 12-15 times eps_phys (nullable, pitched; Eq. 10 with eps' = s I).  *folded
 * (device int) is set to 1 where D <= 0 and left unchanged elsewhere.  For a map without
 * cross term (mg_map_five_point of mg.h: identity, polar, sinh, shear-free affine) eps_xy
 * is written as exactly 0, which Eq. 13 is for it (the general formula would leave rounding
 * residue); D, eps_xx and eps_yy always come from the general formula.
 */
int mgk_eps_analytic(int kind, const double *params4, int nx, int ny, int periodic, double x0,
                     double y0, double hx, double hy, const double *eps_phys, int pitch, double *D,
                     double *exx, double *exy, double *eyy, int *folded, void *stream);

/*
 * Coefficient build from a mapped grid: Jacobian by the central differences of
 * Eqs. 39-42 (one-sided second order at the ends of a non-periodic line; a periodic y
 * line wraps, adding (jump_x, jump_y) across the seam), then as mgk_eps_analytic.
 */
int mgk_eps_grid(int nx, int ny, int periodic, double hx, double hy, const double *xp,
                 const double *yp, double jump_x, double jump_y, const double *eps_phys, int pitch,
                 double *D, double *exx, double *exy, double *eyy, int *folded, void *stream);

/*
 * Fine-level operator A = -L_h from nodal eps (symmetric conservative form of the
 * Eq. 18 stencil): E/N couplings -(face mean of eps_xx / eps_yy)/h^2, corner couplings
 * from (Dx E Dy + Dy E Dx) with E = diag(eps_xy), diagonal = -(sum of the 8 couplings)
 * at unknowns, 1 at Dirichlet nodes.  Couplings missing at the grid edge are 0.  With
 * A->five_point set, eps_xy is taken as zero (it is not read) and cNE, cNW are written as 0.
 */
int mgk_assemble(const mgk_op_f64 *A, double hx, double hy, const double *exx, const double *exy,
                 const double *eyy, void *stream);

/* mgk_assemble for an operator without cross term (A->five_point must be set; eps_xy is not
 * an argument), in one pass that also writes, when B is not NULL, B as mgk_op_to_f32 would
 * with B->dinv = 1 / B->diag computed in FP32.  B has A's sizes and periodicity and its own
 * pitch.  The values are bitwise those of mgk_assemble (and of the FP32 conversion).
 * Returns 1 on a bad argument (A not five_point included), 4 on a launch error. */
int mgk_assemble_five(const mgk_op_f64 *A, const mgk_op_f32 *B, double hx, double hy, const double *exx,
                      const double *eyy, void *stream);

/* b = rho_phys * D at unknowns (Eq. 11), 0 at Dirichlet nodes. */
int mgk_rhs(const mgk_op_f64 *A, const double *rho_phys, const double *D, double *b, void *stream);

/* Tensor of the next coarser level of a rediscretized hierarchy (MG_COARSE_REDISCRETIZE of
 * mg.h): each field e0, e1, e2 (eps_xx, eps_xy, eps_yy on fine's layout) at the coarse nodes
 * (c0, c1, c2 on coarse's layout): full weighting (1/16)[1 2 1; 2 4 2; 1 2 1] about the
 * coincident fine node at coarse unknowns, the coincident fine value on the boundary ring.
 * Only the sizes, periodicity and pitches of fine and coarse (and coarse->five_point: c1 is
 * then written as 0 without reading e1) are used; coarse must be fine's next level.  The
 * coarse operator is then mgk_assemble on coarse with twice the spacing. */
int mgk_coarsen_eps(const mgk_op_f64 *fine, const mgk_op_f64 *coarse, const double *e0, const double *e1,
                    const double *e2, double *c0, double *c1, double *c2, void *stream);

/* Galerkin coarse operator A_H = (1/4) P^T A_h P with bilinear P (Sec. 3: A_H of Eq. 23). */
int mgk_galerkin(const mgk_op_f64 *fine, const mgk_op_f64 *coarse, void *stream);

/* FP32 copy of an operator (rounded to nearest); with src->five_point set, the NE / NW
 * arrays of dst are written as 0 without reading src's.  dst->five_point is not used. */
int mgk_op_to_f32(const mgk_op_f64 *src, const mgk_op_f32 *dst, void *stream);

/* Four-colour Gauss-Seidel (omega = 1, Sec. 2.1), `sweeps` sweeps in colour order
 * (0,0),(1,1),(1,0),(0,1) of (i mod 2, j mod 2), or the reverse order when reverse != 0.
 * phi is updated in place at unknowns. */
int mgk_smooth_f64(const mgk_op_f64 *A, double *phi, const double *b, int sweeps, int reverse,
                   void *stream);
int mgk_smooth_f32(const mgk_op_f32 *A, float *phi, const float *b, int sweeps, int reverse,
                   void *stream);

/* Four-colour successive over-relaxation, the single-level iteration the paper compares
 * against (Sec. 4, omega = 1.875 there): `sweeps` sweeps in the forward colour order; at each
 * unknown of a colour phi += omega (gs - phi), gs its Gauss-Seidel value.  0 < omega < 2. */
int mgk_sor_f64(const mgk_op_f64 *A, double *phi, const double *b, int sweeps, double omega,
                void *stream);
int mgk_sor_f32(const mgk_op_f32 *A, float *phi, const float *b, int sweeps, double omega,
                void *stream);

/* Weighted Jacobi: phi += omega (b - A phi) / diag at unknowns, `sweeps` times; tmp is a
 * pitched scratch array of the same shape. */
int mgk_jacobi_f64(const mgk_op_f64 *A, double *phi, const double *b, double *tmp, int sweeps,
                   double omega, void *stream);

/* r = b - A phi at unknowns, 0 at Dirichlet nodes (Eq. 20). */
int mgk_residual_f64(const mgk_op_f64 *A, const double *phi, const double *b, double *r,
                     void *stream);

/* Residual (Eq. 20) fused with full-weighting restriction r_H = I_h^H r_h (Sec. 3):
 * bH(I,J) = sum of (1/16)[1 2 1; 2 4 2; 1 2 1] r around fine node (2I, 2J); bH has
 * the coarse sizes ((nx-1)/2+1, (ny-1)/2+1) and pitch pitch_c; coarse Dirichlet nodes get 0. */
int mgk_resid_restrict_f64(const mgk_op_f64 *A, const double *phi, const double *b, double *bH,
                           int pitch_c, void *stream);
int mgk_resid_restrict_f32(const mgk_op_f32 *A, const float *phi, const float *b, float *bH,
                           int pitch_c, void *stream);

/* The same restriction for a phi whose odd rows (j odd) were the last ones solved exactly by
 * a zebra x-line half-sweep (Sec. 2.1 smoothing with whole rows as blocks): b - A phi is zero
 * on those rows up to the rounding of the row solves, so it is taken as zero there and
 * bH(I,J) = (1/16)(2 r(2I-1,2J) + 4 r(2I,2J) + 2 r(2I+1,2J)) from the even rows alone.
 * Same arguments, sizes and error returns as mgk_resid_restrict_*; it equals them exactly
 * when the odd rows' residual is exactly zero. */
int mgk_resid_restrict_even_f64(const mgk_op_f64 *A, const double *phi, const double *b,
                                double *bH, int pitch_c, void *stream);
int mgk_resid_restrict_even_f32(const mgk_op_f32 *A, const float *phi, const float *b, float *bH,
                                int pitch_c, void *stream);

/* phi += I_H^h eH (bilinear interpolation, Eq. 24) at fine unknowns; A gives the fine
 * sizes and pitch, eH the coarse array with pitch pitch_c. */
int mgk_prolong_add_f64(const mgk_op_f64 *A, double *phi, const double *eH, int pitch_c,
                        void *stream);
int mgk_prolong_add_f32(const mgk_op_f32 *A, float *phi, const float *eH, int pitch_c,
                        void *stream);

/* Coarsest-level inverse: assembles the dense matrix of the unknowns of A (m <= 256 of
 * them, lexicographic order, i fastest) and inverts it in place by Gauss-Jordan
 * elimination in one CTA; inv holds m*m doubles.  *status (device int) = 0, or 11
 * when a pivot is not positive (operator not SPD). */
int mgk_coarse_factor(const mgk_op_f64 *A, double *inv, int *status, void *stream);

/* x = A^-1 b on the coarsest level using the inverse from mgk_coarse_factor (one CTA);
 * Dirichlet nodes of x are left unchanged. */
int mgk_coarse_solve_f64(const mgk_op_f64 *A, const double *inv, const double *b, double *x,
                         void *stream);
int mgk_coarse_solve_f32(const mgk_op_f32 *A, const double *inv, const float *b, float *x,
                         void *stream);

/* One multigrid V(nu1, nu2) cycle (Sec. 3, Eqs. 19-24) on a caller-built hierarchy of
 * nlev levels: ops[l] the level operators (ops[l+1] the coarsening of ops[l]), x[l], b[l]
 * the iterate and right-hand side of each level, t[l] a scratch array of the same shape,
 * inv the coarsest inverse from mgk_coarse_factor on ops[nlev-1].  Starts from the
 * iterate in x[0] (coarse iterates start from zero) and leaves the result in x[0];
 * smoother: 0 four-colour Gauss-Seidel (forward colours before the coarse-grid
 * correction, reverse after), 1 weighted Jacobi (omega 0.8); the line smoother (2) needs
 * mgk_vcycle_line_*.  Same kernels as mg_solve. */
int mgk_vcycle_f64(int nlev, const mgk_op_f64 *ops, double *const *x, double *const *b,
                   double *const *t, const double *inv, int nu1, int nu2, int smoother,
                   void *stream);
int mgk_vcycle_f32(int nlev, const mgk_op_f32 *ops, float *const *x, float *const *b,
                   float *const *t, const double *inv, int nu1, int nu2, int smoother,
                   void *stream);

/* Fused smoothing launch used inside the V-cycle: xout = mgk_fused_sweeps() four-colour
 * Gauss-Seidel sweeps (Sec. 2.1, omega = 1) applied to xin, or to xin + I_H^h eH (Eq. 24)
 * when eH is not NULL (coarse array of pitch pitch_c); reverse != 0 runs the colours
 * backwards.  xin and xout must be different arrays (neighbouring tiles read xin while
 * others write xout); Dirichlet nodes are copied from xin to xout. */
int mgk_smooth_fused_f64(const mgk_op_f64 *A, const double *xin, double *xout, const double *b,
                         int reverse, const double *eH, int pitch_c, void *stream);
int mgk_smooth_fused_f32(const mgk_op_f32 *A, const float *xin, float *xout, const float *b,
                         int reverse, const float *eH, int pitch_c, void *stream);
/* Number of sweeps one fused launch performs (f32 != 0: FP32 instance). */
int mgk_fused_sweeps(int f32);

/* Persistent pipelined variant of mgk_smooth_fused_*: same result (mgk_pipe_sweeps() sweeps,
 * optional prolongation-correction first), tiles staged by bulk asynchronous copies into
 * two shared-memory stages.  Needs 16-byte aligned arrays and a pitch that keeps every row
 * 16-byte aligned (else returns 1).  *err (device int, nullable) is set to 1 if a copy wait
 * exceeds its bound, in which case the launch stops early. */
int mgk_smooth_pipe_f64(const mgk_op_f64 *A, const double *xin, double *xout, const double *b,
                        int reverse, const double *eH, int pitch_c, int *err, void *stream);
int mgk_smooth_pipe_f32(const mgk_op_f32 *A, const float *xin, float *xout, const float *b,
                        int reverse, const float *eH, int pitch_c, int *err, void *stream);
int mgk_pipe_sweeps(int f32);

/* Row-marching variant for large levels: xout = mgk_march_sweeps() (FP32) or
 * mgk_march_sweeps_f64() (FP64) four-colour Gauss-Seidel sweeps (Sec. 2.1, omega = 1;
 * reverse = 1 reverses the colour order) of xin [+ P eH] (Eq. 24) in one pass over the
 * level.  Each CTA streams a strip of columns upward through a ring of rows in shared
 * memory, so every array is read about once.  Same result as the per-colour kernels
 * (identical operations in the same order per node).  Needs xin != xout, 16-byte aligned
 * arrays and a pitch that keeps rows 16-byte aligned (else returns 1); 4 on a CUDA error. */
int mgk_smooth_march_f32(const mgk_op_f32 *A, const float *xin, float *xout, const float *b,
                         int reverse, const float *eH, int pitch_c, void *stream);
int mgk_smooth_march_f64(const mgk_op_f64 *A, const double *xin, double *xout, const double *b,
                         int reverse, const double *eH, int pitch_c, void *stream);
int mgk_march_sweeps(void);
int mgk_march_sweeps_f64(void);

/* Shapes the autotuner chooses among (mg_autotune).  family: 2 fused tiles, 3 pipelined
 * tiles, 4 row marching (the mg_tune_entry.choice codes).  mgk_smooth_variant_info gives
 * variant `variant` of a family in FP32 (f32 = 1) or FP64: owned tile tile_x x tile_y
 * (marching: tile_x owned strip columns, tile_y 0) and sweeps per launch; returns 1 past the
 * last variant.  mgk_smooth_variant_* runs one launch of that variant exactly as the
 * mgk_smooth_fused_* / mgk_smooth_pipe_* / mgk_smooth_march_* entry points run their default
 * one (same arguments and requirements; err is used by the pipelined tiles only). */
int mgk_smooth_variant_info(int f32, int family, int variant, int *tile_x, int *tile_y, int *sweeps);
int mgk_smooth_variant_f64(const mgk_op_f64 *A, int family, int variant, const double *xin, double *xout,
                           const double *b, int reverse, const double *eH, int pitch_c, int *err,
                           void *stream);
int mgk_smooth_variant_f32(const mgk_op_f32 *A, int family, int variant, const float *xin, float *xout,
                           const float *b, int reverse, const float *eH, int pitch_c, int *err,
                           void *stream);

/* Zebra x-line Gauss-Seidel (an addition to the paper's point smoother for operators whose
 * coupling along x dominates, such as the annulus of Eq. 29 in polar coordinates).  A
 * half-sweep of parity p solves, for every row j with j mod 2 == p, the tridiagonal system
 * of the row's unknowns (diagonal, W and E couplings) with the couplings to rows j-1 and
 * j+1 (N, S, NE, NW, SE, SW) and to the row's two Dirichlet end nodes moved to the
 * right-hand side; rows of one parity are independent.  The row systems are solved by
 * cyclic reduction (row length nx - 2 padded to a power of two) with factors that depend
 * on A only:
 *   mgk_line_factor_elems(nx, ny, periodic): elements (of the operator's precision) that
 *     the factors of an nx x ny level take; 0 for sizes below 3;
 *   mgk_line_factor_*: fills `factors` for every row of A; call it again when A changes;
 *   mgk_line_rows_*: one half-sweep of parity 0 or 1, phi updated in place;
 *   mgk_line_smooth_*: `sweeps` sweeps, each parity 0 then 1 (reverse != 0: 1 then 0).
 * Rows of up to 8192 unknowns in FP64 and 16384 in FP32 (shared-memory bound); longer
 * rows, or a periodic grid with an odd row count, return 1. */
size_t mgk_line_factor_elems(int nx, int ny, int periodic);
int mgk_line_factor_f64(const mgk_op_f64 *A, double *factors, void *stream);
int mgk_line_factor_f32(const mgk_op_f32 *A, float *factors, void *stream);
int mgk_line_rows_f64(const mgk_op_f64 *A, const double *factors, double *phi, const double *b,
                      int parity, void *stream);
int mgk_line_rows_f32(const mgk_op_f32 *A, const float *factors, float *phi, const float *b,
                      int parity, void *stream);
int mgk_line_smooth_f64(const mgk_op_f64 *A, const double *factors, double *phi, const double *b,
                        int sweeps, int reverse, void *stream);
int mgk_line_smooth_f32(const mgk_op_f32 *A, const float *factors, float *phi, const float *b,
                        int sweeps, int reverse, void *stream);

/* mgk_vcycle_* with the zebra x-line smoother (pre-smoothing parity 0 first, post-smoothing
 * parity 1 first) on levels 0 .. nlev-2; factors[l] holds the mgk_line_factor_* result of
 * ops[l] for those levels. */
int mgk_vcycle_line_f64(int nlev, const mgk_op_f64 *ops, double *const *x, double *const *b,
                        double *const *t, const double *inv, double *const *factors, int nu1,
                        int nu2, void *stream);
int mgk_vcycle_line_f32(int nlev, const mgk_op_f32 *ops, float *const *x, float *const *b,
                        float *const *t, const double *inv, float *const *factors, int nu1,
                        int nu2, void *stream);

/* Weighted-Jacobi sweeps exactly as mgk_jacobi_f64, for callers that cannot allocate
 * device memory when they call it (a latency-critical loop where cudaMalloc/cudaFree would
 * synchronise the device, or an application whose device memory all belongs to another
 * allocator).  The paper has no counterpart: this is a deployment variant.  Instead of the
 * caller's tmp array it uses one fixed device array of mgk_jacobi_f64_static_capacity()
 * doubles (8 MiB) that every device loading the library keeps until the process exits.
 * Returns 2 (message in mg_last_error) when pitch * rows exceeds that capacity.  Every call
 * looks up the array's device address in the current context; the first one on a device may
 * load the library's device code, so make it before capturing any stream.  All calls on a
 * device share the array and it keeps the last call's contents; calls that overlap on the
 * GPU race on it. */
int mgk_jacobi_f64_static(const mgk_op_f64 *A, double *phi, const double *b, int sweeps,
                          double omega, void *stream);
size_t mgk_jacobi_f64_static_capacity(void);

/* FMA-rate probe (no counterpart in the paper: it measures the arithmetic peak that the
 * FP64 stencil kernels are reported against, since their bound is the FP64 pipe, not HBM).
 * Launches `blocks` CTAs of 256 threads; every thread runs `chains` (4, 8 or 16)
 * independent chains of `iters` fused multiply-adds in registers (FP64 if f64 != 0, else
 * FP32), in operand pattern `pattern` (0: a = a b + c with two constants shared by all
 * chains; 1: a = x y + a with per-chain x and y, the stencil-sum pattern), and writes one
 * value to out[blocks * 256] (device memory, caller-owned).  Time the launch with CUDA
 * events on `stream`; mgk_fma_rate_flops gives its flop count.  Returns 1 on bad arguments,
 * 4 if the launch fails. */
int mgk_fma_rate(int f64, int pattern, int chains, int blocks, int iters, void *out, void *stream);
double mgk_fma_rate_flops(int chains, int blocks, int iters);

/* Test hook of the request server (mg_serve_*): the next `count` completion queries of
 * in-flight requests report a failure (cudaErrorLaunchFailure) without asking the runtime,
 * so tests can drive the server's failure path on the host, with no fault on the device.
 * A request that meets one finishes with MG_ERR_CUDA, its slot is freed and
 * mg_server_stop still returns.  0 turns it off. */
void mgk_server_fail_event_queries(int count);

#ifdef __cplusplus
}
#endif
#endif /* MG_KERNELS_H_ */
