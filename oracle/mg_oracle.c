/*
 * FP64 CPU oracle for the transformed-coefficient geometric multigrid solver.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path, and it is never a fallback for it.
 *
 * Everything here is plain, slow, loop-by-loop FP64 arithmetic that follows the
 * paper (Gautam & Paradkar, "Multigrid Poisson Solver for Complex Geometries
 * Using Finite Difference Method") equation by equation:
 *   - Jacobian of the map x -> x': analytic, or central differences (Eqs. 39-42)
 *   - permittivity tensor on the computational grid (Eq. 10, components Eqs. 12-15)
 *   - transformed charge density rho = rho' det J (Eq. 11)
 *   - generalized Poisson operator -div(eps grad phi) = rho (Eqs. 7, 16-17), written
 *     in symmetric conservative 9-point form (reading of Eq. 18, see below)
 *   - Gauss-Seidel relaxation with omega = 1 as the smoother (Sec. 2.1, after Eq. 18)
 *   - the residual-correction multigrid cycle (Sec. 3, Eqs. 19-24)
 *   - error norms (Eqs. 25-27) live on the Python side.
 *
 * Readings where the paper is silent or garbled (each also listed in the design notes):
 *   - sign: -div(eps grad phi) = rho (Eq. 7 with E = -grad phi, Eq. 17), so A is SPD.
 *   - Eq. 18 is a non-symmetric lexicographic update; the solver operator is its
 *     symmetric conservative counterpart: arithmetic face means of eps_xx / eps_yy
 *     for the second derivatives and (Dx E Dy + Dy E Dx) with E = diag(eps_xy) for the
 *     mixed derivative.  Eq. 18 itself is also implemented (paper_sor_* below).
 *   - the multigrid transfer operators are not specified (Sec. 3): full weighting
 *     restriction R = P^T / 4, bilinear prolongation P, Galerkin coarse operator
 *     A_H = R A_h P, exact dense solve on the coarsest level.
 *   - "red-black" Gauss-Seidel with a 9-point stencil is done with four colours
 *     (i mod 2, j mod 2), order (0,0),(1,1),(1,0),(0,1) before the coarse-grid
 *     correction and the reverse order after it.
 *   - boundary Jacobian: one-sided second-order differences where a neighbour is
 *     missing; a periodic y-direction wraps.
 *   - Dirichlet values live in the boundary ring of phi (equivalent to moving
 *     coupling * value into b).
 *
 * Grid layout: node (i, j), i = 0..nx-1 along x (xi), j along y (eta), stored at
 * a[i + nx * j].  A periodic-y grid of ny vertices stores nyr = ny - 1 rows (row
 * ny-1 is row 0); otherwise nyr = ny.
 *
 * Operator storage (all levels): for node (i, j),
 *   cE  = A[(i,j),(i+1,j)],  cN = A[(i,j),(i,j+1)],
 *   cNE = A[(i,j),(i+1,j+1)], cNW = A[(i,j),(i-1,j+1)],  diag = A[(i,j),(i,j)].
 * The remaining four entries of a row follow from symmetry:
 *   W = cE(i-1,j), S = cN(i,j-1), SW = cNE(i-1,j-1), SE = cNW(i+1,j-1).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_FOLDED 5
#define ORC_ERR_NOT_SPD 11

enum { MAP_IDENTITY = 0, MAP_SINE_WARP = 1, MAP_POLAR = 2, MAP_SINH = 3, MAP_AFFINE = 4 };

static const double PI = 3.14159265358979323846;

static int wrapj(int j, int nyr) { return (j % nyr + nyr) % nyr; }

/* Is (i, j) an unknown (not on a Dirichlet side)? */
static int is_interior(int i, int j, int nx, int ny, int periodic) {
  if (i < 1 || i > nx - 2) return 0;
  if (periodic) return 1;
  return j >= 1 && j <= ny - 2;
}

/* ------------------------------------------------------------------------ */
/* Jacobian J_ab = d x'_a / d x_b (Eq. 1 in 2-D), analytic maps               */
/* ------------------------------------------------------------------------ */
/*
 * params: SINE_WARP {a}            x' = x + a sin(pi x) sin(pi y), y' = y + a sin(2 pi x) sin(pi y)
 *         POLAR     {}             x' = x cos y, y' = x sin y                  (Eq. 29)
 *         SINH      {s, alpha}     x' = s sinh(alpha x), y' = s sinh(alpha y)  (Eq. 52)
 *         AFFINE    {a11,a12,a21,a22} x' = a11 x + a12 y, y' = a21 x + a22 y
 * Node coordinates: x = x0 + i hx, y = y0 + j hy.
 */
int orc_jacobian_analytic(int kind, const double *prm, int nx, int nyr, double x0, double y0,
                          double hx, double hy, double *Jxx, double *Jxy, double *Jyx,
                          double *Jyy) {
  for (int j = 0; j < nyr; ++j) {
    for (int i = 0; i < nx; ++i) {
      double x = x0 + i * hx, y = y0 + j * hy;
      double a = 1, b = 0, c = 0, d = 1; /* Jxx Jxy Jyx Jyy */
      switch (kind) {
        case MAP_IDENTITY:
          break;
        case MAP_SINE_WARP:
          a = 1 + prm[0] * PI * cos(PI * x) * sin(PI * y);
          b = prm[0] * PI * sin(PI * x) * cos(PI * y);
          c = prm[0] * 2 * PI * cos(2 * PI * x) * sin(PI * y);
          d = 1 + prm[0] * PI * sin(2 * PI * x) * cos(PI * y);
          break;
        case MAP_POLAR:
          a = cos(y);
          b = -x * sin(y);
          c = sin(y);
          d = x * cos(y);
          break;
        case MAP_SINH:
          a = prm[0] * prm[1] * cosh(prm[1] * x);
          b = 0;
          c = 0;
          d = prm[0] * prm[1] * cosh(prm[1] * y);
          break;
        case MAP_AFFINE:
          a = prm[0];
          b = prm[1];
          c = prm[2];
          d = prm[3];
          break;
        default:
          return ORC_ERR_ARG;
      }
      size_t k = (size_t)i + (size_t)nx * j;
      Jxx[k] = a;
      Jxy[k] = b;
      Jyx[k] = c;
      Jyy[k] = d;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Jacobian from a mapped grid by central differences (Eqs. 39-42)            */
/* ------------------------------------------------------------------------ */
/* d f / d x at node (i, j): central difference inside, one-sided second order
 * (-3 f0 + 4 f1 - f2) / (2h) at an end of the line. */
static double ddx(const double *f, int i, int j, int nx, double hx) {
  size_t r = (size_t)nx * j;
  if (i == 0) return (-3 * f[r] + 4 * f[r + 1] - f[r + 2]) / (2 * hx);
  if (i == nx - 1) return (3 * f[r + nx - 1] - 4 * f[r + nx - 2] + f[r + nx - 3]) / (2 * hx);
  return (f[r + i + 1] - f[r + i - 1]) / (2 * hx);
}

/* d f / d y; in a periodic grid the mapped coordinates wrap with an offset
 * (period_x, period_y) added when crossing row nyr -> 0 (zero for a closed polar map). */
static double ddy(const double *f, int i, int j, int nx, int ny, int nyr, int periodic,
                  double hy, double jump) {
  if (periodic) {
    int jp = j + 1, jm = j - 1;
    double fp, fm;
    if (jp >= nyr) fp = f[i + (size_t)nx * (jp - nyr)] + jump; else fp = f[i + (size_t)nx * jp];
    if (jm < 0) fm = f[i + (size_t)nx * (jm + nyr)] - jump; else fm = f[i + (size_t)nx * jm];
    return (fp - fm) / (2 * hy);
  }
  if (j == 0)
    return (-3 * f[i] + 4 * f[i + (size_t)nx] - f[i + 2 * (size_t)nx]) / (2 * hy);
  if (j == ny - 1)
    return (3 * f[i + (size_t)nx * (ny - 1)] - 4 * f[i + (size_t)nx * (ny - 2)] +
            f[i + (size_t)nx * (ny - 3)]) / (2 * hy);
  return (f[i + (size_t)nx * (j + 1)] - f[i + (size_t)nx * (j - 1)]) / (2 * hy);
}

int orc_jacobian_grid(int nx, int ny, int periodic, double hx, double hy, const double *xp,
                      const double *yp, double jump_x, double jump_y, double *Jxx, double *Jxy,
                      double *Jyx, double *Jyy) {
  int nyr = periodic ? ny - 1 : ny;
  if (nx < 3 || nyr < 3) return ORC_ERR_ARG;
  for (int j = 0; j < nyr; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t k = (size_t)i + (size_t)nx * j;
      Jxx[k] = ddx(xp, i, j, nx, hx);                                 /* Eq. 39 */
      Jxy[k] = ddy(xp, i, j, nx, ny, nyr, periodic, hy, jump_x);      /* Eq. 40 */
      Jyx[k] = ddx(yp, i, j, nx, hx);                                 /* Eq. 41 */
      Jyy[k] = ddy(yp, i, j, nx, ny, nyr, periodic, hy, jump_y);      /* Eq. 42 */
    }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Permittivity tensor on the computational grid (Eq. 10 -> Eqs. 12-15)       */
/* ------------------------------------------------------------------------ */
/* eps = det(J) J^-1 eps' J^-T with eps' = s I (s = eps_phys, 1 when NULL).
 * Returns ORC_ERR_FOLDED if det J <= 0 anywhere. */
int orc_eps(size_t nodes, const double *Jxx, const double *Jxy, const double *Jyx,
            const double *Jyy, const double *eps_phys, double *D, double *exx, double *exy,
            double *eyy) {
  int folded = 0;
  for (size_t k = 0; k < nodes; ++k) {
    double det = Jxx[k] * Jyy[k] - Jxy[k] * Jyx[k];
    double s = eps_phys ? eps_phys[k] : 1.0;
    D[k] = det;
    if (!(det > 0)) folded = 1;
    exx[k] = s * (Jyy[k] * Jyy[k] + Jxy[k] * Jxy[k]) / det;     /* Eq. 12 */
    exy[k] = s * (-Jyy[k] * Jyx[k] - Jxy[k] * Jxx[k]) / det;    /* Eq. 13 (= Eq. 14) */
    eyy[k] = s * (Jyx[k] * Jyx[k] + Jxx[k] * Jxx[k]) / det;     /* Eq. 15 */
  }
  return folded ? ORC_ERR_FOLDED : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Fine-level operator A = -L_h (symmetric conservative 9-point form)          */
/* ------------------------------------------------------------------------ */
/*
 * L_h phi = [ex_{i+1/2}(phi_{i+1}-phi_i) - ex_{i-1/2}(phi_i-phi_{i-1})]/hx^2
 *         + [ey_{j+1/2}(phi_{j+1}-phi_j) - ey_{j-1/2}(phi_j-phi_{j-1})]/hy^2
 *         + (Dx E Dy + Dy E Dx) phi,
 * ex_{i+1/2} = (exx_i + exx_{i+1}) / 2, ey likewise, Dx, Dy central differences,
 * E = diag(eps_xy).  The mixed term gives only the four corner couplings.
 * Couplings are defined wherever both nodes exist; the diagonal of every unknown
 * is minus the sum of its eight couplings (zero row sums).  Diagonal entries of
 * Dirichlet nodes are set to 1 and never used.
 */
int orc_assemble(int nx, int ny, int periodic, double hx, double hy, const double *exx,
                 const double *exy, const double *eyy, double *cE, double *cN, double *cNE,
                 double *cNW, double *diag) {
  int nyr = periodic ? ny - 1 : ny;
  double ihx2 = 1.0 / (hx * hx), ihy2 = 1.0 / (hy * hy), ixy4 = 1.0 / (4.0 * hx * hy);
  for (int j = 0; j < nyr; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t k = (size_t)i + (size_t)nx * j;
      int has_up = periodic || j + 1 <= ny - 1;
      int ju = wrapj(j + 1, nyr);
      cE[k] = cN[k] = cNE[k] = cNW[k] = 0.0;
      if (i + 1 <= nx - 1) {
        size_t ke = k + 1;
        cE[k] = -0.5 * (exx[k] + exx[ke]) * ihx2;
      }
      if (has_up) {
        size_t kn = (size_t)i + (size_t)nx * ju;
        cN[k] = -0.5 * (eyy[k] + eyy[kn]) * ihy2;
        if (i + 1 <= nx - 1) /* (i,j)-(i+1,j+1): -(exy(i+1,j) + exy(i,j+1)) / (4 hx hy) */
          cNE[k] = -(exy[k + 1] + exy[kn]) * ixy4;
        if (i - 1 >= 0) /* (i,j)-(i-1,j+1): +(exy(i-1,j) + exy(i,j+1)) / (4 hx hy) */
          cNW[k] = (exy[k - 1] + exy[kn]) * ixy4;
      }
    }
  for (int j = 0; j < nyr; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t k = (size_t)i + (size_t)nx * j;
      if (!is_interior(i, j, nx, ny, periodic)) {
        diag[k] = 1.0;
        continue;
      }
      int jd = wrapj(j - 1, nyr);
      size_t kw = k - 1, ks = (size_t)i + (size_t)nx * jd;
      double s = cE[k] + cE[kw] + cN[k] + cN[ks] + cNE[k] + cNE[ks - 1] + cNW[k] + cNW[ks + 1];
      diag[k] = -s;
    }
  return ORC_OK;
}

/* Right-hand side b = rho' det J at unknowns (Eq. 11), 0 on Dirichlet nodes. */
int orc_rhs(int nx, int ny, int periodic, const double *rho_phys, const double *D, double *b) {
  int nyr = periodic ? ny - 1 : ny;
  for (int j = 0; j < nyr; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t k = (size_t)i + (size_t)nx * j;
      b[k] = is_interior(i, j, nx, ny, periodic) ? rho_phys[k] * D[k] : 0.0;
    }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Stencil helpers                                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
  int nx, ny, nyr, periodic;
  const double *cE, *cN, *cNE, *cNW, *diag;
} op_t;

/* Off-diagonal part of row (i, j) applied to phi: sum over the 8 neighbours. */
static double offdiag_row(const op_t *A, const double *phi, int i, int j) {
  int nx = A->nx, nyr = A->nyr;
  int ju = wrapj(j + 1, nyr), jd = wrapj(j - 1, nyr);
  size_t k = (size_t)i + (size_t)nx * j;
  size_t ru = (size_t)nx * ju, rd = (size_t)nx * jd, r0 = (size_t)nx * j;
  double s = 0.0;
  s += A->cE[k] * phi[r0 + i + 1];           /* E  */
  s += A->cE[r0 + i - 1] * phi[r0 + i - 1];  /* W  */
  s += A->cN[k] * phi[ru + i];               /* N  */
  s += A->cN[rd + i] * phi[rd + i];          /* S  */
  s += A->cNE[k] * phi[ru + i + 1];          /* NE */
  s += A->cNE[rd + i - 1] * phi[rd + i - 1]; /* SW */
  s += A->cNW[k] * phi[ru + i - 1];          /* NW */
  s += A->cNW[rd + i + 1] * phi[rd + i + 1]; /* SE */
  return s;
}

/* r = b - A phi at unknowns, 0 elsewhere (Eq. 20). */
static void residual(const op_t *A, const double *phi, const double *b, double *r) {
  for (int j = 0; j < A->nyr; ++j)
    for (int i = 0; i < A->nx; ++i) {
      size_t k = (size_t)i + (size_t)A->nx * j;
      if (!is_interior(i, j, A->nx, A->ny, A->periodic)) {
        r[k] = 0.0;
        continue;
      }
      r[k] = b[k] - (A->diag[k] * phi[k] + offdiag_row(A, phi, i, j));
    }
}

/* One colour phase of Gauss-Seidel (omega = 1): every unknown of colour (ci, cj)
 * is set to (b - offdiag * phi) / diag.  Nodes of one colour are not coupled by
 * the 9-point stencil, so the order inside a phase does not matter. */
static void gs_colour(const op_t *A, double *phi, const double *b, int ci, int cj) {
  for (int j = cj; j < A->nyr; j += 2)
    for (int i = ci; i < A->nx; i += 2) {
      if (!is_interior(i, j, A->nx, A->ny, A->periodic)) continue;
      size_t k = (size_t)i + (size_t)A->nx * j;
      phi[k] = (b[k] - offdiag_row(A, phi, i, j)) / A->diag[k];
    }
}

static const int COLOUR_ORDER[4][2] = {{0, 0}, {1, 1}, {1, 0}, {0, 1}};

/* sweeps of four-colour Gauss-Seidel; reverse = 1 runs the colours backwards. */
static void gs4(const op_t *A, double *phi, const double *b, int sweeps, int reverse) {
  for (int s = 0; s < sweeps; ++s)
    for (int c = 0; c < 4; ++c) {
      int cc = reverse ? 3 - c : c;
      gs_colour(A, phi, b, COLOUR_ORDER[cc][0], COLOUR_ORDER[cc][1]);
    }
}

/* sweeps of four-colour successive over-relaxation: the colours in the Gauss-Seidel order,
 * and at each node of a colour phi += omega * (gs - phi), gs the node's Gauss-Seidel value
 * (Sec. 2.1 with the over-relaxation of Sec. 4's comparison runs, omega = 1.875 there). */
static void sor4(const op_t *A, double *phi, const double *b, int sweeps, double omega) {
  for (int s = 0; s < sweeps; ++s)
    for (int c = 0; c < 4; ++c)
      for (int j = COLOUR_ORDER[c][1]; j < A->nyr; j += 2)
        for (int i = COLOUR_ORDER[c][0]; i < A->nx; i += 2) {
          if (!is_interior(i, j, A->nx, A->ny, A->periodic)) continue;
          size_t k = (size_t)i + (size_t)A->nx * j;
          double gs = (b[k] - offdiag_row(A, phi, i, j)) / A->diag[k];
          phi[k] += omega * (gs - phi[k]);
        }
}

/* Weighted Jacobi: phi += w * (b - A phi) / diag at every unknown. */
static void jacobi(const op_t *A, double *phi, const double *b, double *tmp, int sweeps, double w) {
  for (int s = 0; s < sweeps; ++s) {
    residual(A, phi, b, tmp);
    for (int j = 0; j < A->nyr; ++j)
      for (int i = 0; i < A->nx; ++i) {
        size_t k = (size_t)i + (size_t)A->nx * j;
        if (is_interior(i, j, A->nx, A->ny, A->periodic)) phi[k] += w * tmp[k] / A->diag[k];
      }
  }
}

/* One half-sweep of x-line Gauss-Seidel in zebra order: every row j of parity par
 * (j mod 2 == par) is solved as a whole.  On that row the couplings to its own unknowns
 * (W and E) stay in a tridiagonal system; the couplings to the rows above and below (N, S
 * and the four diagonals) and to the row's two Dirichlet end nodes go to the right-hand
 * side with the current values of those nodes.  Rows of one parity share no coupling, so
 * they can be solved in any order.  The tridiagonal system is solved by the Thomas
 * algorithm (forward elimination, back substitution). */
static void line_rows(const op_t *A, double *phi, const double *b, int par) {
  const int nx = A->nx, N = nx - 2;
  if (N < 1) return;
  double *cp = (double *)calloc((size_t)N, sizeof(double));
  double *dp = (double *)calloc((size_t)N, sizeof(double));
  for (int j = par; j < A->nyr; j += 2) {
    if (!is_interior(1, j, nx, A->ny, A->periodic)) continue;
    const int ju = A->periodic ? wrapj(j + 1, A->nyr) : j + 1;
    const int jd = A->periodic ? wrapj(j - 1, A->nyr) : j - 1;
    const size_t r0 = (size_t)nx * j, ru = (size_t)nx * ju, rd = (size_t)nx * jd;
    for (int t = 0; t < N; ++t) {
      const int i = t + 1;
      const size_t k = r0 + i;
      /* couplings leaving the row: N, S, NE, SW, NW, SE, and the Dirichlet ends */
      double off = A->cN[k] * phi[ru + i] + A->cN[rd + i] * phi[rd + i];
      off += A->cNE[k] * phi[ru + i + 1] + A->cNE[rd + i - 1] * phi[rd + i - 1];
      off += A->cNW[k] * phi[ru + i - 1] + A->cNW[rd + i + 1] * phi[rd + i + 1];
      if (i == 1) off += A->cE[r0] * phi[r0];
      if (i == nx - 2) off += A->cE[k] * phi[k + 1];
      const double rhs = b[k] - off;
      const double sub = (i - 1 >= 1) ? A->cE[k - 1] : 0.0;
      const double sup = (i + 1 <= nx - 2) ? A->cE[k] : 0.0;
      const double m = (t == 0) ? A->diag[k] : A->diag[k] - sub * cp[t - 1];
      cp[t] = sup / m;
      dp[t] = (t == 0) ? rhs / m : (rhs - sub * dp[t - 1]) / m;
    }
    phi[r0 + N] = dp[N - 1];
    for (int t = N - 2; t >= 0; --t) phi[r0 + t + 1] = dp[t] - cp[t] * phi[r0 + t + 2];
  }
  free(cp);
  free(dp);
}

/* sweeps of zebra x-line Gauss-Seidel: rows of parity 0 then 1 (reverse: 1 then 0). */
static void xline(const op_t *A, double *phi, const double *b, int sweeps, int reverse) {
  for (int s = 0; s < sweeps; ++s)
    for (int h = 0; h < 2; ++h) line_rows(A, phi, b, reverse ? 1 - h : h);
}

/* ------------------------------------------------------------------------ */
/* Grid transfers                                                              */
/* ------------------------------------------------------------------------ */
/* Bilinear interpolation weight of coarse offset for a fine offset d = f - 2c. */
static double pw(int d) {
  if (d == 0) return 1.0;
  if (d == 1 || d == -1) return 0.5;
  return 0.0;
}

/* Full weighting: bH(I,J) = sum over the 3x3 fine neighbourhood of (2I,2J) of
 * (1/16)[1 2 1; 2 4 2; 1 2 1] r  (R = P^T / 4). Coarse Dirichlet nodes get 0. */
static void restrict_fw(const op_t *Af, const double *r, const op_t *Ac, double *bH) {
  for (int J = 0; J < Ac->nyr; ++J)
    for (int I = 0; I < Ac->nx; ++I) {
      size_t K = (size_t)I + (size_t)Ac->nx * J;
      if (!is_interior(I, J, Ac->nx, Ac->ny, Ac->periodic)) {
        bH[K] = 0.0;
        continue;
      }
      double s = 0.0;
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          int fi = 2 * I + di, fj = wrapj(2 * J + dj, Af->nyr);
          s += 0.25 * pw(di) * pw(dj) * r[(size_t)fi + (size_t)Af->nx * fj];
        }
      bH[K] = s;
    }
}

/* phi_h += P e_H (bilinear), at fine unknowns only (Eq. 24). */
static void prolong_add(const op_t *Ac, const double *eH, const op_t *Af, double *phi) {
  for (int j = 0; j < Af->nyr; ++j)
    for (int i = 0; i < Af->nx; ++i) {
      if (!is_interior(i, j, Af->nx, Af->ny, Af->periodic)) continue;
      double s = 0.0;
      int I0 = i / 2, J0 = j / 2;
      for (int I = I0; I <= I0 + 1; ++I)
        for (int J = J0; J <= J0 + 1; ++J) {
          if (I > Ac->nx - 1) continue;
          double w = pw(i - 2 * I) * pw(j - 2 * J);
          if (w == 0.0) continue;
          int Jw = wrapj(J, Ac->nyr);
          if (!Ac->periodic && J > Ac->ny - 1) continue;
          s += w * eH[(size_t)I + (size_t)Ac->nx * Jw];
        }
      phi[(size_t)i + (size_t)Af->nx * j] += s;
    }
}

/* ------------------------------------------------------------------------ */
/* Galerkin coarse operator A_H = (1/4) P^T A_h P as a direct triple sum       */
/* ------------------------------------------------------------------------ */
/* Fine-row entry A[(fi,fj),(fi+di,fj+dj)] read through the symmetric storage. */
static double fine_entry(const op_t *A, int fi, int fj, int di, int dj) {
  int nx = A->nx, nyr = A->nyr;
  size_t r0 = (size_t)nx * fj, rd = (size_t)nx * wrapj(fj - 1, nyr);
  if (di == 0 && dj == 0) return A->diag[r0 + fi];
  if (di == 1 && dj == 0) return A->cE[r0 + fi];
  if (di == -1 && dj == 0) return A->cE[r0 + fi - 1];
  if (di == 0 && dj == 1) return A->cN[r0 + fi];
  if (di == 0 && dj == -1) return A->cN[rd + fi];
  if (di == 1 && dj == 1) return A->cNE[r0 + fi];
  if (di == -1 && dj == -1) return A->cNE[rd + fi - 1];
  if (di == -1 && dj == 1) return A->cNW[r0 + fi];
  /* di == 1 && dj == -1 */
  return A->cNW[rd + fi + 1];
}

/*
 * For every coarse unknown I: row[oI][oJ] = (1/4) sum_k sum_l P(k,I) A(k,l) P(l,I+o)
 * over fine k in the 3x3 support of I and the 9 stencil neighbours l of k.  P is the
 * bilinear interpolation over all coarse nodes.  The coarse entries kept are
 * E, N, NE, NW and the diagonal of each coarse unknown; entries stored at coarse
 * Dirichlet nodes are 0 and their diagonal is 1.
 */
int orc_galerkin(int nxf, int nyf, int periodic, const double *fE, const double *fN,
                 const double *fNE, const double *fNW, const double *fD, double *cE, double *cN,
                 double *cNE, double *cNW, double *cD) {
  if ((nxf - 1) % 2 || (nyf - 1) % 2) return ORC_ERR_ARG;
  int nyrf = periodic ? nyf - 1 : nyf;
  op_t Af = {nxf, nyf, nyrf, periodic, fE, fN, fNE, fNW, fD};
  int nxc = (nxf - 1) / 2 + 1, nyc = (nyf - 1) / 2 + 1;
  int nyrc = periodic ? nyc - 1 : nyc;
  for (int J = 0; J < nyrc; ++J)
    for (int I = 0; I < nxc; ++I) {
      size_t K = (size_t)I + (size_t)nxc * J;
      cE[K] = cN[K] = cNE[K] = cNW[K] = 0.0;
      cD[K] = 1.0;
      if (!is_interior(I, J, nxc, nyc, periodic)) continue;
      double row[3][3] = {{0}};
      for (int kj = -1; kj <= 1; ++kj)
        for (int ki = -1; ki <= 1; ++ki) {
          int fi = 2 * I + ki, fj = wrapj(2 * J + kj, nyrf);
          double wk = pw(ki) * pw(kj);
          for (int lj = -1; lj <= 1; ++lj)
            for (int li = -1; li <= 1; ++li) {
              double a = fine_entry(&Af, fi, fj, li, lj);
              /* offset of l from 2I in fine units; l is interpolated from the coarse
                 nodes I + o with o = floor/ceil of (ki+li)/2, (kj+lj)/2 */
              int dxl = ki + li, dyl = kj + lj; /* in -2..2 */
              for (int oj = -1; oj <= 1; ++oj)
                for (int oi = -1; oi <= 1; ++oi) {
                  double wl = pw(dxl - 2 * oi) * pw(dyl - 2 * oj);
                  if (wl == 0.0) continue;
                  row[oi + 1][oj + 1] += 0.25 * wk * a * wl;
                }
            }
        }
      cD[K] = row[1][1];
      cE[K] = row[2][1];
      cN[K] = row[1][2];
      cNE[K] = row[2][2];
      cNW[K] = row[0][2];
    }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Coarsest level: dense Cholesky of the unknown-unknown block                 */
/* ------------------------------------------------------------------------ */
/* Unknown numbering: lexicographic over unknowns (i fastest). */
static int unknown_index(const op_t *A, int i, int j) {
  int ui = i - 1;
  int uj = A->periodic ? j : j - 1;
  return ui + (A->nx - 2) * uj;
}

static int n_unknowns(const op_t *A) {
  int rows = A->periodic ? A->nyr : A->ny - 2;
  return (A->nx - 2) * rows;
}

/* Build the dense SPD matrix M (m x m, row-major) of the unknowns. */
static void dense_matrix(const op_t *A, double *M) {
  int m = n_unknowns(A);
  memset(M, 0, sizeof(double) * (size_t)m * m);
  for (int j = 0; j < A->nyr; ++j)
    for (int i = 0; i < A->nx; ++i) {
      if (!is_interior(i, j, A->nx, A->ny, A->periodic)) continue;
      int p = unknown_index(A, i, j);
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          int ni = i + di, nj = j + dj;
          if (A->periodic) nj = wrapj(nj, A->nyr);
          if (!is_interior(ni, nj, A->nx, A->ny, A->periodic)) continue;
          int q = unknown_index(A, ni, nj);
          M[(size_t)p * m + q] += fine_entry(A, i, j, di, dj);
        }
    }
}

/* In-place Cholesky M = L L^T (lower triangle kept). */
static int cholesky(double *M, int m) {
  for (int c = 0; c < m; ++c) {
    double d = M[(size_t)c * m + c];
    for (int k = 0; k < c; ++k) d -= M[(size_t)c * m + k] * M[(size_t)c * m + k];
    if (!(d > 0)) return ORC_ERR_NOT_SPD;
    d = sqrt(d);
    M[(size_t)c * m + c] = d;
    for (int r = c + 1; r < m; ++r) {
      double s = M[(size_t)r * m + c];
      for (int k = 0; k < c; ++k) s -= M[(size_t)r * m + k] * M[(size_t)c * m + k];
      M[(size_t)r * m + c] = s / d;
    }
  }
  return ORC_OK;
}

static void cholesky_solve(const double *L, int m, double *x) {
  for (int r = 0; r < m; ++r) {
    double s = x[r];
    for (int k = 0; k < r; ++k) s -= L[(size_t)r * m + k] * x[k];
    x[r] = s / L[(size_t)r * m + r];
  }
  for (int r = m - 1; r >= 0; --r) {
    double s = x[r];
    for (int k = r + 1; k < m; ++k) s -= L[(size_t)k * m + r] * x[k];
    x[r] = s / L[(size_t)r * m + r];
  }
}

/* ------------------------------------------------------------------------ */
/* Hierarchy and multigrid cycle (Sec. 3, Eqs. 19-24)                          */
/* ------------------------------------------------------------------------ */
typedef struct {
  int nx, ny, nyr;
  double *cE, *cN, *cNE, *cNW, *diag;
  double *phi, *b, *r;
} level_t;

typedef struct {
  int nlev, periodic;
  level_t lev[24];
  double *chol; /* coarsest dense factor */
  int m;        /* coarsest unknown count */
  int smoother; /* 0 = four-colour GS, 1 = weighted Jacobi */
  int nu1, nu2;
  double omega_j;
} hier_t;

static op_t op_of(const hier_t *H, int l) {
  const level_t *L = &H->lev[l];
  op_t A = {L->nx, L->ny, L->nyr, H->periodic, L->cE, L->cN, L->cNE, L->cNW, L->diag};
  return A;
}

static int level_unknowns(int nx, int ny, int periodic) {
  return (nx - 2) * (periodic ? ny - 1 : ny - 2);
}

/* Number of levels: coarsen (nx, ny) -> ((nx-1)/2+1, (ny-1)/2+1) while both
 * n-1 are even, the coarse grid still has unknowns in both directions, and the
 * current level has more than coarse_max unknowns. */
int orc_num_levels(int nx, int ny, int periodic, int coarse_max) {
  int L = 1;
  while (1) {
    if (level_unknowns(nx, ny, periodic) <= coarse_max) break;
    if ((nx - 1) % 2 || (ny - 1) % 2) break;
    int nxc = (nx - 1) / 2 + 1, nyc = (ny - 1) / 2 + 1;
    if (nxc < 3 || nyc < 3) break;
    if (periodic && nyc - 1 < 2) break;
    nx = nxc;
    ny = nyc;
    ++L;
    if (L >= 24) break;
  }
  return L;
}

static void *xcalloc(size_t n) { return calloc(n ? n : 1, sizeof(double)); }

static void hier_free(hier_t *H) {
  for (int l = 0; l < H->nlev; ++l) {
    level_t *L = &H->lev[l];
    free(L->cE); free(L->cN); free(L->cNE); free(L->cNW); free(L->diag);
    free(L->phi); free(L->b); free(L->r);
  }
  free(H->chol);
}

/* Build the hierarchy from fine-level couplings (copied). */
static int hier_build(hier_t *H, int nx, int ny, int periodic, const double *cE, const double *cN,
                      const double *cNE, const double *cNW, const double *diag, int coarse_max) {
  memset(H, 0, sizeof(*H));
  H->periodic = periodic;
  H->nlev = orc_num_levels(nx, ny, periodic, coarse_max);
  for (int l = 0; l < H->nlev; ++l) {
    level_t *L = &H->lev[l];
    L->nx = nx;
    L->ny = ny;
    L->nyr = periodic ? ny - 1 : ny;
    size_t n = (size_t)L->nx * L->nyr;
    L->cE = xcalloc(n); L->cN = xcalloc(n); L->cNE = xcalloc(n); L->cNW = xcalloc(n);
    L->diag = xcalloc(n); L->phi = xcalloc(n); L->b = xcalloc(n); L->r = xcalloc(n);
    if (l == 0) {
      memcpy(L->cE, cE, n * sizeof(double)); memcpy(L->cN, cN, n * sizeof(double));
      memcpy(L->cNE, cNE, n * sizeof(double)); memcpy(L->cNW, cNW, n * sizeof(double));
      memcpy(L->diag, diag, n * sizeof(double));
    } else {
      level_t *F = &H->lev[l - 1];
      orc_galerkin(F->nx, F->ny, periodic, F->cE, F->cN, F->cNE, F->cNW, F->diag, L->cE, L->cN,
                   L->cNE, L->cNW, L->diag);
    }
    nx = (nx - 1) / 2 + 1;
    ny = (ny - 1) / 2 + 1;
  }
  op_t Ac = op_of(H, H->nlev - 1);
  H->m = n_unknowns(&Ac);
  H->chol = xcalloc((size_t)H->m * H->m);
  dense_matrix(&Ac, H->chol);
  return cholesky(H->chol, H->m);
}

static void coarse_solve(hier_t *H) {
  int l = H->nlev - 1;
  level_t *L = &H->lev[l];
  op_t A = op_of(H, l);
  double *x = xcalloc(H->m);
  for (int j = 0; j < L->nyr; ++j)
    for (int i = 0; i < L->nx; ++i)
      if (is_interior(i, j, L->nx, L->ny, H->periodic))
        x[unknown_index(&A, i, j)] = L->b[(size_t)i + (size_t)L->nx * j];
  cholesky_solve(H->chol, H->m, x);
  for (int j = 0; j < L->nyr; ++j)
    for (int i = 0; i < L->nx; ++i) {
      size_t k = (size_t)i + (size_t)L->nx * j;
      L->phi[k] = is_interior(i, j, L->nx, L->ny, H->periodic) ? x[unknown_index(&A, i, j)] : 0.0;
    }
  free(x);
}

static void smooth(hier_t *H, int l, int sweeps, int reverse) {
  op_t A = op_of(H, l);
  level_t *L = &H->lev[l];
  if (H->smoother == 1) jacobi(&A, L->phi, L->b, L->r, sweeps, H->omega_j);
  else if (H->smoother == 2) xline(&A, L->phi, L->b, sweeps, reverse);
  else gs4(&A, L->phi, L->b, sweeps, reverse);
}

/* One V(nu1, nu2) cycle on level l: smooth, residual (Eq. 20), restrict (r_H = I_h^H r_h),
 * solve the coarse correction equation (Eq. 23) recursively, prolong and add (Eq. 24),
 * smooth again. */
static void vcycle(hier_t *H, int l) {
  if (l == H->nlev - 1) {
    coarse_solve(H);
    return;
  }
  level_t *L = &H->lev[l], *C = &H->lev[l + 1];
  op_t A = op_of(H, l), Ac = op_of(H, l + 1);
  smooth(H, l, H->nu1, 0);
  residual(&A, L->phi, L->b, L->r);
  restrict_fw(&A, L->r, &Ac, C->b);
  memset(C->phi, 0, sizeof(double) * (size_t)C->nx * C->nyr);
  vcycle(H, l + 1);
  prolong_add(&Ac, C->phi, &A, L->phi);
  smooth(H, l, H->nu2, 1);
}

static double norm2_unknowns(const op_t *A, const double *v) {
  double s = 0.0;
  for (int j = 0; j < A->nyr; ++j)
    for (int i = 0; i < A->nx; ++i)
      if (is_interior(i, j, A->nx, A->ny, A->periodic)) {
        double x = v[(size_t)i + (size_t)A->nx * j];
        s += x * x;
      }
  return sqrt(s);
}

/*
 * Solve A phi = b on the fine level by V(nu1, nu2) cycles.
 * phi: in = initial guess with Dirichlet values in its boundary ring, out = solution.
 * Stops when ||r||_2 / ||r_0||_2 <= rtol (r_0 = residual of the initial guess with zero
 * unknowns, i.e. b with the Dirichlet data moved in), or after max_cycles, or - if
 * stagnate > 0 - when the residual has not decreased for `stagnate` cycles in a row.
 * hist (max_cycles + 1 entries, nullable) receives the relative residual before each cycle.
 * Returns the number of cycles run (negative on error).
 */
int orc_solve(int nx, int ny, int periodic, const double *cE, const double *cN,
              const double *cNE, const double *cNW, const double *diag, const double *b,
              double *phi, int smoother, int nu1, int nu2, double omega_j, int coarse_max,
              double rtol, int max_cycles, int stagnate, double *hist) {
  hier_t H;
  int rc = hier_build(&H, nx, ny, periodic, cE, cN, cNE, cNW, diag, coarse_max);
  if (rc) {
    hier_free(&H);
    return -rc;
  }
  H.smoother = smoother;
  H.nu1 = nu1;
  H.nu2 = nu2;
  H.omega_j = omega_j;
  level_t *L = &H.lev[0];
  op_t A = op_of(&H, 0);
  size_t n = (size_t)L->nx * L->nyr;
  memcpy(L->b, b, n * sizeof(double));
  memcpy(L->phi, phi, n * sizeof(double));
  /* reference norm: residual with the unknowns set to zero */
  double *z = xcalloc(n);
  memcpy(z, phi, n * sizeof(double));
  for (int j = 0; j < L->nyr; ++j)
    for (int i = 0; i < L->nx; ++i)
      if (is_interior(i, j, L->nx, L->ny, periodic)) z[(size_t)i + (size_t)L->nx * j] = 0.0;
  residual(&A, z, L->b, L->r);
  double r0 = norm2_unknowns(&A, L->r);
  free(z);
  if (r0 == 0.0) r0 = 1.0;
  int cyc = 0, since_best = 0;
  double best = INFINITY;
  while (1) {
    residual(&A, L->phi, L->b, L->r);
    double rel = norm2_unknowns(&A, L->r) / r0;
    if (hist) hist[cyc] = rel;
    if (rel <= rtol || cyc >= max_cycles) break;
    if (stagnate > 0) {
      if (rel < best) {
        best = rel;
        since_best = 0;
      } else if (++since_best >= stagnate) {
        break;
      }
    }
    vcycle(&H, 0);
    ++cyc;
  }
  memcpy(phi, L->phi, n * sizeof(double));
  hier_free(&H);
  return cyc;
}

/* ------------------------------------------------------------------------ */
/* Single-step entry points (for per-kernel comparisons)                       */
/* ------------------------------------------------------------------------ */
int orc_residual(int nx, int ny, int periodic, const double *cE, const double *cN,
                 const double *cNE, const double *cNW, const double *diag, const double *phi,
                 const double *b, double *r) {
  op_t A = {nx, ny, periodic ? ny - 1 : ny, periodic, cE, cN, cNE, cNW, diag};
  residual(&A, phi, b, r);
  return ORC_OK;
}

int orc_smooth(int nx, int ny, int periodic, const double *cE, const double *cN,
               const double *cNE, const double *cNW, const double *diag, double *phi,
               const double *b, int smoother, int sweeps, int reverse, double omega_j) {
  op_t A = {nx, ny, periodic ? ny - 1 : ny, periodic, cE, cN, cNE, cNW, diag};
  if (smoother == 1) {
    double *tmp = xcalloc((size_t)nx * A.nyr);
    jacobi(&A, phi, b, tmp, sweeps, omega_j);
    free(tmp);
  } else if (smoother == 2) {
    xline(&A, phi, b, sweeps, reverse);
  } else if (smoother == 3) {
    sor4(&A, phi, b, sweeps, omega_j);
  } else {
    gs4(&A, phi, b, sweeps, reverse);
  }
  return ORC_OK;
}

/* One half-sweep of zebra x-line Gauss-Seidel on the rows of parity par only. */
int orc_line_rows(int nx, int ny, int periodic, const double *cE, const double *cN,
                  const double *cNE, const double *cNW, const double *diag, double *phi,
                  const double *b, int par) {
  op_t A = {nx, ny, periodic ? ny - 1 : ny, periodic, cE, cN, cNE, cNW, diag};
  line_rows(&A, phi, b, par);
  return ORC_OK;
}

/* One colour phase only (colour index into the forward order). */
int orc_gs_colour(int nx, int ny, int periodic, const double *cE, const double *cN,
                  const double *cNE, const double *cNW, const double *diag, double *phi,
                  const double *b, int colour) {
  op_t A = {nx, ny, periodic ? ny - 1 : ny, periodic, cE, cN, cNE, cNW, diag};
  gs_colour(&A, phi, b, COLOUR_ORDER[colour][0], COLOUR_ORDER[colour][1]);
  return ORC_OK;
}

int orc_restrict(int nxf, int nyf, int periodic, const double *r, double *bH) {
  int nxc = (nxf - 1) / 2 + 1, nyc = (nyf - 1) / 2 + 1;
  op_t Af = {nxf, nyf, periodic ? nyf - 1 : nyf, periodic, 0, 0, 0, 0, 0};
  op_t Ac = {nxc, nyc, periodic ? nyc - 1 : nyc, periodic, 0, 0, 0, 0, 0};
  restrict_fw(&Af, r, &Ac, bH);
  return ORC_OK;
}

/* Rediscretized coarse levels (the alternative to the Galerkin product): a nodal field f of
 * the fine grid (the tensor components eps_xx, eps_xy, eps_yy) at the coarse nodes, full
 * weighting (1/16)[1 2 1; 2 4 2; 1 2 1] about the coincident fine node (2I, 2J) at coarse nodes
 * whose eight fine neighbours exist (rows wrap when periodic), and injection (the coincident
 * fine value) on the coarse boundary ring.  The coarse operator is then assembled from the
 * coarsened tensor on the coarse grid (spacing 2h) exactly as the fine one (orc_assemble). */
int orc_coarsen_nodal(int nxf, int nyf, int periodic, const double *f, double *fc) {
  const int nxc = (nxf - 1) / 2 + 1, nyc = (nyf - 1) / 2 + 1;
  const int nyrf = periodic ? nyf - 1 : nyf, nyrc = periodic ? nyc - 1 : nyc;
  for (int J = 0; J < nyrc; ++J)
    for (int I = 0; I < nxc; ++I) {
      const int fi = 2 * I, fj = 2 * J;
      const int inner_x = I >= 1 && I <= nxc - 2;
      const int inner_y = periodic || (J >= 1 && J <= nyc - 2);
      double v;
      if (inner_x && inner_y) {
        const int jd = fj == 0 ? nyrf - 1 : fj - 1, ju = fj + 1 == nyrf ? 0 : fj + 1;
        const double *r0 = f + (size_t)nxf * fj, *rd = f + (size_t)nxf * jd, *ru = f + (size_t)nxf * ju;
        v = (4.0 * r0[fi] + 2.0 * (r0[fi - 1] + r0[fi + 1] + rd[fi] + ru[fi]) +
             (rd[fi - 1] + rd[fi + 1] + ru[fi - 1] + ru[fi + 1])) / 16.0;
      } else {
        v = f[(size_t)nxf * fj + fi];
      }
      fc[(size_t)nxc * J + I] = v;
    }
  return ORC_OK;
}

int orc_prolong_add(int nxf, int nyf, int periodic, const double *eH, double *phi) {
  int nxc = (nxf - 1) / 2 + 1, nyc = (nyf - 1) / 2 + 1;
  op_t Af = {nxf, nyf, periodic ? nyf - 1 : nyf, periodic, 0, 0, 0, 0, 0};
  op_t Ac = {nxc, nyc, periodic ? nyc - 1 : nyc, periodic, 0, 0, 0, 0, 0};
  prolong_add(&Ac, eH, &Af, phi);
  return ORC_OK;
}

/* Dense solve of A x = b on one level (x, b node arrays; Dirichlet nodes of x = 0). */
int orc_dense_solve(int nx, int ny, int periodic, const double *cE, const double *cN,
                    const double *cNE, const double *cNW, const double *diag, const double *b,
                    double *x) {
  op_t A = {nx, ny, periodic ? ny - 1 : ny, periodic, cE, cN, cNE, cNW, diag};
  int m = n_unknowns(&A);
  double *M = xcalloc((size_t)m * m), *v = xcalloc(m);
  dense_matrix(&A, M);
  int rc = cholesky(M, m);
  if (!rc) {
    for (int j = 0; j < A.nyr; ++j)
      for (int i = 0; i < nx; ++i)
        if (is_interior(i, j, nx, ny, periodic))
          v[unknown_index(&A, i, j)] = b[(size_t)i + (size_t)nx * j];
    cholesky_solve(M, m, v);
    for (int j = 0; j < A.nyr; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t k = (size_t)i + (size_t)nx * j;
        x[k] = is_interior(i, j, nx, ny, periodic) ? v[unknown_index(&A, i, j)] : 0.0;
      }
  }
  free(M);
  free(v);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* The paper's own update, Eq. 18, taken literally (non-symmetric operator)    */
/* ------------------------------------------------------------------------ */
/*
 * Lexicographic SOR sweeps with the k1..k6 coefficients of Eq. 18, read as the
 * Gauss-Seidel row update  phi_new = (k1 phi_E + k3 phi_W + k4 phi_N + k5 phi_S
 *   + k6 (phi_NE - phi_NW - phi_SE + phi_SW) + rho) / k2,
 * i.e. with every term divided by k2 (the printed equation divides only rho) and
 * the right-hand-side sign of Eq. 17.  i is the inner (fast) index.  Then
 * phi = phi_old + omega (phi_new - phi_old) (Sec. 2.1).  Used for the paper-operator
 * consistency check and as the SOR reference (omega = 1.875, tol 1e-10, Sec. 4).
 * Dirichlet non-periodic grids only.  Returns sweeps run; tol applies to
 * max |phi_new - phi_old|.
 */
/*
 * Four-colour SOR on A phi = b until ||r||_2 / ||r_0||_2 <= rtol (r_0 as in orc_solve),
 * checked every `check` sweeps, or max_sweeps.  hist (nullable, max_sweeps / check + 1
 * entries) receives the relative residual at every check.  Returns the sweeps run.
 */
int orc_sor_solve(int nx, int ny, int periodic, const double *cE, const double *cN,
                  const double *cNE, const double *cNW, const double *diag, const double *b,
                  double *phi, double omega, double rtol, int max_sweeps, int check, double *hist) {
  op_t A = {nx, ny, periodic ? ny - 1 : ny, periodic, cE, cN, cNE, cNW, diag};
  size_t n = (size_t)nx * A.nyr;
  double *z = xcalloc(n), *r = xcalloc(n);
  memcpy(z, phi, n * sizeof(double));
  for (int j = 0; j < A.nyr; ++j)
    for (int i = 0; i < nx; ++i)
      if (is_interior(i, j, nx, ny, periodic)) z[(size_t)i + (size_t)nx * j] = 0.0;
  residual(&A, z, b, r);
  double r0 = norm2_unknowns(&A, r);
  if (r0 == 0.0) r0 = 1.0;
  int sweeps = 0, q = 0;
  if (check < 1) check = 1;
  while (1) {
    residual(&A, phi, b, r);
    double rel = norm2_unknowns(&A, r) / r0;
    if (hist) hist[q] = rel;
    ++q;
    if (rel <= rtol || sweeps >= max_sweeps) break;
    sor4(&A, phi, b, check, omega);
    sweeps += check;
  }
  free(z);
  free(r);
  return sweeps;
}

int orc_paper_sor(int nx, int ny, double hx, double hy, const double *exx, const double *exy,
                  const double *eyy, const double *rho, double *phi, double omega, double tol,
                  int max_sweeps) {
  double dx2 = hx * hx, dy2 = hy * hy, dxy = hx * hy;
  int it;
  for (it = 0; it < max_sweeps; ++it) {
    double change = 0.0;
    for (int j = 1; j < ny - 1; ++j)
      for (int i = 1; i < nx - 1; ++i) {
        size_t k = (size_t)i + (size_t)nx * j;
        size_t ke = k + 1, kw = k - 1, kn = k + nx, ks = k - nx;
        double k2 = 2.0 * (exx[k] / dx2 + eyy[k] / dy2);
        double k1 = exx[k] / dx2 + (exx[ke] - exx[kw]) / (4 * dx2) + (exy[kn] - exy[ks]) / (4 * dxy);
        double k3 = exx[k] / dx2 - (exx[ke] - exx[kw]) / (4 * dx2) - (exy[kn] - exy[ks]) / (4 * dxy);
        double k4 = eyy[k] / dy2 + (eyy[kn] - eyy[ks]) / (4 * dy2) + (exy[ke] - exy[kw]) / (4 * dxy);
        double k5 = eyy[k] / dy2 - (eyy[kn] - eyy[ks]) / (4 * dy2) - (exy[ke] - exy[kw]) / (4 * dxy);
        double k6 = exy[k] / (2 * dxy);
        double nw = k1 * phi[ke] + k3 * phi[kw] + k4 * phi[kn] + k5 * phi[ks] +
                    k6 * (phi[kn + 1] - phi[kn - 1] - phi[ks + 1] + phi[ks - 1]) + rho[k];
        nw /= k2;
        double d = nw - phi[k];
        phi[k] += omega * d;
        if (fabs(d) > change) change = fabs(d);
      }
    if (change <= tol) return it + 1;
  }
  return it;
}

/* ------------------------------------------------------------------------ */
/* Multigrid as a preconditioner; preconditioned conjugate gradients          */
/* ------------------------------------------------------------------------ */
/* Opaque hierarchy for repeated V-cycles on the same operator. */
void *orc_hier_create(int nx, int ny, int periodic, const double *cE, const double *cN,
                      const double *cNE, const double *cNW, const double *diag, int smoother,
                      int nu1, int nu2, double omega_j, int coarse_max) {
  hier_t *H = (hier_t *)calloc(1, sizeof(hier_t));
  if (hier_build(H, nx, ny, periodic, cE, cN, cNE, cNW, diag, coarse_max)) {
    hier_free(H);
    free(H);
    return NULL;
  }
  H->smoother = smoother;
  H->nu1 = nu1;
  H->nu2 = nu2;
  H->omega_j = omega_j;
  return H;
}

void orc_hier_free(void *h) {
  if (!h) return;
  hier_free((hier_t *)h);
  free(h);
}

/* z = one V-cycle applied to A z = r from z = 0 (the multigrid preconditioner B r). */
void orc_hier_vcycle(void *h, const double *r, double *z) {
  hier_t *H = (hier_t *)h;
  level_t *L = &H->lev[0];
  size_t n = (size_t)L->nx * L->nyr;
  memcpy(L->b, r, n * sizeof(double));
  memset(L->phi, 0, n * sizeof(double));
  vcycle(H, 0);
  memcpy(z, L->phi, n * sizeof(double));
}

static double dot_unknowns(const op_t *A, const double *u, const double *v) {
  double s = 0.0;
  for (int j = 0; j < A->nyr; ++j)
    for (int i = 0; i < A->nx; ++i)
      if (is_interior(i, j, A->nx, A->ny, A->periodic)) {
        size_t k = (size_t)i + (size_t)A->nx * j;
        s += u[k] * v[k];
      }
  return s;
}

/* A u at unknowns with u = 0 on Dirichlet nodes. */
static void apply_A(const op_t *A, const double *u, double *out) {
  for (int j = 0; j < A->nyr; ++j)
    for (int i = 0; i < A->nx; ++i) {
      size_t k = (size_t)i + (size_t)A->nx * j;
      out[k] = is_interior(i, j, A->nx, A->ny, A->periodic)
                   ? A->diag[k] * u[k] + offdiag_row(A, u, i, j) : 0.0;
    }
}

/*
 * Conjugate gradients on the unknowns, preconditioned by one V-cycle per iteration
 * (symmetric cycle: the colour order after the correction is the reverse of the one
 * before it, R = P^T / 4, Galerkin coarse operators, exact coarsest solve).
 * phi: in = initial guess with Dirichlet values in the boundary ring, out = solution.
 * Same stopping rules and history convention as orc_solve.
 */
int orc_pcg_solve(int nx, int ny, int periodic, const double *cE, const double *cN,
                  const double *cNE, const double *cNW, const double *diag, const double *b,
                  double *phi, int smoother, int nu1, int nu2, double omega_j, int coarse_max,
                  double rtol, int max_iters, int stagnate, double *hist) {
  hier_t *H = (hier_t *)orc_hier_create(nx, ny, periodic, cE, cN, cNE, cNW, diag, smoother, nu1,
                                        nu2, omega_j, coarse_max);
  if (!H) return -ORC_ERR_NOT_SPD;
  op_t A = op_of(H, 0);
  size_t n = (size_t)nx * A.nyr;
  double *r = xcalloc(n), *z = xcalloc(n), *p = xcalloc(n), *q = xcalloc(n), *z0 = xcalloc(n);
  memcpy(z0, phi, n * sizeof(double));
  for (int j = 0; j < A.nyr; ++j)
    for (int i = 0; i < nx; ++i)
      if (is_interior(i, j, nx, ny, periodic)) z0[(size_t)i + (size_t)nx * j] = 0.0;
  residual(&A, z0, b, r);
  double r0 = norm2_unknowns(&A, r);
  if (r0 == 0.0) r0 = 1.0;
  residual(&A, phi, b, r);
  double *rt = xcalloc(n);
  double rz = 0.0, best = INFINITY;
  int it = 0, since_best = 0;
  while (1) {
    /* stopping test on the true residual b - A phi (the recursively updated r drifts
       away from it once it reaches rounding level) */
    residual(&A, phi, b, rt);
    double rel = norm2_unknowns(&A, rt) / r0;
    if (hist) hist[it] = rel;
    if (rel <= rtol || it >= max_iters) break;
    if (stagnate > 0) {
      if (rel < best) {
        best = rel;
        since_best = 0;
      } else if (++since_best >= stagnate) {
        break;
      }
    }
    orc_hier_vcycle(H, r, z);
    double rz_new = dot_unknowns(&A, r, z);
    if (!(rz_new > 0.0) || !isfinite(rz_new)) break; /* breakdown at rounding level */
    if (it == 0) {
      memcpy(p, z, n * sizeof(double));
    } else {
      double beta = rz_new / rz;
      for (size_t k = 0; k < n; ++k) p[k] = z[k] + beta * p[k];
    }
    rz = rz_new;
    apply_A(&A, p, q);
    double pq = dot_unknowns(&A, p, q);
    if (!(pq > 0.0) || !isfinite(pq)) break;
    double alpha = rz / pq;
    for (int j = 0; j < A.nyr; ++j)
      for (int i = 0; i < nx; ++i)
        if (is_interior(i, j, nx, ny, periodic)) {
          size_t k = (size_t)i + (size_t)nx * j;
          phi[k] += alpha * p[k];
          r[k] -= alpha * q[k];
        }
    ++it;
  }
  free(r); free(z); free(p); free(q); free(z0); free(rt);
  orc_hier_free(H);
  return it;
}

/* ------------------------------------------------------------------------------------
 * Numerical grid generation with internal Dirichlet nodes (Sec. 4.2, Eqs. 36-37).
 * The coordinate x' (or y') is discrete-harmonic for the operator given (the identity
 * map's 5-point Laplacian) at every free unknown; at unknowns with fixed[k] != 0 it equals
 * v[k].  Rewrites the system so that the solver can treat every unknown alike: b[k] = v[k]
 * and row k = e_k at fixed unknowns; at free unknowns b[k] = -(sum over fixed unknown
 * neighbours m of A_km v[m]); every matrix entry between a fixed unknown and any other
 * node is set to zero (the matrix stays symmetric).  Boundary-ring couplings of free nodes
 * are kept: the ring carries its own Dirichlet values in phi.
 * ------------------------------------------------------------------------------------ */
void orc_mask_dirichlet(int nx, int ny, int periodic, double *cE, double *cN, double *cNE,
                        double *cNW, double *diag, const unsigned char *fixed, const double *v,
                        double *b) {
  const int nyr = periodic ? ny - 1 : ny;
  /* neighbour offsets and where the coupling to it is stored: (di, dj, array, storing node) */
  for (int j = 0; j < nyr; ++j)
    for (int i = 0; i < nx; ++i) {
      const size_t k = (size_t)i + (size_t)nx * j;
      b[k] = 0.0;
      if (!is_interior(i, j, nx, ny, periodic)) continue;
      if (fixed[k]) {
        b[k] = v[k];
        continue;
      }
      double s = 0.0;
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          if (di == 0 && dj == 0) continue;
          int jj = j + dj, ii = i + di;
          if (periodic) jj = (jj + nyr) % nyr;
          if (!is_interior(ii, jj, nx, ny, periodic)) continue;
          const size_t m = (size_t)ii + (size_t)nx * jj;
          if (!fixed[m]) continue;
          /* the entry A_km: stored at k for E, N, NE, NW; at m for W, S, SW, SE */
          double c;
          if (dj == 0) c = (di > 0) ? cE[k] : cE[m];
          else if (di == 0) c = (dj > 0) ? cN[k] : cN[m];
          else if (di == dj) c = (dj > 0) ? cNE[k] : cNE[m];
          else c = (dj > 0) ? cNW[k] : cNW[m];
          s += c * v[m];
        }
      b[k] = -s;
    }
  /* remove every entry that touches a fixed unknown; identity rows there */
  for (int j = 0; j < nyr; ++j)
    for (int i = 0; i < nx; ++i) {
      const size_t k = (size_t)i + (size_t)nx * j;
      const int kf = is_interior(i, j, nx, ny, periodic) && fixed[k];
      int ju = j + 1;
      int has_up = 1;
      if (ju == nyr) {
        if (periodic) ju = 0;
        else has_up = 0;
      }
      const size_t ke = k + 1, kn = (size_t)i + (size_t)nx * ju;
      if (i + 1 < nx && (kf || (is_interior(i + 1, j, nx, ny, periodic) && fixed[ke]))) cE[k] = 0.0;
      if (has_up) {
        if (kf || (is_interior(i, ju, nx, ny, periodic) && fixed[kn])) cN[k] = 0.0;
        if (i + 1 < nx && (kf || (is_interior(i + 1, ju, nx, ny, periodic) && fixed[kn + 1])))
          cNE[k] = 0.0;
        if (i >= 1 && (kf || (is_interior(i - 1, ju, nx, ny, periodic) && fixed[kn - 1]))) cNW[k] = 0.0;
      }
      if (kf) diag[k] = 1.0;
    }
}
