"""FP64 CPU oracle for the transformed-coefficient multigrid solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The product
path (the CUDA library and its Python binding) never imports it and never falls
back to it.  It shares no code with the CUDA path; the only common module is the
seeded input generator ``paper_2602_01888_gb300.inputs``, which holds no solver
arithmetic.

The arithmetic lives in ``mg_oracle.c`` (plain FP64 loops, one function per paper
equation or step); this module compiles it with gcc, loads it with ctypes and adds
numpy glue plus the paper's error norms (Eqs. 25-27).

Pins (checked by ``tests/test_oracle_*.py`` against things other than the oracle
itself): identity map -> textbook 5-point Laplacian; det(eps) = 1 for eps' = I;
closed-form polar tensor; O(h^2) agreement of the central-difference and analytic
tensors; exact symmetry and zero row sums; exact solutions for quadratics under
affine maps; agreement with an independently assembled dense solve; Galerkin
operator equal to a sparse-matrix triple product built independently; the
adjoint relation R = P^T/4; the Gauss-Seidel colour-phase property; second-order
convergence on manufactured and paper validation solutions (Sec. 4).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, replace
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_handle = None

SMOOTHER_GS4 = 0
SMOOTHER_JACOBI = 1
SMOOTHER_XLINE = 2  # zebra x-line Gauss-Seidel
SMOOTHER_SOR4 = 3   # four-colour SOR (single-level iteration; factor in omega_j)
DEFAULT_COARSE_MAX = 64


def build(force: bool = False) -> str:
    """Compile mg_oracle.c into liboracle.so (plain, portable C; no FMA contraction)."""
    with _lock:
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
            return _SO
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
        return _SO


def lib():
    global _handle
    if _handle is None:
        build()
        h = ctypes.CDLL(_SO)
        D = ctypes.POINTER(ctypes.c_double)
        i, d, sz = ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        sigs = {
            "orc_jacobian_analytic": [i, D, i, i, d, d, d, d, D, D, D, D],
            "orc_jacobian_grid": [i, i, i, d, d, D, D, d, d, D, D, D, D],
            "orc_eps": [sz, D, D, D, D, D, D, D, D, D],
            "orc_assemble": [i, i, i, d, d, D, D, D, D, D, D, D, D],
            "orc_rhs": [i, i, i, D, D, D],
            "orc_galerkin": [i, i, i, D, D, D, D, D, D, D, D, D, D],
            "orc_num_levels": [i, i, i, i],
            "orc_solve": [i, i, i, D, D, D, D, D, D, D, i, i, i, d, i, d, i, i, D],
            "orc_residual": [i, i, i, D, D, D, D, D, D, D, D],
            "orc_smooth": [i, i, i, D, D, D, D, D, D, D, i, i, i, d],
            "orc_gs_colour": [i, i, i, D, D, D, D, D, D, D, i],
            "orc_restrict": [i, i, i, D, D],
            "orc_coarsen_nodal": [i, i, i, D, D],
            "orc_prolong_add": [i, i, i, D, D],
            "orc_dense_solve": [i, i, i, D, D, D, D, D, D, D],
            "orc_paper_sor": [i, i, d, d, D, D, D, D, D, d, d, i],
            "orc_pcg_solve": [i, i, i, D, D, D, D, D, D, D, i, i, i, d, i, d, i, i, D],
            "orc_line_rows": [i, i, i, D, D, D, D, D, D, D, i],
            "orc_sor_solve": [i, i, i, D, D, D, D, D, D, D, d, d, i, i, D],
            "orc_mask_dirichlet": [i, i, i, D, D, D, D, D, ctypes.POINTER(ctypes.c_ubyte), D, D],
            "orc_hier_free": [ctypes.c_void_p],
            "orc_hier_vcycle": [ctypes.c_void_p, D, D],
        }
        for name, args in sigs.items():
            f = getattr(h, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        h.orc_hier_create.argtypes = [i, i, i, D, D, D, D, D, i, i, i, d, i]
        h.orc_hier_create.restype = ctypes.c_void_p
        h.orc_hier_free.restype = None
        h.orc_hier_vcycle.restype = None
        h.orc_mask_dirichlet.restype = None
        _handle = h
    return _handle


def _p(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle arrays are C-contiguous float64"
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


MAP_CODES = {"identity": 0, "sine_warp": 1, "polar": 2, "sinh": 3, "affine": 4}


# ---------------------------------------------------------------- coefficient build
def jacobian(grid, mapspec):
    """(Jxx, Jxy, Jyx, Jyy) at every stored node: analytic derivatives of the map, or
    central differences of the mapped grid (Eqs. 39-42)."""
    out = [np.zeros(grid.shape) for _ in range(4)]
    if mapspec.kind == "grid":
        xp, yp = _f64(mapspec.xp), _f64(mapspec.yp)
        rc = lib().orc_jacobian_grid(grid.nx, grid.ny, int(grid.periodic_y), grid.hx, grid.hy,
                                     _p(xp), _p(yp), float(mapspec.jump[0]), float(mapspec.jump[1]),
                                     *[_p(a) for a in out])
    else:
        prm = _f64(list(mapspec.params) + [0.0] * 4)
        rc = lib().orc_jacobian_analytic(MAP_CODES[mapspec.kind], _p(prm), grid.nx, grid.nyr,
                                         grid.x0, grid.y0, grid.hx, grid.hy, *[_p(a) for a in out])
    if rc:
        raise RuntimeError(f"oracle jacobian failed ({rc})")
    return tuple(out)


def eps_tensor(J, eps_phys=None):
    """(D, exx, exy, eyy): det J and the computational-domain tensor, Eqs. 10, 12-15."""
    Jxx, Jxy, Jyx, Jyy = (_f64(a) for a in J)
    shape = Jxx.shape
    D, exx, exy, eyy = (np.zeros(shape) for _ in range(4))
    ep = None if eps_phys is None else _f64(eps_phys)
    rc = lib().orc_eps(Jxx.size, _p(Jxx), _p(Jxy), _p(Jyx), _p(Jyy), _p(ep), _p(D), _p(exx),
                       _p(exy), _p(eyy))
    return D, exx, exy, eyy, rc


@dataclass
class Operator:
    """One level's operator in symmetric 9-point storage (see mg_oracle.c)."""

    nx: int
    ny: int
    periodic: bool
    cE: np.ndarray
    cN: np.ndarray
    cNE: np.ndarray
    cNW: np.ndarray
    diag: np.ndarray

    @property
    def nyr(self):
        return self.ny - 1 if self.periodic else self.ny

    def arrays(self):
        return (self.cE, self.cN, self.cNE, self.cNW, self.diag)

    def _args(self):
        return (self.nx, self.ny, int(self.periodic)) + tuple(_p(a) for a in self.arrays())


def assemble(grid, exx, exy, eyy) -> Operator:
    arrs = [np.zeros(grid.shape) for _ in range(5)]
    lib().orc_assemble(grid.nx, grid.ny, int(grid.periodic_y), grid.hx, grid.hy, _p(_f64(exx)),
                       _p(_f64(exy)), _p(_f64(eyy)), *[_p(a) for a in arrs])
    return Operator(grid.nx, grid.ny, grid.periodic_y, *arrs)


def rhs(grid, rho_phys, D):
    b = np.zeros(grid.shape)
    lib().orc_rhs(grid.nx, grid.ny, int(grid.periodic_y), _p(_f64(rho_phys)), _p(_f64(D)), _p(b))
    return b


def galerkin(A: Operator) -> Operator:
    nxc, nyc = (A.nx - 1) // 2 + 1, (A.ny - 1) // 2 + 1
    nyrc = nyc - 1 if A.periodic else nyc
    arrs = [np.zeros((nyrc, nxc)) for _ in range(5)]
    rc = lib().orc_galerkin(A.nx, A.ny, int(A.periodic), *[_p(a) for a in A.arrays()],
                            *[_p(a) for a in arrs])
    if rc:
        raise RuntimeError("oracle galerkin: grid not coarsenable")
    return Operator(nxc, nyc, A.periodic, *arrs)


def num_levels(nx, ny, periodic, coarse_max=DEFAULT_COARSE_MAX):
    return lib().orc_num_levels(nx, ny, int(periodic), coarse_max)


def hierarchy(A0: Operator, coarse_max=DEFAULT_COARSE_MAX):
    ops = [A0]
    for _ in range(num_levels(A0.nx, A0.ny, A0.periodic, coarse_max) - 1):
        ops.append(galerkin(ops[-1]))
    return ops


def coarsen_nodal(nxf, nyf, periodic, f):
    """A nodal field at the coarse nodes: full weighting inside, injection on the boundary."""
    nxc, nyc = (nxf - 1) // 2 + 1, (nyf - 1) // 2 + 1
    fc = np.zeros(((nyc - 1) if periodic else nyc, nxc))
    lib().orc_coarsen_nodal(nxf, nyf, int(periodic), _p(_f64(f)), _p(fc))
    return fc


def rediscretized_hierarchy(grid, exx, exy, eyy, coarse_max=DEFAULT_COARSE_MAX):
    """Operators of every level assembled from the tensor coarsened level by level
    (coarsen_nodal) on grids of twice the spacing: the alternative to the Galerkin product.
    The grid is the one the operator lives on (the doubled periodic grid for Neumann sides)."""
    levels = num_levels(grid.nx, grid.ny, grid.periodic_y, coarse_max)
    g, e = grid, (exx, exy, eyy)
    ops = [assemble(g, *e)]
    for _ in range(levels - 1):
        e = tuple(coarsen_nodal(g.nx, g.ny, g.periodic_y, a) for a in e)
        g = replace(g, nx=(g.nx - 1) // 2 + 1, ny=(g.ny - 1) // 2 + 1)
        ops.append(assemble(g, *e))
    return ops


# ---------------------------------------------------------------- single steps
def residual(A: Operator, phi, b):
    r = np.zeros(A.cE.shape)
    lib().orc_residual(*A._args(), _p(_f64(phi)), _p(_f64(b)), _p(r))
    return r


def smooth(A: Operator, phi, b, sweeps=1, reverse=False, smoother=SMOOTHER_GS4, omega_j=0.8):
    out = _f64(phi).copy()
    lib().orc_smooth(*A._args(), _p(out), _p(_f64(b)), smoother, sweeps, int(reverse), omega_j)
    return out


def sor_solve(A: Operator, b, phi0, omega=1.875, rtol=1e-10, max_sweeps=200000, check=16):
    """Four-colour SOR (single-level) to a relative residual rtol, checked every `check`
    sweeps.  Returns (phi, sweeps, history of relative residuals at the checks)."""
    phi = _f64(phi0).copy()
    hist = np.zeros(max_sweeps // max(check, 1) + 2)
    sw = lib().orc_sor_solve(*A._args(), _p(_f64(b)), _p(phi), omega, rtol, max_sweeps, check, _p(hist))
    return phi, sw, hist[:sw // max(check, 1) + 1].copy()


def line_rows(A: Operator, phi, b, parity):
    """One half-sweep of zebra x-line Gauss-Seidel on the rows j with j mod 2 == parity."""
    out = _f64(phi).copy()
    lib().orc_line_rows(*A._args(), _p(out), _p(_f64(b)), parity)
    return out


def gs_colour(A: Operator, phi, b, colour):
    out = _f64(phi).copy()
    lib().orc_gs_colour(*A._args(), _p(out), _p(_f64(b)), colour)
    return out


def restrict(nxf, nyf, periodic, r):
    nxc, nyc = (nxf - 1) // 2 + 1, (nyf - 1) // 2 + 1
    bH = np.zeros(((nyc - 1) if periodic else nyc, nxc))
    lib().orc_restrict(nxf, nyf, int(periodic), _p(_f64(r)), _p(bH))
    return bH


def prolong_add(nxf, nyf, periodic, eH, phi):
    out = _f64(phi).copy()
    lib().orc_prolong_add(nxf, nyf, int(periodic), _p(_f64(eH)), _p(out))
    return out


def dense_solve(A: Operator, b):
    x = np.zeros(A.cE.shape)
    rc = lib().orc_dense_solve(*A._args(), _p(_f64(b)), _p(x))
    if rc:
        raise RuntimeError(f"oracle dense solve failed ({rc}): operator not SPD")
    return x


def solve(A: Operator, b, phi0, rtol=1e-14, max_cycles=200, stagnate=3, smoother=SMOOTHER_GS4,
          nu1=2, nu2=2, omega_j=0.8, coarse_max=DEFAULT_COARSE_MAX):
    """V(nu1, nu2) cycles from phi0 (Dirichlet values in its boundary ring).  Returns
    (phi, cycles, history of relative residuals)."""
    phi = _f64(phi0).copy()
    hist = np.zeros(max_cycles + 1)
    cyc = lib().orc_solve(*A._args(), _p(_f64(b)), _p(phi), smoother, nu1, nu2, omega_j,
                          coarse_max, rtol, max_cycles, stagnate, _p(hist))
    if cyc < 0:
        raise RuntimeError(f"oracle solve failed ({-cyc})")
    return phi, cyc, hist[:cyc + 1].copy()


def pcg_solve(A: Operator, b, phi0, rtol=1e-14, max_iters=200, stagnate=3, smoother=SMOOTHER_GS4,
              nu1=2, nu2=2, omega_j=0.8, coarse_max=DEFAULT_COARSE_MAX):
    """Conjugate gradients preconditioned by one V(nu1, nu2) cycle.  Returns
    (phi, iterations, history of relative residuals)."""
    phi = _f64(phi0).copy()
    hist = np.zeros(max_iters + 1)
    it = lib().orc_pcg_solve(*A._args(), _p(_f64(b)), _p(phi), smoother, nu1, nu2, omega_j,
                             coarse_max, rtol, max_iters, stagnate, _p(hist))
    if it < 0:
        raise RuntimeError(f"oracle pcg failed ({-it})")
    return phi, it, hist[:it + 1].copy()


class Hierarchy:
    """Multigrid hierarchy kept alive for repeated preconditioner applications."""

    def __init__(self, A: Operator, smoother=SMOOTHER_GS4, nu1=2, nu2=2, omega_j=0.8,
                 coarse_max=DEFAULT_COARSE_MAX):
        self.A = A
        self._h = lib().orc_hier_create(*A._args(), smoother, nu1, nu2, omega_j, coarse_max)
        if not self._h:
            raise RuntimeError("oracle hierarchy: coarsest operator not SPD")

    def vcycle(self, r):
        z = np.zeros(self.A.cE.shape)
        lib().orc_hier_vcycle(self._h, _p(_f64(r)), _p(z))
        return z

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_hier_free(self._h)
            self._h = None


def paper_sor(grid, exx, exy, eyy, rho, phi0, omega=1.875, tol=1e-10, max_sweeps=100000):
    """The paper's Eq. 18 update with SOR (Sec. 2.1, settings of Sec. 4)."""
    phi = _f64(phi0).copy()
    it = lib().orc_paper_sor(grid.nx, grid.ny, grid.hx, grid.hy, _p(_f64(exx)), _p(_f64(exy)),
                             _p(_f64(eyy)), _p(_f64(rho)), _p(phi), omega, tol, max_sweeps)
    return phi, it


# ---------------------------------------------------------------- problem pipeline
@dataclass
class Prepared:
    J: tuple
    D: np.ndarray
    exx: np.ndarray
    exy: np.ndarray
    eyy: np.ndarray
    A: Operator
    b: np.ndarray
    phi0: np.ndarray
    status: int
    take: Optional[np.ndarray] = None  # Neumann grids: row of the doubled system per grid row

    def extract(self, phi):
        """The solution on the instance's own grid from a solution of the system A."""
        return np.asarray(phi) if self.take is None else np.asarray(phi)[self.take]


def boundary_ring(grid, bc):
    """Node array that is bc on Dirichlet nodes and 0 at unknowns."""
    phi0 = np.zeros(grid.shape)
    if bc is not None:
        m = ~grid.interior_mask()
        phi0[m] = np.asarray(bc)[m]
    return phi0


def doubled_grid(g):
    """The periodic grid of twice the height on which a grid with Neumann y sides is solved:
    y in [y0 - ly, y0 + ly), 2 (ny - 1) stored rows."""
    return replace(g, ny=2 * (g.ny - 1) + 1, y0=g.y0 - g.ly, ly=2.0 * g.ly, periodic_y=True, neumann_y=False)


def neumann_rows(ny):
    """Even reflection of an ny-row grid into the doubled periodic grid: for each row of the
    doubled grid the row of the original it copies and the factor applied to eps_xy there
    (+1 in the original half, -1 in the mirrored half, 0 on the two Neumann rows, where an odd
    function vanishes); and for each original row its row in the doubled grid."""
    n = ny - 1
    jd = np.arange(2 * n)
    src = np.where(jd >= n, jd - n, n - jd)
    sign = np.where(jd >= n, 1.0, -1.0)
    sign[0] = sign[n] = 0.0
    take = np.where(np.arange(ny) < n, np.arange(ny) + n, 0)
    return src, sign, take


def prepare(inst) -> Prepared:
    """Coefficient build (Eqs. 10-15, 39-42), operator and right-hand side (Eq. 11).

    A grid with Neumann y sides (Eq. 28) is solved as the periodic problem on the doubled
    grid whose coefficients, charge, Dirichlet data and D are the even reflection of the
    original ones (eps_xy odd): its solution is even about both sides, so its normal
    derivative there vanishes, and the boundary rows carry the standard mirror-node
    discretization of the Neumann condition."""
    g = inst.grid
    if getattr(g, "neumann_y", False):
        g0 = replace(g, neumann_y=False)
        J = jacobian(g0, inst.map)  # one-sided differences on the Neumann rows (grid maps)
        D, exx, exy, eyy, st = eps_tensor(J, inst.eps_phys)
        src, sign, take = neumann_rows(g.ny)
        gd = doubled_grid(g)
        A = assemble(gd, exx[src], exy[src] * sign[:, None], eyy[src])
        b = rhs(gd, np.asarray(inst.rho_phys)[src], D[src])
        phi0 = boundary_ring(gd, None if inst.bc is None else np.asarray(inst.bc)[src])
        return Prepared(J, D, exx, exy, eyy, A, b, phi0, st, take=take)
    J = jacobian(g, inst.map)
    D, exx, exy, eyy, st = eps_tensor(J, inst.eps_phys)
    A = assemble(g, exx, exy, eyy)
    b = rhs(g, inst.rho_phys, D)
    return Prepared(J, D, exx, exy, eyy, A, b, boundary_ring(g, inst.bc), st)


def solve_instance(inst, rtol=1e-14, max_cycles=200, stagnate=3, **kw):
    P = prepare(inst)
    if P.status:
        raise RuntimeError(f"map folded (det J <= 0), status {P.status}")
    phi, cyc, hist = solve(P.A, P.b, P.phi0, rtol=rtol, max_cycles=max_cycles, stagnate=stagnate,
                           **kw)
    return phi, cyc, hist, P


# ---------------------------------------------------------------- error norms
def mask_dirichlet(A: Operator, fixed, v):
    """Operator and right-hand side with Dirichlet values v at the unknowns where fixed is
    set (Sec. 4.2 grid generation with an internal boundary); returns (A', b)."""
    B = Operator(A.nx, A.ny, A.periodic, *[a.copy() for a in A.arrays()])
    fx = np.ascontiguousarray(np.asarray(fixed, dtype=np.uint8))
    b = np.zeros(B.cE.shape)
    lib().orc_mask_dirichlet(B.nx, B.ny, int(B.periodic), *[_p(a) for a in B.arrays()],
                             fx.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), _p(_f64(v)), _p(b))
    return B, b


def harmonic_grid(grid, fixed, xp, yp, rtol=0.0, max_iters=400, stagnate=10):
    """Numerical grid generation (Sec. 4.2, Eqs. 36-37): x' and y' discrete-harmonic for the
    identity map's operator (the 5-point Laplacian, eps = I), Dirichlet data on the outer
    ring and at the fixed unknowns, solved by the oracle's MG-PCG from the given arrays
    (rtol 0: to FP64 stagnation).  Returns (xp', yp', iterations)."""
    ones = np.ones(grid.shape)
    A = assemble(grid, ones, np.zeros(grid.shape), ones)
    out, its = [], []
    for v in (xp, yp):
        B, b = mask_dirichlet(A, fixed, v)
        phi, it, _ = pcg_solve(B, b, np.array(v, dtype=np.float64), rtol=rtol, max_iters=max_iters,
                               stagnate=stagnate)
        out.append(phi)
        its.append(it)
    return out[0], out[1], its


def error_norms(exact, numerical):
    """(L_inf, L_2, L_1) over all N^2 nodes, Eqs. 25-27."""
    d = np.abs(np.asarray(exact) - np.asarray(numerical))
    n2 = d.size
    return float(d.max()), float(np.sqrt((d * d).sum() / n2)), float(d.sum() / n2)


def rel_l2(a, b, mask=None):
    a = np.asarray(a)
    b = np.asarray(b)
    if mask is not None:
        a, b = a[mask], b[mask]
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))
