"""Seeded synthetic inputs for the transformed-coefficient multigrid solver.

This module is shared by the CUDA path, the oracle, the tests and the benchmark.
It holds grid descriptions, the coordinates x'(x, y), y'(x, y) of each map, the
physical sources rho', physical material eps', Dirichlet data and exact solutions.
It holds none of the solver's arithmetic: no Jacobians, no permittivity tensor, no
operator.  Those are computed independently by the CUDA kernels and by the oracle.

Workloads (all synthetic; the paper uses no dataset):

* ``config1``  129^2 unit square, analytic sine-warp map, manufactured
  phi' = sin(pi x') sin(pi y'), rho' = 2 pi^2 phi' (sign: -div(eps grad phi) = rho).
* ``config2``  1025^2 unit square with a circular inclusion of radius 0.25 at the
  centre, handled by a local boundary-fitted map: the inner square [0.5-r, 0.5+r]^2
  of the computational grid is mapped onto the disc by the side-to-quadrant map of
  Eq. 44, the outer boundary is the identity, and x', y' are discrete harmonic
  elsewhere (Eqs. 36-37).  eps' = 10 inside, 1 outside, 5.5 on the ring; 16 seeded
  Gaussian blobs (sigma 0.02, centres U[0,1]^2, amplitudes U[-1,1]); phi = 0 on the
  outer boundary.
* ``config3``  8193^2 full annulus r in [0.2, 1] by the polar map of Eq. 29
  (x' = x cos y, y' = x sin y, computational x in [0.2, 1], y in [0, 2 pi), periodic
  in y); phi = 0 at r = 0.2 and r = 1; 64 seeded Fourier modes with |k| <= 16 and
  amplitude ~ N(0,1) |k|^-2.
* ``config4``  512 instances, sides uniform over {65, 129, 257, 513}, geometry of
  config2 with radius U[0.1, 0.35] and eps' ratio U[1, 50].
* ``config5``  a Poisson-arrival request stream; sides log-uniform in [129, 2049]
  snapped to m 2^k + 1 with m in [8, 16]; geometry of config4 with the inclusion radius
  drawn from a catalogue of four values (each distinct mapped grid costs a harmonic solve
  on the host); eps' ratio U[1, 50], seeded blob sources.

Validation cases from the paper's Sec. 4: circle with uniform source (Eq. 43),
circle Laplace with phi = sin(8 theta) (Eq. 45), full annulus with the logarithmic
solution of Eq. 28-a, plus affine maps with quadratic solutions.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from functools import lru_cache
from typing import Optional, Sequence

import numpy as np

MAP_KINDS = {"identity": 0, "sine_warp": 1, "polar": 2, "sinh": 3, "affine": 4, "grid": 5}


@dataclass(frozen=True)
class Grid:
    """Uniform computational grid of nx x ny vertices on [x0, x0+lx] x [y0, y0+ly].

    Arrays are row-major (nyr, nx) with i (x) contiguous.  A grid periodic in y has
    ny - 1 stored rows (row ny-1 coincides with row 0).  With neumann_y the two y sides
    carry a homogeneous Neumann condition (their nodes are unknowns); the x sides stay
    Dirichlet.
    """

    nx: int
    ny: int
    x0: float = 0.0
    y0: float = 0.0
    lx: float = 1.0
    ly: float = 1.0
    periodic_y: bool = False
    neumann_y: bool = False

    @property
    def hx(self) -> float:
        return self.lx / (self.nx - 1)

    @property
    def hy(self) -> float:
        return self.ly / (self.ny - 1)

    @property
    def nyr(self) -> int:
        return self.ny - 1 if self.periodic_y else self.ny

    @property
    def shape(self):
        return (self.nyr, self.nx)

    @property
    def unknowns(self) -> int:
        return (self.nx - 2) * (self.nyr if (self.periodic_y or self.neumann_y) else self.ny - 2)

    def coords(self):
        x = self.x0 + self.hx * np.arange(self.nx)
        y = self.y0 + self.hy * np.arange(self.nyr)
        return np.meshgrid(x, y)  # (nyr, nx) each

    def interior_mask(self):
        m = np.zeros(self.shape, dtype=bool)
        if self.periodic_y or self.neumann_y:
            m[:, 1:-1] = True
        else:
            m[1:-1, 1:-1] = True
        return m


@dataclass
class MapSpec:
    """A coordinate map x -> x' (Eq. 1).  Analytic kinds carry parameters; kind
    'grid' carries the mapped node coordinates xp, yp of shape (nyr, nx).

    jump: for a periodic-y mapped grid, the offset added to (x', y') when row
    nyr wraps back to row 0 (zero for a closed map such as the full annulus).
    """

    kind: str
    params: tuple = ()
    xp: Optional[np.ndarray] = None
    yp: Optional[np.ndarray] = None
    jump: tuple = (0.0, 0.0)

    @property
    def code(self) -> int:
        return MAP_KINDS[self.kind]

    def physical(self, grid: Grid):
        """Physical coordinates (x', y') of every stored node."""
        if self.kind == "grid":
            return self.xp, self.yp
        x, y = grid.coords()
        p = self.params
        if self.kind == "identity":
            return x.copy(), y.copy()
        if self.kind == "sine_warp":
            a = p[0]
            return (x + a * np.sin(np.pi * x) * np.sin(np.pi * y),
                    y + a * np.sin(2 * np.pi * x) * np.sin(np.pi * y))
        if self.kind == "polar":  # Eq. 29
            return x * np.cos(y), x * np.sin(y)
        if self.kind == "sinh":  # Eq. 52
            s, al = p
            return s * np.sinh(al * x), s * np.sinh(al * y)
        if self.kind == "affine":
            a11, a12, a21, a22 = p
            return a11 * x + a12 * y, a21 * x + a22 * y
        raise ValueError(self.kind)


@dataclass
class Instance:
    """One solve: grid, map, optional eps' (nodal scalar), rho' at the nodes,
    Dirichlet data (node array whose boundary ring is used; None = 0) and, where
    known, the exact continuum solution at the nodes."""

    name: str
    grid: Grid
    map: MapSpec
    rho_phys: np.ndarray
    eps_phys: Optional[np.ndarray] = None
    bc: Optional[np.ndarray] = None
    exact: Optional[np.ndarray] = None
    rtol: float = 1e-10
    meta: dict = field(default_factory=dict)


# --------------------------------------------------------------------------
# Discrete harmonic grid generation (Eqs. 36-37) with an internal Dirichlet ring
# --------------------------------------------------------------------------
def _lap_apply(u, hx, hy):
    """5-point Laplacian at interior nodes of a (ny, nx) array (boundary rows/cols 0)."""
    out = np.zeros_like(u)
    out[1:-1, 1:-1] = ((u[1:-1, 2:] - 2 * u[1:-1, 1:-1] + u[1:-1, :-2]) / (hx * hx)
                       + (u[2:, 1:-1] - 2 * u[1:-1, 1:-1] + u[:-2, 1:-1]) / (hy * hy))
    return out


def _rb_sweep(u, f, free, hx, hy, parity_masks):
    wx, wy = 1.0 / (hx * hx), 1.0 / (hy * hy)
    wd = 2 * wx + 2 * wy
    for pm in parity_masks:
        nb = np.zeros_like(u)
        nb[1:-1, 1:-1] = (wx * (u[1:-1, 2:] + u[1:-1, :-2]) + wy * (u[2:, 1:-1] + u[:-2, 1:-1]))
        upd = free & pm
        u[upd] = ((nb + f) / wd)[upd]   # Laplacian u = -f form: (sum nb - wd u) = -f


def _mg_level_masks(shape):
    ny, nx = shape
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    red = (ii + jj) % 2 == 0
    return [red, ~red]


def _harmonic_mg(u, fixed, hx, hy, depth):
    """Solve the 5-point Laplace equation for u at the nodes where fixed is False,
    with u given where fixed is True, by multigrid V(2,2) cycles; the coarsest level
    (after `depth` halvings) is solved by a sparse direct solve."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    levels = [(fixed, hx, hy)]
    for _ in range(depth):
        f, a, b = levels[-1]
        levels.append((f[::2, ::2].copy(), 2 * a, 2 * b))

    def direct(rhs, fx, a, b):
        ny, nx = fx.shape
        free = ~fx
        idx = -np.ones(fx.shape, dtype=np.int64)
        idx[free] = np.arange(int(free.sum()))
        rows, cols, vals = [], [], []
        wx, wy = 1 / (a * a), 1 / (b * b)
        jj, ii = np.nonzero(free)
        p = idx[jj, ii]
        rows.append(p); cols.append(p); vals.append(np.full(p.shape, 2 * wx + 2 * wy))
        for dj, di, w in ((0, 1, wx), (0, -1, wx), (1, 0, wy), (-1, 0, wy)):
            q = idx[jj + dj, ii + di]
            ok = q >= 0
            rows.append(p[ok]); cols.append(q[ok]); vals.append(np.full(int(ok.sum()), -w))
        M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(p.size, p.size))
        x = np.zeros(fx.shape)
        x[free] = spla.spsolve(M.tocsc(), rhs[free])
        return x

    def vcycle(l, e, r):
        fx, a, b = levels[l]
        if l == len(levels) - 1:
            return direct(r, fx, a, b)
        pm = _mg_level_masks(fx.shape)
        free = ~fx
        for _ in range(2):
            _rb_sweep(e, r, free, a, b, pm)
        res = np.zeros_like(e)
        res[free] = (r + _lap_apply(e, a, b))[free]
        rc = np.zeros(levels[l + 1][0].shape)
        rc[1:-1, 1:-1] = (4 * res[2:-2:2, 2:-2:2]
                          + 2 * (res[1:-3:2, 2:-2:2] + res[3:-1:2, 2:-2:2]
                                 + res[2:-2:2, 1:-3:2] + res[2:-2:2, 3:-1:2])
                          + res[1:-3:2, 1:-3:2] + res[1:-3:2, 3:-1:2]
                          + res[3:-1:2, 1:-3:2] + res[3:-1:2, 3:-1:2]) / 16.0
        rc[levels[l + 1][0]] = 0.0
        ec = vcycle(l + 1, np.zeros_like(rc), rc)
        fine = np.zeros_like(e)
        fine[::2, ::2] = ec
        fine[1::2, ::2] = 0.5 * (ec[:-1, :] + ec[1:, :])
        fine[::2, 1::2] = 0.5 * (ec[:, :-1] + ec[:, 1:])
        fine[1::2, 1::2] = 0.25 * (ec[:-1, :-1] + ec[1:, :-1] + ec[:-1, 1:] + ec[1:, 1:])
        e[free] += fine[free]
        for _ in range(2):
            _rb_sweep(e, r, free, a, b, pm[::-1])
        return e

    free = ~fixed
    scale = max(1.0, float(np.abs(u).max()))
    for _ in range(60):
        r = np.zeros_like(u)
        r[free] = _lap_apply(u, hx, hy)[free]          # residual of -Lap u = 0 is +Lap u
        rmax = np.abs(r).max() * hx * hy / scale
        if rmax < 1e-15:
            break
        e = vcycle(0, np.zeros_like(u), r)
        u[free] += e[free]
    return u


def _eq44_boundary(u, v, b):
    """Eq. 44: the sides of the square [-b, b]^2 onto the quadrants of the circle of
    radius b.  (u, v) lie on the square's boundary."""
    xp = np.empty_like(u)
    yp = np.empty_like(u)
    on_x = np.isclose(np.abs(u), b) & ~np.isclose(np.abs(v), b)
    on_y = ~on_x
    # sides y = -b, y = b (and corners)
    xp[on_y] = u[on_y] / math.sqrt(2.0)
    yp[on_y] = np.sign(v[on_y]) * b * np.sqrt(np.maximum(0.0, 1 - u[on_y] ** 2 / (2 * b * b)))
    # sides x = -b, x = b
    xp[on_x] = np.sign(u[on_x]) * b * np.sqrt(np.maximum(0.0, 1 - v[on_x] ** 2 / (2 * b * b)))
    yp[on_x] = v[on_x] / math.sqrt(2.0)
    return xp, yp


def inclusion_ring_data(n: int, i0: int):
    """Dirichlet data of the inclusion grid: the ring of the inner square [i0, n-1-i0]^2
    carries the Eq. 44 square-to-circle map, the outer boundary the identity.  Returns the
    ring mask and x', y' arrays holding the identity everywhere except on the ring (the
    initial guess of the harmonic solve)."""
    grid = Grid(n, n)
    x, y = grid.coords()
    xp, yp = x.copy(), y.copy()
    i1 = n - 1 - i0
    ring = np.zeros(grid.shape, dtype=bool)
    ring[i0:i1 + 1, i0] = ring[i0:i1 + 1, i1] = True
    ring[i0, i0:i1 + 1] = ring[i1, i0:i1 + 1] = True
    b = (i1 - i0) / 2 * grid.hx
    c = 0.5 * (x[0, i0] + x[0, i1])
    bx, by = _eq44_boundary(x[ring] - c, y[ring] - c, b)
    xp[ring] = c + bx
    yp[ring] = c + by
    return ring, xp, yp


@lru_cache(maxsize=64)
def _inclusion_grid_cached(n: int, i0: int):
    grid = Grid(n, n)
    ring, xp, yp = inclusion_ring_data(n, i0)
    fixed = ring.copy()
    fixed[0, :] = fixed[-1, :] = fixed[:, 0] = fixed[:, -1] = True
    # first guess: the identity outside the ring, the same square-to-disc boundary
    # data scaled inwards inside it (any guess converges; this one saves cycles)
    depth = _harmonic_depth(n, i0)
    xp = _harmonic_mg(xp, fixed, grid.hx, grid.hy, depth)
    yp = _harmonic_mg(yp, fixed, grid.hx, grid.hy, depth)
    xp.setflags(write=False)
    yp.setflags(write=False)
    return xp, yp


def _harmonic_depth(n: int, i0: int) -> int:
    """Number of halvings for the grid generator: keep the ring on coarse grid lines
    and stop at a coarsest side of at most 129."""
    d = 0
    m = n - 1
    while m % 2 == 0 and i0 % (2 ** (d + 1)) == 0 and m // 2 >= 16 and m > 128:
        m //= 2
        d += 1
    return d


def snap_ring(n: int, r: float) -> int:
    """Index i0 of the inner square [i0, n-1-i0]^2 for a requested radius r (as a
    fraction of the unit square): rounded so that the ring sits on grid lines of a
    few coarser levels."""
    g = 1
    while (n - 1) % (2 * g) == 0 and (n - 1) // (2 * g) >= 64:
        g *= 2
    i0 = int(round((0.5 - r) * (n - 1) / g)) * g
    return max(g, min(i0, (n - 1) // 2 - g))


def inclusion_grid(n: int, r: float):
    """Mapped grid (x', y') for the unit square with a circular inclusion of radius
    ~r at its centre; returns (xp, yp, i0, r_snapped)."""
    i0 = snap_ring(n, r)
    if (n, i0) in _SEEDED:
        xp, yp = _SEEDED[(n, i0)]
    else:
        xp, yp = _inclusion_grid_cached(n, i0)
    return xp, yp, i0, 0.5 - i0 / (n - 1)


def _grid_job(args):
    n, i0, nsrc, seed = args
    xp, yp = _inclusion_grid_cached(n, i0)
    src = [gaussian_blobs(xp, yp, np.random.default_rng(seed + 7919 * v)) for v in range(nsrc)]
    return n, i0, np.array(xp), np.array(yp), src


def prefetch_inclusion_grids(pairs, workers: int = 0, sources: int = 0, seed: int = 0):
    """Generate the mapped grids of many (side, radius) pairs in parallel worker
    processes (started with 'spawn') and seed the in-process cache with them.  With
    sources > 0 also draw that many seeded 16-blob sources per grid (served by
    ``cached_source``).  Call it from a script's main guard."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os

    jobs = sorted({(n, snap_ring(n, r)) for n, r in pairs})
    todo = [j for j in jobs if j not in _SEEDED or len(_SOURCES.get(j, ())) < sources]
    if not todo:
        return
    workers = workers or max(1, min(16, (os.cpu_count() or 2) - 1))
    todo.sort(key=lambda j: -j[0])  # largest first: they dominate the wall time
    args = [(n, i0, sources, seed + 1009 * n + i0) for n, i0 in todo]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        for n, i0, xp, yp, src in ex.map(_grid_job, args):
            xp.setflags(write=False)
            yp.setflags(write=False)
            _SEEDED[(n, i0)] = (xp, yp)
            if sources:
                _SOURCES[(n, i0)] = src


def cached_source(n: int, i0: int, variant: int) -> np.ndarray:
    """One of the pre-drawn sources of grid (n, i0) (see prefetch_inclusion_grids)."""
    src = _SOURCES[(n, i0)]
    return src[variant % len(src)]


_SEEDED: dict = {}
_SOURCES: dict = {}


def inclusion_eps(n: int, i0: int, ratio: float) -> np.ndarray:
    """eps' = ratio strictly inside the inner square, 1 outside, (1+ratio)/2 on its ring."""
    e = np.ones((n, n))
    i1 = n - 1 - i0
    e[i0:i1 + 1, i0:i1 + 1] = 0.5 * (1 + ratio)
    e[i0 + 1:i1, i0 + 1:i1] = ratio
    return e


def gaussian_blobs(xp, yp, rng, count=16, sigma=0.02, box=(0.0, 1.0)):
    cx = rng.uniform(box[0], box[1], count)
    cy = rng.uniform(box[0], box[1], count)
    amp = rng.uniform(-1.0, 1.0, count)
    rho = np.zeros_like(xp)
    for k in range(count):
        rho += amp[k] * np.exp(-((xp - cx[k]) ** 2 + (yp - cy[k]) ** 2) / (2 * sigma * sigma))
    return rho


def fourier_source(xp, yp, rng, modes=64, kmax=16):
    """sum_m A_m cos(pi (kx x' + ky y') + phase), integer k with 1 <= |k| <= kmax drawn
    uniformly, A ~ N(0,1) |k|^-2, phase ~ U[0, 2 pi)."""
    ks = [(a, b) for a in range(-kmax, kmax + 1) for b in range(-kmax, kmax + 1)
          if 1 <= math.hypot(a, b) <= kmax]
    pick = rng.choice(len(ks), size=modes, replace=False)
    rho = np.zeros_like(xp)
    for m in pick:
        kx, ky = ks[m]
        kk = math.hypot(kx, ky)
        amp = rng.standard_normal() / (kk * kk)
        ph = rng.uniform(0.0, 2 * math.pi)
        rho += amp * np.cos(math.pi * (kx * xp + ky * yp) + ph)
    return rho


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------
def config1(n: int = 129) -> Instance:
    grid = Grid(n, n)
    mp = MapSpec("sine_warp", (0.1,))
    xp, yp = mp.physical(grid)
    exact = np.sin(np.pi * xp) * np.sin(np.pi * yp)
    rho = 2 * np.pi ** 2 * exact
    return Instance(f"sine_warp_{n}", grid, mp, rho, exact=exact, rtol=1e-10)


def inclusion_instance(n: int, r: float, ratio: float, seed: int, blobs: int = 16,
                       sigma: float = 0.02, name: str | None = None) -> Instance:
    xp, yp, i0, rs = inclusion_grid(n, r)
    rng = np.random.default_rng(seed)
    rho = gaussian_blobs(xp, yp, rng, blobs, sigma)
    grid = Grid(n, n)
    return Instance(name or f"inclusion_{n}_r{rs:.4f}_e{ratio:.2f}", grid,
                    MapSpec("grid", (), np.asarray(xp), np.asarray(yp)), rho,
                    eps_phys=inclusion_eps(n, i0, ratio), rtol=1e-10,
                    meta={"r": rs, "ratio": ratio, "i0": i0, "seed": seed})


def config2(n: int = 1025, seed: int = 2) -> Instance:
    return inclusion_instance(n, 0.25, 10.0, seed, name=f"inclusion_{n}")


def annulus_grid(n: int) -> Grid:
    return Grid(n, n, x0=0.2, y0=0.0, lx=0.8, ly=2 * math.pi, periodic_y=True)


def config3(n: int = 8193, seed: int = 3) -> Instance:
    grid = annulus_grid(n)
    mp = MapSpec("polar")
    xp, yp = mp.physical(grid)
    rng = np.random.default_rng(seed)
    rho = fourier_source(xp, yp, rng)
    return Instance(f"annulus_{n}", grid, mp, rho, rtol=1e-9)


def config4_specs(count: int = 512, seed0: int = 4000) -> list:
    """(side, radius, ratio, seed) per instance of the batched workload."""
    out = []
    for k in range(count):
        rng = np.random.default_rng(seed0 + k)
        n = int(rng.choice([65, 129, 257, 513]))
        r = float(rng.uniform(0.1, 0.35))
        ratio = float(rng.uniform(1.0, 50.0))
        out.append((n, r, ratio, seed0 + k))
    return out


def config4(count: int = 512, seed0: int = 4000) -> list:
    return [inclusion_instance(n, r, e, s) for (n, r, e, s) in config4_specs(count, seed0)]


def snap_side(side: float) -> int:
    """Nearest m 2^k + 1 with m in [8, 16]."""
    best = None
    for k in range(0, 12):
        for m in range(8, 17):
            v = m * 2 ** k + 1
            if best is None or abs(v - side) < abs(best - side):
                best = v
    return best


def config5_stream(count: int = 20000, seed: int = 5, rate: float = 100.0,
                   side_range=(129, 2049), radii: Sequence[float] | None = None) -> list:
    """Request stream: list of (arrival_time_s, side, radius, ratio, source_seed); the
    inclusion radius is drawn U[0.1, 0.35] per request unless a catalogue `radii` is given."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    lo, hi = math.log(side_range[0]), math.log(side_range[1])
    out = []
    for q in range(count):
        side = snap_side(math.exp(rng.uniform(lo, hi)))
        if radii is None:
            r = float(rng.uniform(0.1, 0.35))
        else:
            r = float(radii[int(rng.integers(len(radii)))])
        ratio = float(rng.uniform(1.0, 50.0))
        out.append((float(t[q]), side, r, ratio, int(seed * 1_000_003 + q)))
    return out


# --------------------------------------------------------------------------
# Validation cases (Sec. 4) and small structured cases
# --------------------------------------------------------------------------
def identity_poisson(n: int, ny: int | None = None) -> Instance:
    ny = ny or n
    grid = Grid(n, ny)
    mp = MapSpec("identity")
    x, y = mp.physical(grid)
    exact = np.sin(np.pi * x) * np.sin(np.pi * y)
    return Instance(f"identity_{n}x{ny}", grid, mp, 2 * np.pi ** 2 * exact, exact=exact)


def affine_quadratic(n: int, a=(1.0, 0.3, -0.2, 1.1)) -> Instance:
    """Affine map with phi' = x'^2 + y'^2, rho' = -4: the 9-point stencil is exact
    for quadratics, so the discrete solution equals the nodal values."""
    grid = Grid(n, n)
    mp = MapSpec("affine", tuple(a))
    xp, yp = mp.physical(grid)
    exact = xp ** 2 + yp ** 2
    return Instance(f"affine_{n}", grid, mp, np.full(grid.shape, -4.0), bc=exact.copy(),
                    exact=exact)


@lru_cache(maxsize=16)
def _circle_grid_cached(n: int, b: float):
    grid = Grid(n, n, x0=-b, y0=-b, lx=2 * b, ly=2 * b)
    x, y = grid.coords()
    xp, yp = x.copy(), y.copy()
    fixed = np.zeros(grid.shape, dtype=bool)
    fixed[0, :] = fixed[-1, :] = fixed[:, 0] = fixed[:, -1] = True
    bx, by = _eq44_boundary(x[fixed], y[fixed], b)
    xp[fixed] = bx
    yp[fixed] = by
    depth = 0
    m = n - 1
    while m % 2 == 0 and m > 128:
        m //= 2
        depth += 1
    xp = _harmonic_mg(xp, fixed, grid.hx, grid.hy, depth)
    yp = _harmonic_mg(yp, fixed, grid.hx, grid.hy, depth)
    xp.setflags(write=False)
    yp.setflags(write=False)
    return grid, xp, yp


def circle_poisson(n: int, b: float = 2.0) -> Instance:
    """Sec. 4.2.1: circle of radius b, exact phi = (x'^2 + y'^2)/4 (Eq. 43); with the
    sign convention -div(eps grad phi) = rho the source is rho' = -1."""
    grid, xp, yp = _circle_grid_cached(n, b)
    exact = (xp ** 2 + yp ** 2) / 4.0
    return Instance(f"circle_poisson_{n}", grid, MapSpec("grid", (), np.asarray(xp), np.asarray(yp)),
                    np.full(grid.shape, -1.0), bc=exact.copy(), exact=exact)


def circle_laplace(n: int, mode: int = 8) -> Instance:
    """Sec. 4.2.2: unit circle, phi = sin(n theta) on r = 1, exact r^n sin(n theta) (Eq. 45)."""
    grid, xp, yp = _circle_grid_cached(n, 1.0)
    r = np.hypot(xp, yp)
    th = np.arctan2(yp, xp)
    exact = r ** mode * np.sin(mode * th)
    return Instance(f"circle_laplace_{n}", grid, MapSpec("grid", (), np.asarray(xp), np.asarray(yp)),
                    np.zeros(grid.shape), bc=exact.copy(), exact=exact)


def annulus_log(n: int) -> Instance:
    """Full annulus r in [0.2, 1] (polar map Eq. 29, periodic in theta), phi = 1 at
    r = 0.2 and 0 at r = 1: exact ln(1/r)/ln(1/0.2), the form of Eq. 28-a."""
    grid = annulus_grid(n)
    mp = MapSpec("polar")
    x, _ = grid.coords()
    exact = np.log(1.0 / x) / np.log(1.0 / 0.2)
    return Instance(f"annulus_log_{n}", grid, mp, np.zeros(grid.shape), bc=exact.copy(),
                    exact=exact)


def semi_annulus(n: int, a: float = 2.0, R: float = 5.0, phi0: float = 1.0) -> Instance:
    """The semi-annulus of Sec. 4.1 (Eq. 28): r in [a, R], theta in [0, pi] by the polar map
    (Eq. 29), phi = phi0 at r = a, 0 at r = R, zero normal derivative at theta = 0 and pi,
    charge-free; exact solution phi0 ln(R/r) / ln(R/a) (Eq. 28-a)."""
    grid = Grid(n, n, x0=a, y0=0.0, lx=R - a, ly=math.pi, neumann_y=True)
    x, _ = grid.coords()
    exact = phi0 * np.log(R / x) / np.log(R / a)
    return Instance(f"semi_annulus_{n}", grid, MapSpec("polar"), np.zeros(grid.shape), bc=exact.copy(),
                    exact=exact)


def neumann_manufactured(n: int) -> Instance:
    """Unit square, identity map, phi = sin(pi x) cos(pi y): zero at x = 0, 1 and zero normal
    derivative at y = 0, 1; rho = 2 pi^2 phi."""
    grid = Grid(n, n, neumann_y=True)
    x, y = grid.coords()
    exact = np.sin(np.pi * x) * np.cos(np.pi * y)
    return Instance(f"neumann_mms_{n}", grid, MapSpec("identity"), 2 * np.pi ** 2 * exact, bc=np.zeros(grid.shape),
                    exact=exact)


def random_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, shape)


def _gaussian_potential(r: np.ndarray, rho0: float, sigma: float) -> np.ndarray:
    """Radially symmetric potential of the charge -rho0 exp(-r^2 / (2 sigma^2)) in the plane
    under -lap(phi) = rho: r phi'(r) = rho0 sigma^2 (1 - exp(-u)), u = r^2 / (2 sigma^2), so
    phi = (rho0 sigma^2 / 2) (ln(2 sigma^2) + ln u + E1(u)) up to a constant.  ln u + E1(u)
    is -gamma + Ein(u) with Ein(u) = sum_k (-1)^(k+1) u^k / (k k!), summed directly for small u
    (finite at the beam centre), by scipy's E1 elsewhere."""
    from scipy.special import exp1
    u = np.asarray(r, dtype=np.float64) ** 2 / (2.0 * sigma * sigma)
    g = np.empty_like(u)
    small = u < 1.0
    us = u[small]
    ein = np.zeros_like(us)
    term = np.ones_like(us)
    for k in range(1, 40):
        term = term * (-us) / k  # (-u)^k / k!
        ein -= term / k
    g[small] = -np.euler_gamma + ein
    ub = u[~small]
    g[~small] = np.log(ub) + exp1(ub)
    return 0.5 * rho0 * sigma * sigma * (math.log(2.0 * sigma * sigma) + g)


def sinh_beam(n: int = 129, s: float = 5.0, alpha: float = 0.6, rho0: float = 100.0,
              sigma: float = 0.5) -> Instance:
    """The stretched-grid example of Sec. 5.1: computational square [-3, 3]^2 (Lx = Ly = 6),
    map x' = s sinh(alpha x), y' = s sinh(alpha y) (Eq. 52, s = 5, alpha = 0.6), Gaussian beam
    rho' = -rho0 exp(-(x'^2 + y'^2) / (2 sigma^2)) at the origin (Eq. 53, rho0 = 100,
    sigma = 0.5).  The paper does not state its boundary condition; here the Dirichlet data
    are the beam's free-space potential, which is then the exact solution."""
    grid = Grid(n, n, x0=-3.0, y0=-3.0, lx=6.0, ly=6.0)
    mp = MapSpec("sinh", (s, alpha))
    xp, yp = mp.physical(grid)
    r2 = xp * xp + yp * yp
    rho = -rho0 * np.exp(-r2 / (2.0 * sigma * sigma))
    exact = _gaussian_potential(np.sqrt(r2), rho0, sigma)
    return Instance(f"sinh_beam_{n}", grid, mp, rho, bc=exact.copy(), exact=exact)
