"""Pins of the FP64 oracle against facts that do not come from the oracle itself
(closed forms, an independent sparse-matrix construction of the operator, dense direct
solves, adjoint identities, orders of accuracy, the paper's own Eq. 18 update)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2602_01888_gb300 import inputs as I
import _indep as X


def _eps_of(O, inst):
    P = O.prepare(inst)
    return P


# ---------------------------------------------------------------- coefficient build
def test_identity_map_is_the_textbook_five_point_laplacian(oracle):
    inst = I.identity_poisson(9)
    P = oracle.prepare(inst)
    assert np.all(P.D == 1.0) and np.all(P.exx == 1.0) and np.all(P.eyy == 1.0)
    assert np.all(P.exy == 0.0)
    h2 = 1.0 / inst.grid.hx ** 2
    A = P.A
    assert np.all(A.cNE == 0.0) and np.all(A.cNW == 0.0)
    assert np.all(A.cE[:, :-1] == -h2) and np.all(A.cN[:-1, :] == -h2)
    assert np.all(A.diag[1:-1, 1:-1] == 4 * h2)


def test_eps_matches_matrix_form_of_eq10(oracle):
    """Components (Eqs. 12-15) vs eps = det(J) J^-1 eps' J^-T evaluated as matrices."""
    rng = np.random.default_rng(7)
    for _ in range(5):
        a11, a22 = rng.uniform(0.5, 2.0, 2)
        a12, a21 = rng.uniform(-0.4, 0.4, 2)
        inst = I.affine_quadratic(9, (a11, a12, a21, a22))
        s = rng.uniform(0.5, 20.0, inst.grid.shape)
        J = oracle.jacobian(inst.grid, inst.map)
        D, exx, exy, eyy, st = oracle.eps_tensor(J, s)
        assert st == 0
        Jm = np.array([[a11, a12], [a21, a22]])
        Ji = np.linalg.inv(Jm)
        E = np.linalg.det(Jm) * Ji @ Ji.T
        assert np.allclose(exx, s * E[0, 0], rtol=1e-14, atol=0)
        assert np.allclose(exy, s * E[0, 1], rtol=1e-14, atol=1e-15)
        assert np.allclose(eyy, s * E[1, 1], rtol=1e-14, atol=0)


def test_det_eps_is_one_for_identity_material(oracle):
    for inst in (I.config1(33), I.annulus_log(33), I.inclusion_instance(65, 0.25, 1.0, 1),
                 I.circle_poisson(33)):
        P = oracle.prepare(inst)
        det = P.exx * P.eyy - P.exy ** 2
        assert np.abs(det - 1).max() < 1e-12, inst.name


def test_polar_closed_form(oracle):
    inst = I.annulus_log(33)
    P = oracle.prepare(inst)
    r, _ = inst.grid.coords()
    assert np.allclose(P.exx, r, rtol=1e-14)
    assert np.allclose(P.eyy, 1.0 / r, rtol=1e-14)
    assert np.abs(P.exy).max() < 1e-15
    assert np.allclose(P.D, r, rtol=1e-14)


def test_polar_cross_term_residue_moves_the_solution_by_rounding_only(oracle):
    """Reading r13: for the polar map Eq. 13 vanishes identically and the general formula
    leaves only rounding residue in eps_xy; the 5-point operator (eps_xy = 0) then has the
    same discrete solution up to rounding.  At 257^2 dropping the residue moves the oracle's
    annulus solution by 2e-14 (the solver's own stagnation level; 1.9e-13 at 2049^2), while
    the closed-form tensor, whose few-ulp differences from the general formula are systematic
    along theta, moves it by 4e-13, a gap that grows like n^2 (1.4e-12 at 513^2, 2.9e-10 at
    8193^2, where it would break the FP64 bound)."""
    inst = I.annulus_log(257)
    g = inst.grid
    P = oracle.prepare(inst)
    emag = max(np.abs(P.exx).max(), np.abs(P.eyy).max())
    assert np.abs(P.exy).max() <= 1e-15 * emag          # residue only
    assert np.count_nonzero(P.exy) > 0                    # ... but not exactly zero
    r, _ = g.coords()
    kw = dict(rtol=0.0, max_iters=60, stagnate=4, smoother=oracle.SMOOTHER_XLINE, nu1=1, nu2=1)
    sol = {}
    for name, (exx, exy, eyy) in {"general": (P.exx, P.exy, P.eyy),
                                  "no_residue": (P.exx, np.zeros_like(P.exy), P.eyy),
                                  "closed_form": (r, np.zeros_like(r), 1.0 / r)}.items():
        A = oracle.assemble(g, exx, exy, eyy)
        sol[name], _, _ = oracle.pcg_solve(A, P.b, P.phi0, **kw)
    m = g.interior_mask()
    d_res = oracle.rel_l2(sol["no_residue"], sol["general"], m)
    d_closed = oracle.rel_l2(sol["closed_form"], sol["general"], m)
    assert d_res < 1e-13
    assert 5 * d_res < d_closed < 1e-11


def test_sinh_closed_form_offdiagonal_vanishes(oracle):
    g = I.Grid(33, 33, -3.0, -3.0, 6.0, 6.0)
    mp = I.MapSpec("sinh", (5.0, 0.6))
    D, exx, exy, eyy, st = oracle.eps_tensor(oracle.jacobian(g, mp))
    x, y = g.coords()
    cx, cy = np.cosh(0.6 * x), np.cosh(0.6 * y)
    assert np.all(exy == 0.0)
    assert np.allclose(exx, cy / cx, rtol=1e-14) and np.allclose(eyy, cx / cy, rtol=1e-14)
    assert np.allclose(D, 9.0 * cx * cy, rtol=1e-14)


def test_central_difference_tensor_converges_at_second_order(oracle):
    errs = []
    for n in (33, 65, 129):
        inst = I.config1(n)
        xp, yp = inst.map.physical(inst.grid)
        Pa = oracle.prepare(inst)
        gm = I.MapSpec("grid", (), xp, yp)
        D, exx, exy, eyy, _ = oracle.eps_tensor(oracle.jacobian(inst.grid, gm))
        errs.append(max(np.abs(exx - Pa.exx).max(), np.abs(exy - Pa.exy).max(),
                        np.abs(eyy - Pa.eyy).max(), np.abs(D - Pa.D).max()))
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(1.9 < o < 2.15 for o in orders), orders


def test_folded_map_is_reported(oracle):
    inst = I.affine_quadratic(9, (1.0, 0.0, 0.0, -1.0))
    _, _, _, _, st = oracle.eps_tensor(oracle.jacobian(inst.grid, inst.map))
    assert st == 5


def test_charge_conservation_eq11(oracle):
    """sum b hx hy = integral of rho' over the physical domain (= 8 for config 1) + O(h^2)."""
    errs = []
    for n in (33, 65, 129):
        inst = I.config1(n)
        P = oracle.prepare(inst)
        errs.append(abs(P.b.sum() * inst.grid.hx * inst.grid.hy - 8.0))
    assert errs[-1] < 1e-3
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


# ---------------------------------------------------------------- operator
@pytest.mark.parametrize("case", ["sine", "inclusion", "annulus", "rect"])
def test_operator_equals_difference_matrix_construction(oracle, case):
    inst = {"sine": lambda: I.config1(17),
            "inclusion": lambda: I.inclusion_instance(33, 0.25, 10.0, 3),
            "annulus": lambda: I.annulus_log(17),
            "rect": lambda: I.Instance("rect", I.Grid(17, 9, 0.0, 0.0, 1.0, 0.6),
                                       I.MapSpec("sine_warp", (0.08,)), np.ones((9, 17)))}[case]()
    P = oracle.prepare(inst)
    A_ref = X.full_operator(inst.grid, P.exx, P.exy, P.eyy)
    u = X.unknown_ids(inst.grid)
    # every stored coupling of an unknown row equals the matrix entry
    A_or = X.coupling_matrix(inst.grid, P.A)
    Aref_uu = A_ref[u][:, u]
    assert abs(A_or - Aref_uu).max() <= 1e-10 * abs(Aref_uu).max()
    # diagonal = minus the sum of all eight couplings (Dirichlet columns included)
    rows = A_ref[u]
    assert np.abs(np.asarray(rows.sum(axis=1)).ravel()).max() <= 1e-9 * abs(Aref_uu).max()
    # symmetric
    assert abs(A_or - A_or.T).max() == 0.0


def test_affine_quadratic_is_reproduced_exactly(oracle):
    for a in ((1.0, 0.3, -0.2, 1.1), (1.3, -0.5, 0.4, 0.9)):
        inst = I.affine_quadratic(33, a)
        phi, cyc, hist, P = oracle.solve_instance(inst, rtol=1e-14)
        err = np.abs(phi - inst.exact).max() / np.abs(inst.exact).max()
        assert err < 1e-12, (a, err)


@pytest.mark.parametrize("n,case", [(9, "sine"), (17, "sine"), (17, "inclusion"), (17, "annulus")])
def test_multigrid_solution_equals_dense_direct_solve(oracle, n, case):
    inst = {"sine": lambda: I.config1(n),
            "inclusion": lambda: I.inclusion_instance(n, 0.25, 25.0, 4),
            "annulus": lambda: I.annulus_log(n)}[case]()
    P = oracle.prepare(inst)
    Auu, rhs = X.system(inst.grid, P.exx, P.exy, P.eyy, P.b, P.phi0)
    x = np.linalg.solve(Auu.toarray(), rhs)
    np.linalg.cholesky(Auu.toarray())  # SPD
    phi, cyc, hist = oracle.solve(P.A, P.b, P.phi0, rtol=1e-14, coarse_max=4)
    assert cyc >= 1
    m = inst.grid.interior_mask()
    assert np.abs(phi[m] - x).max() <= 1e-12 * np.abs(x).max()
    # and through flexible-free PCG
    phi2, _, _ = oracle.pcg_solve(P.A, P.b, P.phi0, rtol=1e-14, coarse_max=4)
    assert np.abs(phi2[m] - x).max() <= 1e-12 * np.abs(x).max()


# ---------------------------------------------------------------- transfers / coarse operator
@pytest.mark.parametrize("periodic", [False, True])
def test_restriction_is_a_quarter_of_the_prolongation_transpose(oracle, periodic):
    gf = I.annulus_grid(33) if periodic else I.Grid(33, 17)
    nxc, nyc = (gf.nx - 1) // 2 + 1, (gf.ny - 1) // 2 + 1
    gc = I.Grid(nxc, nyc, gf.x0, gf.y0, gf.lx, gf.ly, gf.periodic_y)
    rng = np.random.default_rng(3)
    r = rng.standard_normal(gf.shape) * gf.interior_mask()
    e = rng.standard_normal(gc.shape) * gc.interior_mask()
    Rr = oracle.restrict(gf.nx, gf.ny, periodic, r)
    Pe = oracle.prolong_add(gf.nx, gf.ny, periodic, e, np.zeros(gf.shape))
    lhs = 4.0 * np.sum(Rr * e)
    rhs = np.sum(r * Pe)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)
    # P against the independent sparse bilinear matrix
    Psp = X.prolongation(gf, gc)
    assert np.allclose(Pe[gf.interior_mask()], Psp @ e[gc.interior_mask()], rtol=0, atol=1e-14)


@pytest.mark.parametrize("case", ["sine", "inclusion", "annulus"])
def test_galerkin_equals_sparse_triple_product(oracle, case):
    inst = {"sine": lambda: I.config1(33), "inclusion": lambda: I.inclusion_instance(33, 0.25, 10.0, 5),
            "annulus": lambda: I.annulus_log(33)}[case]()
    P = oracle.prepare(inst)
    gf = inst.grid
    gc = I.Grid((gf.nx - 1) // 2 + 1, (gf.ny - 1) // 2 + 1, gf.x0, gf.y0, gf.lx, gf.ly, gf.periodic_y)
    Ac = oracle.galerkin(P.A)
    Af = X.full_operator(gf, P.exx, P.exy, P.eyy)
    u = X.unknown_ids(gf)
    Pm = X.prolongation(gf, gc)
    AH = 0.25 * (Pm.T @ Af[u][:, u] @ Pm)
    AH_or = X.coupling_matrix(gc, Ac)
    assert abs(AH_or - AH).max() <= 1e-11 * abs(AH).max()


# ---------------------------------------------------------------- smoother
def test_gauss_seidel_colour_phase_zeroes_its_residual(oracle):
    inst = I.inclusion_instance(33, 0.25, 10.0, 6)
    P = oracle.prepare(inst)
    rng = np.random.default_rng(0)
    phi = rng.standard_normal(inst.grid.shape) * inst.grid.interior_mask()
    for c, (ci, cj) in enumerate(((0, 0), (1, 1), (1, 0), (0, 1))):
        phi = oracle.gs_colour(P.A, phi, P.b, c)
        r = oracle.residual(P.A, phi, P.b)
        sel = np.zeros(inst.grid.shape, dtype=bool)
        sel[cj::2, ci::2] = True
        sel &= inst.grid.interior_mask()
        scale = np.abs(P.A.diag[inst.grid.interior_mask()]).max() * np.abs(phi).max()
        assert np.abs(r[sel]).max() <= 1e-14 * scale
        other = inst.grid.interior_mask() & ~sel
        assert np.abs(r[other]).max() > 1e-6 * scale  # the property is not trivially true


def test_vcycle_contraction_in_textbook_range(oracle):
    inst = I.identity_poisson(65)
    phi, cyc, hist, _ = oracle.solve_instance(inst, rtol=1e-12)
    rho = hist[2:8] / hist[1:7]
    assert 0.02 < np.median(rho) < 0.2


# ---------------------------------------------------------------- accuracy (Sec. 4)
def _orders(oracle, make, sizes):
    errs = []
    for n in sizes:
        inst = make(n)
        phi, *_ = oracle.solve_instance(inst, rtol=1e-13)
        errs.append(oracle.error_norms(inst.exact, phi))
    return [[math.log2(errs[k][q] / errs[k + 1][q]) for q in range(3)] for k in range(len(sizes) - 1)]


def test_second_order_manufactured_sine_warp(oracle):
    o = _orders(oracle, I.config1, (33, 65, 129))
    assert all(1.9 < v < 2.1 for v in o[-1]), o


def test_second_order_annulus_log_solution(oracle):
    o = _orders(oracle, I.annulus_log, (33, 65, 129))
    assert all(1.9 < v < 2.1 for v in o[-1]), o


def test_second_order_circle_poisson_eq43(oracle):
    """L2 and L1 converge at second order; L_inf approaches it more slowly (about 1.6 at
    these sizes) because the square-to-circle boundary map of Eq. 44 makes det J vanish
    at the four corners of the computational square."""
    o = _orders(oracle, I.circle_poisson, (65, 129, 257))
    assert 1.8 < o[-1][1] < 2.2 and 1.8 < o[-1][2] < 2.2, o
    assert o[-1][0] > 1.5, o


def test_second_order_circle_laplace_eq45(oracle):
    o = _orders(oracle, I.circle_laplace, (65, 129, 257))
    assert all(1.8 < v < 2.2 for v in o[-1]), o


def test_paper_eq18_operator_converges_to_the_same_solution(oracle):
    """The literal Eq. 18 update (non-symmetric) with SOR converges at second order to the
    continuum solution, like the symmetric form the solver uses."""
    errs = []
    for n in (17, 33, 65):
        inst = I.config1(n)
        P = oracle.prepare(inst)
        rho = inst.rho_phys * P.D
        phi, it = oracle.paper_sor(inst.grid, P.exx, P.exy, P.eyy, rho, P.phi0, omega=1.875, tol=1e-13)
        errs.append(np.abs(phi - inst.exact).max())
        sym, *_ = oracle.solve_instance(inst, rtol=1e-13)
        assert np.abs(phi - sym).max() < 5 * np.abs(sym - inst.exact).max() + 1e-12
    assert math.log2(errs[-2] / errs[-1]) > 1.85


# ---------------------------------------------------------------- input generators
def test_inclusion_grid_boundary_data_and_positivity(oracle):
    inst = I.inclusion_instance(129, 0.25, 10.0, 1)
    xp, yp = inst.map.xp, inst.map.yp
    i0 = inst.meta["i0"]
    n = 129
    i1 = n - 1 - i0
    g = inst.grid
    x, y = g.coords()
    # outer boundary: identity
    for sl in (np.s_[0, :], np.s_[-1, :], np.s_[:, 0], np.s_[:, -1]):
        assert np.all(xp[sl] == x[sl]) and np.all(yp[sl] == y[sl])
    # ring: on the circle of radius r (Eq. 44)
    r = inst.meta["r"]
    ring = np.zeros(g.shape, bool)
    ring[i0:i1 + 1, i0] = ring[i0:i1 + 1, i1] = ring[i0, i0:i1 + 1] = ring[i1, i0:i1 + 1] = True
    rad = np.hypot(xp[ring] - 0.5, yp[ring] - 0.5)
    assert np.allclose(rad, r, rtol=1e-13)
    # discrete harmonic elsewhere
    lap = I._lap_apply(np.array(xp), g.hx, g.hy) * g.hx * g.hy
    free = ~ring
    free[0, :] = free[-1, :] = free[:, 0] = free[:, -1] = False
    assert np.abs(lap[free]).max() < 1e-12
    P = oracle.prepare(inst)
    assert P.status == 0 and P.D.min() > 0


# ---------------------------------------------------------------- grid generation (Sec. 4.2)
def _affine(x, y):
    return 1.3 * x + 0.4 * y + 0.1, -0.2 * x + 0.9 * y - 0.05


def test_harmonic_grid_reproduces_affine_maps_with_internal_dirichlet_nodes(oracle):
    """Affine functions are discrete-harmonic for the 5-point Laplacian: with affine data on
    the outer ring and at scattered fixed interior nodes, the generated grid is that map
    at every node (and the fixed nodes keep their values)."""
    g = I.Grid(33, 29, 0.0, 0.0, 1.0, 0.875)
    x, y = g.coords()
    ax, ay = _affine(x, y)
    rng = np.random.default_rng(5)
    fixed = (rng.random(g.shape) < 0.05) & g.interior_mask()
    fixed[10, 5:20] = True  # a wall of fixed nodes
    xp0 = np.where(fixed | ~g.interior_mask(), ax, 0.0)
    yp0 = np.where(fixed | ~g.interior_mask(), ay, 0.0)
    xo, yo, _ = oracle.harmonic_grid(g, fixed, xp0, yp0)
    assert np.abs(xo - ax).max() < 1e-12 and np.abs(yo - ay).max() < 1e-12


def test_harmonic_grid_matches_the_independent_masked_multigrid_of_the_inputs(oracle):
    """The inclusion grid (ring carrying the Eq. 44 map) from the oracle's masked operator
    and MG-PCG against the numpy red-black multigrid that generates the workloads' grids."""
    n = 65
    i0 = I.snap_ring(n, 0.25)
    xref, yref = I._inclusion_grid_cached(n, i0)
    g = I.Grid(n, n)
    fixed, xp0, yp0 = I.inclusion_ring_data(n, i0)
    xo, yo, _ = oracle.harmonic_grid(g, fixed, xp0, yp0)
    assert np.abs(xo - xref).max() < 1e-11 and np.abs(yo - yref).max() < 1e-11


def test_harmonic_grid_obeys_the_discrete_maximum_principle(oracle):
    g = I.Grid(41, 41)
    rng = np.random.default_rng(9)
    data = rng.standard_normal(g.shape)
    fixed = np.zeros(g.shape, dtype=bool)
    fixed[20, 20] = True
    v = np.where(fixed | ~g.interior_mask(), data, 0.0)
    xo, _, _ = oracle.harmonic_grid(g, fixed, v, v)
    lo, hi = data[fixed | ~g.interior_mask()].min(), data[fixed | ~g.interior_mask()].max()
    assert xo.min() >= lo - 1e-12 and xo.max() <= hi + 1e-12
    assert xo[20, 20] == data[20, 20]


# ---------------------------------------------------------------- x-line smoothing
def _rows_residual(oracle, A, phi, b, parity):
    r = oracle.residual(A, phi, b)
    rows = np.zeros(r.shape, dtype=bool)
    rows[parity::2, :] = True
    return np.abs(r[rows]).max(), np.abs(r[~rows]).max()


@pytest.mark.parametrize("case", ["sine", "annulus", "inclusion"])
@pytest.mark.parametrize("parity", [0, 1])
def test_line_half_sweep_zeroes_the_residual_on_its_rows(oracle, case, parity):
    """A line half-sweep solves every row of its parity exactly: afterwards the residual
    vanishes (to rounding) on those rows, for 9-point operators (sine warp, inclusion) and
    a periodic one (annulus), and not on the other rows."""
    inst = {"sine": lambda: I.config1(33), "annulus": lambda: I.annulus_log(33),
            "inclusion": lambda: I.inclusion_instance(65, 0.25, 10.0, 3)}[case]()
    P = oracle.prepare(inst)
    rng = np.random.default_rng(3)
    phi0 = P.phi0 + rng.standard_normal(P.phi0.shape) * inst.grid.interior_mask()
    phi = oracle.line_rows(P.A, phi0, P.b, parity)
    on, off = _rows_residual(oracle, P.A, phi, P.b, parity)
    scale = np.abs(P.A.diag).max() * np.abs(phi).max()
    assert on < 1e-12 * scale and off > 1e-6 * scale, (on, off, scale)
    # Dirichlet ring untouched, the other parity's rows untouched
    keep = ~inst.grid.interior_mask()
    other = np.zeros_like(keep)
    other[1 - parity::2, :] = True
    assert np.array_equal(phi[keep | other], phi0[keep | other])


@pytest.mark.parametrize("case", ["sine", "annulus", "inclusion"])
def test_zebra_sweep_leaves_a_residual_on_the_even_rows_only(oracle, case):
    """After a zebra sweep (even rows, then odd rows) the residual is rounding residue on the
    odd rows, so full weighting of it reduces to the even rows: at coarse node (I, J),
    (2 r(2I-1, 2J) + 4 r(2I, 2J) + 2 r(2I+1, 2J)) / 16.  The restriction after line
    pre-smoothing relies on this; here it is the oracle's full weighting of the whole
    residual against that one-row sum written out."""
    inst = {"sine": lambda: I.config1(33), "annulus": lambda: I.annulus_log(33),
            "inclusion": lambda: I.inclusion_instance(65, 0.25, 10.0, 3)}[case]()
    P = oracle.prepare(inst)
    g = inst.grid
    rng = np.random.default_rng(4)
    phi0 = P.phi0 + rng.standard_normal(P.phi0.shape) * g.interior_mask()
    phi = oracle.smooth(P.A, phi0, P.b, sweeps=1, smoother=oracle.SMOOTHER_XLINE)
    r = oracle.residual(P.A, phi, P.b)
    scale = np.abs(P.A.diag).max() * np.abs(phi).max()
    assert np.abs(r[1::2, :]).max() < 1e-12 * scale < np.abs(r[0::2, :]).max()
    full = oracle.restrict(g.nx, g.ny, g.periodic_y, r)
    gc = I.Grid((g.nx - 1) // 2 + 1, (g.ny - 1) // 2 + 1, periodic_y=g.periodic_y)
    even = np.zeros(gc.shape)
    ev = r[0::2, :]
    even[:, 1:-1] = (2 * ev[: gc.shape[0], 1:-2:2] + 4 * ev[: gc.shape[0], 2:-1:2] + 2 * ev[: gc.shape[0], 3::2]) / 16
    even *= gc.interior_mask()
    assert np.abs(full - even).max() < 1e-12 * scale
    assert np.abs(full).max() > 1e-3 * scale


def test_line_smoothing_of_decoupled_rows_is_an_exact_solve(oracle):
    """With every coupling between rows removed the rows are independent one-dimensional
    problems; one zebra sweep solves them exactly (compared with numpy's dense solve)."""
    inst = I.config1(17)
    P = oracle.prepare(inst)
    A = oracle.Operator(P.A.nx, P.A.ny, P.A.periodic, P.A.cE.copy(), np.zeros_like(P.A.cN),
                        np.zeros_like(P.A.cNE), np.zeros_like(P.A.cNW), P.A.diag.copy())
    b = np.random.default_rng(8).standard_normal(P.b.shape) * inst.grid.interior_mask()
    phi = oracle.smooth(A, np.zeros_like(b), b, sweeps=1, smoother=oracle.SMOOTHER_XLINE)
    for j in range(1, A.ny - 1):
        N = A.nx - 2
        M = np.diag(A.diag[j, 1:-1]) + np.diag(A.cE[j, 1:-2], 1) + np.diag(A.cE[j, 1:-2], -1)
        assert np.allclose(phi[j, 1:-1], np.linalg.solve(M, b[j, 1:-1]), rtol=1e-12, atol=1e-14)


def test_line_smoothing_makes_the_annulus_cycle_robust(oracle):
    """On the anisotropic annulus (strong coupling along x) the x-line V(1,1) preconditioner
    needs a handful of CG iterations where the point smoother needs over twenty."""
    inst = I.config3(257)
    P = oracle.prepare(inst)
    _, it_pt, _ = oracle.pcg_solve(P.A, P.b, P.phi0, rtol=1e-8, max_iters=200, nu1=1, nu2=1)
    _, it_ln, _ = oracle.pcg_solve(P.A, P.b, P.phi0, rtol=1e-8, max_iters=200, nu1=1, nu2=1,
                                   smoother=oracle.SMOOTHER_XLINE)
    assert it_ln <= 8 and it_pt >= 3 * it_ln, (it_ln, it_pt)


# ---------------------------------------------------------------- SOR (Sec. 4 comparison method)
def _rows_decoupled_laplacian(N, rows=1):
    """1-D Poisson rows (diag 2, E/W -1) with every coupling between rows removed."""
    import oracle as O
    nx, ny = N + 2, rows + 2
    cE = np.zeros((ny, nx))
    cE[:, :-1] = -1.0
    z = np.zeros((ny, nx))
    diag = np.full((ny, nx), 2.0)
    return O.Operator(nx, ny, False, cE, z.copy(), z.copy(), z.copy(), diag)


@pytest.mark.parametrize("omega", [1.5, 1.9])
def test_sor_contraction_factor_matches_youngs_theorem(oracle, omega):
    """On one row of the 1-D Poisson matrix the four-colour order is red-black, a consistent
    ordering, so Young's theorem gives SOR's asymptotic contraction factor from the Jacobi
    spectral radius mu = cos(pi h): (omega mu + sqrt(omega^2 mu^2 - 4 (omega - 1)))^2 / 4 below
    the optimal omega, omega - 1 above it.  The measured per-sweep residual contraction
    (geometric mean over the last sweeps) must match."""
    N = 31
    A = _rows_decoupled_laplacian(N)
    mu = np.cos(np.pi / (N + 1))
    w_opt = 2.0 / (1.0 + np.sqrt(1.0 - mu * mu))
    if omega < w_opt:
        rho = ((omega * mu + np.sqrt(omega * omega * mu * mu - 4.0 * (omega - 1.0))) / 2.0) ** 2
    else:
        rho = omega - 1.0
    rng = np.random.default_rng(4)
    phi0 = np.zeros(A.cE.shape)
    phi0[1, 1:-1] = rng.standard_normal(N)
    _, sw, hist = oracle.sor_solve(A, np.zeros(A.cE.shape), phi0, omega=omega, rtol=0.0, max_sweeps=400,
                                   check=1)
    assert sw == 400
    rate = (hist[400] / hist[200]) ** (1.0 / 200)
    assert abs(rate - rho) < 2e-3 * rho, (rate, rho)


def test_sor_with_unit_factor_is_gauss_seidel(oracle):
    inst = I.config1(33)
    P = oracle.prepare(inst)
    rng = np.random.default_rng(6)
    phi = rng.standard_normal(P.A.cE.shape)
    gs = oracle.smooth(P.A, phi, P.b, sweeps=2, smoother=oracle.SMOOTHER_GS4)
    sor = oracle.smooth(P.A, phi, P.b, sweeps=2, smoother=oracle.SMOOTHER_SOR4, omega_j=1.0)
    assert np.abs(gs - sor).max() < 1e-13 * np.abs(gs).max()


def test_sor_solve_reaches_the_dense_solution(oracle):
    """SOR at the paper's omega = 1.875 on a warped 17^2 grid, to rtol 1e-12, against numpy's
    dense solve of the same system."""
    inst = I.config1(17)
    P = oracle.prepare(inst)
    phi, sw, hist = oracle.sor_solve(P.A, P.b, P.phi0, omega=1.875, rtol=1e-12, max_sweeps=20000, check=4)
    ref = oracle.dense_solve(P.A, P.b) + P.phi0 * ~inst.grid.interior_mask()
    assert hist[-1] <= 1e-12 and sw < 20000
    m = inst.grid.interior_mask()
    assert np.abs(phi[m] - ref[m]).max() < 1e-10 * np.abs(ref[m]).max()


# ---------------------------------------------------------------- Neumann sides (Sec. 4.1, Eq. 28)
def _neumann_solution(oracle, inst, rtol=1e-14):
    P = oracle.prepare(inst)
    phi, _, _ = oracle.pcg_solve(P.A, P.b, P.phi0, rtol=rtol, max_iters=400, stagnate=5)
    return P.extract(phi)


@pytest.mark.parametrize("n", [17, 33, 65])
def test_semi_annulus_is_the_one_dimensional_radial_solution(oracle, n):
    """The polar map gives eps = diag(r, 1/r) and rows that are all alike, so with zero normal
    derivative on the two straight sides the discrete solution cannot depend on theta: every
    row equals the solution of the 1-D radial problem -d/dr(r dphi/dr) = 0 discretized with
    the same face means (r_i + r_{i+1}) / 2, solved here by numpy."""
    inst = I.semi_annulus(n)
    phi = _neumann_solution(oracle, inst)
    g = inst.grid
    r = g.x0 + g.hx * np.arange(g.nx)
    e = 0.5 * (r[:-1] + r[1:])
    N = g.nx - 2
    M = np.zeros((N, N))
    rhs = np.zeros(N)
    for k in range(N):
        M[k, k] = e[k] + e[k + 1]
        if k > 0:
            M[k, k - 1] = -e[k]
        if k < N - 1:
            M[k, k + 1] = -e[k + 1]
    rhs[0] += e[0] * 1.0  # phi0 = 1 at r = a; 0 at r = R
    ref = np.concatenate([[1.0], np.linalg.solve(M, rhs), [0.0]])
    assert np.abs(phi - ref[None, :]).max() < 1e-12


def test_semi_annulus_converges_at_second_order_to_eq_28a(oracle):
    errs = []
    for n in (33, 65, 129):
        inst = I.semi_annulus(n)
        phi = _neumann_solution(oracle, inst)
        errs.append(np.abs(phi - inst.exact).max())
    assert errs[0] / errs[1] > 3.6 and errs[1] / errs[2] > 3.6, errs


def test_neumann_manufactured_solution_converges_at_second_order(oracle):
    """phi = sin(pi x) cos(pi y) varies along the Neumann sides: the boundary rows are
    exercised, not only the interior."""
    errs = []
    for n in (17, 33, 65):
        inst = I.neumann_manufactured(n)
        phi = _neumann_solution(oracle, inst)
        errs.append(np.abs(phi - inst.exact).max())
    assert errs[0] / errs[1] > 3.6 and errs[1] / errs[2] > 3.6, errs


def _skew_map(x, y):
    return x + 0.08 * np.sin(np.pi * x) * np.cos(np.pi * y), y + 0.08 * np.sin(np.pi * x) * np.sin(np.pi * y)


@pytest.mark.parametrize("n", [33, 65])
def test_neumann_reflection_equals_the_doubled_problem_of_a_skewed_grid(oracle, n):
    """A skewed mapped grid (eps_xy != 0 inside) that is itself mirror-symmetric about both y
    sides: the Neumann problem on [0,1]^2 must equal the periodic problem on y in [-1, 1)
    built directly from the map (central differences everywhere, y' jumping by 2 across the
    seam).  The two differ only by the one-sided Jacobian on the Neumann rows, O(h^2); an
    eps_xy of the wrong sign in the mirrored half would leave an O(1) difference."""
    g = I.Grid(n, n, neumann_y=True)
    x, y = g.coords()
    xp, yp = _skew_map(x, y)
    rho = 1.0 + xp * np.cos(np.pi * yp)
    inst = I.Instance("skew", g, I.MapSpec("grid", xp=xp, yp=yp), rho, bc=np.zeros(g.shape))
    phi = _neumann_solution(oracle, inst)
    gd = oracle.doubled_grid(g)
    xd, yd = gd.coords()
    xpd, ypd = _skew_map(xd, yd)
    direct = I.Instance("skew2", gd, I.MapSpec("grid", xp=xpd, yp=ypd, jump=(0.0, 2.0)),
                        1.0 + xpd * np.cos(np.pi * ypd), bc=np.zeros(gd.shape))
    Pd = oracle.prepare(direct)
    phid, _, _ = oracle.pcg_solve(Pd.A, Pd.b, Pd.phi0, rtol=1e-14, max_iters=400, stagnate=5)
    _, _, take = oracle.neumann_rows(n)
    diff = np.abs(phi - phid[take]).max() / np.abs(phi).max()
    assert diff < 2.0 * g.hx ** 2, diff


# ---------------------------------------------------------------- weighted Jacobi (smoother 1)
@pytest.mark.parametrize("case", ["inclusion", "annulus"])
def test_jacobi_sweep_equals_the_matrix_definition(oracle, case):
    """One weighted-Jacobi sweep (Sec. 3's smoother choice, omega_J = 4/5) is
    x + omega diag(A)^-1 (b - A x) at the unknowns, the boundary ring untouched.  A and its
    diagonal come from the independent sparse construction, not from the oracle's couplings;
    a wrong sign, a missing omega or a wrong diagonal fails here."""
    inst = {"inclusion": lambda: I.inclusion_instance(33, 0.25, 10.0, 8),
            "annulus": lambda: I.annulus_log(33)}[case]()
    g = inst.grid
    P = oracle.prepare(inst)
    A = X.full_operator(g, P.exx, P.exy, P.eyy)
    d = A.diagonal()
    rng = np.random.default_rng(21)
    x = rng.standard_normal(g.shape)
    b = rng.standard_normal(g.shape) * np.abs(d).max()
    u = X.unknown_ids(g)
    want = x.ravel().copy()
    r = b.ravel() - A @ x.ravel()
    want[u] += 0.8 * r[u] / d[u]
    got = oracle.smooth(P.A, x, b, sweeps=1, smoother=oracle.SMOOTHER_JACOBI, omega_j=0.8).ravel()
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-14 * scale * 10, np.abs(got - want).max() / scale
    m = ~g.interior_mask().ravel()
    assert np.array_equal(got[m], x.ravel()[m])
    # two sweeps are the map applied twice
    y = want.reshape(g.shape)
    want2 = y.ravel().copy()
    want2[u] += 0.8 * (b.ravel() - A @ y.ravel())[u] / d[u]
    got2 = oracle.smooth(P.A, x, b, sweeps=2, smoother=oracle.SMOOTHER_JACOBI, omega_j=0.8).ravel()
    assert np.abs(got2 - want2).max() <= 1e-13 * np.abs(want2).max()


@pytest.mark.parametrize("omega", [0.8, 1.2])
def test_jacobi_contraction_factor_matches_the_one_dimensional_spectrum(oracle, omega):
    """On a row of the 1-D Poisson matrix (diag 2, neighbours -1; rows decoupled) the
    weighted-Jacobi iteration matrix I - omega D^-1 A has the eigenvalues
    1 - omega (1 - cos(k pi h)), k = 1..N, h = 1/(N+1).  With b = 0 the iterate is the error;
    its measured asymptotic growth per sweep must equal the largest |eigenvalue|: the
    smoothest mode for omega = 0.8 (0.9846 at N = 15), the most oscillatory one for
    omega = 1.2 (1.377: the iteration diverges)."""
    N = 15
    A = _rows_decoupled_laplacian(N)
    h = 1.0 / (N + 1)
    lam = 1.0 - omega * (1.0 - np.cos(np.arange(1, N + 1) * np.pi * h))
    rho = np.abs(lam).max()
    rng = np.random.default_rng(9)
    phi = np.zeros(A.cE.shape)
    phi[1, 1:-1] = rng.standard_normal(N)
    b = np.zeros(A.cE.shape)
    norms = []
    for _ in range(600):
        phi = oracle.smooth(A, phi, b, sweeps=1, smoother=oracle.SMOOTHER_JACOBI, omega_j=omega)
        norms.append(np.linalg.norm(phi))
    rate = (norms[-1] / norms[299]) ** (1.0 / 300)
    assert abs(rate - rho) < 1e-6 * rho, (rate, rho)


# ---------------------------------------------------------------- stretched grid (Sec. 5.1)
def test_sinh_beam_converges_at_second_order(oracle):
    """The Gaussian beam (Eq. 53) on the sinh-stretched grid (Eq. 52) with the beam's
    free-space potential as Dirichlet data (closed form through the exponential integral,
    checked against its own ODE in the next test): the oracle's solution converges to it at
    second order in L1, L2 and Linf (Eqs. 25-27) over 65, 129, 257, 513."""
    o = _orders(oracle, I.sinh_beam, (65, 129, 257, 513))
    assert all(1.9 < v < 2.1 for v in o[-1]), o
    assert all(1.8 < v < 2.2 for v in o[-2]), o


def test_gaussian_potential_solves_the_radial_equation():
    """The closed form used as exact solution satisfies (1/r) (r phi')' = rho0 exp(-r^2/(2
    sigma^2)), i.e. -lap(phi) = rho' of Eq. 53, checked by fourth-order finite differences in
    r; and it is finite and smooth through the beam centre."""
    rho0, sigma = 100.0, 0.5
    f = lambda r: I._gaussian_potential(np.asarray(r, dtype=float), rho0, sigma)
    d = 1e-3
    for r in (0.2, 0.5, 0.7071, 0.9, 1.5, 3.0, 8.0):
        rr = r + d * np.arange(-2, 3)
        p = f(rr)
        d1 = (p[0] - 8 * p[1] + 8 * p[3] - p[4]) / (12 * d)
        d2 = (-p[0] + 16 * p[1] - 30 * p[2] + 16 * p[3] - p[4]) / (12 * d * d)
        lap = d2 + d1 / r
        want = rho0 * np.exp(-r * r / (2 * sigma * sigma))
        assert abs(lap - want) < 1e-6 * max(1.0, want), (r, lap, want)
    c = f([0.0, 1e-4])
    assert abs(c[1] - c[0]) < 1e-5


@pytest.mark.parametrize("periodic", [False, True])
def test_nodal_coarsening_is_full_weighting_inside_and_injection_on_the_ring(oracle, periodic):
    """The tensor coarsening of the rediscretized hierarchy: at coarse unknowns it is the
    full-weighting restriction (pinned by R = P^T / 4), on the boundary ring the coincident
    fine value, and it reproduces a linear field exactly inside."""
    rng = np.random.default_rng(5)
    g = I.Grid(33, 33, periodic_y=periodic)
    gc = I.Grid(17, 17, periodic_y=periodic)
    f = rng.standard_normal(g.shape)
    fc = oracle.coarsen_nodal(g.nx, g.ny, periodic, f)
    inner = gc.interior_mask()
    r = oracle.restrict(g.nx, g.ny, periodic, f)
    assert np.abs(fc[inner] - r[inner]).max() < 1e-15 * np.abs(f).max()
    ring = ~inner
    assert np.array_equal(fc[ring], f[::2, ::2][: fc.shape[0]][ring])
    x, y = g.coords()
    lin = 0.3 + 1.7 * x - 0.9 * y if not periodic else 0.3 + 1.7 * x  # periodic rows: no y trend
    xc, yc = gc.coords()
    lin_c = 0.3 + 1.7 * xc - 0.9 * yc if not periodic else 0.3 + 1.7 * xc
    assert np.abs(oracle.coarsen_nodal(g.nx, g.ny, periodic, lin) - lin_c).max() < 1e-14


@pytest.mark.parametrize("periodic", [False, True])
def test_rediscretized_identity_levels_are_textbook_laplacians(oracle, periodic):
    """For the identity map every rediscretized level is the 5-point Laplacian of its own
    spacing (the coarsened tensor stays the identity)."""
    g = I.Grid(65, 65, 0.0, 0.0, 1.0, 2.0, periodic_y=periodic)
    P = oracle.prepare(I.Instance("id", g, I.MapSpec("identity"), np.zeros(g.shape)))
    ops = oracle.rediscretized_hierarchy(g, P.exx, P.exy, P.eyy)
    assert len(ops) >= 3
    hx, hy = g.hx, g.hy
    for A in ops:
        gl = I.Grid(A.nx, A.ny, 0.0, 0.0, 1.0, 2.0, periodic_y=periodic)
        m = gl.interior_mask()
        assert np.allclose(A.diag[m], 2 / hx ** 2 + 2 / hy ** 2, rtol=1e-13)
        inner_e = m.copy()
        inner_e[:, -2:] = False
        assert np.allclose(A.cE[inner_e], -1 / hx ** 2, rtol=1e-13)
        assert np.abs(A.cNE).max() == 0 and np.abs(A.cNW).max() == 0
        hx, hy = 2 * hx, 2 * hy
