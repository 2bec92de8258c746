"""Zebra x-line Gauss-Seidel on the GPU (mgk_line_*: cyclic reduction of every row with
factors computed once per operator) against the oracle's line smoother (Thomas algorithm
per row: oracle.line_rows, oracle.smooth with SMOOTHER_XLINE), then the line-smoothed
V-cycle (mgk_vcycle_line_*) against oracle.Hierarchy(smoother=SMOOTHER_XLINE), and line-
smoothed solves through mg_solve / mg_batch_solve.

Tolerances.  Both sides solve the same diagonally dominant tridiagonal row systems.  On
these cases the dominance margin (the cross-row coupling) keeps their condition numbers
small (about 2 + 2 (x coupling / y coupling), below 130 on the annulus of Eq. 29), and the
two orders of elimination agree to a small multiple of cond * eps.  FP64: 1e-12 relative to
max |phi|.  FP32: the operator and data are rounded to FP32 (relative 6e-8) and the rows
solved in FP32, so 2e-5 relative, as for the FP32 point smoother."""
import ctypes as C

import numpy as np
import pytest

from paper_2602_01888_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _rect(nx, ny, mp=("affine", (1.0, 0.25, -0.1, 1.05)), ly=0.5):
    return lambda: I.Instance("r", I.Grid(nx, ny, 0.0, 0.0, 1.0, ly), I.MapSpec(*mp), np.ones((ny, nx)))


CASES = {
    "sine_129": lambda: I.config1(129),
    "annulus_129": lambda: I.annulus_log(129),
    "incl_257": lambda: I.inclusion_instance(257, 0.25, 10.0, 21),
    "ragged_193x97": _rect(193, 97),
    "one_unknown_3x9": _rect(3, 9),          # rows of one unknown (N = 1, padded to 2)
    "two_unknowns_4x7": _rect(4, 7),         # N = 2 = padded length
    "pow2_34x33": _rect(34, 33, ("sine_warp", (0.05,))),   # N = 32 exactly
    "pow2p1_35x17": _rect(35, 17, ("sine_warp", (0.05,))),  # N = 33: padded to 64
    "annulus_513": lambda: I.annulus_log(513),
}


def _dev(torch, a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def _op(libmg, torch, A, dt):
    t = [_dev(torch, a, dt) for a in (A.cE, A.cN, A.cNE, A.cNW, A.diag, 1.0 / A.diag)]
    return t, libmg.op_struct(t, A.nx, A.ny, A.periodic, f32=(dt == torch.float32))


def _factors(libmg, torch, A, s, dt, tag):
    n = libmg.lib().mgk_line_factor_elems(A.nx, A.ny, int(A.periodic))
    f = torch.zeros(max(n, 1), dtype=dt, device="cuda")
    libmg.mgk(f"mgk_line_factor_{tag}", C.byref(s), f.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return f


def _data(A, seed):
    rng = np.random.default_rng(seed)
    phi = rng.standard_normal(A.cE.shape)  # random Dirichlet ring too: the row ends matter
    b = rng.standard_normal(A.cE.shape) * np.abs(A.diag).max()
    return phi, b


def _rel(got, ref):
    return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_half_sweeps_match_oracle(libmg, oracle, cuda, case, prec):
    torch = cuda
    inst = CASES[case]()
    A = oracle.prepare(inst).A
    dt = torch.float64 if prec == "f64" else torch.float32
    keep, s = _op(libmg, torch, A, dt)
    f = _factors(libmg, torch, A, s, dt, prec)
    phi, b = _data(A, 5)
    bd = _dev(torch, b, dt)
    stream = torch.cuda.current_stream().cuda_stream
    for par in (0, 1):
        x = _dev(torch, phi, dt)
        libmg.mgk(f"mgk_line_rows_{prec}", C.byref(s), f.data_ptr(), x.data_ptr(), bd.data_ptr(), par, stream)
        torch.cuda.synchronize()
        got = x.double().cpu().numpy()
        ref = oracle.line_rows(A, phi, b, par)
        err = _rel(got, ref)
        assert err < (1e-12 if prec == "f64" else 2e-5), (case, prec, par, err)
        # only the unknowns of rows of this parity change: the rest is untouched (bitwise)
        moved = np.zeros(A.cE.shape, bool)
        moved[par::2, 1:-1] = True
        if not A.periodic:
            moved[0, :] = moved[-1, :] = False
        start = phi.astype(np.float32).astype(np.float64) if prec == "f32" else phi
        assert np.array_equal(got[~moved], start[~moved]), (case, prec, par)


@pytest.mark.parametrize("case", ["sine_129", "annulus_129", "ragged_193x97", "pow2p1_35x17"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("sweeps,rev", [(1, 0), (2, 1), (3, 0)])
def test_sweeps_match_oracle(libmg, oracle, cuda, case, prec, sweeps, rev):
    torch = cuda
    inst = CASES[case]()
    A = oracle.prepare(inst).A
    dt = torch.float64 if prec == "f64" else torch.float32
    keep, s = _op(libmg, torch, A, dt)
    f = _factors(libmg, torch, A, s, dt, prec)
    phi, b = _data(A, 7)
    x, b_d = _dev(torch, phi, dt), _dev(torch, b, dt)
    libmg.mgk(f"mgk_line_smooth_{prec}", C.byref(s), f.data_ptr(), x.data_ptr(), b_d.data_ptr(),
              sweeps, rev, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    ref = oracle.smooth(A, phi, b, sweeps=sweeps, reverse=bool(rev), smoother=oracle.SMOOTHER_XLINE)
    err = _rel(x.double().cpu().numpy(), ref)
    assert err < (1e-12 if prec == "f64" else 2e-5), (case, prec, sweeps, rev, err)


@pytest.mark.parametrize("prec,nx", [("f64", 8193), ("f32", 16385)])
def test_longest_rows(libmg, oracle, cuda, prec, nx):
    """The longest rows each precision supports (8192 / 16384 unknowns: the factor kernel's
    three row arrays fill 192 KB of shared memory); one node more is refused.  Square cells
    keep the row systems well conditioned (with hy >> hx their condition number grows like
    (hy / hx)^2, and FP32 rows then differ from FP64 by that times 6e-8)."""
    torch = cuda
    inst = _rect(nx, 9, ("sine_warp", (0.05,)), ly=8.0 / (nx - 1))()
    A = oracle.prepare(inst).A
    dt = torch.float64 if prec == "f64" else torch.float32
    keep, s = _op(libmg, torch, A, dt)
    f = _factors(libmg, torch, A, s, dt, prec)
    phi, b = _data(A, 9)
    x = _dev(torch, phi, dt)
    stream = torch.cuda.current_stream().cuda_stream
    b_d = _dev(torch, b, dt)
    libmg.mgk(f"mgk_line_smooth_{prec}", C.byref(s), f.data_ptr(), x.data_ptr(), b_d.data_ptr(), 1, 0, stream)
    torch.cuda.synchronize()
    ref = oracle.smooth(A, phi, b, sweeps=1, smoother=oracle.SMOOTHER_XLINE)
    assert _rel(x.double().cpu().numpy(), ref) < (1e-12 if prec == "f64" else 2e-5)
    big = _rect(nx + 2, 5, ("sine_warp", (0.05,)))()
    Ab = oracle.prepare(big).A
    kb, sb = _op(libmg, torch, Ab, dt)
    fb = torch.zeros(8, dtype=dt, device="cuda")
    rc = getattr(libmg.lib(), f"mgk_line_factor_{prec}")(C.byref(sb), fb.data_ptr(), stream)
    assert rc == 1


def _gpu_vcycle_line(libmg, torch, ops, r, prec, nu):
    dt = torch.float64 if prec == "f64" else torch.float32
    keep, X, B, T, F = [], [], [], [], []
    arr = ((libmg.mgk_op_f64 if prec == "f64" else libmg.mgk_op_f32) * len(ops))()
    for l, A in enumerate(ops):
        t, s = _op(libmg, torch, A, dt)
        keep.append(t)
        arr[l] = s
        shape = A.cE.shape
        X.append(torch.zeros(shape, dtype=dt, device="cuda"))
        B.append(_dev(torch, r, dt) if l == 0 else torch.zeros(shape, dtype=dt, device="cuda"))
        T.append(torch.zeros(shape, dtype=dt, device="cuda"))
        if l < len(ops) - 1:
            F.append(_factors(libmg, torch, A, s, dt, prec))
    Ac = ops[-1]
    m = (Ac.nx - 2) * (Ac.nyr if Ac.periodic else Ac.ny - 2)
    inv = torch.zeros(m * m, dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    t64, s64 = _op(libmg, torch, Ac, torch.float64)
    stream = torch.cuda.current_stream().cuda_stream
    libmg.mgk("mgk_coarse_factor", C.byref(s64), inv.data_ptr(), status.data_ptr(), stream)
    ptrs = lambda L: (C.c_void_p * len(L))(*[t.data_ptr() for t in L])
    libmg.mgk(f"mgk_vcycle_line_{prec}", len(ops), arr, ptrs(X), ptrs(B), ptrs(T), inv.data_ptr(),
              ptrs(F), nu[0], nu[1], stream)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return X[0].double().cpu().numpy()


@pytest.mark.parametrize("case", ["sine_129", "annulus_129", "incl_257", "ragged_193x97", "annulus_513"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("nu", [(2, 2), (1, 1), (0, 1)])
def test_vcycle_line_matches_oracle(libmg, oracle, cuda, case, prec, nu):
    inst = CASES[case]()
    P = oracle.prepare(inst)
    ops = oracle.hierarchy(P.A)
    H = oracle.Hierarchy(P.A, smoother=oracle.SMOOTHER_XLINE, nu1=nu[0], nu2=nu[1])
    rng = np.random.default_rng(33)
    r = rng.standard_normal(inst.grid.shape) * inst.grid.interior_mask() * np.abs(P.A.diag).max()
    ref = H.vcycle(r)
    got = _gpu_vcycle_line(libmg, cuda, ops, r, prec, nu)
    assert _rel(got, ref) < (1e-12 if prec == "f64" else 2e-5), (case, prec, nu)


@pytest.fixture(scope="module")
def ctx(libmg, cuda):
    c = libmg.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_line_solve_on_annulus(libmg, oracle, ctx, prec):
    """FCG preconditioned by the line-smoothed V(2,2) on the annulus of Eq. 29 (x coupling
    up to 62 times the y coupling): the oracle's PCG with the same cycle takes the same
    number of iterations (FP64), the solution matches the oracle's, and the point smoother
    needs several times more iterations on the same problem."""
    inst = I.annulus_log(257)
    P = oracle.prepare(inst)
    ref, it_ref, _ = oracle.pcg_solve(P.A, P.b, P.phi0, rtol=1e-10, max_iters=100, stagnate=0,
                                      smoother=oracle.SMOOTHER_XLINE)
    pr = libmg.Problem(ctx, inst, libmg.make_opts(prec, "fcg", rtol=1e-10, smoother="xline"))
    phi, st = pr.solve()
    _, st_gs = pr.solve(opts=libmg.make_opts(prec, "fcg", rtol=1e-10, smoother="gs4"))
    pr.close()
    m = inst.grid.interior_mask()
    assert oracle.rel_l2(phi, ref, m) < 1e-8
    if prec == "fp64":
        assert abs(st.iters - it_ref) <= 1, (st.iters, it_ref)
    assert st.iters <= 8 and 3 * st.iters <= st_gs.iters, (st.iters, st_gs.iters)


def test_factors_follow_update_transform_and_batch(libmg, ctx):
    """A problem first solved with the point smoother gets its line factors on its first
    line-smoothed solve; mg_update_transform recomputes them (the moved problem solves
    bitwise like a fresh one); a batch of line-smoothed solves equals the single solves."""
    a = [I.inclusion_instance(*s) for s in I.config4_specs(4, seed0=7300)]
    b = [I.inclusion_instance(x.grid.nx, r, e, sd) for x, (_, r, e, sd) in zip(a, I.config4_specs(4, seed0=7400))]
    lo = libmg.make_opts("mixed", "fcg", rtol=1e-9, smoother="xline")
    go = libmg.make_opts("mixed", "fcg", rtol=1e-9, smoother="gs4")
    moved = [libmg.Problem(ctx, x, go) for x in a]
    for p in moved:
        p.solve()
        p.solve(opts=lo)
    for p, x in zip(moved, b):
        libmg.mg_update_transform(p.h, x.grid, x.map, np.ascontiguousarray(x.eps_phys))
        p.inst = x
    alone = []
    for p, x in zip(moved, b):
        fresh = libmg.Problem(ctx, x, lo)
        want, _ = fresh.solve()
        got, st = p.solve(opts=lo)
        assert np.array_equal(want, got) and st.rel_residual <= 1e-9
        alone.append(got)
        fresh.close()
    phis = [np.zeros(x.grid.shape) for x in b]
    stats = libmg.mg_batch_solve(ctx.h, [p.h for p in moved], [np.ascontiguousarray(x.rho_phys) for x in b],
                                 None, phis, lo)
    for k, (w, g) in enumerate(zip(alone, phis)):
        assert np.array_equal(w, g), k
    assert all(s.rel_residual <= 1e-9 for s in stats)
    for p in moved:
        p.close()


def test_line_smoother_refuses_too_long_rows(libmg, ctx):
    """Rows of 8255 unknowns exceed the FP64 line kernels (8192 at most): the solve is refused
    with MG_ERR_SIZE before anything runs, and the point smoother still solves the problem."""
    g = I.Grid(8257, 129, 0.0, 0.0, 1.0, 0.0155)  # coarsens to 130 x 3 (128 unknowns)
    inst = I.Instance("w", g, I.MapSpec("identity", ()), np.zeros(g.shape), bc=np.ones(g.shape))
    p = libmg.Problem(ctx, inst, libmg.make_opts("fp64", "fcg", coarse_max=256))
    with pytest.raises(libmg.MGError) as e:
        p.solve(opts=libmg.make_opts("fp64", "fcg", coarse_max=256, smoother="xline"))
    assert e.value.status == libmg.MG_ERR_SIZE
    phi, st = p.solve()
    assert st.rel_residual <= 1e-10
    p.close()


# Rows of 1025 to 4095 unknowns (padded lengths 2048 and 4096) are solved by the partition
# method: segments of Np / 256 unknowns whose interiors are eliminated per thread, then the
# separator system by cyclic reduction.  Square cells keep FP32 rows well conditioned.
PART_CASES = {
    "rect_1027x9": _rect(1027, 9, ("sine_warp", (0.05,)), ly=8.0 / 1026),    # N = 1025: S = 8, most padded
    "rect_2049x9": _rect(2049, 9, ("sine_warp", (0.05,)), ly=8.0 / 2048),    # S = 8
    "rect_3073x9": _rect(3073, 9, ("affine", (1.0, 0.2, -0.1, 1.05)), ly=8.0 / 3072),  # S = 16, padded
    "rect_4097x9": _rect(4097, 9, ("sine_warp", (0.05,)), ly=8.0 / 4096),    # S = 16
    "annulus_2049": lambda: I.annulus_log(2049),                            # periodic, S = 8
}


@pytest.mark.parametrize("case", list(PART_CASES))
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_partition_half_sweeps_match_oracle(libmg, oracle, cuda, case, prec):
    torch = cuda
    inst = PART_CASES[case]()
    A = oracle.prepare(inst).A
    dt = torch.float64 if prec == "f64" else torch.float32
    keep, s = _op(libmg, torch, A, dt)
    f = _factors(libmg, torch, A, s, dt, prec)
    phi, b = _data(A, 15)
    bd = _dev(torch, b, dt)
    stream = torch.cuda.current_stream().cuda_stream
    for par in (0, 1):
        x = _dev(torch, phi, dt)
        libmg.mgk(f"mgk_line_rows_{prec}", C.byref(s), f.data_ptr(), x.data_ptr(), bd.data_ptr(), par, stream)
        torch.cuda.synchronize()
        got = x.double().cpu().numpy()
        ref = oracle.line_rows(A, phi, b, par)
        err = _rel(got, ref)
        assert err < (1e-12 if prec == "f64" else 2e-5), (case, prec, par, err)
        moved = np.zeros(A.cE.shape, bool)
        moved[par::2, 1:-1] = True
        if not A.periodic:
            moved[0, :] = moved[-1, :] = False
        start = phi.astype(np.float32).astype(np.float64) if prec == "f32" else phi
        assert np.array_equal(got[~moved], start[~moved]), (case, prec, par)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("nu", [(1, 1), (2, 2)])
def test_partition_vcycle_matches_oracle(libmg, oracle, cuda, prec, nu):
    """A line-smoothed V-cycle whose finest level (2049 wide) uses the partition solver in all
    three half-sweep forms (stored iterate, zero iterate, coarse correction interpolated in)
    and whose coarser levels use cyclic reduction, against the oracle's cycle."""
    inst = I.annulus_log(2049)
    P = oracle.prepare(inst)
    ops = oracle.hierarchy(P.A)
    H = oracle.Hierarchy(P.A, smoother=oracle.SMOOTHER_XLINE, nu1=nu[0], nu2=nu[1])
    rng = np.random.default_rng(35)
    r = rng.standard_normal(inst.grid.shape) * inst.grid.interior_mask() * np.abs(P.A.diag).max()
    ref = H.vcycle(r)
    got = _gpu_vcycle_line(libmg, cuda, ops, r, prec, nu)
    assert _rel(got, ref) < (1e-12 if prec == "f64" else 2e-5), (prec, nu)
