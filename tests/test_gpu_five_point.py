"""5-point forms of the finest-level kernels.  A map whose transformed tensor has no cross
term (the polar map of Eq. 29, the sinh stretching of Eq. 52, the identity) gives an
operator with zero NE / NW couplings (the coefficient build writes eps_xy = 0 exactly for
them); the library then runs kernels that skip those couplings.  Adding a zero product
changes no floating-point sum, so every 5-point form must equal the 9-point form on the same
arrays exactly.  The coefficient build of those maps is checked against the oracle in
test_gpu_kernels, and whole solves here against the oracle's phi*."""
import ctypes as C

import numpy as np
import pytest

from paper_2602_01888_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = {
    "annulus_65": lambda: I.annulus_log(65),            # polar, periodic in theta
    "semi_annulus_33": lambda: I.semi_annulus(33),      # polar, Neumann sides (reflected grid)
    "sinh_65": lambda: I.sinh_beam(65),                 # sinh stretching
    "identity_33x17": lambda: I.Instance("identity", I.Grid(33, 17, 0.0, 0.0, 1.0, 0.5),
                                         I.MapSpec("identity"), I.random_field((17, 33), 3)),
}


def _stream(torch):
    return torch.cuda.current_stream().cuda_stream


def _operator(libmg, torch, inst, five, pitch):
    """Finest operator of an analytic-map instance built by the library's kernels, with the
    5-point flag as given; returns the op struct and its six arrays."""
    g = inst.grid
    z = lambda: torch.zeros((g.nyr, pitch), dtype=torch.float64, device="cuda")
    D, exx, exy, eyy = z(), z(), z(), z()
    folded = torch.zeros(1, dtype=torch.int32, device="cuda")
    prm = (C.c_double * 4)(*(list(inst.map.params) + [0.0] * 4)[:4])
    libmg.mgk("mgk_eps_analytic", libmg.MAP_CODES[inst.map.kind], prm, g.nx, g.ny, int(g.periodic_y),
              g.x0, g.y0, g.hx, g.hy, None, pitch, D.data_ptr(), exx.data_ptr(), exy.data_ptr(),
              eyy.data_ptr(), folded.data_ptr(), _stream(torch))
    ops = [z() for _ in range(6)]
    st = libmg.op_struct(ops, g.nx, g.ny, g.periodic_y, five_point=five)
    libmg.mgk("mgk_assemble", C.byref(st), g.hx, g.hy, exx.data_ptr(), exy.data_ptr(), eyy.data_ptr(),
              _stream(torch))
    torch.cuda.synchronize()
    assert int(folded.item()) == 0
    assert torch.count_nonzero(exy).item() == 0  # eps_xy written as exact zeros for these maps
    return st, ops


def _grid_of(inst):
    # Neumann sides are handled by the solver's reflected grid; the kernels here take the
    # caller's grid as a Dirichlet or periodic one, which is all these checks need
    return inst.grid


@pytest.mark.parametrize("case", list(CASES))
def test_library_classifies_the_maps(libmg, case):
    inst = CASES[case]()
    assert libmg.map_five_point(inst.map)
    assert not libmg.map_five_point(I.MapSpec("sine_warp", (0.1,)))
    assert not libmg.map_five_point(I.MapSpec("affine", (1.1, 0.2, -0.1, 0.9)))
    assert libmg.map_five_point(I.MapSpec("affine", (1.1, 0.0, 0.0, 0.9)))


@pytest.mark.parametrize("case", list(CASES))
def test_five_point_assembly_equals_the_nine_point_form(libmg, cuda, case):
    torch = cuda
    inst = CASES[case]()
    g = _grid_of(inst)
    pitch = (g.nx + 31) // 32 * 32
    st9, ops9 = _operator(libmg, torch, inst, False, pitch)
    st5, ops5 = _operator(libmg, torch, inst, True, pitch)
    for a, b in zip(ops9, ops5):
        assert torch.equal(a, b)
    assert torch.count_nonzero(ops5[2]).item() == 0 and torch.count_nonzero(ops5[3]).item() == 0
    z32 = lambda: torch.zeros((g.nyr, pitch), dtype=torch.float32, device="cuda")
    o9, o5 = [z32() for _ in range(6)], [torch.full((g.nyr, pitch), 7.0, dtype=torch.float32, device="cuda")
                                         for _ in range(6)]
    s9 = libmg.op_struct(o9, g.nx, g.ny, g.periodic_y, f32=True)
    s5 = libmg.op_struct(o5, g.nx, g.ny, g.periodic_y, f32=True, five_point=True)
    libmg.mgk("mgk_op_to_f32", C.byref(st9), C.byref(s9), _stream(torch))
    libmg.mgk("mgk_op_to_f32", C.byref(st5), C.byref(s5), _stream(torch))
    torch.cuda.synchronize()
    for a, b in zip(o9, o5):
        assert torch.equal(a[:, : g.nx], b[:, : g.nx])


@pytest.mark.parametrize("case", list(CASES))
def test_one_pass_assembly_equals_the_separate_kernels(libmg, cuda, case):
    """mgk_assemble_five (couplings, diagonal and the FP32 copy of the level in one pass, which
    the solver uses for maps without cross term) against mgk_assemble followed by
    mgk_op_to_f32 on the same tensor: bitwise equal arrays; the FP32 reciprocal diagonal
    equals the FP32 division of the FP32 diagonal.  A 9-point operator is refused."""
    torch = cuda
    inst = CASES[case]()
    g = inst.grid
    pitch = (g.nx + 31) // 32 * 32
    pf = pitch + 32  # the FP32 copy with a pitch of its own
    st = _stream(torch)
    z = lambda: torch.zeros((g.nyr, pitch), dtype=torch.float64, device="cuda")
    D, exx, exy, eyy = z(), z(), z(), z()
    folded = torch.zeros(1, dtype=torch.int32, device="cuda")
    prm = (C.c_double * 4)(*(list(inst.map.params) + [0.0] * 4)[:4])
    libmg.mgk("mgk_eps_analytic", libmg.MAP_CODES[inst.map.kind], prm, g.nx, g.ny, int(g.periodic_y), g.x0, g.y0,
              g.hx, g.hy, None, pitch, D.data_ptr(), exx.data_ptr(), exy.data_ptr(), eyy.data_ptr(),
              folded.data_ptr(), st)
    ref = [z() for _ in range(6)]
    sref = libmg.op_struct(ref, g.nx, g.ny, g.periodic_y, five_point=True)
    libmg.mgk("mgk_assemble", C.byref(sref), g.hx, g.hy, exx.data_ptr(), exy.data_ptr(), eyy.data_ptr(), st)
    ref32 = [torch.zeros((g.nyr, pf), dtype=torch.float32, device="cuda") for _ in range(6)]
    sref32 = libmg.op_struct(ref32, g.nx, g.ny, g.periodic_y, f32=True, five_point=True)
    libmg.mgk("mgk_op_to_f32", C.byref(sref), C.byref(sref32), st)
    full = lambda shape, dt: torch.full(shape, 7.0, dtype=dt, device="cuda")
    got = [full((g.nyr, pitch), torch.float64) for _ in range(6)]
    got32 = [full((g.nyr, pf), torch.float32) for _ in range(6)]
    alone = [full((g.nyr, pitch), torch.float64) for _ in range(6)]
    sgot = libmg.op_struct(got, g.nx, g.ny, g.periodic_y, five_point=True)
    sgot32 = libmg.op_struct(got32, g.nx, g.ny, g.periodic_y, f32=True, five_point=True)
    salone = libmg.op_struct(alone, g.nx, g.ny, g.periodic_y, five_point=True)
    libmg.mgk("mgk_assemble_five", C.byref(sgot), C.byref(sgot32), g.hx, g.hy, exx.data_ptr(), eyy.data_ptr(), st)
    libmg.mgk("mgk_assemble_five", C.byref(salone), None, g.hx, g.hy, exx.data_ptr(), eyy.data_ptr(), st)
    torch.cuda.synchronize()
    n = g.nx
    for a, b, c in zip(ref, got, alone):
        assert torch.equal(a[:, :n], b[:, :n]) and torch.equal(a[:, :n], c[:, :n])
    for a, b in zip(ref32[:5], got32[:5]):
        assert torch.equal(a[:, :n], b[:, :n])
    assert torch.equal(got32[5][:, :n], 1.0 / got32[4][:, :n])
    assert torch.count_nonzero(got[2][:, :n]).item() == 0 and torch.count_nonzero(got32[3][:, :n]).item() == 0
    s9 = libmg.op_struct(got, g.nx, g.ny, g.periodic_y, five_point=False)
    with pytest.raises(Exception):
        libmg.mgk("mgk_assemble_five", C.byref(s9), None, g.hx, g.hy, exx.data_ptr(), eyy.data_ptr(), st)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_five_point_kernels_equal_the_nine_point_forms(libmg, cuda, case, prec):
    """Gauss-Seidel sweeps, residual + restriction and zebra line sweeps on one operator,
    once with the 5-point flag and once without: bitwise equal results."""
    torch = cuda
    inst = CASES[case]()
    g = _grid_of(inst)
    pitch = (g.nx + 31) // 32 * 32
    st, ops = _operator(libmg, torch, inst, False, pitch)
    dt = torch.float64 if prec == "f64" else torch.float32
    if prec == "f32":
        o32 = [torch.zeros((g.nyr, pitch), dtype=torch.float32, device="cuda") for _ in range(6)]
        s32 = libmg.op_struct(o32, g.nx, g.ny, g.periodic_y, f32=True)
        libmg.mgk("mgk_op_to_f32", C.byref(st), C.byref(s32), _stream(torch))
        ops, st = o32, s32
    s9 = libmg.op_struct(ops, g.nx, g.ny, g.periodic_y, f32=prec == "f32")
    s5 = libmg.op_struct(ops, g.nx, g.ny, g.periodic_y, f32=prec == "f32", five_point=True)
    gen = torch.Generator(device="cuda").manual_seed(7)
    x0 = torch.randn((g.nyr, pitch), dtype=torch.float64, device="cuda", generator=gen).to(dt)
    b = torch.randn((g.nyr, pitch), dtype=torch.float64, device="cuda", generator=gen).to(dt)
    nc, mc = (g.nx - 1) // 2 + 1, (g.ny - 1) // 2 + 1
    pc = (nc + 31) // 32 * 32
    out = {}
    for tag, s in (("9", s9), ("5", s5)):
        x = x0.clone()
        libmg.mgk(f"mgk_smooth_{prec}", C.byref(s), x.data_ptr(), b.data_ptr(), 2, 0, _stream(torch))
        bH = torch.zeros((mc, pc), dtype=dt, device="cuda")
        libmg.mgk(f"mgk_resid_restrict_{prec}", C.byref(s), x.data_ptr(), b.data_ptr(), bH.data_ptr(), pc,
                  _stream(torch))
        xl = x0.clone()
        fac = torch.zeros(libmg.lib().mgk_line_factor_elems(g.nx, g.ny, int(g.periodic_y)), dtype=dt,
                          device="cuda")
        libmg.mgk(f"mgk_line_factor_{prec}", C.byref(s), fac.data_ptr(), _stream(torch))
        libmg.mgk(f"mgk_line_smooth_{prec}", C.byref(s), fac.data_ptr(), xl.data_ptr(), b.data_ptr(), 2, 0,
                  _stream(torch))
        torch.cuda.synchronize()
        out[tag] = (x, bH, xl)
    for a, c in zip(out["9"], out["5"]):
        assert torch.equal(a, c)
    assert not torch.equal(out["5"][0], x0)  # the sweeps did change the iterate


@pytest.mark.parametrize("case", ["annulus_65", "sinh_65", "identity_33x17"])
def test_five_point_galerkin_equals_the_nine_point_form(libmg, cuda, case):
    """The coarse operator from a 5-point fine operator skips the zero products: same arrays."""
    torch = cuda
    inst = CASES[case]()
    g = _grid_of(inst)
    pitch = (g.nx + 31) // 32 * 32
    st, ops = _operator(libmg, torch, inst, False, pitch)
    nc, mc = (g.nx - 1) // 2 + 1, (g.ny - 1) // 2 + 1
    mrc = mc - 1 if g.periodic_y else mc
    pc = (nc + 31) // 32 * 32
    out = {}
    for five in (False, True):
        fine = libmg.op_struct(ops, g.nx, g.ny, g.periodic_y, five_point=five)
        co = [torch.full((mrc, pc), 3.0, dtype=torch.float64, device="cuda") for _ in range(6)]
        cs = libmg.op_struct(co, nc, mc, g.periodic_y)
        libmg.mgk("mgk_galerkin", C.byref(fine), C.byref(cs), _stream(torch))
        torch.cuda.synchronize()
        out[five] = [a[:, :nc] for a in co]
    for a, b in zip(out[False], out[True]):
        assert torch.equal(a, b)
    assert torch.count_nonzero(out[True][2]).item() > 0  # the coarse level is 9-point


def _ref(oracle, inst):
    P = oracle.prepare(inst)
    phi, it, hist = oracle.pcg_solve(P.A, P.b, P.phi0, rtol=0.0, max_iters=400, stagnate=10)
    return phi


@pytest.fixture(scope="module")
def ctx(libmg, cuda):
    c = libmg.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("precision,smoother", [("mixed", "xline"), ("fp64", "gs4"), ("fp64", "xline")])
def test_update_between_five_and_nine_point_maps(libmg, oracle, ctx, precision, smoother):
    """One problem on the annulus grid moved polar -> sine warp -> polar by
    mg_update_transform: each solve equals a fresh problem's bitwise (the graphs captured
    for the other stencil are not reused) and the oracle's phi* within the path's bound."""
    polar = I.annulus_log(129)
    g = polar.grid
    warped = I.Instance("warped_annulus", g, I.MapSpec("sine_warp", (0.02,)),
                        I.random_field(g.shape, 5), bc=polar.bc)
    nu = (1, 1) if smoother == "xline" else (2, 2)
    # the random charge makes the warped problem's error exceed its residual: solve to 1e-12
    opts = libmg.make_opts(precision, "fcg", rtol=1e-12, max_iters=200, nu1=nu[0], nu2=nu[1],
                           smoother=smoother)
    tol = 1e-10 if precision == "fp64" else 1e-9
    prob = libmg.Problem(ctx, polar, opts)
    assert libmg.problem_five_point(prob.h)
    phi_a, _ = prob.solve()
    seq = [(warped, False), (polar, True)]
    for inst, five in seq:
        eps = None if inst.eps_phys is None else np.ascontiguousarray(inst.eps_phys)
        libmg.mg_update_transform(prob.h, g, inst.map, eps)
        assert libmg.problem_five_point(prob.h) == five
        phi, st = prob.solve(rho=np.ascontiguousarray(inst.rho_phys))
        fresh = libmg.Problem(ctx, inst, opts)
        phi_f, _ = fresh.solve()
        fresh.close()
        assert np.array_equal(phi, phi_f), inst.name
        err = oracle.rel_l2(phi, _ref(oracle, inst), g.interior_mask())
        assert err <= tol, (inst.name, err, st.iters)
    assert np.array_equal(phi, phi_a)
    prob.close()
