"""Rediscretized coarse operators (MG_COARSE_REDISCRETIZE): the tensor coarsening and the
coarse assembly through the C ABI against the oracle's rediscretized hierarchy level by level,
and whole solves with such hierarchies against the oracle's phi* (the finest operator, hence
phi*, is the same as with Galerkin coarse levels)."""
import ctypes as C

import numpy as np
import pytest

from paper_2602_01888_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-9

CASES = {
    "sine_warp_65": lambda: I.config1(65),
    "annulus_65": lambda: I.annulus_log(65),
    "inclusion_129": lambda: I.inclusion_instance(129, 0.25, 10.0, 7),
    "rect_65x33": lambda: I.Instance("rect", I.Grid(65, 33, 0.0, 0.0, 1.0, 0.5),
                                     I.MapSpec("sine_warp", (0.05,)), I.random_field((33, 65), 1)),
}


def _stream(torch):
    return torch.cuda.current_stream().cuda_stream


def _dev(torch, a, pitch):
    a = np.asarray(a, dtype=np.float64)
    t = torch.zeros((a.shape[0], pitch), dtype=torch.float64, device="cuda")
    t[:, : a.shape[1]] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t


@pytest.mark.parametrize("case", list(CASES))
def test_coarsening_and_coarse_assembly_match_the_oracle(libmg, oracle, cuda, case):
    torch = cuda
    inst = CASES[case]()
    g = inst.grid
    P = oracle.prepare(inst)
    ref = oracle.rediscretized_hierarchy(g, P.exx, P.exy, P.eyy)
    assert len(ref) >= 3
    e = [P.exx, P.exy, P.eyy]
    nx, ny, hx, hy = g.nx, g.ny, g.hx, g.hy
    pitch = (nx + 31) // 32 * 32
    ed = [_dev(torch, a, pitch) for a in e]
    scratch = [torch.zeros_like(ed[0]) for _ in range(6)]
    fine = libmg.op_struct(scratch, nx, ny, g.periodic_y)
    for lvl, A in enumerate(ref[1:], start=1):
        nxc, nyc = (nx - 1) // 2 + 1, (ny - 1) // 2 + 1
        nyrc = nyc - 1 if g.periodic_y else nyc
        pc = (nxc + 31) // 32 * 32
        cd = [torch.full((nyrc, pc), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]
        ops = [torch.zeros((nyrc, pc), dtype=torch.float64, device="cuda") for _ in range(6)]
        coarse = libmg.op_struct(ops, nxc, nyc, g.periodic_y)
        assert libmg.lib().mgk_coarsen_eps(C.byref(fine), C.byref(coarse), *[a.data_ptr() for a in ed],
                                            *[a.data_ptr() for a in cd], _stream(torch)) == 0
        hx, hy = 2 * hx, 2 * hy
        libmg.mgk("mgk_assemble", C.byref(coarse), hx, hy, cd[0].data_ptr(), cd[1].data_ptr(),
                  cd[2].data_ptr(), _stream(torch))
        torch.cuda.synchronize()
        scale = np.abs(A.diag).max()
        for got, want in zip(ops[:5], A.arrays()):
            assert np.abs(got[:, :nxc].cpu().numpy() - want).max() <= 1e-13 * scale, (case, lvl)
        nx, ny, pitch, fine, ed = nxc, nyc, pc, coarse, cd
    with pytest.raises(Exception):
        libmg.mgk("mgk_coarsen_eps", C.byref(fine), C.byref(fine), *[a.data_ptr() for a in ed],
                  *[a.data_ptr() for a in ed], _stream(torch))


def _ref(oracle, inst):
    P = oracle.prepare(inst)
    phi, _, _ = oracle.pcg_solve(P.A, P.b, P.phi0, rtol=0.0, max_iters=400, stagnate=10)
    return P.extract(phi)


@pytest.fixture(scope="module")
def ctx(libmg, cuda):
    c = libmg.Context(0)
    yield c
    c.close()


# residual tolerances of the Galerkin solve tests for the same instances
SOLVES = {
    "sine_warp_129": (lambda: I.config1(129), "gs4", (2, 2), 1e-10),
    "annulus_129": (lambda: I.annulus_log(129), "xline", (1, 1), 1e-11),
    "inclusion_257": (lambda: I.inclusion_instance(257, 0.25, 10.0, 2), "gs4", (2, 2), 1e-10),
    "semi_annulus_65": (lambda: I.semi_annulus(65), "gs4", (2, 2), 1e-12),
}


@pytest.mark.parametrize("case", list(SOLVES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_rediscretized_solves_match_oracle(libmg, oracle, ctx, case, precision):
    make, smoother, nu, rtol = SOLVES[case]
    inst = make()
    opts = libmg.make_opts(precision, "fcg", rtol=rtol, max_iters=300, smoother=smoother, nu1=nu[0],
                           nu2=nu[1], coarse_op="rediscretize")
    prob = libmg.Problem(ctx, inst, opts)
    phi, st = prob.solve()
    err = oracle.rel_l2(phi, _ref(oracle, inst), inst.grid.interior_mask())
    assert err <= (FP64_TOL if precision == "fp64" else MIXED_TOL), (case, precision, err, st.iters)
    # a solve asking for the other coarse operator is refused
    with pytest.raises(Exception):
        prob.solve(opts=libmg.make_opts(precision, "fcg", rtol=rtol, smoother=smoother, nu1=nu[0],
                                        nu2=nu[1], coarse_op="galerkin"))
    prob.close()


def test_bad_coarse_operator_is_rejected(libmg, ctx):
    inst = I.config1(33)
    opts = libmg.make_opts("fp64", "fcg")
    opts.coarse_op = 7
    with pytest.raises(Exception):
        libmg.Problem(ctx, inst, opts)
