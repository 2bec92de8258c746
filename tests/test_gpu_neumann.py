"""Homogeneous Neumann y sides (Eq. 28) on the GPU: the library reflects the coefficients
built on the caller's grid into the periodic grid of twice the height (k_mirror_eps), maps
the caller's charge, Dirichlet data and warm start through the reflection, and returns the
caller's rows.  Compared with the oracle's independent reflection (oracle.prepare +
Prepared.extract): the paper's semi-annulus (Sec. 4.1), a manufactured solution varying
along the Neumann sides, and a skewed mirror-symmetric mapped grid (eps_xy != 0, odd in the
mirrored half).  Both sides solve to 1e-12 (FP64) or the mixed path to 1e-11; nodes agree to
1e-10 relative."""
import numpy as np
import pytest

from paper_2602_01888_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(libmg, cuda):
    c = libmg.Context(0)
    yield c
    c.close()


def _skew(n):
    g = I.Grid(n, n, neumann_y=True)
    x, y = g.coords()
    xp = x + 0.08 * np.sin(np.pi * x) * np.cos(np.pi * y)
    yp = y + 0.08 * np.sin(np.pi * x) * np.sin(np.pi * y)
    return I.Instance("skew", g, I.MapSpec("grid", xp=xp, yp=yp), 1.0 + xp * np.cos(np.pi * yp),
                      bc=np.zeros(g.shape))


CASES = {
    "semi_annulus_65": lambda: I.semi_annulus(65),
    "semi_annulus_129": lambda: I.semi_annulus(129),
    "manufactured_65": lambda: I.neumann_manufactured(65),
    "skew_65": lambda: _skew(65),
    "rect_129x33": lambda: I.Instance("r", I.Grid(129, 33, 0.0, 0.0, 2.0, 0.5, neumann_y=True),
                                      I.MapSpec("sine_warp", (0.05,)),
                                      I.random_field((33, 129), 3), bc=I.random_field((33, 129), 4)),
}


def _oracle(oracle, inst):
    P = oracle.prepare(inst)
    phi, _, _ = oracle.pcg_solve(P.A, P.b, P.phi0, rtol=1e-14, max_iters=400, stagnate=5)
    return P.extract(phi)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec,smoother", [("fp64", "gs4"), ("mixed", "gs4"), ("fp64", "xline")])
def test_neumann_solve_matches_oracle(libmg, oracle, ctx, case, prec, smoother):
    inst = CASES[case]()
    ref = _oracle(oracle, inst)
    rtol = 1e-12 if prec == "fp64" else 1e-11
    pr = libmg.Problem(ctx, inst, libmg.make_opts(prec, "fcg", rtol=rtol, max_iters=400, smoother=smoother))
    phi, st = pr.solve()
    pr.close()
    assert phi.shape == inst.grid.shape and st.rel_residual <= rtol
    err = np.abs(phi - ref).max() / np.abs(ref).max()
    assert err < 1e-10, (case, prec, smoother, err, st.iters)


def test_semi_annulus_second_order_on_the_gpu(libmg, ctx):
    """Eq. 28-a: the GPU solution's max error falls about 4x per halving of h."""
    errs = []
    for n in (65, 129, 257):
        inst = I.semi_annulus(n)
        pr = libmg.Problem(ctx, inst, libmg.make_opts("fp64", "fcg", rtol=1e-12))
        phi, _ = pr.solve()
        pr.close()
        errs.append(np.abs(phi - inst.exact).max())
    assert errs[0] / errs[1] > 3.6 and errs[1] / errs[2] > 3.6, errs


def test_neumann_device_inputs_warm_start_and_batch(libmg, ctx, cuda):
    """Device arrays in the caller's layout, a warm start through the reflection (the converged
    solution stays put), and a batch of Neumann and Dirichlet problems equal to single solves."""
    torch = cuda
    inst = CASES["rect_129x33"]()
    opts = libmg.make_opts("fp64", "fcg", rtol=1e-12)
    pr = libmg.Problem(ctx, inst, opts, device_inputs=True)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rho, bc = d(inst.rho_phys), d(inst.bc)
    phi = torch.zeros(inst.grid.shape, dtype=torch.float64, device="cuda")
    libmg.mg_solve(pr.h, rho, bc, phi, opts)
    host, _ = pr.solve()
    assert np.array_equal(phi.cpu().numpy(), host)
    warm = libmg.make_opts("fp64", "fcg", rtol=1e-12, warm_start=True)
    st = libmg.mg_solve(pr.h, rho, bc, phi, warm)
    assert st.iters <= 1 and np.abs(phi.cpu().numpy() - host).max() < 1e-12 * np.abs(host).max()
    others = [I.semi_annulus(65), I.config1(65), I.neumann_manufactured(33)]
    probs = [libmg.Problem(ctx, x, opts) for x in others]
    alone = [p.solve()[0] for p in probs]
    phis = [np.zeros(x.grid.shape) for x in others]
    bcs = [None if x.bc is None else np.ascontiguousarray(x.bc) for x in others]
    libmg.mg_batch_solve(ctx.h, [p.h for p in probs], [np.ascontiguousarray(x.rho_phys) for x in others],
                         bcs, phis, opts)
    for a, b in zip(alone, phis):
        assert np.array_equal(a, b)
    for p in probs + [pr]:
        p.close()


def test_neumann_arguments(libmg, ctx):
    g = I.Grid(33, 33, periodic_y=True, neumann_y=True)
    inst = I.Instance("bad", g, I.MapSpec("identity"), np.zeros(g.shape))
    with pytest.raises(libmg.MGError) as e:
        libmg.Problem(ctx, inst, libmg.make_opts("fp64", "fcg"))
    assert e.value.status == libmg.MG_ERR_ARG
    gn = I.Grid(33, 33, neumann_y=True)
    z = np.zeros(gn.shape)
    with pytest.raises(libmg.MGError) as e:
        libmg.mg_harmonic_grid(ctx.h, gn, np.zeros(gn.shape, np.uint8), z, z, z.copy(), z.copy(), rtol=1e-12)
    assert e.value.status == libmg.MG_ERR_ARG
