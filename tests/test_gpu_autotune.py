"""The smoother autotuner (mg_autotune): every family it times can run at that size, its
choice is the fastest it measured, and solves on a tuned context return exactly what they
return on an untuned one (the families compute the same values)."""
import numpy as np
import pytest

from paper_2602_01888_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = [lambda: I.inclusion_instance(513, 0.25, 10.0, 4), lambda: I.annulus_log(1025),
         lambda: I.config1(129)]


def _solve_all(libmg, ctx):
    out = []
    for make in CASES:
        inst = make()
        for prec in ("fp64", "mixed"):
            p = libmg.Problem(ctx, inst, libmg.make_opts(prec, "fcg", rtol=1e-10, max_iters=400))
            phi, st = p.solve()
            out.append((phi, st.iters))
            p.close()
    return out


def test_tuned_choice_is_fastest_and_results_unchanged(libmg, cuda):
    ctx = libmg.Context(0)
    before = _solve_all(libmg, ctx)
    table = libmg.mg_autotune(ctx.h, 1025)
    assert {(prec, side) for prec, side, _, _ in table} == \
        {(p, s) for p in ("fp64", "mixed") for s in (33, 65, 129, 257, 513, 1025)}
    for prec, side, ms, choice in table:
        assert ms and choice == min(ms, key=ms.get), (prec, side, ms, choice)
        assert "colour" in ms
    after = _solve_all(libmg, ctx)
    for (a, ia), (b, ib) in zip(before, after):
        assert ia == ib and np.array_equal(a, b)
    ctx.close()


VARIANT_CASES = {
    "sine_385x257": lambda: I.Instance("s", I.Grid(385, 257, 0.0, 0.0, 1.5, 1.0),
                                       I.MapSpec("sine_warp", (0.08,)), np.ones((257, 385))),
    "annulus_257": lambda: I.annulus_log(257),
}


@pytest.mark.parametrize("case", list(VARIANT_CASES))
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("prolong", [False, True])
def test_every_tuned_variant_matches_the_oracle(libmg, oracle, cuda, case, prec, prolong):
    """Each shape the autotuner may pick (tile sizes and sweeps per launch of the fused and
    pipelined tiles, sweeps per pass of row marching), one launch, against the oracle's
    sweeps, with and without the fused coarse correction; the FP64 variants agree with each
    other bitwise (the same operations per node in the same order)."""
    import ctypes as C
    torch = cuda
    inst = VARIANT_CASES[case]()
    P = oracle.prepare(inst)
    g = inst.grid
    pitch = (g.nx + 31) // 32 * 32
    dt = torch.float64 if prec == "f64" else torch.float32
    rng = np.random.default_rng(71)
    phi0 = rng.standard_normal(g.shape)
    b = rng.standard_normal(g.shape) * np.abs(P.A.diag).max()

    def padded(a):
        t = torch.zeros((g.nyr, pitch), dtype=dt, device="cuda")
        t[:, : g.nx] = torch.from_numpy(np.array(a)).to("cuda", dt)
        return t

    ops = [padded(a) for a in (P.A.cE, P.A.cN, P.A.cNE, P.A.cNW, P.A.diag, 1.0 / P.A.diag)]
    st = libmg.op_struct(ops, g.nx, g.ny, g.periodic_y, f32=(prec == "f32"))
    start, eH_d, pc = phi0.copy(), None, 0
    if prolong:
        gc = I.Grid((g.nx - 1) // 2 + 1, (g.ny - 1) // 2 + 1, g.x0, g.y0, g.lx, g.ly, g.periodic_y)
        eH = rng.standard_normal(gc.shape) * gc.interior_mask()
        start = oracle.prolong_add(g.nx, g.ny, g.periodic_y, eH, phi0)
        pc = (gc.nx + 31) // 32 * 32
        eH_d = torch.zeros((gc.nyr, pc), dtype=dt, device="cuda")
        eH_d[:, : gc.nx] = torch.from_numpy(eH).to("cuda", dt)
    stream = torch.cuda.current_stream().cuda_stream
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    refs, by_sweeps = {}, {}
    ran = 0
    for family in (2, 3, 4):
        for v, tile, ns in libmg.smooth_variants(prec == "f32", family):
            if ns not in refs:
                refs[ns] = oracle.smooth(P.A, start, b, sweeps=ns)
            xin, b_d = padded(phi0), padded(b)
            xout = torch.full((g.nyr, pitch), float("nan"), dtype=dt, device="cuda")
            libmg.mgk(f"mgk_smooth_variant_{prec}", C.byref(st), family, v, xin.data_ptr(), xout.data_ptr(),
                      b_d.data_ptr(), 0, eH_d.data_ptr() if eH_d is not None else None, pc, err.data_ptr(), stream)
            torch.cuda.synchronize()
            assert int(err.item()) == 0
            got = xout[:, : g.nx].double().cpu().numpy()
            e = np.abs(got - refs[ns]).max() / np.abs(refs[ns]).max()
            assert e < (1e-13 if prec == "f64" else 1e-5), (family, tile, ns, e)
            if prec == "f64":
                first = by_sweeps.setdefault(ns, got)
                assert np.array_equal(first, got), (family, tile, ns)
            ran += 1
    assert ran >= (12 if prec == "f64" else 14)


def test_tuner_reports_tile_shape_and_depth(libmg, cuda):
    ctx = libmg.Context(0)
    table = libmg.mg_autotune(ctx.h, 513, variants=True)
    for prec, side, ms, choice, var in table:
        tx, ty = var["tile"]
        if choice in ("fused", "pipelined"):
            assert (tx, ty) in ((32, 32), (64, 16), (64, 24)) and var["sweeps"] in (1, 2), (prec, side, var)
        elif choice == "marching":
            assert ty == 0 and tx > 0 and var["sweeps"] in (1, 2)
        else:
            assert choice == "colour"
    ctx.close()
