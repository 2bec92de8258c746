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
