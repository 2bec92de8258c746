"""The stretched-grid example of Sec. 5.1 on the GPU: the Gaussian beam (Eq. 53) on the sinh
map (Eq. 52, s = 5, alpha = 0.6, computational square [-3, 3]^2), Dirichlet data equal to the
beam's free-space potential (the exact solution, a closed form).

* The GPU's FP64 and mixed solutions match the oracle's phi* (1e-10 / 1e-9).
* The GPU's discretization error against the exact solution falls at second order in L1,
  L2 and Linf (Eqs. 25-27) over 65, 129, 257, 513, and equals the oracle's error norms."""
import math

import numpy as np
import pytest

from paper_2602_01888_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(libmg, cuda):
    c = libmg.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sinh_beam_matches_oracle(libmg, oracle, ctx, prec):
    inst = I.sinh_beam(129)
    P = oracle.prepare(inst)
    ref, _, _ = oracle.pcg_solve(P.A, P.b, P.phi0, rtol=0.0, max_iters=400, stagnate=10)
    prob = libmg.Problem(ctx, inst, libmg.make_opts(prec, "fcg", rtol=1e-11, max_iters=400))
    phi, st = prob.solve()
    err = oracle.rel_l2(phi, ref, inst.grid.interior_mask())
    assert err <= (1e-10 if prec == "fp64" else 1e-9), (prec, err, st.iters)
    prob.close()


def test_sinh_beam_second_order_on_the_gpu(libmg, oracle, ctx):
    errs = []
    for n in (65, 129, 257, 513):
        inst = I.sinh_beam(n)
        prob = libmg.Problem(ctx, inst, libmg.make_opts("fp64", "fcg", rtol=1e-12, max_iters=400))
        phi, st = prob.solve()
        prob.close()
        e = oracle.error_norms(inst.exact, phi)
        ref, *_ = oracle.solve_instance(inst, rtol=1e-13)
        assert np.allclose(e, oracle.error_norms(inst.exact, ref), rtol=1e-6), (n, e)
        errs.append(e)
    orders = [[math.log2(errs[k][q] / errs[k + 1][q]) for q in range(3)] for k in range(3)]
    assert all(1.9 < v < 2.1 for v in orders[-1]), orders
    assert all(1.8 < v < 2.2 for v in orders[-2]), orders
