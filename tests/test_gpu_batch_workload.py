"""The batched workload (inclusion instances, sides {65,129,257,513}, radius U[0.1,0.35],
eps' ratio U[1,50]) at the settings the benchmark uses: flexible CG to rtol 1e-9.

* For the instance with the largest ratio and the median ratio of each side, the batched
  solution's error against the oracle's phi* is within the 1e-9 target (mixed and FP64).
* A 64-instance batch (one graph launch) returns, for every instance, exactly what a
  single mg_solve of that instance returns."""
import numpy as np
import pytest

from paper_2602_01888_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RTOL = 1e-9
# FP64 rows aim at the FP64 path's 1e-10 error bound.  At rtol 1e-9 the oracle's own MG-PCG
# leaves up to 8.2e-11 on these instances (129^2, ratio 49); at 5e-10 at most 1.5e-11.
RTOL_FP64 = 5e-10


@pytest.fixture(scope="module")
def ctx(libmg, cuda):
    c = libmg.Context(0)
    yield c
    c.close()


def _picks():
    specs = I.config4_specs(512)
    out = []
    for n in (65, 129, 257, 513):
        s = sorted([x for x in specs if x[0] == n], key=lambda x: -x[2])
        out += [s[0], s[len(s) // 2]]
    return out


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batched_instances_match_oracle(libmg, oracle, ctx, prec):
    insts = [I.inclusion_instance(*s) for s in _picks()]
    rtol = RTOL_FP64 if prec == "fp64" else RTOL
    opts = libmg.make_opts(prec, "fcg", rtol=rtol, max_iters=400)
    probs = [libmg.Problem(ctx, x, opts) for x in insts]
    phis = [np.zeros(x.grid.shape) for x in insts]
    stats = libmg.mg_batch_solve(ctx.h, [p.h for p in probs],
                                 [np.ascontiguousarray(x.rho_phys) for x in insts], None, phis, opts)
    for x, phi, st in zip(insts, phis, stats):
        P = oracle.prepare(x)
        ref, _, _ = oracle.pcg_solve(P.A, P.b, P.phi0, rtol=0.0, max_iters=400, stagnate=10)
        err = oracle.rel_l2(phi, ref, x.grid.interior_mask())
        assert st.rel_residual <= rtol
        assert err <= (1e-10 if prec == "fp64" else 1e-9), (x.name, prec, err, st.iters)
    for p in probs:
        p.close()


def test_batch_of_64_equals_single_solves(libmg, ctx, cuda):
    torch = cuda
    specs = I.config4_specs(64, seed0=9000)
    insts = [I.inclusion_instance(*s) for s in specs]
    opts = libmg.make_opts("mixed", "fcg", rtol=RTOL, max_iters=400)
    probs = [libmg.Problem(ctx, x, opts, device_inputs=True) for x in insts]
    rhos = [torch.from_numpy(np.ascontiguousarray(x.rho_phys)).cuda() for x in insts]
    alone = []
    for p, r, x in zip(probs, rhos, insts):
        phi = torch.zeros(x.grid.shape, dtype=torch.float64, device="cuda")
        libmg.mg_solve(p.h, r, None, phi, opts)
        alone.append(phi)
    phis = [torch.zeros(x.grid.shape, dtype=torch.float64, device="cuda") for x in insts]
    for _ in range(2):  # the second call replays the cached batch graph
        for t in phis:
            t.zero_()
        stats = libmg.mg_batch_solve(ctx.h, [p.h for p in probs], rhos, None, phis, opts)
        torch.cuda.synchronize()
        for k, (a, b) in enumerate(zip(alone, phis)):
            assert torch.equal(a, b), k
        assert all(s.rel_residual <= RTOL for s in stats)
    for p in probs:
        p.close()


def test_batch_update_transform_equals_fresh_setup(libmg, ctx):
    """Problems set up for one geometry and moved to another by one mg_batch_update_transform
    solve exactly like problems set up for the second geometry; a folding map in the batch
    fails alone, with its own status."""
    a = [I.inclusion_instance(*s) for s in I.config4_specs(6, seed0=7000)]
    b = [I.inclusion_instance(x.grid.nx, r, e, sd) for x, (_, r, e, sd) in
         zip(a, I.config4_specs(6, seed0=7100))]
    opts = libmg.make_opts("mixed", "fcg", rtol=RTOL, max_iters=400)
    moved = [libmg.Problem(ctx, x, opts) for x in a]
    st = libmg.mg_batch_update_transform(ctx.h, [p.h for p in moved], [x.map for x in b],
                                         [np.ascontiguousarray(x.eps_phys) for x in b])
    assert st == [0] * len(b)
    for p, x in zip(moved, b):
        fresh = libmg.Problem(ctx, x, opts)
        want, _ = fresh.solve()
        got = np.zeros(x.grid.shape)
        libmg.mg_solve(p.h, np.ascontiguousarray(x.rho_phys), None, got, opts)
        assert np.array_equal(want, got), x.name
        fresh.close()
    # instance 2 gets a mirrored (orientation-reversing) map: only it reports the fold
    maps = [x.map for x in b]
    maps[2] = I.MapSpec("affine", (-1.0, 0.0, 0.0, 1.0))
    st = libmg.mg_batch_update_transform(ctx.h, [p.h for p in moved], maps,
                                         [np.ascontiguousarray(x.eps_phys) for x in b],
                                         raise_on_error=False)
    assert st[2] == libmg.MG_ERR_MAP_FOLDED
    assert all(s == 0 for k, s in enumerate(st) if k != 2)
    for p in moved:
        p.close()
