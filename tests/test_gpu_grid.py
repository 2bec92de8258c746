"""Numerical grid generation on the GPU (mg_harmonic_grid, Sec. 4.2 Eqs. 36-37) against the
oracle's masked operator + MG-PCG (oracle.harmonic_grid), with internal Dirichlet nodes:
the inclusion ring carrying the Eq. 44 boundary map, scattered fixed nodes, a periodic
grid with a fixed column.  Both sides solve to FP64 accuracy; nodes agree to 1e-11."""
import numpy as np
import pytest

from paper_2602_01888_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(libmg, cuda):
    c = libmg.Context(0)
    yield c
    c.close()


def _inclusion_case(n, r):
    i0 = I.snap_ring(n, r)
    ring, xp0, yp0 = I.inclusion_ring_data(n, i0)
    xref, yref = I._inclusion_grid_cached(n, i0)  # the workload's grid (numpy multigrid)
    return I.Grid(n, n), ring.astype(np.uint8), xp0, yp0, xref, yref


@pytest.mark.parametrize("n,r", [(65, 0.25), (129, 0.3), (257, 0.15)])
@pytest.mark.parametrize("mem", ["host", "device"])
def test_inclusion_grid_matches_oracle(libmg, oracle, ctx, cuda, n, r, mem):
    torch = cuda
    g, fixed, xp0, yp0, _, _ = _inclusion_case(n, r)
    xo_ref, yo_ref, _ = oracle.harmonic_grid(g, fixed, xp0, yp0)
    if mem == "host":
        xo, yo = np.zeros(g.shape), np.zeros(g.shape)
        stats = libmg.mg_harmonic_grid(ctx.h, g, fixed, xp0, yp0, xo, yo, rtol=1e-13)
    else:
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        xo_d = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        yo_d = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        fx, xi, yi = d(fixed), d(xp0), d(yp0)
        stats = libmg.mg_harmonic_grid(ctx.h, g, fx, xi, yi, xo_d, yo_d, rtol=1e-13)
        torch.cuda.synchronize()
        xo, yo = xo_d.cpu().numpy(), yo_d.cpu().numpy()
    assert np.abs(xo - xo_ref).max() < 1e-11, np.abs(xo - xo_ref).max()
    assert np.abs(yo - yo_ref).max() < 1e-11, np.abs(yo - yo_ref).max()
    f = fixed.astype(bool)
    assert np.array_equal(xo[f], xp0[f]) and np.array_equal(yo[f], yp0[f])
    assert all(s.rel_residual <= 1e-13 for s in stats)


def test_scattered_and_periodic_fixed_nodes_match_oracle(libmg, oracle, ctx):
    # periodic in y (polar-like annulus data on the two rings), a fixed column and scattered
    # fixed nodes inside
    g = I.Grid(65, 65, 0.2, 0.0, 0.8, 2 * np.pi, periodic_y=True)
    x, y = g.coords()
    rng = np.random.default_rng(17)
    fixed = ((rng.random(g.shape) < 0.03) & g.interior_mask()).astype(np.uint8)
    fixed[:, 33] = 1
    data = fixed.astype(bool) | ~g.interior_mask()
    xp0 = np.where(data, x * np.cos(y), 0.0)
    yp0 = np.where(data, x * np.sin(y), 0.0)
    xo_ref, yo_ref, _ = oracle.harmonic_grid(g, fixed, xp0, yp0)
    xo, yo = np.zeros(g.shape), np.zeros(g.shape)
    libmg.mg_harmonic_grid(ctx.h, g, fixed, xp0, yp0, xo, yo, rtol=1e-13)
    assert np.abs(xo - xo_ref).max() < 1e-11 and np.abs(yo - yo_ref).max() < 1e-11


def test_full_size_inclusion_grid_matches_workload_grid(libmg, ctx):
    """The 1025^2 inclusion grid of the benchmark workload, generated on the GPU, against the
    numpy multigrid that the workload inputs come from (an independent implementation)."""
    g, fixed, xp0, yp0, xref, yref = _inclusion_case(1025, 0.25)
    xo, yo = np.zeros(g.shape), np.zeros(g.shape)
    libmg.mg_harmonic_grid(ctx.h, g, fixed, xp0, yp0, xo, yo, rtol=1e-13)
    assert np.abs(xo - xref).max() < 1e-10 and np.abs(yo - yref).max() < 1e-10


def test_bad_arguments(libmg, ctx):
    g = I.Grid(33, 33)
    z = np.zeros(g.shape)
    with pytest.raises(libmg.MGError) as e:
        libmg.mg_harmonic_grid(ctx.h, g, np.zeros(g.shape, np.uint8), z, z, z.copy(), z.copy(), rtol=0.0)
    assert e.value.status == libmg.MG_ERR_ARG
