"""Annulus workload (polar map Eq. 29, periodic in theta, 64-mode Fourier source).

* At 1025^2 the whole solution is compared with the oracle's phi* (mixed and FP64, at the
  rtol the benchmark uses for this workload): relative L2 error <= 1e-9 (mixed) and
  <= 1e-10 (FP64).
* At the benchmark's full size (8193^2) the oracle cannot solve in test time.  Its phi* at
  seeded sample nodes is stored under tests/golden/ (written from the oracle alone) and the
  GPU solution is compared with it; independently, the test checks the GPU solution node by node: at seeded sample nodes it rebuilds the operator on a 5x5
  patch from the map (its own Jacobian, tensor and assembly) and evaluates b - A phi with
  the GPU's phi.  Since ||r||_2 <= rtol ||r_0||_2 over all nodes, every sampled |r_i| must be
  below rtol ||r_0||_2, where ||r_0|| = ||b|| (zero Dirichlet data) is also computed by the
  oracle."""
import functools

import numpy as np
import pytest

from paper_2602_01888_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RTOL = 6e-10  # 1025^2 cases
# rtol of the 8193^2 benchmark workload per precision.  The FP64 residual floor there is
# about 1e-9 (b - A phi evaluated in FP64 at phi*: the oracle's own solution stalls at
# 1.05e-9), far above the error it corresponds to: at rtol 1e-8 the mixed solution is
# within ~1e-10 of the oracle's phi*; the FP64 path, held to 1e-10, stops at 2e-9 (x-line
# V(1,1) at 1e-8 left 3.4e-10), twice the floor.  Both checked below against the stored
# samples.
RTOL_FULL = 1e-8
RTOL_FULL_FP64 = 2e-9


@functools.lru_cache(maxsize=1)
def _full():
    """The 8193^2 workload's inputs, generated once for every full-size test here."""
    return I.config3(8193)


@pytest.fixture(scope="module")
def ctx(libmg, cuda):
    c = libmg.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("smoother", ["gs4", "xline"])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_annulus_recipe_1025_matches_oracle(libmg, oracle, ctx, prec, smoother):
    inst = I.config3(1025)
    P = oracle.prepare(inst)
    ref, it, hist = oracle.pcg_solve(P.A, P.b, P.phi0, rtol=0.0, max_iters=400, stagnate=3)
    prob = libmg.Problem(ctx, inst, libmg.make_opts(prec, "fcg", rtol=RTOL, max_iters=400, smoother=smoother))
    phi, st = prob.solve()
    err = oracle.rel_l2(phi, ref, inst.grid.interior_mask())
    assert err <= (1e-10 if prec == "fp64" else 1e-9), (prec, err, st.iters)
    prob.close()


def _patch_residual(oracle, inst, phi_gpu, i, j):
    """b - A phi at node (i, j) from a 5x5 patch rebuilt by the oracle."""
    g = inst.grid
    pg = I.Grid(5, 5, g.x0 + (i - 2) * g.hx, g.y0 + (j - 2) * g.hy, 4 * g.hx, 4 * g.hy)
    J = oracle.jacobian(pg, inst.map)
    D, exx, exy, eyy, st = oracle.eps_tensor(J, None)
    A = oracle.assemble(pg, exx, exy, eyy)
    rows = [(j + d) % g.nyr for d in range(-2, 3)]
    phi = np.array([[phi_gpu[r, i + d] for d in range(-2, 3)] for r in rows])
    rho = np.array([[inst.rho_phys[r, i + d] for d in range(-2, 3)] for r in rows])
    b = oracle.rhs(pg, rho, D)
    r = oracle.residual(A, phi, b)
    return r[2, 2], b[2, 2]


def test_annulus_full_size_sampled_residuals(libmg, oracle, ctx, cuda):
    torch = cuda
    inst = _full()
    g = inst.grid
    prob = libmg.Problem(ctx, inst, libmg.make_opts("mixed", "fcg", rtol=RTOL_FULL, max_iters=400))
    rho = torch.from_numpy(np.ascontiguousarray(inst.rho_phys)).cuda()
    phi = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    _, st = prob.solve(rho=rho, phi=phi)
    torch.cuda.synchronize()
    assert st.rel_residual <= RTOL_FULL
    prob.close()
    phi_h = phi.cpu().numpy()
    del phi, rho
    # ||r_0|| = ||b|| over the unknowns, computed by the oracle on the full grid
    J = oracle.jacobian(g, inst.map)
    D, *_ = oracle.eps_tensor(J, None)
    del J
    b = oracle.rhs(g, inst.rho_phys, D)
    r0 = float(np.linalg.norm(b))
    del b, D
    rng = np.random.default_rng(77)
    worst = 0.0
    for _ in range(256):
        i = int(rng.integers(1, g.nx - 1))
        j = int(rng.integers(0, g.nyr))
        r, bb = _patch_residual(oracle, inst, phi_h, i, j)
        worst = max(worst, abs(r))
    assert worst <= RTOL_FULL * r0, (worst, RTOL_FULL * r0)
    # and the solution is not trivially small: it carries the source's scale
    assert np.abs(phi_h).max() > 1e-6


@pytest.mark.parametrize("prec,smoother,nu", [("mixed", "gs4", 2), ("mixed", "xline", 2), ("mixed", "xline", 1),
                                              ("fp64", "xline", 1), ("fp64", "gs4", 2)])
def test_annulus_full_size_matches_oracle_golden(libmg, ctx, cuda, prec, smoother, nu):
    """8193^2 annulus at the benchmark's rtol (point smoother V(2,2), line smoother V(2,2)
    and V(1,1)), against the oracle's phi* at 4096 seeded sample nodes
    (tests/golden/annulus_8193_samples.npz, written by tests/golden/make_golden.py from the
    oracle alone): relative L2 error over the samples within 1e-9 for the mixed path and
    1e-10 for the FP64 path."""
    import os
    torch = cuda
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden", "annulus_8193_samples.npz"))
    inst = _full()
    g = inst.grid
    rtol = RTOL_FULL_FP64 if prec == "fp64" else RTOL_FULL
    prob = libmg.Problem(ctx, inst, libmg.make_opts(prec, "fcg", rtol=rtol, max_iters=400,
                                                    smoother=smoother, nu1=nu, nu2=nu))
    rho = torch.from_numpy(np.ascontiguousarray(inst.rho_phys)).cuda()
    phi = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    _, st = prob.solve(rho=rho, phi=phi)
    jj = torch.from_numpy(gold["j"]).cuda()
    ii = torch.from_numpy(gold["i"]).cuda()
    got = phi[jj, ii].cpu().numpy()
    prob.close()
    ref = gold["phi"]
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= (1e-10 if prec == "fp64" else 1e-9), (prec, err, st.iters, st.rel_residual)
