"""Four-colour SOR on the GPU, the single-level iteration the paper compares multigrid with
(Sec. 4, omega = 1.875): the sweep kernel (mgk_sor_*) against the oracle's sor4
(oracle.smooth with SMOOTHER_SOR4), and the MG_OUTER_SOR solve against oracle.sor_solve
(same residual test every nu1 sweeps).

Tolerances: FP64 1e-12 relative to max |phi| (the same operations, rounding order aside;
three sweeps at omega up to 1.875 amplify rounding by a small factor); FP32 2e-5 relative,
as for the other FP32 smoothers."""
import ctypes as C

import numpy as np
import pytest

from paper_2602_01888_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = {
    "sine_129": lambda: I.config1(129),
    "annulus_129": lambda: I.annulus_log(129),
    "incl_257": lambda: I.inclusion_instance(257, 0.25, 10.0, 21),
    "ragged_193x97": lambda: I.Instance("g", I.Grid(193, 97, 0.0, 0.0, 1.0, 0.5),
                                        I.MapSpec("affine", (1.0, 0.25, -0.1, 1.05)), np.ones((97, 193))),
}


def _dev(torch, a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("omega,sweeps", [(1.0, 1), (1.5, 3), (1.875, 2)])
def test_sor_sweeps_match_oracle(libmg, oracle, cuda, case, prec, omega, sweeps):
    torch = cuda
    A = oracle.prepare(CASES[case]()).A
    dt = torch.float64 if prec == "f64" else torch.float32
    t = [_dev(torch, a, dt) for a in (A.cE, A.cN, A.cNE, A.cNW, A.diag, 1.0 / A.diag)]
    s = libmg.op_struct(t, A.nx, A.ny, A.periodic, f32=(prec == "f32"))
    rng = np.random.default_rng(11)
    phi = rng.standard_normal(A.cE.shape)
    b = rng.standard_normal(A.cE.shape) * np.abs(A.diag).max()
    x, b_d = _dev(torch, phi, dt), _dev(torch, b, dt)
    libmg.mgk(f"mgk_sor_{prec}", C.byref(s), x.data_ptr(), b_d.data_ptr(), sweeps, omega,
              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    ref = oracle.smooth(A, phi, b, sweeps=sweeps, smoother=oracle.SMOOTHER_SOR4, omega_j=omega)
    err = np.abs(x.double().cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < (1e-12 if prec == "f64" else 2e-5), (case, prec, omega, sweeps, err)


@pytest.fixture(scope="module")
def ctx(libmg, cuda):
    c = libmg.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("case,n", [("sine", 65), ("annulus", 65), ("incl", 129)])
def test_sor_solve_matches_oracle(libmg, oracle, ctx, case, n):
    """Same residual test every 16 sweeps on both sides: the same number of sweeps to rtol
    1e-10 (one check either way where the residual lands on the threshold) and the same
    solution, which is also the multigrid solution."""
    inst = {"sine": lambda: I.config1(n), "annulus": lambda: I.annulus_log(n),
            "incl": lambda: I.inclusion_instance(n, 0.25, 10.0, 5)}[case]()
    P = oracle.prepare(inst)
    ref, sw, hist = oracle.sor_solve(P.A, P.b, P.phi0, omega=1.875, rtol=1e-10, max_sweeps=400000, check=16)
    opts = libmg.make_opts("fp64", "sor", rtol=1e-10, max_iters=25000, nu1=16, omega_j=1.875)
    pr = libmg.Problem(ctx, inst, opts)
    phi, st = pr.solve()
    mg_phi, _ = pr.solve(opts=libmg.make_opts("fp64", "fcg", rtol=1e-12))
    pr.close()
    assert st.rel_residual <= 1e-10
    assert abs(16 * st.iters - sw) <= 16, (st.iters * 16, sw)
    m = inst.grid.interior_mask()
    scale = np.abs(ref[m]).max()
    assert np.abs(phi[m] - ref[m]).max() < 1e-9 * scale
    assert np.abs(phi[m] - mg_phi[m]).max() < 1e-7 * scale  # both within their residual tolerance


def test_sor_options_are_checked(libmg, ctx):
    inst = I.config1(33)
    pr = libmg.Problem(ctx, inst, libmg.make_opts("fp64", "fcg"))
    for kw in (dict(nu1=0), dict(nu1=17), dict(omega_j=2.0), dict(omega_j=0.0)):
        with pytest.raises(libmg.MGError) as e:
            pr.solve(opts=libmg.make_opts("fp64", "sor", **kw))
        assert e.value.status == libmg.MG_ERR_ARG, kw
    pr.close()
    mixed = libmg.Problem(ctx, inst, libmg.make_opts("mixed", "fcg"))
    with pytest.raises(libmg.MGError):
        mixed.solve(opts=libmg.make_opts("mixed", "sor", nu1=8, omega_j=1.875))
    mixed.close()
