"""Per-kernel parity: each CUDA kernel (called through the mgk_* C ABI) against the FP64
oracle on the same seeded inputs.  FP64 kernels must agree to rounding (1e-13 relative
to the magnitude of the compared quantity, 1e-12 for the Galerkin triple sum); FP32
kernels to a few FP32 ulps of the terms involved (1e-5)."""
import ctypes as C

import numpy as np
import pytest

from paper_2602_01888_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = {
    "sine_97x65": lambda: I.Instance("s", I.Grid(97, 65), I.MapSpec("sine_warp", (0.1,)),
                                     np.ones((65, 97))),
    "incl_129": lambda: I.inclusion_instance(129, 0.25, 10.0, 11),
    "annulus_65": lambda: I.annulus_log(65),
    "rect_33x17": lambda: I.Instance("r", I.Grid(33, 17, 0.0, 0.0, 1.0, 0.5),
                                     I.MapSpec("affine", (1.1, 0.2, -0.1, 0.9)), np.ones((17, 33))),
    "tiny_5": lambda: I.config1(5),
    "periodic_17": lambda: I.annulus_log(17),
    # the stretched grid of Sec. 5.1 (Eq. 52, s = 5, alpha = 0.6) on [-3, 3]^2
    "sinh_65": lambda: I.sinh_beam(65),
}


def _dev(torch, a, pitch=None, dtype=None):
    a = np.array(a)  # writable copy
    dtype = dtype or torch.float64
    if pitch is None or pitch == a.shape[1]:
        return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)
    t = torch.full((a.shape[0], pitch), float("nan"), dtype=dtype, device="cuda")
    t[:, : a.shape[1]] = torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)
    return t


def _host(t, nx):
    return t[:, :nx].double().cpu().numpy()


def _op_tensors(torch, A, pitch=None, dtype=None):
    arrs = [A.cE, A.cN, A.cNE, A.cNW, A.diag, 1.0 / A.diag]
    return [_dev(torch, a, pitch, dtype) for a in arrs]


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _stream(torch):
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("case", list(CASES))
def test_coefficient_build_matches_oracle(libmg, oracle, cuda, case):
    torch = cuda
    inst = CASES[case]()
    g = inst.grid
    pitch = g.nx + 3  # a row pitch larger than nx
    D, exx, exy, eyy = (torch.zeros((g.nyr, pitch), dtype=torch.float64, device="cuda") for _ in range(4))
    folded = torch.zeros(1, dtype=torch.int32, device="cuda")
    eps = None if inst.eps_phys is None else _dev(torch, inst.eps_phys, pitch)
    if inst.map.kind == "grid":
        xp, yp = _dev(torch, inst.map.xp, pitch), _dev(torch, inst.map.yp, pitch)
        libmg.mgk("mgk_eps_grid", g.nx, g.ny, int(g.periodic_y), g.hx, g.hy, xp.data_ptr(),
                  yp.data_ptr(), 0.0, 0.0, eps.data_ptr() if eps is not None else None, pitch,
                  D.data_ptr(), exx.data_ptr(), exy.data_ptr(), eyy.data_ptr(), folded.data_ptr(),
                  _stream(torch))
    else:
        prm = (C.c_double * 4)(*(list(inst.map.params) + [0.0] * 4)[:4])
        libmg.mgk("mgk_eps_analytic", libmg.MAP_CODES[inst.map.kind], prm, g.nx, g.ny,
                  int(g.periodic_y), g.x0, g.y0, g.hx, g.hy,
                  eps.data_ptr() if eps is not None else None, pitch, D.data_ptr(), exx.data_ptr(),
                  exy.data_ptr(), eyy.data_ptr(), folded.data_ptr(), _stream(torch))
    torch.cuda.synchronize()
    P = oracle.prepare(inst)
    assert int(folded.item()) == 0
    assert _rel(_host(D, g.nx), P.D) < 1e-13
    emag = max(np.abs(P.exx).max(), np.abs(P.eyy).max())  # size of the tensor
    for got, ref in ((exx, P.exx), (exy, P.exy), (eyy, P.eyy)):
        assert np.abs(_host(got, g.nx) - ref).max() < 1e-13 * emag
    # operator from the device tensor
    ops = [torch.zeros((g.nyr, pitch), dtype=torch.float64, device="cuda") for _ in range(6)]
    s = libmg.op_struct(ops, g.nx, g.ny, g.periodic_y)
    # keep every device input referenced until the asynchronous kernels have run
    ex_d, exy_d, ey_d = (_dev(torch, a, pitch) for a in (P.exx, P.exy, P.eyy))
    libmg.mgk("mgk_assemble", C.byref(s), g.hx, g.hy, ex_d.data_ptr(), exy_d.data_ptr(),
              ey_d.data_ptr(), _stream(torch))
    b = torch.zeros((g.nyr, pitch), dtype=torch.float64, device="cuda")
    rho_d, D_d = _dev(torch, inst.rho_phys, pitch), _dev(torch, P.D, pitch)
    libmg.mgk("mgk_rhs", C.byref(s), rho_d.data_ptr(), D_d.data_ptr(), b.data_ptr(), _stream(torch))
    torch.cuda.synchronize()
    scale = np.abs(P.A.diag).max()
    for got, ref in zip(ops[:5], P.A.arrays()):
        assert np.abs(_host(got, g.nx) - ref).max() <= 1e-13 * scale
    assert _rel(_host(b, g.nx), P.b) < 1e-14


def test_folded_map_flag(libmg, cuda):
    torch = cuda
    g = I.Grid(9, 9)
    t = [torch.zeros((9, 9), dtype=torch.float64, device="cuda") for _ in range(4)]
    folded = torch.zeros(1, dtype=torch.int32, device="cuda")
    prm = (C.c_double * 4)(1.0, 0.0, 0.0, -1.0)
    libmg.mgk("mgk_eps_analytic", 4, prm, 9, 9, 0, 0.0, 0.0, g.hx, g.hy, None, 9,
              *[x.data_ptr() for x in t], folded.data_ptr(), _stream(torch))
    torch.cuda.synchronize()
    assert int(folded.item()) == 1


def _coarse_grid(g):
    return I.Grid((g.nx - 1) // 2 + 1, (g.ny - 1) // 2 + 1, g.x0, g.y0, g.lx, g.ly, g.periodic_y)


@pytest.mark.parametrize("case", ["sine_97x65", "incl_129", "annulus_65", "rect_33x17", "periodic_17"])
def test_galerkin_matches_oracle(libmg, oracle, cuda, case):
    torch = cuda
    inst = CASES[case]()
    P = oracle.prepare(inst)
    A, g = P.A, inst.grid
    for _ in range(2):
        if (g.nx - 1) % 2 or (g.ny - 1) % 2 or g.nx < 5:
            break
        gc = _coarse_grid(g)
        ref = oracle.galerkin(A)
        fine = _op_tensors(torch, A)
        coarse = [torch.zeros(gc.shape, dtype=torch.float64, device="cuda") for _ in range(6)]
        sf = libmg.op_struct(fine, g.nx, g.ny, g.periodic_y)
        sc = libmg.op_struct(coarse, gc.nx, gc.ny, gc.periodic_y)
        libmg.mgk("mgk_galerkin", C.byref(sf), C.byref(sc), _stream(torch))
        torch.cuda.synchronize()
        scale = np.abs(ref.diag).max()
        for got, r in zip(coarse[:5], ref.arrays()):
            assert np.abs(_host(got, gc.nx) - r).max() <= 1e-12 * scale
        A, g = ref, gc


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("reverse", [0, 1])
def test_smoother_matches_oracle(libmg, oracle, cuda, case, reverse):
    torch = cuda
    inst = CASES[case]()
    P = oracle.prepare(inst)
    g = inst.grid
    rng = np.random.default_rng(5)
    phi0 = rng.standard_normal(g.shape)
    b = rng.standard_normal(g.shape) * np.abs(P.A.diag).max()
    ref = oracle.smooth(P.A, phi0, b, sweeps=2, reverse=bool(reverse))
    ops = _op_tensors(torch, P.A)
    s = libmg.op_struct(ops, g.nx, g.ny, g.periodic_y)
    x, b_d = _dev(torch, phi0), _dev(torch, b)
    libmg.mgk("mgk_smooth_f64", C.byref(s), x.data_ptr(), b_d.data_ptr(), 2, reverse, _stream(torch))
    torch.cuda.synchronize()
    assert _rel(_host(x, g.nx), ref) < 1e-13
    # FP32 instance
    ops32 = _op_tensors(torch, P.A, dtype=torch.float32)
    s32 = libmg.op_struct(ops32, g.nx, g.ny, g.periodic_y, f32=True)
    x32, b32 = _dev(torch, phi0, dtype=torch.float32), _dev(torch, b, dtype=torch.float32)
    libmg.mgk("mgk_smooth_f32", C.byref(s32), x32.data_ptr(), b32.data_ptr(), 2, reverse,
              _stream(torch))
    torch.cuda.synchronize()
    assert _rel(_host(x32, g.nx), ref) < 1e-5


@pytest.mark.parametrize("case", ["sine_97x65", "incl_129", "annulus_65", "rect_33x17", "periodic_17"])
def test_jacobi_and_residual_match_oracle(libmg, oracle, cuda, case):
    torch = cuda
    inst = CASES[case]()
    P = oracle.prepare(inst)
    g = inst.grid
    rng = np.random.default_rng(8)
    phi0 = rng.standard_normal(g.shape)
    b = rng.standard_normal(g.shape) * np.abs(P.A.diag).max()
    ops = _op_tensors(torch, P.A)
    s = libmg.op_struct(ops, g.nx, g.ny, g.periodic_y)
    r = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    p_d, b_d = _dev(torch, phi0), _dev(torch, b)
    libmg.mgk("mgk_residual_f64", C.byref(s), p_d.data_ptr(), b_d.data_ptr(), r.data_ptr(),
              _stream(torch))
    x = _dev(torch, phi0)
    tmp = torch.zeros_like(x)
    libmg.mgk("mgk_jacobi_f64", C.byref(s), x.data_ptr(), b_d.data_ptr(), tmp.data_ptr(), 3, 0.8,
              _stream(torch))
    torch.cuda.synchronize()
    rref = oracle.residual(P.A, phi0, b)
    scale = np.abs(P.A.diag).max() * np.abs(phi0).max()
    assert np.abs(_host(r, g.nx) - rref).max() <= 1e-13 * scale
    ref = oracle.smooth(P.A, phi0, b, sweeps=3, smoother=oracle.SMOOTHER_JACOBI, omega_j=0.8)
    assert _rel(_host(x, g.nx), ref) < 1e-13


@pytest.mark.parametrize("case", ["sine_97x65", "incl_129", "annulus_65", "rect_33x17", "tiny_5", "periodic_17"])
def test_residual_restriction_and_prolongation_match_oracle(libmg, oracle, cuda, case):
    torch = cuda
    inst = CASES[case]()
    P = oracle.prepare(inst)
    g = inst.grid
    gc = _coarse_grid(g)
    rng = np.random.default_rng(9)
    phi0 = rng.standard_normal(g.shape)
    b = rng.standard_normal(g.shape) * np.abs(P.A.diag).max()
    ref_bH = oracle.restrict(g.nx, g.ny, g.periodic_y, oracle.residual(P.A, phi0, b))
    pc = gc.nx + 5
    for dt, tol, f32 in ((torch.float64, 1e-13, False), (torch.float32, 2e-6, True)):
        ops = _op_tensors(torch, P.A, dtype=dt)
        s = libmg.op_struct(ops, g.nx, g.ny, g.periodic_y, f32=f32)
        bH = torch.zeros((gc.nyr, pc), dtype=dt, device="cuda")
        p_d, b_d = _dev(torch, phi0, dtype=dt), _dev(torch, b, dtype=dt)
        libmg.mgk("mgk_resid_restrict_f32" if f32 else "mgk_resid_restrict_f64", C.byref(s),
                  p_d.data_ptr(), b_d.data_ptr(), bH.data_ptr(), pc, _stream(torch))
        eH = rng.standard_normal(gc.shape) * gc.interior_mask()
        x, eH_d = _dev(torch, phi0, dtype=dt), _dev(torch, eH, pc, dtype=dt)
        libmg.mgk("mgk_prolong_add_f32" if f32 else "mgk_prolong_add_f64", C.byref(s), x.data_ptr(),
                  eH_d.data_ptr(), pc, _stream(torch))
        torch.cuda.synchronize()
        scale = np.abs(P.A.diag).max() * np.abs(phi0).max()
        assert np.abs(_host(bH, gc.nx) - ref_bH).max() <= tol * scale
        ref_x = oracle.prolong_add(g.nx, g.ny, g.periodic_y, eH, phi0)
        assert np.abs(_host(x, g.nx) - ref_x).max() <= tol * 10


@pytest.mark.parametrize("case", ["sine_97x65", "incl_129", "annulus_65", "rect_33x17", "tiny_5", "periodic_17",
                                  "sinh_65"])
def test_even_row_restriction_matches_oracle(libmg, oracle, cuda, case):
    """mgk_resid_restrict_even (the restriction after zebra x-line pre-smoothing): on any
    iterate it is the oracle's full weighting of the residual with the odd rows set to zero;
    after one oracle zebra sweep (even rows, then odd rows) it is the oracle's full weighting
    of the true residual, whose odd rows are then rounding residue."""
    torch = cuda
    inst = CASES[case]()
    P = oracle.prepare(inst)
    g = inst.grid
    gc = _coarse_grid(g)
    rng = np.random.default_rng(12)
    phi0 = rng.standard_normal(g.shape)
    b = rng.standard_normal(g.shape) * np.abs(P.A.diag).max()
    r0 = oracle.residual(P.A, phi0, b)
    r0[1::2, :] = 0.0
    phi1 = oracle.smooth(P.A, phi0, b, sweeps=1, smoother=oracle.SMOOTHER_XLINE)
    refs = ((phi0, oracle.restrict(g.nx, g.ny, g.periodic_y, r0)),
            (phi1, oracle.restrict(g.nx, g.ny, g.periodic_y, oracle.residual(P.A, phi1, b))))
    pc = gc.nx + 5
    for dt, tol, f32 in ((torch.float64, 1e-13, False), (torch.float32, 2e-6, True)):
        ops = _op_tensors(torch, P.A, dtype=dt)
        s = libmg.op_struct(ops, g.nx, g.ny, g.periodic_y, f32=f32)
        for phi, ref in refs:
            bH = torch.full((gc.nyr, pc), float("nan"), dtype=dt, device="cuda")
            p_d, b_d = _dev(torch, phi, dtype=dt), _dev(torch, b, dtype=dt)  # held until the launch ran
            libmg.mgk("mgk_resid_restrict_even_f32" if f32 else "mgk_resid_restrict_even_f64", C.byref(s),
                      p_d.data_ptr(), b_d.data_ptr(), bH.data_ptr(), pc, _stream(torch))
            torch.cuda.synchronize()
            scale = np.abs(P.A.diag).max() * np.abs(phi).max()
            assert np.abs(_host(bH, gc.nx) - ref).max() <= tol * scale, (case, f32)
    with pytest.raises(Exception):  # missing arrays are refused before any launch
        libmg.mgk("mgk_resid_restrict_even_f64", C.byref(libmg.op_struct(_op_tensors(torch, P.A), g.nx, g.ny,
                                                                           g.periodic_y)),
                  None, None, None, pc, _stream(torch))


@pytest.mark.parametrize("case", ["tiny_5", "periodic_17", "rect_33x17"])
def test_coarsest_inverse_solve_matches_dense_oracle(libmg, oracle, cuda, case):
    torch = cuda
    inst = CASES[case]()
    P = oracle.prepare(inst)
    A = P.A
    ops = oracle.hierarchy(A, coarse_max=256)
    Ac = ops[-1]
    gc = I.Grid(Ac.nx, Ac.ny, periodic_y=Ac.periodic)
    m = (Ac.nx - 2) * (Ac.nyr if Ac.periodic else Ac.ny - 2)
    assert m <= 256
    rng = np.random.default_rng(10)
    b = rng.standard_normal(gc.shape) * gc.interior_mask()
    ref = oracle.dense_solve(Ac, b)
    t = _op_tensors(torch, Ac)
    s = libmg.op_struct(t, Ac.nx, Ac.ny, Ac.periodic)
    inv = torch.zeros(m * m, dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    libmg.mgk("mgk_coarse_factor", C.byref(s), inv.data_ptr(), status.data_ptr(), _stream(torch))
    for dt, f32, tol in ((torch.float64, False, 1e-12), (torch.float32, True, 1e-6)):
        x = torch.zeros(gc.shape, dtype=dt, device="cuda")
        ops_x = _op_tensors(torch, Ac, dtype=dt)
        sx = libmg.op_struct(ops_x, Ac.nx, Ac.ny, Ac.periodic, f32=f32)
        b_d = _dev(torch, b, dtype=dt)
        libmg.mgk("mgk_coarse_solve_f32" if f32 else "mgk_coarse_solve_f64", C.byref(sx),
                  inv.data_ptr(), b_d.data_ptr(), x.data_ptr(), _stream(torch))
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert _rel(_host(x, Ac.nx), ref) < tol


def test_bad_arguments_are_rejected(libmg, cuda):
    s = libmg.mgk_op_f64()
    s.nx, s.ny, s.pitch = 9, 9, 4  # pitch < nx
    assert libmg.lib().mgk_smooth_f64(C.byref(s), None, None, 1, 0, None) == 1
