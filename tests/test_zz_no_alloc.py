"""The allocation-free Jacobi smoother (mgk_jacobi_f64_static) against the ordinary one
(mgk_jacobi_f64, caller-provided scratch): the same result on two calls in a row.

It exists for callers that cannot allocate device memory when they smooth (a
latency-critical loop, or device memory owned entirely by another allocator): its scratch
is a fixed device array inside the library.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_2602_01888_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _dev(torch, a):
    return torch.from_numpy(np.array(a)).to("cuda", torch.float64)


def _operator(oracle, torch, inst, libmg):
    P = oracle.prepare(inst)
    ops = [_dev(torch, a) for a in (P.A.cE, P.A.cN, P.A.cNE, P.A.cNW, P.A.diag, 1.0 / P.A.diag)]
    g = inst.grid
    return P, ops, libmg.op_struct(ops, g.nx, g.ny, g.periodic_y)


@pytest.mark.parametrize("case", ["inclusion_129", "annulus_65"])
def test_static_scratch_jacobi_equals_caller_scratch_jacobi(libmg, oracle, cuda, case):
    torch = cuda
    inst = {"inclusion_129": lambda: I.inclusion_instance(129, 0.25, 10.0, 51),
            "annulus_65": lambda: I.annulus_log(65)}[case]()
    P, ops, st = _operator(oracle, torch, inst, libmg)
    g = inst.grid
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(52)
    for call in range(2):  # two calls in a row share (and reuse) the static array
        phi0 = rng.standard_normal(g.shape)
        b = rng.standard_normal(g.shape) * np.abs(P.A.diag).max()
        b_d = _dev(torch, b)
        x_ref, x_new = _dev(torch, phi0), _dev(torch, phi0)
        tmp = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        libmg.mgk("mgk_jacobi_f64", C.byref(st), x_ref.data_ptr(), b_d.data_ptr(), tmp.data_ptr(), 3,
                  0.8, stream)
        libmg.mgk("mgk_jacobi_f64_static", C.byref(st), x_new.data_ptr(), b_d.data_ptr(), 3, 0.8,
                  stream)
        torch.cuda.synchronize()
        ref, got = x_ref.cpu().numpy(), x_new.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), (case, call)


def test_static_scratch_rejects_grids_beyond_its_capacity(libmg, cuda):
    cap = libmg.lib().mgk_jacobi_f64_static_capacity()
    s = libmg.mgk_op_f64()
    s.nx, s.ny, s.periodic, s.pitch = 2049, 2049, 0, 2080  # 2080 * 2049 > 2^20
    assert 2080 * 2049 > cap
    dummy = cuda.zeros(8, dtype=cuda.float64, device="cuda")
    for name in ("cE", "cN", "cNE", "cNW", "diag", "dinv"):
        setattr(s, name, dummy.data_ptr())
    rc = libmg.lib().mgk_jacobi_f64_static(C.byref(s), dummy.data_ptr(), dummy.data_ptr(), 1, 0.8, None)
    assert rc == 2
    assert "static array" in libmg.mg_last_error()


def _random_pitched_operator(torch, libmg, nx, ny, pitch, seed):
    """A diagonally dominant random 9-point operator in pitched device arrays (the two entry
    points are compared with each other, so any operator with a nonzero diagonal serves)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    off = [(-torch.rand((ny, pitch), generator=g, dtype=torch.float64)).cuda() for _ in range(4)]
    diag = (8.0 + torch.rand((ny, pitch), generator=g, dtype=torch.float64)).cuda()
    ops = off + [diag, 1.0 / diag]
    return ops, libmg.op_struct(ops, nx, ny, False)


def test_static_scratch_accepts_a_grid_of_exactly_its_capacity(libmg, cuda):
    """pitch x rows equal to the capacity (1024 x 1024 = 2^20, nx = 1000) is accepted and
    gives bitwise the caller-scratch result on two calls in a row; zero sweeps leave phi
    unchanged."""
    torch = cuda
    nx, ny, pitch = 1000, 1024, 1024
    assert pitch * ny == libmg.lib().mgk_jacobi_f64_static_capacity()
    ops, st = _random_pitched_operator(torch, libmg, nx, ny, pitch, 61)
    stream = torch.cuda.current_stream().cuda_stream
    g = torch.Generator(device="cpu").manual_seed(62)
    for call in range(2):
        phi0 = torch.randn((ny, pitch), generator=g, dtype=torch.float64).cuda()
        b = torch.randn((ny, pitch), generator=g, dtype=torch.float64).cuda()
        x_ref, x_new = phi0.clone(), phi0.clone()
        tmp = torch.zeros((ny, pitch), dtype=torch.float64, device="cuda")
        libmg.mgk("mgk_jacobi_f64", C.byref(st), x_ref.data_ptr(), b.data_ptr(), tmp.data_ptr(), 2, 0.8,
                  stream)
        libmg.mgk("mgk_jacobi_f64_static", C.byref(st), x_new.data_ptr(), b.data_ptr(), 2, 0.8, stream)
        torch.cuda.synchronize()
        assert torch.equal(x_new, x_ref), call
        assert not torch.equal(x_new, phi0)
        x0 = phi0.clone()
        libmg.mgk("mgk_jacobi_f64_static", C.byref(st), x0.data_ptr(), b.data_ptr(), 0, 0.8, stream)
        torch.cuda.synchronize()
        assert torch.equal(x0, phi0)
