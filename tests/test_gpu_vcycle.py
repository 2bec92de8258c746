"""One complete V-cycle on the GPU (mgk_vcycle_*: fused tile smoothers on the large
levels, the single-CTA tail kernel on the small ones, the coarsest dense inverse) against
one V-cycle of the oracle on the same hierarchy, right-hand side and zero start.
FP64: agreement to rounding (1e-12 relative); FP32: 2e-5 relative."""
import ctypes as C
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2602_01888_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = {
    "sine_129": lambda: I.config1(129),
    "incl_257": lambda: I.inclusion_instance(257, 0.25, 10.0, 21),
    "annulus_129": lambda: I.annulus_log(129),
    "rect_129x65": lambda: I.Instance("r", I.Grid(129, 65, 0.0, 0.0, 1.0, 0.5),
                                      I.MapSpec("sine_warp", (0.07,)), np.ones((65, 129))),
    "tiny_17": lambda: I.config1(17),
    "ragged_193x97": lambda: I.Instance("g", I.Grid(193, 97, 0.0, 0.0, 1.0, 0.5),
                                        I.MapSpec("affine", (1.0, 0.25, -0.1, 1.05)),
                                        np.ones((97, 193))),
    "annulus_513": lambda: I.annulus_log(513),
    "ragged_769x385": lambda: I.Instance("g", I.Grid(769, 385, 0.0, 0.0, 1.0, 0.5),
                                         I.MapSpec("sine_warp", (0.05,)), np.ones((385, 769))),
}


def _dev(torch, a, dtype):
    return torch.from_numpy(np.array(a)).to("cuda", dtype)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("nu", [(2, 2), (1, 1), (3, 1)])
def test_vcycle_matches_oracle(libmg, oracle, cuda, case, prec, nu):
    torch = cuda
    inst = CASES[case]()
    P = oracle.prepare(inst)
    ops = oracle.hierarchy(P.A)
    H = oracle.Hierarchy(P.A, nu1=nu[0], nu2=nu[1])
    rng = np.random.default_rng(31)
    r = rng.standard_normal(inst.grid.shape) * inst.grid.interior_mask() * np.abs(P.A.diag).max()
    ref = H.vcycle(r)
    dt = torch.float64 if prec == "f64" else torch.float32
    keep = []
    structs = (libmg.mgk_op_f64 if prec == "f64" else libmg.mgk_op_f32) * len(ops)
    arr = structs()
    X, B, T = [], [], []
    for l, A in enumerate(ops):
        t = [_dev(torch, a, dt) for a in (A.cE, A.cN, A.cNE, A.cNW, A.diag, 1.0 / A.diag)]
        keep.append(t)
        arr[l] = libmg.op_struct(t, A.nx, A.ny, A.periodic, f32=(prec == "f32"))
        shape = A.cE.shape
        X.append(torch.zeros(shape, dtype=dt, device="cuda"))
        B.append(_dev(torch, r, dt) if l == 0 else torch.zeros(shape, dtype=dt, device="cuda"))
        T.append(torch.zeros(shape, dtype=dt, device="cuda"))
    Ac = ops[-1]
    m = (Ac.nx - 2) * (Ac.nyr if Ac.periodic else Ac.ny - 2)
    inv = torch.zeros(m * m, dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    t64 = [_dev(torch, a, torch.float64) for a in (Ac.cE, Ac.cN, Ac.cNE, Ac.cNW, Ac.diag, 1.0 / Ac.diag)]
    s64 = libmg.op_struct(t64, Ac.nx, Ac.ny, Ac.periodic)
    stream = torch.cuda.current_stream().cuda_stream
    libmg.mgk("mgk_coarse_factor", C.byref(s64), inv.data_ptr(), status.data_ptr(), stream)
    ptrs = lambda L: (C.c_void_p * len(L))(*[t.data_ptr() for t in L])
    libmg.mgk(f"mgk_vcycle_{prec}", len(ops), arr, ptrs(X), ptrs(B), ptrs(T), inv.data_ptr(),
              nu[0], nu[1], 0, stream)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    got = X[0].double().cpu().numpy()
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < (1e-12 if prec == "f64" else 2e-5), (case, prec, nu, err)


def test_host_loop_mode_matches_graph_mode(libmg):
    """MG_SOLVE_LOOP=host (used for per-kernel profiling) runs the same kernels: bitwise
    equal results and iteration counts."""
    code = r"""
import sys, numpy as np
sys.path.insert(0, %r)
from paper_2602_01888_gb300 import inputs as I, mg
ctx = mg.Context(0)
out = []
for prec, outer in (("fp64", "fcg"), ("mixed", "fcg"), ("fp64", "vcycle")):
    inst = I.inclusion_instance(129, 0.25, 10.0, 3)
    p = mg.Problem(ctx, inst, mg.make_opts(prec, outer, rtol=1e-10))
    phi, st = p.solve()
    out.append((phi, st.iters))
np.save(sys.argv[1], np.stack([o[0] for o in out]))
print(" ".join(str(o[1]) for o in out))
""" % os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    import tempfile
    res = {}
    with tempfile.TemporaryDirectory() as d:
        for mode in ("graph", "host"):
            env = dict(os.environ)
            if mode == "host":
                env["MG_SOLVE_LOOP"] = "host"
            f = os.path.join(d, mode + ".npy")
            r = subprocess.run([sys.executable, "-c", code, f], env=env, capture_output=True, text=True,
                               timeout=600)
            assert r.returncode == 0, r.stderr
            res[mode] = (np.load(f), r.stdout.strip())
    assert res["graph"][1] == res["host"][1]
    assert np.array_equal(res["graph"][0], res["host"][0])


PIPE_CASES = {
    "sine_385x257": lambda: I.Instance("s", I.Grid(385, 257, 0.0, 0.0, 1.5, 1.0),
                                       I.MapSpec("sine_warp", (0.08,)), np.ones((257, 385))),
    "incl_257": lambda: I.inclusion_instance(257, 0.3, 30.0, 22),
    "annulus_257": lambda: I.annulus_log(257),
    "ragged_301x199": lambda: I.Instance("g", I.Grid(301, 199, 0.0, 0.0, 1.0, 0.66),
                                         I.MapSpec("affine", (1.0, 0.2, -0.15, 1.1)),
                                         np.ones((199, 301))),
}


@pytest.mark.parametrize("case", list(PIPE_CASES))
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("rev", [0, 1])
@pytest.mark.parametrize("prolong", [False, True])
def test_pipelined_and_tile_smoothers_match_oracle(libmg, oracle, cuda, case, prec, rev, prolong):
    """k_smooth_pipe, k_smooth_fused and k_smooth_march, one launch each, against the oracle's
    sweeps, with and without the fused prolongation-correction; rows padded to a 32-multiple
    pitch."""
    torch = cuda
    inst = PIPE_CASES[case]()
    P = oracle.prepare(inst)
    g = inst.grid
    pitch = (g.nx + 31) // 32 * 32
    dt = torch.float64 if prec == "f64" else torch.float32
    rng = np.random.default_rng(41)
    phi0 = rng.standard_normal(g.shape)
    b = rng.standard_normal(g.shape) * np.abs(P.A.diag).max()

    def padded(a):
        t = torch.zeros((g.nyr, pitch), dtype=dt, device="cuda")
        t[:, : g.nx] = torch.from_numpy(np.array(a)).to("cuda", dt)
        return t

    ops = [padded(a) for a in (P.A.cE, P.A.cN, P.A.cNE, P.A.cNW, P.A.diag, 1.0 / P.A.diag)]
    st = libmg.op_struct(ops, g.nx, g.ny, g.periodic_y, f32=(prec == "f32"))
    start = phi0.copy()
    eH_d, pc = None, 0
    if prolong and (g.nx - 1) % 2 == 0 and (g.ny - 1) % 2 == 0:
        gc = I.Grid((g.nx - 1) // 2 + 1, (g.ny - 1) // 2 + 1, g.x0, g.y0, g.lx, g.ly, g.periodic_y)
        eH = rng.standard_normal(gc.shape) * gc.interior_mask()
        start = oracle.prolong_add(g.nx, g.ny, g.periodic_y, eH, phi0)
        pc = (gc.nx + 31) // 32 * 32
        eH_d = torch.zeros((gc.nyr, pc), dtype=dt, device="cuda")
        eH_d[:, : gc.nx] = torch.from_numpy(eH).to("cuda", dt)
    elif prolong:
        pytest.skip("odd grid: no coarse level")
    stream = torch.cuda.current_stream().cuda_stream
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    kinds = ("pipe", "fused", "march")
    for kind in kinds:
        sweeps = {"pipe": lambda: libmg.lib().mgk_pipe_sweeps(int(prec == "f32")),
                  "fused": lambda: libmg.lib().mgk_fused_sweeps(int(prec == "f32")),
                  "march": lambda: (libmg.lib().mgk_march_sweeps() if prec == "f32"
                                    else libmg.lib().mgk_march_sweeps_f64())}[kind]()
        ref = oracle.smooth(P.A, start, b, sweeps=sweeps, reverse=bool(rev))
        xin, xout, b_d = padded(phi0), torch.zeros((g.nyr, pitch), dtype=dt, device="cuda"), padded(b)
        args = [C.byref(st), xin.data_ptr(), xout.data_ptr(), b_d.data_ptr(), rev,
                eH_d.data_ptr() if eH_d is not None else None, pc]
        if kind == "pipe":
            libmg.mgk(f"mgk_smooth_pipe_{prec}", *args, err.data_ptr(), stream)
        elif kind == "march":
            libmg.mgk(f"mgk_smooth_march_{prec}", *args, stream)
        else:
            libmg.mgk(f"mgk_smooth_fused_{prec}", *args, stream)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        got = xout[:, : g.nx].double().cpu().numpy()
        e = np.abs(got - ref).max() / np.abs(ref).max()
        assert e < (1e-13 if prec == "f64" else 1e-5), (kind, case, prec, rev, prolong, e)


MARCH_CASES = {
    "annulus_1025": lambda: I.annulus_log(1025),
    "sine_1537x769": lambda: I.Instance("s", I.Grid(1537, 769, 0.0, 0.0, 2.0, 1.0),
                                        I.MapSpec("sine_warp", (0.06,)), np.ones((769, 1537))),
    "ragged_483x131": lambda: I.Instance("g", I.Grid(483, 131, 0.0, 0.0, 1.0, 0.27),
                                         I.MapSpec("affine", (1.0, 0.2, -0.15, 1.1)),
                                         np.ones((131, 483))),
}


@pytest.mark.parametrize("case", list(MARCH_CASES))
@pytest.mark.parametrize("rev", [0, 1])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_march_smoother_multi_strip_matches_oracle(libmg, oracle, cuda, case, rev, prec):
    """The row-marching smoother (FP32: two sweeps a pass, FP64: one) on grids of several
    strips and segments (and the periodic seam of the annulus) against the oracle's sweeps;
    every node of xout written."""
    torch = cuda
    inst = MARCH_CASES[case]()
    P = oracle.prepare(inst)
    g = inst.grid
    pitch = (g.nx + 31) // 32 * 32
    dt = torch.float32 if prec == "f32" else torch.float64
    rng = np.random.default_rng(43)
    phi0 = rng.standard_normal(g.shape)
    b = rng.standard_normal(g.shape) * np.abs(P.A.diag).max()

    def padded(a):
        t = torch.zeros((g.nyr, pitch), dtype=dt, device="cuda")
        t[:, : g.nx] = torch.from_numpy(np.array(a)).to("cuda", dt)
        return t

    ops = [padded(a) for a in (P.A.cE, P.A.cN, P.A.cNE, P.A.cNW, P.A.diag, 1.0 / P.A.diag)]
    st = libmg.op_struct(ops, g.nx, g.ny, g.periodic_y, f32=(prec == "f32"))
    ns = libmg.lib().mgk_march_sweeps() if prec == "f32" else libmg.lib().mgk_march_sweeps_f64()
    ref = oracle.smooth(P.A, phi0, b, sweeps=ns, reverse=bool(rev))
    xin, b_d = padded(phi0), padded(b)
    xout = torch.full((g.nyr, pitch), float("nan"), dtype=dt, device="cuda")
    libmg.mgk(f"mgk_smooth_march_{prec}", C.byref(st), xin.data_ptr(), xout.data_ptr(), b_d.data_ptr(), rev,
              None, 0, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = xout[:, : g.nx].double().cpu().numpy()
    assert np.isfinite(got).all()
    e = np.abs(got - ref).max() / np.abs(ref).max()
    assert e < (1e-5 if prec == "f32" else 1e-13), (case, rev, e)
    if prec == "f64":
        # bitwise the per-colour kernels' sweep (same operations in the same order per node)
        x2 = padded(phi0)
        libmg.mgk("mgk_smooth_f64", C.byref(st), x2.data_ptr(), b_d.data_ptr(), ns, rev,
                  torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert torch.equal(x2[:, : g.nx], xout[:, : g.nx])
