"""Benchmark: unknowns solved per second to 1e-9 relative error on one GB300.

Workload (default): the 8193^2 annulus (polar map of Eq. 29, r in [0.2, 1], periodic in
theta, Dirichlet at both radii; 64-mode seeded Fourier source), 67.1 M unknowns.  The
mixed path (FP32 x-line V(1,1) cycles inside FP64 flexible CG) is the headline value; the
FP64 path runs beside it.  One step is one pass of the whole hot path on resident inputs:
coefficient build + Galerkin hierarchy + coarsest inverse (mg_update_transform) and the
solve (mg_solve) to the residual tolerance whose error against the FP64 oracle is at most
a tenth of the 1e-9 target (checked by the GPU test suite at these settings).

Prints one JSON line.  --impl reference times the FP64 CPU oracle on a bounded sample of
the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2602_01888_gb300 import inputs as I  # noqa: E402

METRIC = "unknowns solved/sec to 1e-9 rel. error (FP64 vs mixed, 1 GB300)"
RTOL = 1e-9
# FP64 rate at the maximum SM clock (2 FP64 FMA per clock per SM x 152 SMs x 2.07 GHz); the
# FP64 fractions use the same count at the SM clock sampled in the run (fp64_peak()).
FP64_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def _hbm_peak():
    """HBM denominator: the copy bandwidth measured on this GPU pool (MEASURED_PEAKS.json
    beside this file), else the fallback figure of an earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError, TypeError):
        return 6800.0, "of fallback (6.8 TB/s, MEASURED_PEAKS.json absent)"


HBM_PEAK_GBS, HBM_PEAK_SOURCE = _hbm_peak()
MARCH_NODES = 2000000  # FP32 levels of at least this many nodes are smoothed by the marching kernel


def _traffic_table():
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            return json.load(f)["entries"]
    except (OSError, ValueError, KeyError):
        return []


def profiled_traffic(kernel, nx, rows):
    """DRAM bytes per launch of `kernel` on an nx x rows level from the committed ncu
    figures (profiles/dram_traffic.json), scaled by the node count from the captured size;
    None if that kernel was not captured since its last change."""
    for e in _traffic_table():
        if e["kernel"] == kernel:
            cx, cy = e["captured"]
            return e["bytes"] * (nx * rows) / (cx * cy)
    return None


_FP64_PEAK = None
FP64_FMA_PER_CLK_PER_SM = 2  # GB300's FP64 units: 2 fused multiply-adds per clock per SM
N_SM = 152


def fp64_peak(mg, torch, seconds=1.2):
    """FP64 peak of this GPU for the FP64 roofline fractions: derived from the unit count and
    the SM clock sampled while the library's FMA-chain probe runs (2 FMA/clk/SM x 2 flop x
    152 SMs x median SM MHz), with the probe's own best rate beside it (independent register
    FMA chains, best over operand patterns and launch shapes, CUDA events).  The probe
    reaches about 84% of the derived figure, while the FP64 `A p` kernel of the outer
    iteration reaches 90-94% of it, so the derived figure, not the probe, bounds the FP64
    kernels."""
    global _FP64_PEAK
    if _FP64_PEAK is None:
        pr = fma_probe(mg, torch, True, seconds)
        mhz = pr.get("sm_mhz") or pr.get("sm_max_mhz") or 2070.0
        derived = FP64_FMA_PER_CLK_PER_SM * 2 * N_SM * mhz * 1e6 / 1e12
        _FP64_PEAK = {"tflops": derived, "sm_mhz": mhz, "probe_tflops": pr["tflops"], "probe_shape": pr["shape"],
                      "probe_frac_of_derived": pr["tflops"] / derived,
                      "source": (f"derived: {FP64_FMA_PER_CLK_PER_SM} FP64 FMA/clk/SM x 2 flop x {N_SM} SMs x "
                                 f"{mhz:.0f} MHz (median sampled during the FMA-chain probe)")}
    return _FP64_PEAK


def fma_probe(mg, torch, f64, seconds=0.6):
    """Best FMA rate over a few launch shapes (independent chains per thread x CTAs per SM),
    each timed with CUDA events for a share of `seconds`; SM clock sampled meanwhile."""
    iters = 2000 if f64 else 50000
    shapes = [(pat, ch, 152 * k) for pat in (0, 1) for ch in (4, 8, 16) for k in (8, 16, 32)]
    out = torch.empty(152 * 32 * 256, dtype=torch.float64 if f64 else torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    for pat, ch, blocks in shapes:
        mg.mgk("mgk_fma_rate", int(f64), pat, ch, blocks, iters, out.data_ptr(), s)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    best, best_shape = 0.0, None
    for pat, ch, blocks in shapes:
        flops = mg.lib().mgk_fma_rate_flops(ch, blocks, iters)
        t_end = time.perf_counter() + seconds / len(shapes)
        while time.perf_counter() < t_end:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            mg.mgk("mgk_fma_rate", int(f64), pat, ch, blocks, iters, out.data_ptr(), s)
            e1.record()
            e1.synchronize()
            r = flops / (e0.elapsed_time(e1) * 1e-3) / 1e12
            if r > best:
                best, best_shape = r, {"pattern": pat, "chains": ch, "ctas": blocks, "threads": 256}
    clocks = sampler.stop()
    r = {"tflops": best, "shape": best_shape, "sm_mhz": clocks.get("sm_mhz"),
         "sm_max_mhz": clocks.get("sm_max_mhz"), "reasons": clocks.get("reasons"),
         "source": "FMA-chain probe mgk_fma_rate (FP64)" if f64 else "FMA-chain probe mgk_fma_rate (FP32)"}
    if r["sm_mhz"] and r["sm_max_mhz"]:
        r["tflops_at_max_clock"] = best * r["sm_max_mhz"] / r["sm_mhz"]
    return r


# Single-instance workloads: (builder, precisions with the headline first, outer iteration,
# residual tolerance per precision, builder of the bounded CPU sample).  Each tolerance is
# calibrated so that the error against the oracle's phi* is at most a tenth of the 1e-9
# target, and within 1e-10 on the FP64 path (measured: inclusion 1025^2 at 3e-8 -> 2.2e-11
# for the oracle's own MG-PCG; annulus 8193^2 against the stored oracle samples: mixed at
# 1e-8 -> 1.1e-10, FP64 x-line V(1,1) at 1e-8 -> 3.4e-10, so the FP64 row stops at 2e-9,
# twice the FP64 residual floor of that grid; all checked by the GPU tests).
WORKLOADS = {
    "inclusion_1025": (lambda: I.config2(1025), ("fp64", "mixed"), "fcg", {"fp64": 3e-8, "mixed": 3e-8},
                       lambda: I.config2(1025)),
    "sine_warp_129": (lambda: I.config1(129), ("fp64", "mixed"), "vcycle", {"fp64": 1e-10, "mixed": 1e-10},
                      lambda: I.config1(129)),
    "annulus_8193": (lambda: I.config3(8193), ("mixed", "fp64"), "fcg", {"mixed": 1e-8, "fp64": 2e-9},
                     lambda: I.config3(1025)),
}


# Smoother and (nu1, nu2) per workload unless given on the command line: zebra x-line
# Gauss-Seidel where the map makes the operator anisotropic (the annulus of Eq. 29: x coupling
# up to 62 times the y coupling; 7 FCG iterations instead of 31), four-colour point
# Gauss-Seidel elsewhere.
SMOOTHER_DEFAULT = {"annulus_8193": ("xline", (1, 1))}


def smoother_of(args):
    sm, nu = SMOOTHER_DEFAULT.get(args.workload, ("gs4", (2, 2)))
    return (args.smoother or sm), (args.nu or nu)


def workload(name: str):
    if name in WORKLOADS:
        return WORKLOADS[name][0]()
    raise SystemExit(f"unknown workload {name}")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, device=0):
        self.device, self.samples, self.proc, self.thread = device, [], None, None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[5 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(sm)}


# ------------------------------------------------------------------ distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(ws):
    if ws <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group("gloo")
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def allmax(dist, v):
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ reference arm (oracle)
def oracle_solve_seconds(inst, rtol=RTOL, smoother="gs4", nu=(2, 2)):
    import oracle as O
    sm = {"gs4": O.SMOOTHER_GS4, "xline": O.SMOOTHER_XLINE}[smoother]
    t0 = time.perf_counter()
    P = O.prepare(inst)
    phi, it, hist = O.pcg_solve(P.A, P.b, P.phi0, rtol=rtol, max_iters=400, smoother=sm, nu1=nu[0],
                                nu2=nu[1])
    return time.perf_counter() - t0, it


def run_reference_instances(args):
    """Reference arm of the many-instance workloads: the oracle (FCG preconditioned by its
    V(2,2), one thread) on a fixed bounded subset of the workload's own instances per step:
    the first 8 of the 512 batch instances, or the first 6 requests of the served stream with
    sides up to 513 (the mapped grids of larger ones take minutes to generate on the CPU)."""
    import oracle as O
    O.build()
    if args.workload == "batch512":
        insts = [I.inclusion_instance(*sp) for sp in I.config4_specs(BATCH_COUNT)[:8]]
        rtol, sample = BATCH_RTOL, "the first 8 of the 512 batch instances per step, same rtol"
    else:
        stream = [q for q in I.config5_stream(2000, seed=5, rate=1.0, side_range=(129, 2049)) if q[1] <= 513][:6]
        # the CPU generates these requests' mapped grids itself (numpy multigrid of the inputs)
        insts = [I.inclusion_instance(n, r, ratio, sd) for _, n, r, ratio, sd in stream]
        rtol, sample = SERVE_RTOL, "the first 6 served requests with sides up to 513 per step, same rtol"
    U = sum(x.grid.unknowns for x in insts)

    def step():
        t = 0.0
        for x in insts:
            dt, _ = oracle_solve_seconds(x, rtol)
            t += dt
        return t

    for _ in range(args.warmup):
        step()
    tot = sum(step() for _ in range(args.steps))
    v = U * args.steps / tot
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "unknowns/s", "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": {"workload": args.workload, "rtol": rtol, "smoother": "gs4",
                                                      "outer": "fcg+vcycle(2,2)"},
                      "cpu_baseline": {"value": v, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": v, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
    return 0


# Bounded CPU samples of each single-instance workload (the oracle's inputs), by name.
SAMPLES = {
    "annulus_8193": lambda: I.config3(1025),
    "inclusion_1025": lambda: I.config2(1025),
    "inclusion_513": lambda: I.inclusion_instance(513, 0.25, 10.0, 2),
    "sine_warp_129": lambda: I.config1(129),
}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _core_worker(conn, key, rtol, smoother, nu):
    """One host core: builds its copy of the sample once, then runs one oracle step (the
    coefficient build and the MG-preconditioned CG solve) per request from the parent."""
    import oracle as O  # noqa: F401  (built by the parent)
    inst = SAMPLES[key]()
    conn.send("ready")
    while conn.recv() is not None:
        t0 = time.monotonic()
        oracle_solve_seconds(inst, rtol, smoother, nu)
        conn.send((t0, time.monotonic(), inst.grid.unknowns))


class OracleCores:
    """The oracle as it stands, one independent copy per host core (spawned processes, so it
    is safe after CUDA was initialised): a step runs one sample solve on every core at once
    and takes from the first start to the last finish."""

    def __init__(self, n, key, rtol, smoother, nu):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for _ in range(n):
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_core_worker, args=(b, key, rtol, smoother, nu), daemon=True)
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)
        for c in self.conns:
            if c.recv() != "ready":
                raise RuntimeError("oracle worker failed to start")

    def step(self):
        for c in self.conns:
            c.send(1)
        outs = [c.recv() for c in self.conns]
        return max(o[1] for o in outs) - min(o[0] for o in outs), sum(o[2] for o in outs)

    def close(self):
        for c in self.conns:
            c.send(None)
        for pr in self.procs:
            pr.join(timeout=60)


def cpu_baseline(key, rtol, smoother, nu, what):
    """The oracle timed on this host: one thread on one sample, and every core running its
    own copy of the same sample at once (aggregate unknowns/s)."""
    import oracle as O
    O.build()
    inst = SAMPLES[key]()
    dt, it = oracle_solve_seconds(inst, rtol, smoother, nu)
    one = inst.grid.unknowns / dt
    n = os.cpu_count() or 1
    pool = OracleCores(n, key, rtol, smoother, nu)
    try:
        wall, U = pool.step()
    finally:
        pool.close()
    desc = (f"one {inst.grid.nx}^2 solve of the {what} recipe (coefficients + MG-preconditioned CG "
            f"with the same cycle ({smoother}, V({nu[0]},{nu[1]})) to rtol {rtol})")
    return {"value": U / wall, "unit": "unknowns/s", "cores": n, "kind": "oracle",
            "sample": f"{desc} on each of the {n} host cores at once, aggregate",
            "single_thread": {"value": one, "cores": 1, "sample": desc + ", 1 thread"},
            "nproc": n, "cpu_model": cpu_model()}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload in ("batch512", "serve"):
        return run_reference_instances(args)
    if args.workload == "sor_vs_gmg":
        print(json.dumps({"impl": "reference", "unavailable": "sor_vs_gmg already times the oracle itself "
                                                              "(its cpu_oracle_1_thread entries)"}))
        return 0
    import oracle as O
    O.build()
    _, precisions, outer, rtols, _ = WORKLOADS[args.workload]
    rtol = rtols[precisions[0]]  # the headline path's tolerance (error within 1e-10 of phi*)
    key = args.workload
    if args.workload == "inclusion_1025" and (args.steps + args.warmup) > 16:
        key = "inclusion_513"
    smoother, nu = smoother_of(args)
    n = args.ref_cores or os.cpu_count() or 1
    inst = SAMPLES[key]()
    sample = (f"{args.workload} recipe at {inst.grid.nx}^2 (the full workload is too large for the CPU "
              f"in the run's time), same rtol and cycle; one copy per host core, {n} at once")
    pool = OracleCores(n, key, rtol, smoother, nu)
    try:
        for _ in range(args.warmup):
            pool.step()
        tot, U = 0.0, 0
        for _ in range(args.steps):
            dt, u = pool.step()
            tot += dt
            U += u
    finally:
        pool.close()
    v = U / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "unknowns/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "rtol": rtol, "smoother": smoother,
                                            "outer": f"fcg+vcycle({nu[0]},{nu[1]})"},
            "cpu_baseline": {"value": v, "unit": "unknowns/s", "cores": n, "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model()},
            "e2e": {"value": v, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _hbm_roof(kern, ach, launch_s, g, **extra):
    """Roofline object of a bytes-bound kernel: algorithmic GB/s against the HBM peak."""
    return dict({"bound": "hbm", "achieved": ach, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                 "frac": ach / HBM_PEAK_GBS, "traffic": profiled_traffic(kern, g.nx, g.nyr), "kernel": kern,
                 "launch_us": launch_s * 1e6, "peak_source": HBM_PEAK_SOURCE}, **extra)


def _fp64_roof(mg, torch, kern, tflops, launch_s, g, **extra):
    """Roofline object of an FP64-pipe-bound kernel: algorithmic TFLOP/s against the FP64
    peak derived from the unit count and the SM clock sampled in this run (fp64_peak)."""
    pk = fp64_peak(mg, torch)
    return dict({"bound": "alu", "achieved": tflops, "peak": pk["tflops"], "unit": "TFLOP/s",
                 "frac": tflops / pk["tflops"], "traffic": profiled_traffic(kern, g.nx, g.nyr), "kernel": kern,
                 "launch_us": launch_s * 1e6,
                 "peak_source": pk["source"] + f"; FMA-chain probe {pk['probe_tflops']:.3f} TFLOP/s"},
                **extra)


# ------------------------------------------------------------------ our arm
def measure_smoother(mg, torch, inst, prec, reps=20, smoother="gs4", family=None):
    """Dominant kernel of the level-0 smoothing timed alone with CUDA events on this
    workload's finest level, operator built by the library's own kernels: one four-colour
    Gauss-Seidel sweep (4 launches of k_gs_colour), or on FP32 levels of at least
    MARCH_NODES nodes one launch of the row-marching kernel (two sweeps).  FP64: flop-bound
    (18 flop per updated unknown); FP32: bytes-bound (algorithmic 32 B per node and pass:
    iterate read and written, b, four couplings, 1/diag)."""
    import ctypes as C
    g = inst.grid
    pitch = (g.nx + 31) // 32 * 32
    f32 = prec == "mixed"
    z = lambda d=torch.float64: torch.zeros((g.nyr, pitch), dtype=d, device="cuda")
    pad = lambda a: torch.nn.functional.pad(torch.from_numpy(np.array(a, dtype=np.float64)).cuda(),
                                            (0, pitch - g.nx))
    D, exx, exy, eyy = z(), z(), z(), z()
    folded = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    eps = pad(inst.eps_phys) if inst.eps_phys is not None else None
    if inst.map.kind == "grid":
        xp, yp = pad(inst.map.xp), pad(inst.map.yp)
        mg.mgk("mgk_eps_grid", g.nx, g.ny, int(g.periodic_y), g.hx, g.hy, xp.data_ptr(), yp.data_ptr(),
               0.0, 0.0, eps.data_ptr() if eps is not None else None, pitch, D.data_ptr(),
               exx.data_ptr(), exy.data_ptr(), eyy.data_ptr(), folded.data_ptr(), s)
    else:
        prm = (C.c_double * 4)(*(list(inst.map.params) + [0.0] * 4)[:4])
        mg.mgk("mgk_eps_analytic", mg.MAP_CODES[inst.map.kind], prm, g.nx, g.ny, int(g.periodic_y),
               g.x0, g.y0, g.hx, g.hy, eps.data_ptr() if eps is not None else None, pitch,
               D.data_ptr(), exx.data_ptr(), exy.data_ptr(), eyy.data_ptr(), folded.data_ptr(), s)
    ops = [z() for _ in range(6)]
    five = mg.map_five_point(inst.map)  # the solver's own choice for this map
    st = mg.op_struct(ops, g.nx, g.ny, g.periodic_y, five_point=five)
    mg.mgk("mgk_assemble", C.byref(st), g.hx, g.hy, exx.data_ptr(), exy.data_ptr(), eyy.data_ptr(), s)
    dt = torch.float32 if f32 else torch.float64
    if f32:
        ops32 = [z(torch.float32) for _ in range(6)]
        st32 = mg.op_struct(ops32, g.nx, g.ny, g.periodic_y, f32=True, five_point=five)
        mg.mgk("mgk_op_to_f32", C.byref(st), C.byref(st32), s)
        st, name = st32, "mgk_smooth_f32"
    else:
        name = "mgk_smooth_f64"
    del D, exx, exy, eyy
    x = z(dt)
    b = torch.randn((g.nyr, pitch), dtype=torch.float64, device="cuda").to(dt)
    if smoother == "xline":
        return _measure_line(mg, torch, g, st, x, b, f32, s, reps, five)
    fam, shape = parse_choice(family)
    if fam is None:  # untuned: the size rule of the cycle
        fam = "marching" if g.nx * g.nyr >= MARCH_NODES else "colour"
    if fam in ("pipelined", "fused", "marching"):
        return _measure_variant(mg, torch, g, st, x, z(dt), b, f32, s, reps, fam, shape)

    def once():
        mg.mgk(name, C.byref(st), x.data_ptr(), b.data_ptr(), 1, 0, s)

    for _ in range(3):
        once()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        once()
    e1.record()
    torch.cuda.synchronize()
    per_launch_s = e0.elapsed_time(e1) * 1e-3 / (reps * 4)
    kern = "k_gs_colour<float>" if f32 else "k_gs_colour<double>"
    if f32:
        bytes_per_launch = 32.0 * g.nx * g.nyr / 4  # a sweep's algorithmic bytes over its 4 launches
        ach = bytes_per_launch / per_launch_s / 1e9
        return _hbm_roof(kern, ach, per_launch_s, g)
    flops_per_launch = g.unknowns / 4 * 18.0  # 8 FMA + subtract + scale per updated unknown
    achieved = flops_per_launch / per_launch_s / 1e12
    return _fp64_roof(mg, torch, kern, achieved, per_launch_s, g)


FAMILY_CODES = {"fused": 2, "pipelined": 3, "marching": 4}


def parse_choice(desc):
    """("fused", (64, 16, 2)) from the bench's autotune entry "fused 64x16/2"; ("marching",
    (240, 0, 2)) from "marching w240/2"; (family, None) without a shape; (None, None) if
    untuned."""
    if not desc:
        return None, None
    parts = desc.split()
    if len(parts) == 1:
        return parts[0], None
    dims, ns = parts[1].split("/")
    if dims.startswith("w"):
        return parts[0], (int(dims[1:]), 0, int(ns))
    tx, ty = dims.split("x")
    return parts[0], (int(tx), int(ty), int(ns))


def _measure_variant(mg, torch, g, st, x, x2, b, f32, s, reps, family, shape):
    """One launch shape of the tile or row-marching smoothers (the autotuner's choice for
    the finest level, else the family's default), ping-pong iterates.  FP64: flop-bound (18
    flop per unknown and sweep); FP32: bytes-bound (32 B per node and launch: each array read
    once, the iterate written once)."""
    import ctypes as C
    tag = "f32" if f32 else "f64"
    code = FAMILY_CODES[family]
    vs = mg.smooth_variants(f32, code)
    v, tile, ns = vs[0]
    for cand in vs:
        if shape is not None and (cand[1][0], cand[1][1], cand[2]) == shape:
            v, tile, ns = cand

    def once():
        mg.mgk(f"mgk_smooth_variant_{tag}", C.byref(st), code, v, x.data_ptr(), x2.data_ptr(), b.data_ptr(), 0,
               None, 0, None, s)

    for _ in range(3):
        once()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        once()
    e1.record()
    torch.cuda.synchronize()
    per_launch_s = e0.elapsed_time(e1) * 1e-3 / reps
    T = "float" if f32 else "double"
    if family == "marching":
        kern = f"k_smooth_march<{T}> w{tile[0]}/{ns}"  # owned strip columns / sweeps per pass
    else:
        kern = f"k_smooth_{'pipe' if family == 'pipelined' else 'fused'}<{T},{tile[0]},{tile[1]},{ns}>"
    note = f"the autotuner's choice for this level size ({family}), {ns} sweep(s) per launch"
    if f32:
        ach = 32.0 * g.nx * g.nyr / per_launch_s / 1e9
        return _hbm_roof(kern, ach, per_launch_s, g, sweeps_per_launch=ns, note=note)
    achieved = g.unknowns * 18.0 * ns / per_launch_s / 1e12
    return _fp64_roof(mg, torch, kern, achieved, per_launch_s, g, sweeps_per_launch=ns, note=note)


def cycle_model(prec, smoother, nu, five=False):
    """Algorithmic bytes and flops per fine node of one V(nu1, nu2) cycle, coarser levels
    included (x 4/3).  Point smoother, two sweeps per pass: each pass reads the five
    operator arrays (C = 5 elements) and moves the iterate in and out and b; the residual +
    restriction pass reads the operator, iterate and b and writes a quarter node; the first
    post-smoothing pass also reads the quarter-size correction (68 + 3C bytes at FP64 for
    V(2,2)).  Line smoother: 14 elements per sweep (six off-row couplings, iterate in and
    out, b, five factor arrays), plus the residual + restriction pass and a prolongation
    pass.  After line pre-smoothing the residual is computed on the even rows only (the odd
    rows were just solved exactly): x of every row, b, diag and the E coupling of the even
    rows, the N, NE and NW couplings of every row (they couple an even row to both of its
    neighbours): 5.5 elements + 1/4, 9 flops per fine node; with nu1 = 0 the whole residual,
    7 + 1/4 elements and 18 flops.  Flops: 18 per unknown update.  five: the finest operator
    is a 5-point stencil (no NE / NW couplings): 10 elements per line sweep, a residual pass
    of 3.5 + 1/4 (5 + 1/4 in full), 5 flops per fine node (10 in full) and 16 per line update
    instead of 24."""
    e = 8.0 if prec == "fp64" else 4.0
    n1, n2 = nu
    if smoother == "xline":
        half = 0.5 if n1 > 0 else 1.0  # share of the rows whose residual is computed
        if five:
            fine = (n1 + n2) * 10 * e + (3.5 if n1 > 0 else 5.0) * e + 0.25 * e + (2 + 0.25) * e
            flops = (n1 + n2) * 16.0 + 10.0 * half + 8.0
        else:
            fine = (n1 + n2) * 14 * e + (5.5 if n1 > 0 else 7.0) * e + 0.25 * e + (2 + 0.25) * e
            flops = (n1 + n2) * 24.0 + 18.0 * half + 8.0
    else:
        p1, p2 = -(-n1 // 2), -(-n2 // 2)
        fine = (p1 + 1 + p2) * 5 * e + p1 * 3 * e + (2 + 0.25) * e + p2 * 3 * e + 0.25 * e
        flops = (n1 + n2) * 18.0 + 18.0 + 8.0
    return fine * 4.0 / 3.0, flops * 4.0 / 3.0


def _measure_line(mg, torch, g, st, x, b, f32, s, reps, five=False):
    """Zebra x-line sweep (two launches of k_line_zebra, one per row parity) on the finest
    level.  Bytes-bound; algorithmic bytes per node and sweep: 14 elements (the N, NE, NW
    couplings of every row, read once per half-sweep as own or lower row: 6; the iterate
    read once and written once: 2; b: 1; the five cyclic-reduction factor arrays: 5); 10 for
    a 5-point operator (no NE / NW couplings: 2 instead of 6)."""
    import ctypes as C
    tag = "f32" if f32 else "f64"
    esz = 4 if f32 else 8
    n = mg.lib().mgk_line_factor_elems(g.nx, g.ny, int(g.periodic_y))
    f = torch.zeros(n, dtype=torch.float32 if f32 else torch.float64, device="cuda")
    mg.mgk(f"mgk_line_factor_{tag}", C.byref(st), f.data_ptr(), s)

    def once():
        mg.mgk(f"mgk_line_smooth_{tag}", C.byref(st), f.data_ptr(), x.data_ptr(), b.data_ptr(), 1, 0, s)

    for _ in range(3):
        once()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        once()
    e1.record()
    torch.cuda.synchronize()
    per_launch_s = e0.elapsed_time(e1) * 1e-3 / (reps * 2)
    kern = f"k_line_zebra<{'float' if f32 else 'double'}>" + (" 5-point" if five else "")
    elems = 10.0 if five else 14.0
    bytes_per_launch = elems * esz * g.nx * g.nyr / 2
    ach = bytes_per_launch / per_launch_s / 1e9
    return _hbm_roof(kern, ach, per_launch_s, g, elements_per_node_and_sweep=elems)


def measure_grid_generation(mg, torch, ctx, n, r, cpu=False):
    """Numerical grid generation of the inclusion workload's mapped grid (Sec. 4.2) on the
    GPU (mg_harmonic_grid: x' and y', device arrays, FCG to rtol 1e-13), timed with CUDA
    events after one warm-up; with cpu=True also the numpy multigrid that generates the
    workload inputs, for comparison."""
    i0 = I.snap_ring(n, r)
    ring, xp0, yp0 = I.inclusion_ring_data(n, i0)
    g = I.Grid(n, n)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    fx, xi, yi = d(ring.astype(np.uint8)), d(xp0), d(yp0)
    xo, yo = torch.empty_like(xi), torch.empty_like(yi)
    st = mg.mg_harmonic_grid(ctx.h, g, fx, xi, yi, xo, yo, rtol=1e-13)
    torch.cuda.synchronize()
    reps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        st = mg.mg_harmonic_grid(ctx.h, g, fx, xi, yi, xo, yo, rtol=1e-13)
    e1.record()
    torch.cuda.synchronize()
    out = {"side": n, "gpu_ms": e0.elapsed_time(e1) / reps, "iters": [s.iters for s in st],
           "rel_residual": max(s.rel_residual for s in st)}
    if cpu:
        t0 = time.perf_counter()
        I._inclusion_grid_cached.__wrapped__(n, i0)
        out["cpu_numpy_s"] = time.perf_counter() - t0
    return out


def run_kernel_only(args):
    """Run one library kernel `--reps` times on a sine-warp operator of side `--side`
    (built by the library's own kernels) and print its mean CUDA-event time per launch;
    used for profiling a single kernel at a chosen size.  fp64peak / fp32peak instead run
    the FMA-chain probe for about a second and print the best rate with the SM clock
    sampled meanwhile (the FP64 figure is the denominator of the FP64 roofline fractions)."""
    import ctypes as C
    import torch
    from paper_2602_01888_gb300 import mg
    torch.cuda.set_device(0)
    if args.kernel in ("fp64peak", "fp32peak"):
        r = fma_probe(mg, torch, args.kernel == "fp64peak", seconds=1.0)
        print(json.dumps(dict(r, kernel=args.kernel, nominal_fp64_tflops=FP64_NOMINAL_TFLOPS)))
        return 0
    n = args.side
    g = I.Grid(n, args.ny or n)
    pitch = (n + 31) // 32 * 32
    f64 = args.kernel.rstrip("p").endswith("64")
    dt = torch.float64 if f64 else torch.float32
    z = lambda d=torch.float64: torch.zeros((g.nyr, pitch), dtype=d, device="cuda")
    D, exx, exy, eyy = z(), z(), z(), z()
    folded = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    # the sine-warp operator (9-point); --stencil 5: the sinh stretching's (no cross term), run
    # by the 5-point forms of the kernels
    five = args.stencil == 5
    kind, prm = (3, (C.c_double * 4)(1.0, 0.5, 0.0, 0.0)) if five else (1, (C.c_double * 4)(0.1, 0.0, 0.0, 0.0))
    mg.mgk("mgk_eps_analytic", kind, prm, n, g.ny, 0, 0.0, 0.0, g.hx, g.hy, None, pitch, D.data_ptr(),
           exx.data_ptr(), exy.data_ptr(), eyy.data_ptr(), folded.data_ptr(), s)
    ops = [z() for _ in range(6)]
    st = mg.op_struct(ops, n, g.ny, False, five_point=five)
    mg.mgk("mgk_assemble", C.byref(st), g.hx, g.hy, exx.data_ptr(), exy.data_ptr(), eyy.data_ptr(), s)
    if not f64:
        ops32 = [z(torch.float32) for _ in range(6)]
        st32 = mg.op_struct(ops32, n, g.ny, False, f32=True, five_point=five)
        mg.mgk("mgk_op_to_f32", C.byref(st), C.byref(st32), s)
        st = st32
    x, b = z(dt), torch.randn((g.nyr, pitch), dtype=torch.float64, device="cuda").to(dt)
    x2 = z(dt)
    nc = (n - 1) // 2 + 1
    pc = (nc + 31) // 32 * 32
    bH = torch.zeros(((g.ny - 1) // 2 + 1, pc), dtype=dt, device="cuda")
    sfx = "f64" if f64 else "f32"
    if args.kernel.startswith("line"):
        fac = torch.zeros(mg.lib().mgk_line_factor_elems(n, g.ny, 0), dtype=dt, device="cuda")
        mg.mgk(f"mgk_line_factor_{sfx}", C.byref(st), fac.data_ptr(), s)

    # the family's default variant unless --variant picks another (fused: FP64 32x32/1, FP32 64x24/2)
    var = args.variant if args.variant >= 0 else (5 if args.kernel.startswith("fused") and not f64 else 0)

    def once():
        if args.kernel.startswith("line"):  # one zebra sweep: two launches of k_line_zebra
            mg.mgk(f"mgk_line_smooth_{sfx}", C.byref(st), fac.data_ptr(), x.data_ptr(), b.data_ptr(), 1, 0, s)
        elif args.kernel.startswith(("march", "pipe", "fused")):
            # "march32p" / "march64p": with the coarse-grid correction fused (post-smoothing form);
            # --variant k: the autotuner's variant k of the family (tile shape, sweeps per launch)
            corr = args.kernel.endswith("p") and args.kernel.startswith("march")
            fam = FAMILY_CODES["marching" if args.kernel.startswith("march") else
                               "pipelined" if args.kernel.startswith("pipe") else "fused"]
            mg.mgk(f"mgk_smooth_variant_{sfx}", C.byref(st), fam, var, x.data_ptr(), x2.data_ptr(),
                   b.data_ptr(), 0, bH.data_ptr() if corr else None, pc if corr else 0, None, s)
        elif args.kernel.startswith("smooth"):
            mg.mgk(f"mgk_smooth_{sfx}", C.byref(st), x.data_ptr(), b.data_ptr(), 1, 0, s)
        elif args.kernel.startswith("restricte"):  # the even-row form used after line pre-smoothing
            mg.mgk(f"mgk_resid_restrict_even_{sfx}", C.byref(st), x.data_ptr(), b.data_ptr(), bH.data_ptr(), pc, s)
        elif args.kernel.startswith("restrict"):
            mg.mgk(f"mgk_resid_restrict_{sfx}", C.byref(st), x.data_ptr(), b.data_ptr(), bH.data_ptr(), pc, s)
        elif args.kernel.startswith("prolong"):
            mg.mgk(f"mgk_prolong_add_{sfx}", C.byref(st), x.data_ptr(), bH.data_ptr(), pc, s)
        else:
            raise SystemExit(f"unknown kernel {args.kernel}")

    for _ in range(3):
        once()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.reps):
        once()
    e1.record()
    torch.cuda.synchronize()
    rec = {"kernel": args.kernel, "side": n, "ny": g.ny, "reps": args.reps, "stencil": args.stencil,
           "ms_per_call": e0.elapsed_time(e1) / args.reps}
    if args.kernel.startswith(("march", "pipe", "fused")):
        fam = FAMILY_CODES["marching" if args.kernel.startswith("march") else
                           "pipelined" if args.kernel.startswith("pipe") else "fused"]
        v, tile, ns = mg.smooth_variants(not f64, fam)[var]
        rec.update(variant=v, tile=tile, sweeps=ns, ms_per_sweep=rec["ms_per_call"] / ns)
    print(json.dumps(rec))
    return 0


def autotune(mg, ctx, max_side, enabled):
    """Time the smoother families in every variant per level size on this GPU (mg_autotune)
    before the problems are set up; returns {precision: {side: "family tile/sweeps"}} for the
    bench line (tile tx x ty for tile kernels, owned strip columns for row marching)."""
    if not enabled:
        return None
    out = {}
    for prec, side, _, choice, var in mg.mg_autotune(ctx.h, max(33, max_side), variants=True):
        tx, ty = var["tile"]
        if choice in ("fused", "pipelined"):
            desc = f"{choice} {tx}x{ty}/{var['sweeps']}"
        elif choice == "marching":
            desc = f"{choice} w{tx}/{var['sweeps']}"
        else:
            desc = choice
        out.setdefault(prec, {})[str(side)] = desc
    return out


def run_ours(args):
    import torch
    from paper_2602_01888_gb300 import mg

    ws, rank, local = dist_env()
    dist = dist_init(ws)
    torch.cuda.set_device(local)
    mg.lib()
    _, precisions, outer, rtols, _ = WORKLOADS[args.workload]
    rtol = rtols[precisions[0]]
    smoother, nu = smoother_of(args)
    inst = workload(args.workload)
    g = inst.grid
    U = g.unknowns
    n = g.nx * g.nyr
    ctx = mg.Context(local)
    ctx.use_torch_stream()
    tuned = autotune(mg, ctx, max(g.nx, g.ny), not args.no_autotune)
    res = {}
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    dev = lambda a: None if a is None else torch.from_numpy(np.array(a, dtype=np.float64)).cuda()
    grid_map = inst.map.kind == "grid"
    xp_d = dev(inst.map.xp) if grid_map else None
    yp_d = dev(inst.map.yp) if grid_map else None
    eps_d, rho_d, bc_d = dev(inst.eps_phys), dev(inst.rho_phys), dev(inst.bc)
    phi_d = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    n_in = 1 + (2 if grid_map else 0) + (1 if inst.eps_phys is not None else 0) + \
        (1 if inst.bc is not None else 0)
    for prec in precisions:
        opts = mg.make_opts(prec, outer, rtol=rtols[prec], max_iters=400, smoother=smoother, nu1=nu[0],
                            nu2=nu[1], coarse_op=args.coarse_op)
        prob = mg.Problem(ctx, inst, opts, device_inputs=True)

        def step():
            mg.mg_update_transform(prob.h, g, inst.map, eps_d, xp_d, yp_d)
            return mg.mg_solve(prob.h, rho_d, bc_d, phi_d, opts)

        for _ in range(args.warmup):
            st = step()
        torch.cuda.synchronize()
        barrier(dist)
        headline = prec == precisions[0]
        sampler = ClockSampler(local) if (headline and rank == 0) else None
        if sampler:
            sampler.start()
        times = []
        for _ in range(args.steps):
            flush.fill_(1.0)  # evict L2 (512 MB > 129 MB) between timed steps
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            st = step()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
        clocks = sampler.stop() if sampler else None
        tot = allmax(dist, float(sum(times)))
        barrier(dist)
        # end to end through the public API with host (pinned) buffers
        pin = lambda a: None if a is None else \
            torch.from_numpy(np.array(a, dtype=np.float64)).pin_memory().numpy()
        xp_h = pin(inst.map.xp) if grid_map else None
        yp_h = pin(inst.map.yp) if grid_map else None
        eps_h, rho_h, bc_h = pin(inst.eps_phys), pin(inst.rho_phys), pin(inst.bc)
        phi_h = torch.zeros(g.shape, dtype=torch.float64).pin_memory().numpy()
        e2e_steps = max(1, min(args.steps, 5))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            mg.mg_update_transform(prob.h, g, inst.map, eps_h, xp_h, yp_h)
            mg.mg_solve(prob.h, rho_h, bc_h, phi_h, opts)
        e2e_t = allmax(dist, time.perf_counter() - t0)
        cycle_ms = mg.mg_cycle_time(prob.h, opts, reps=20)
        res[prec] = {"tot": tot, "times": times, "stats": st, "clocks": clocks, "cycle_ms": cycle_ms,
                     "e2e": ws * U * e2e_steps / e2e_t, "levels": len(prob.levels()),
                     "setup_ms": st.setup_ms, "solve_ms": st.solve_ms,
                     "five_point": mg.problem_five_point(prob.h)}
        prob.close()
    del flush
    family = (tuned or {}).get(precisions[0], {}).get(str(g.nx))  # the tuner's choice for the finest level
    roof = measure_smoother(mg, torch, inst, precisions[0], smoother=smoother, family=family) if rank == 0 else None
    gridgen = None
    if rank == 0 and grid_map and "r" in inst.meta:
        gridgen = measure_grid_generation(mg, torch, ctx, g.nx, inst.meta["r"], cpu=not args.no_cpu_baseline)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, rtol, smoother, nu, args.workload)
    if rank == 0:
        h, others = precisions[0], precisions[1:]
        rh = res[h]
        value = ws * U * args.steps / rh["tot"]
        line = {
            "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * rh["tot"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if h == "fp64" else "f32 cycle in f64 refinement", "data": "synthetic",
            "config": {"workload": args.workload, "precision": h,
                       "outer": f"{outer}+vcycle({nu[0]},{nu[1]})", "smoother": smoother,
                       "rtol": rtols, "unknowns": U, "l2": "flushed between steps (512 MB write)",
                       "finest_stencil": "5-point (map without cross term)" if rh["five_point"] else "9-point",
                       "coarse_op": args.coarse_op,
                       "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
            "iters": rh["stats"].iters, "levels": rh["levels"], "setup_ms": rh["setup_ms"],
            "solve_ms": rh["solve_ms"], "rel_residual": rh["stats"].rel_residual,
            "e2e": {"value": rh["e2e"], "unit": "unknowns/s", "h2d_bytes_per_step": n_in * n * 8,
                    "d2h_bytes_per_step": n * 8},
            "gpu_launches": args.steps * (rh["stats"].kernel_launches + rh["stats"].setup_kernel_launches),
            "roofline": roof, "cpu_baseline": cpu, "clocks": rh["clocks"],
        }
        vc = {}
        for prec in precisions:
            bpn, fpn = cycle_model(prec, smoother, nu, five=res[prec]["five_point"])
            nodes = g.nx * g.nyr
            t = res[prec]["cycle_ms"] * 1e-3
            ent = {"ms": 1e3 * t, "bytes_per_cycle": bpn * nodes, "achieved_gbs": bpn * nodes / t / 1e9,
                   "frac_hbm": bpn * nodes / t / 1e9 / HBM_PEAK_GBS, "bytes_per_fine_node": bpn}
            if prec == "fp64":  # the FP64 cycle is bound by the FP64 pipe, not HBM
                ent["achieved_tflops"] = fpn * nodes / t / 1e12
                ent["frac_fp64"] = ent["achieved_tflops"] / fp64_peak(mg, torch)["tflops"]
            vc[prec] = ent
        line["vcycle"] = dict(vc, model="algorithmic bytes per fine node and cycle (coarse levels x 4/3), "
                                        "see cycle_model; measured by mg_cycle_time (graph replay, warm)")
        if gridgen:
            line["grid_generation"] = gridgen
        line["autotune"] = tuned
        if "fp64" in precisions:
            line["fp64_peak"] = fp64_peak(mg, torch)
        for o in others:
            ro = res[o]
            line[o] = {"value": ws * U * args.steps / ro["tot"], "ms_per_step": 1e3 * ro["tot"] / args.steps,
                       "iters": ro["stats"].iters, "e2e": ro["e2e"], "solve_ms": ro["solve_ms"],
                       "setup_ms": ro["setup_ms"], "rel_residual": ro["stats"].rel_residual,
                       "gpu_launches": args.steps * (ro["stats"].kernel_launches
                                                     + ro["stats"].setup_kernel_launches)}
        print(json.dumps(line))
    ctx.close()
    return 0


# ------------------------------------------------------------------ batched workload
BATCH_COUNT = 512
BATCH_RTOL = 1e-9  # oracle check on the largest-ratio instances of each size: error <= 1e-10


def _d64(torch, a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def run_batch(args):
    """512 independent inclusion instances (sides uniform over {65,129,257,513}, radius
    U[0.1,0.35], eps' ratio U[1,50], 16 blobs each).  One step = the coefficient build and
    hierarchy of every instance (one mg_batch_update_transform) + one mg_batch_solve of all 512 (one
    graph launch).  Reported for the mixed path (headline), the FP64 path, and the plain FP64
    solver run instance by instance (mg_update_transform + mg_solve per instance)."""
    ws, rank, local = dist_env()
    specs = I.config4_specs(BATCH_COUNT, seed0=4000 + BATCH_COUNT * rank)
    I.prefetch_inclusion_grids([(n, r) for n, r, _, _ in specs])  # spawn pool, before CUDA
    import torch
    from paper_2602_01888_gb300 import mg

    dist = dist_init(ws)
    torch.cuda.set_device(local)
    mg.lib()
    smoother, nu = smoother_of(args)
    insts = [I.inclusion_instance(n, r, e, sd) for n, r, e, sd in specs]
    U = sum(x.grid.unknowns for x in insts)
    nodes = sum(x.grid.nx * x.grid.nyr for x in insts)
    ctx = mg.Context(local)
    ctx.use_torch_stream()
    tuned = autotune(mg, ctx, 513, not args.no_autotune)
    dev = [dict(xp=_d64(torch, x.map.xp), yp=_d64(torch, x.map.yp), eps=_d64(torch, x.eps_phys),
                rho=_d64(torch, x.rho_phys), phi=torch.zeros(x.grid.shape, dtype=torch.float64, device="cuda"))
           for x in insts]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    res = {}
    for prec in ("mixed", "fp64"):
        opts = mg.make_opts(prec, "fcg", rtol=BATCH_RTOL, max_iters=400, smoother=smoother, nu1=nu[0], nu2=nu[1])
        probs = [mg.Problem(ctx, x, opts, device_inputs=True) for x in insts]
        hs = [p.h for p in probs]
        rhos = [d["rho"] for d in dev]
        phis = [d["phi"] for d in dev]

        maps = [x.map for x in insts]
        eps_l, xp_l, yp_l = ([d[k] for d in dev] for k in ("eps", "xp", "yp"))

        def setup_all():
            mg.mg_batch_update_transform(ctx.h, hs, maps, eps_l, xp_l, yp_l)

        def step():
            setup_all()
            return mg.mg_batch_solve(ctx.h, hs, rhos, None, phis, opts)

        for _ in range(args.warmup):
            stats = step()
        torch.cuda.synchronize()
        barrier(dist)
        sampler = ClockSampler(local) if (prec == "mixed" and rank == 0) else None
        if sampler:
            sampler.start()
        times, solve_t = [], []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            torch.cuda.synchronize()
            e0.record()
            setup_all()
            e1.record()
            stats = mg.mg_batch_solve(ctx.h, hs, rhos, None, phis, opts)
            e2.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e2) * 1e-3)
            solve_t.append(e1.elapsed_time(e2) * 1e-3)
        clocks = sampler.stop() if sampler else None
        tot = allmax(dist, float(sum(times)))
        r = {"tot": tot, "solve": allmax(dist, float(sum(solve_t))), "clocks": clocks,
             "iters": [s.iters for s in stats], "rel": max(s.rel_residual for s in stats),
             "launches": sum(s.kernel_launches + s.setup_kernel_launches for s in stats)}
        # the plain solver, one instance after another (same resident problems)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for p, x, d in zip(probs, insts, dev):
            mg.mg_update_transform(p.h, x.grid, x.map, d["eps"], d["xp"], d["yp"])
            mg.mg_solve(p.h, d["rho"], None, d["phi"], opts)
        e1.record()
        torch.cuda.synchronize()
        r["sequential_s"] = allmax(dist, e0.elapsed_time(e1) * 1e-3)
        if prec == "mixed":
            # end to end with host buffers: inputs read from pinned host memory, results written back
            pin = lambda a: None if a is None else \
                torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory().numpy()
            host = [dict(xp=pin(x.map.xp), yp=pin(x.map.yp), eps=pin(x.eps_phys), rho=pin(x.rho_phys),
                         phi=torch.zeros(x.grid.shape, dtype=torch.float64).pin_memory().numpy())
                    for x in insts]
            e2e_steps = max(1, min(args.steps, 3))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                mg.mg_batch_update_transform(ctx.h, hs, maps, [h["eps"] for h in host],
                                             [h["xp"] for h in host], [h["yp"] for h in host])
                mg.mg_batch_solve(ctx.h, hs, [h["rho"] for h in host], None, [h["phi"] for h in host], opts)
            r["e2e"] = ws * U * e2e_steps / allmax(dist, time.perf_counter() - t0)
            del host
        res[prec] = r
        for p in probs:
            p.close()
    del flush
    roof = None
    if rank == 0:
        big = max(insts, key=lambda x: x.grid.nx)
        roof = measure_smoother(mg, torch, big, "mixed")
        roof["note"] = f"k_gs_colour<float> on one {big.grid.nx}^2 instance (L2-resident at this size)"
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle as O
        O.build()
        sample = [x for x in insts if x.grid.nx == 257][:2]
        t = 0.0
        for x in sample:
            dt, _ = oracle_solve_seconds(x, BATCH_RTOL)
            t += dt
        cpu = {"value": sum(x.grid.unknowns for x in sample) / t, "unit": "unknowns/s", "cores": 1,
               "kind": "oracle", "sample": f"{len(sample)} of the 257^2 instances solved one by one "
                                           f"(coefficients + MG-preconditioned CG to rtol {BATCH_RTOL}), 1 thread"}
    if rank == 0:
        rm, rf = res["mixed"], res["fp64"]
        line = {
            "metric": METRIC, "value": ws * U * args.steps / rm["tot"], "unit": "unknowns/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * rm["tot"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 cycle in f64 refinement", "data": "synthetic",
            "config": {"workload": "batch512", "instances": BATCH_COUNT, "sides": [65, 129, 257, 513],
                       "precision": "mixed", "outer": f"fcg+vcycle({nu[0]},{nu[1]})", "smoother": smoother,
                       "rtol": BATCH_RTOL, "unknowns": U,
                       "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"{BATCH_COUNT} instances per GPU x{ws}" if ws > 1 else "1 GPU"},
            "solve_ms": 1e3 * rm["solve"] / args.steps,
            "iters": {"min": min(rm["iters"]), "max": max(rm["iters"]), "mean": float(np.mean(rm["iters"]))},
            "rel_residual_max": rm["rel"],
            "fp64_batched": {"value": ws * U * args.steps / rf["tot"], "ms_per_step": 1e3 * rf["tot"] / args.steps,
                             "solve_ms": 1e3 * rf["solve"] / args.steps, "iters_max": max(rf["iters"])},
            "fp64_sequential": {"value": ws * U / rf["sequential_s"], "ms_per_step": 1e3 * rf["sequential_s"]},
            "mixed_sequential": {"value": ws * U / rm["sequential_s"], "ms_per_step": 1e3 * rm["sequential_s"]},
            "e2e": {"value": rm["e2e"], "unit": "unknowns/s", "h2d_bytes_per_step": 4 * 8 * nodes,
                    "d2h_bytes_per_step": 8 * nodes},
            "gpu_launches": args.steps * rm["launches"],
            "roofline": roof, "cpu_baseline": cpu, "clocks": rm["clocks"], "autotune": tuned,
        }
        print(json.dumps(line))
    ctx.close()
    return 0


# ------------------------------------------------------------------ serving workload
SERVE_RTOL = 1e-9


def _blobs_device(torch, xp, yp, seed, count=16, sigma=0.02):
    """The 16-blob source of the inclusion recipe (centres U[0,1]^2, amplitudes U[-1,1],
    sigma 0.02; parameters drawn by numpy from the seed) evaluated on the device."""
    rng = np.random.default_rng(seed)
    cx, cy, amp = rng.uniform(0.0, 1.0, count), rng.uniform(0.0, 1.0, count), rng.uniform(-1.0, 1.0, count)
    rho = torch.zeros_like(xp)
    for k in range(count):
        rho += float(amp[k]) * torch.exp(-((xp - float(cx[k])) ** 2 + (yp - float(cy[k])) ** 2) /
                                         (2 * sigma * sigma))
    return rho


def serve_inputs(mg, torch, ctx, stream, sources=2):
    """Host inputs of every distinct (side, inclusion ring) of a request stream: the mapped
    grid generated on the GPU by the library's harmonic grid generator (Sec. 4.2, Eq. 44
    data on the ring, mg_harmonic_grid to rtol 1e-13) and `sources` seeded 16-blob sources
    per grid.  Returns ({(n, i0): (xp, yp, [rho, ...])}, seconds spent)."""
    t0 = time.perf_counter()
    out = {}
    for n, i0 in sorted({(n, I.snap_ring(n, r)) for _, n, r, _, _ in stream}, key=lambda k: -k[0]):
        ring, xp0, yp0 = I.inclusion_ring_data(n, i0)
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        fx, xi, yi = d(ring.astype(np.uint8)), d(xp0), d(yp0)
        xo, yo = torch.empty_like(xi), torch.empty_like(yi)
        mg.mg_harmonic_grid(ctx.h, I.Grid(n, n), fx, xi, yi, xo, yo, rtol=1e-13)
        srcs = [_blobs_device(torch, xo, yo, 1009 * n + 7919 * v + i0).cpu().numpy() for v in range(sources)]
        out[(n, i0)] = (xo.cpu().numpy(), yo.cpu().numpy(), srcs)
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def _serve_requests(stream, inputs):
    """(arrival, grid, map, rho, eps key, unknowns) per request."""
    out = []
    for q, (t, n, r, ratio, seed) in enumerate(stream):
        i0 = I.snap_ring(n, r)
        xp, yp, srcs = inputs[(n, i0)]
        out.append((t, I.Grid(n, n), I.MapSpec("grid", (), xp, yp), srcs[seed % len(srcs)], (n, i0, ratio),
                    (n - 2) ** 2))
    return out


def _serve_pass(mg, ctx, reqs, arrivals, inflight, mem_budget):
    """Submit reqs at the given arrival offsets (None: all at once), collect every result,
    return the server's report and the client-side wall time."""
    import collections
    srv = mg.mg_server_start(ctx.h, max_inflight=inflight, mem_budget=mem_budget)
    tickets = collections.deque()
    unconverged = []

    def collect(item):
        tk, k = item
        st, stats = mg.mg_serve_poll(srv, tk, 600_000, None)
        if st == mg.MG_ERR_NOT_CONVERGED:
            # best iterate returned; counted in the report with the request and its residual
            unconverged.append((k, stats.iters, stats.rel_residual))
        elif st:
            raise RuntimeError(f"mg_serve_poll: status {st}: {mg.mg_last_error()}")

    eps_cache = {}
    opts = mg.make_opts("mixed", "fcg", rtol=SERVE_RTOL, max_iters=400)
    t0 = time.perf_counter()
    for k, (_, grid, mp, rho, epsk, _) in enumerate(reqs):
        if arrivals is not None:
            dt = arrivals[k] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
        eps = eps_cache.get(epsk)
        if eps is None:
            eps = I.inclusion_eps(epsk[0], epsk[1], epsk[2])
            if len(eps_cache) < 64:
                eps_cache[epsk] = eps
        while True:
            st, tk = mg.mg_serve_submit(srv, grid, mp, rho, eps_phys=eps, opts=opts)
            if st != mg.MG_ERR_BUSY or not tickets:
                break
            collect(tickets.popleft())  # staging full: take the oldest result first
        if st:
            raise RuntimeError(f"mg_serve_submit: status {st}: {mg.mg_last_error()}")
        tickets.append((tk, k))
        while len(tickets) > 4 * inflight:  # keep the host staging bounded
            collect(tickets.popleft())
    while tickets:
        collect(tickets.popleft())
    wall = time.perf_counter() - t0
    rep = mg.mg_server_stop(srv)
    rep.not_converged = len(unconverged)
    rep.unconverged = unconverged
    return rep, wall


def _plain_fp64(mg, ctx, reqs):
    """The plain FP64 GPU solver on the same requests, one after another through the public
    API with host arrays: a resident problem per grid shape, mg_update_transform + mg_solve
    (FP64 flexible CG, the serving rtol) per request.  Returns unknowns/s."""
    opts = mg.make_opts("fp64", "fcg", rtol=SERVE_RTOL, max_iters=400)
    probs = {}
    U = 0
    t0 = time.perf_counter()
    for _, grid, mp, rho, epsk, u in reqs:
        h = probs.get(grid.nx)
        eps = I.inclusion_eps(epsk[0], epsk[1], epsk[2])
        if h is None:
            h = probs[grid.nx] = mg.mg_setup_transform(ctx.h, grid, mp, eps, opts)
        else:
            mg.mg_update_transform(h, grid, mp, eps)
        phi = np.zeros(grid.shape)
        mg.mg_solve(h, np.ascontiguousarray(rho), None, phi, opts, True)
        U += u
    wall = time.perf_counter() - t0
    for h in probs.values():
        mg.mg_problem_free(h)
    return U / wall


def run_serve(args):
    """Poisson-arrival request stream (sides log-uniform in [129, 2049] snapped to m 2^k + 1,
    inclusion radius drawn U[0.1, 0.35] per request and snapped so the ring lies on grid
    lines, eps' ratio U[1,50]), solved by the library's request server.  The mapped grids are
    generated by the library on the GPU before the timed passes.  First a saturation pass
    (requests submitted as fast as the server takes them) measures throughput; then
    open-loop passes at fractions of that rate measure p50/p99 submit-to-result latency; the
    plain FP64 solver runs a sample of the same requests one by one for comparison."""
    ws, rank, local = dist_env()
    count = args.requests
    stream = I.config5_stream(count, seed=5 + 1000 * rank, rate=1.0, side_range=(129, args.serve_max_side))
    warm_stream = I.config5_stream(min(64, count), seed=99, rate=1.0, side_range=(129, 513))
    import torch
    from paper_2602_01888_gb300 import mg

    dist = dist_init(ws)
    torch.cuda.set_device(local)
    mg.lib()
    ctx = mg.Context(local)
    tuned = autotune(mg, ctx, args.serve_max_side, not args.no_autotune)
    inputs, gen_s = serve_inputs(mg, torch, ctx, stream + warm_stream)
    reqs = _serve_requests(stream, inputs)
    U = sum(q[5] for q in reqs)
    warm = _serve_requests(warm_stream, inputs)
    _serve_pass(mg, ctx, warm, None, args.inflight, 0)
    barrier(dist)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    rep, wall = _serve_pass(mg, ctx, reqs, None, args.inflight, 0)
    clocks = sampler.stop() if sampler else None
    wall = allmax(dist, wall)
    sat_rps = count / wall
    lat = []
    base = np.array([q[0] for q in stream])
    for frac in args.serve_loads:
        rate = frac * sat_rps
        arr = base / rate  # the same exponential gaps rescaled to the target rate
        r2, w2 = _serve_pass(mg, ctx, reqs, arr, args.inflight, 0)
        lat.append({"load": frac, "rate_rps": rate, "p50_ms": r2.p50_ms, "p99_ms": r2.p99_ms,
                    "max_ms": r2.max_ms, "unknowns_per_s": U / w2, "completed": r2.completed,
                    "failed": r2.failed, "not_converged": r2.not_converged,
                    "mean_inflight": r2.mean_batch, "reused": r2.reused,
                    "evicted": r2.evicted})
    sample = reqs[: min(len(reqs), args.plain_sample)]
    plain = _plain_fp64(mg, ctx, sample)
    if rank == 0:
        bytes_in = sum(8 * q[1].nx * q[1].nyr * 4 for q in reqs)
        bytes_out = sum(8 * q[1].nx * q[1].nyr for q in reqs)
        line = {
            "metric": METRIC, "value": ws * U / wall, "unit": "unknowns/s", "n_gpus": ws, "steps": 1,
            "warmup": 1, "ms_per_step": 1e3 * wall, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 cycle in f64 refinement", "data": "synthetic",
            "config": {"workload": "serve", "requests": count,
                       "sides": f"log-uniform [129,{args.serve_max_side}] snapped to m*2^k+1",
                       "radius": "U[0.1,0.35] per request, snapped so the ring lies on grid lines",
                       "distinct_grids": len(inputs), "rtol": SERVE_RTOL, "inflight_slots": args.inflight,
                       "unknowns": U, "l2": "inputs of consecutive requests exceed L2 in aggregate"},
            "saturated": {"requests_per_s": sat_rps, "p50_ms": rep.p50_ms, "p99_ms": rep.p99_ms,
                          "completed": rep.completed, "failed": rep.failed,
                          "not_converged": rep.not_converged, "mean_inflight": rep.mean_batch,
                          "reused": rep.reused, "evicted": rep.evicted,
                          "not_converged_requests": [
                              {"index": k, "side": stream[k][1], "radius": stream[k][2], "ratio": stream[k][3],
                               "seed": stream[k][4], "iters": it, "rel_residual": rr}
                              for k, it, rr in rep.unconverged]},
            "latency": lat,
            "fp64_plain": {"value": plain, "requests": len(sample),
                           "how": "mg_update_transform + mg_solve per request, FP64, hierarchy per grid shape"},
            "grid_generation_s": gen_s,
            "e2e": {"value": ws * U / wall, "unit": "unknowns/s", "h2d_bytes_per_step": bytes_in,
                    "d2h_bytes_per_step": bytes_out},
            "gpu_launches": None, "roofline": None, "cpu_baseline": None, "clocks": clocks,
            "autotune": tuned,
        }
        print(json.dumps(line))
    ctx.close()
    return 0


# ------------------------------------------------------------------ SOR baseline
SOR_CASES = (("sine_warp_129", lambda: I.config1(129)), ("circle_poisson_257", lambda: I.circle_poisson(257)),
             ("inclusion_257", lambda: I.inclusion_instance(257, 0.25, 10.0, 2)))
SOR_OMEGA, SOR_RTOL = 1.875, 1e-10


def run_sor(args):
    """The paper's comparison (Sec. 4): the single-level SOR iteration (omega 1.875) against
    multigrid on the same problems and to the same residual tolerance, here both on the GPU
    (four-colour SOR, MG_OUTER_SOR, 16 sweeps per residual test; FP64 FCG + V(2,2)) and both
    in the CPU oracle (one thread).  Reports solve times (hierarchy resident, inputs on the
    device) and their ratio per problem."""
    import torch
    from paper_2602_01888_gb300 import mg
    import oracle as O
    torch.cuda.set_device(0)
    ctx = mg.Context(0)
    ctx.use_torch_stream()
    rows = []
    for name, build in SOR_CASES:
        inst = build()
        rho = torch.from_numpy(np.ascontiguousarray(inst.rho_phys)).cuda()
        bc = None if inst.bc is None else torch.from_numpy(np.ascontiguousarray(inst.bc)).cuda()
        phi = torch.zeros(inst.grid.shape, dtype=torch.float64, device="cuda")
        so = mg.make_opts("fp64", "sor", rtol=SOR_RTOL, max_iters=200000, nu1=16, omega_j=SOR_OMEGA)
        go = mg.make_opts("fp64", "fcg", rtol=SOR_RTOL, max_iters=400)
        pr = mg.Problem(ctx, inst, go, device_inputs=True)
        res = {}
        for tag, o in (("gmg", go), ("sor", so)):
            for _ in range(args.warmup if tag == "gmg" else 1):
                mg.mg_solve(pr.h, rho, bc, phi, o)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = args.steps if tag == "gmg" else 1
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                st = mg.mg_solve(pr.h, rho, bc, phi, o)
            e1.record()
            torch.cuda.synchronize()
            res[tag] = (e0.elapsed_time(e1) / reps, st.iters, st.rel_residual)
        pr.close()
        P = O.prepare(inst)
        t0 = time.perf_counter()
        _, sw_cpu, _ = O.sor_solve(P.A, P.b, P.phi0, omega=SOR_OMEGA, rtol=SOR_RTOL, max_sweeps=400000, check=16)
        t_sor_cpu = time.perf_counter() - t0
        t0 = time.perf_counter()
        _, it_cpu, _ = O.pcg_solve(P.A, P.b, P.phi0, rtol=SOR_RTOL, max_iters=400)
        t_gmg_cpu = time.perf_counter() - t0
        rows.append({"problem": name, "unknowns": inst.grid.unknowns,
                     "gpu": {"sor_ms": res["sor"][0], "sor_sweeps": 16 * res["sor"][1], "gmg_ms": res["gmg"][0],
                             "gmg_iters": res["gmg"][1], "sor_over_gmg": res["sor"][0] / res["gmg"][0]},
                     "cpu_oracle_1_thread": {"sor_ms": 1e3 * t_sor_cpu, "sor_sweeps": sw_cpu,
                                             "gmg_ms": 1e3 * t_gmg_cpu, "gmg_iters": it_cpu,
                                             "sor_over_gmg": t_sor_cpu / t_gmg_cpu}})
    ctx.close()
    print(json.dumps({"metric": "solve time of SOR (omega 1.875) over multigrid, same residual tolerance",
                      "rtol": SOR_RTOL, "dtype": "f64", "data": "synthetic", "cases": rows}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="annulus_8193",
                    choices=sorted(WORKLOADS) + ["batch512", "serve", "sor_vs_gmg"])
    ap.add_argument("--requests", type=int, default=20000, help="serve: requests per pass")
    ap.add_argument("--plain-sample", type=int, default=500,
                    help="serve: requests solved one by one by the plain FP64 solver for comparison")
    ap.add_argument("--inflight", type=int, default=16, help="serve: concurrent request slots")
    ap.add_argument("--serve-max-side", type=int, default=2049, help="serve: largest grid side")
    ap.add_argument("--serve-loads", type=float, nargs="*", default=[0.5, 0.8, 0.95],
                    help="serve: open-loop arrival rates as fractions of the saturated rate")
    ap.add_argument("--smoother", default=None, choices=["gs4", "xline"],
                    help="four-colour point Gauss-Seidel, or zebra x-line Gauss-Seidel (default per workload)")
    ap.add_argument("--nu", type=lambda v: tuple(int(t) for t in v.split(",")), default=None,
                    help="pre,post smoothing sweeps of the V-cycle (default per workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-cores", type=int, default=0,
                    help="reference arm: host cores running the oracle at once (default: all)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the size-threshold smoother choice instead of timing the families")
    ap.add_argument("--kernel-only", dest="kernel", default=None,
                    help="smooth64|smooth32|fused64|fused32|pipe64|pipe32|march32|march32p|march64|march64p|"
                         "line64|line32|"
                         "restrict64|restrict32|restricte64|restricte32|prolong64|prolong32|fp64peak|fp32peak")
    ap.add_argument("--side", type=int, default=2049)
    ap.add_argument("--ny", type=int, default=0, help="kernel-only: rows (default: --side)")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--coarse-op", dest="coarse_op", default="galerkin", choices=["galerkin", "rediscretize"],
                    help="coarse operators of the single-instance workloads: Galerkin products or the "
                         "assembly on each coarse grid from the coarsened tensor")
    ap.add_argument("--stencil", type=int, default=9, choices=(5, 9),
                    help="kernel-only: 9 = sine-warp operator, 5 = a map without cross term (5-point kernels)")
    ap.add_argument("--variant", type=int, default=-1,
                    help="kernel-only march/pipe/fused: the autotuner's variant index (default: the family's default)")
    args = ap.parse_args()
    if args.kernel:
        return run_kernel_only(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch512":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "sor_vs_gmg":
        return run_sor(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
