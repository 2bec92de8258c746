"""Benchmark: unknowns solved per second to 1e-9 relative error on one GB300.

Workload (default): the 1025^2 unit square with a circular inclusion of radius 0.25
(local boundary-fitted map, Jacobian by central differences of the mapped grid, eps'
ratio 10, 16 seeded Gaussian blobs, phi = 0 on the boundary).  One step is one pass of
the whole hot path on resident inputs: coefficient build + Galerkin hierarchy + coarsest
inverse (mg_update_transform) and the solve to rtol 1e-9 (mg_solve), whose error
against the FP64 oracle is <= 1e-9 (checked by the GPU test suite at these settings).

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the same workload.
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
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12  # 2 FP64 FMA/clk/SM x 152 SMs x 2.07 GHz


def workload(name: str):
    if name == "inclusion_1025":
        return I.config2(1025)
    if name == "sine_warp_129":
        return I.config1(129)
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
def oracle_solve_seconds(inst):
    import oracle as O
    t0 = time.perf_counter()
    P = O.prepare(inst)
    phi, it, hist = O.pcg_solve(P.A, P.b, P.phi0, rtol=RTOL, max_iters=400)
    return time.perf_counter() - t0, it


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    O.build()
    side = 1025 if (args.steps + args.warmup) <= 16 else 513
    inst = workload(args.workload) if side == 1025 else I.inclusion_instance(513, 0.25, 10.0, 2)
    U = inst.grid.unknowns
    for _ in range(args.warmup):
        oracle_solve_seconds(inst)
    tot = 0.0
    for _ in range(args.steps):
        dt, it = oracle_solve_seconds(inst)
        tot += dt
    v = U * args.steps / tot
    sample = (f"full {args.workload} workload per step" if side == 1025 else
              "inclusion recipe at 513^2 per step (1/4 of the unknowns), same rtol")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "unknowns/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "rtol": RTOL},
            "cpu_baseline": {"value": v, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ our arm
def measure_smoother(mg, torch, inst, reps=20):
    """Dominant FP64 kernel timed alone: one four-colour Gauss-Seidel sweep (4 launches)
    on the fine level of this workload, operator built by the library's own kernels."""
    import ctypes as C
    g = inst.grid
    pitch = (g.nx + 31) // 32 * 32
    dev = lambda a=None: (torch.zeros((g.nyr, pitch), dtype=torch.float64, device="cuda") if a is None
                          else torch.nn.functional.pad(torch.from_numpy(np.array(a)).cuda(),
                                                       (0, pitch - g.nx)))
    xp, yp, eps = dev(inst.map.xp), dev(inst.map.yp), dev(inst.eps_phys)
    D, exx, exy, eyy = dev(), dev(), dev(), dev()
    folded = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    mg.mgk("mgk_eps_grid", g.nx, g.ny, 0, g.hx, g.hy, xp.data_ptr(), yp.data_ptr(), 0.0, 0.0,
           eps.data_ptr(), pitch, D.data_ptr(), exx.data_ptr(), exy.data_ptr(), eyy.data_ptr(),
           folded.data_ptr(), s)
    ops = [dev() for _ in range(6)]
    st = mg.op_struct(ops, g.nx, g.ny, False)
    mg.mgk("mgk_assemble", C.byref(st), g.hx, g.hy, exx.data_ptr(), exy.data_ptr(), eyy.data_ptr(), s)
    x = dev()
    b = torch.randn((g.nyr, pitch), dtype=torch.float64, device="cuda")
    for _ in range(3):
        mg.mgk("mgk_smooth_f64", C.byref(st), x.data_ptr(), b.data_ptr(), 1, 0, s)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        mg.mgk("mgk_smooth_f64", C.byref(st), x.data_ptr(), b.data_ptr(), 1, 0, s)
    e1.record()
    torch.cuda.synchronize()
    per_launch_s = e0.elapsed_time(e1) * 1e-3 / (reps * 4)
    flops_per_launch = g.unknowns / 4 * 18.0  # 8 FMA + subtract + scale per updated unknown
    achieved = flops_per_launch / per_launch_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
            "kernel": "k_gs_colour<double>", "launch_us": per_launch_s * 1e6,
            "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2.07 GHz (probe: 1.20 TFLOP/s at 1.99 GHz)"}


def run_kernel_only(args):
    """Run one library kernel `--reps` times on a sine-warp operator of side `--side`
    (built by the library's own kernels) and print its mean CUDA-event time per launch;
    used for profiling a single kernel at a chosen size."""
    import ctypes as C
    import torch
    from paper_2602_01888_gb300 import mg
    torch.cuda.set_device(0)
    n = args.side
    g = I.Grid(n, n)
    pitch = (n + 31) // 32 * 32
    f64 = args.kernel.endswith("64")
    dt = torch.float64 if f64 else torch.float32
    z = lambda d=torch.float64: torch.zeros((g.nyr, pitch), dtype=d, device="cuda")
    D, exx, exy, eyy = z(), z(), z(), z()
    folded = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    prm = (C.c_double * 4)(0.1, 0.0, 0.0, 0.0)
    mg.mgk("mgk_eps_analytic", 1, prm, n, n, 0, 0.0, 0.0, g.hx, g.hy, None, pitch, D.data_ptr(),
           exx.data_ptr(), exy.data_ptr(), eyy.data_ptr(), folded.data_ptr(), s)
    ops = [z() for _ in range(6)]
    st = mg.op_struct(ops, n, n, False)
    mg.mgk("mgk_assemble", C.byref(st), g.hx, g.hy, exx.data_ptr(), exy.data_ptr(), eyy.data_ptr(), s)
    if not f64:
        ops32 = [z(torch.float32) for _ in range(6)]
        st32 = mg.op_struct(ops32, n, n, False, f32=True)
        mg.mgk("mgk_op_to_f32", C.byref(st), C.byref(st32), s)
        st = st32
    x, b = z(dt), torch.randn((g.nyr, pitch), dtype=torch.float64, device="cuda").to(dt)
    x2 = z(dt)
    nc = (n - 1) // 2 + 1
    pc = (nc + 31) // 32 * 32
    bH = torch.zeros((nc, pc), dtype=dt, device="cuda")
    sfx = "f64" if f64 else "f32"

    def once():
        if args.kernel.startswith("pipe"):
            mg.mgk(f"mgk_smooth_pipe_{sfx}", C.byref(st), x.data_ptr(), x2.data_ptr(), b.data_ptr(), 0,
                   None, 0, None, s)
        elif args.kernel.startswith("fused"):
            mg.mgk(f"mgk_smooth_fused_{sfx}", C.byref(st), x.data_ptr(), x2.data_ptr(), b.data_ptr(), 0,
                   None, 0, s)
        elif args.kernel.startswith("smooth"):
            mg.mgk(f"mgk_smooth_{sfx}", C.byref(st), x.data_ptr(), b.data_ptr(), 1, 0, s)
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
    print(json.dumps({"kernel": args.kernel, "side": n, "reps": args.reps,
                      "ms_per_call": e0.elapsed_time(e1) / args.reps}))
    return 0


def run_ours(args):
    import torch
    from paper_2602_01888_gb300 import mg

    ws, rank, local = dist_env()
    dist = dist_init(ws)
    torch.cuda.set_device(local)
    mg.lib()
    inst = workload(args.workload)
    g = inst.grid
    U = g.unknowns
    n = g.nx * g.nyr
    ctx = mg.Context(local)
    ctx.use_torch_stream()
    res = {}
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    dev = lambda a: torch.from_numpy(np.array(a, dtype=np.float64)).cuda()
    xp_d, yp_d, eps_d, rho_d = dev(inst.map.xp), dev(inst.map.yp), dev(inst.eps_phys), dev(inst.rho_phys)
    phi_d = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    for prec in ("fp64", "mixed"):
        opts = mg.make_opts(prec, "fcg", rtol=RTOL, max_iters=400)
        prob = mg.Problem(ctx, inst, opts, device_inputs=True)

        def step():
            mg.mg_update_transform(prob.h, g, inst.map, eps_d, xp_d, yp_d)
            return mg.mg_solve(prob.h, rho_d, None, phi_d, opts)

        for _ in range(args.warmup):
            st = step()
        torch.cuda.synchronize()
        barrier(dist)
        sampler = ClockSampler(local) if (prec == "fp64" and rank == 0) else None
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
        # end to end through the public API with host buffers (pinned)
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory().numpy()
        xp_h, yp_h, eps_h, rho_h = pin(inst.map.xp), pin(inst.map.yp), pin(inst.eps_phys), pin(inst.rho_phys)
        phi_h = torch.zeros(g.shape, dtype=torch.float64).pin_memory().numpy()
        e2e_steps = max(1, min(args.steps, 5))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            mg.mg_update_transform(prob.h, g, inst.map, eps_h, xp_h, yp_h)
            mg.mg_solve(prob.h, rho_h, None, phi_h, opts)
        e2e_t = allmax(dist, time.perf_counter() - t0)
        res[prec] = {"tot": tot, "times": times, "stats": st, "clocks": clocks,
                     "e2e": ws * U * e2e_steps / e2e_t, "levels": len(prob.levels()),
                     "setup_ms": st.setup_ms, "solve_ms": st.solve_ms}
        prob.close()
    roof = measure_smoother(mg, torch, inst) if rank == 0 else None
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle as O
        O.build()
        dt, it = oracle_solve_seconds(inst)
        cpu = {"value": U / dt, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
               "sample": f"one full {args.workload} solve (coefficients + PCG to rtol {RTOL}), 1 thread"}
    if rank == 0:
        r64, rmx = res["fp64"], res["mixed"]
        value = ws * U * args.steps / r64["tot"]
        mixed_value = ws * U * args.steps / rmx["tot"]
        line = {
            "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * r64["tot"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "precision": "fp64", "outer": "fcg+vcycle(2,2)",
                       "rtol": RTOL, "unknowns": U, "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
            "mixed": {"value": mixed_value, "ms_per_step": 1e3 * rmx["tot"] / args.steps,
                      "iters": rmx["stats"].iters, "dtype": "f32 cycle in f64 refinement",
                      "gpu_launches": args.steps * (rmx["stats"].kernel_launches
                                                    + rmx["stats"].setup_kernel_launches),
                      "e2e": rmx["e2e"], "solve_ms": rmx["solve_ms"], "setup_ms": rmx["setup_ms"]},
            "iters": r64["stats"].iters, "levels": r64["levels"],
            "setup_ms": r64["setup_ms"], "solve_ms": r64["solve_ms"],
            "rel_residual": r64["stats"].rel_residual,
            "e2e": {"value": r64["e2e"], "unit": "unknowns/s", "h2d_bytes_per_step": 4 * n * 8,
                    "d2h_bytes_per_step": n * 8},
            "gpu_launches": args.steps * (r64["stats"].kernel_launches + r64["stats"].setup_kernel_launches),
            "roofline": roof, "cpu_baseline": cpu, "clocks": r64["clocks"],
        }
        print(json.dumps(line))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="inclusion_1025", choices=["inclusion_1025", "sine_warp_129"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel-only", dest="kernel", default=None,
                    help="smooth64|smooth32|fused64|fused32|pipe64|pipe32|restrict64|restrict32|prolong64|prolong32")
    ap.add_argument("--side", type=int, default=2049)
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()
    if args.kernel:
        return run_kernel_only(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
