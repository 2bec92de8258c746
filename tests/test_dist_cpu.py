"""The benchmark's multi-rank plumbing on CPU with two gloo ranks (no GPU): the barrier and
max-over-ranks reduction that bench.py uses under torchrun, and the reference arm launched
by torchrun, where rank 0 alone prints the JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    ws, r, _ = bench.dist_env()
    dist = bench.dist_init(ws)
    v = bench.allmax(dist, 10.0 * (r + 1))
    bench.barrier(dist)
    with open(os.path.join(out, f"r{r}.txt"), "w") as f:
        f.write(repr((ws, r, v)))
    dist.destroy_process_group()


def test_gloo_barrier_and_allmax_two_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    got = sorted(open(tmp_path / f"r{k}.txt").read() for k in range(2))
    assert got == [repr((2, 0, 20.0)), repr((2, 1, 20.0))]


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--workload", "sine_warp_129", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_of_the_batch_workload():
    """The oracle on the batch workload's own instances (a fixed bounded subset per step),
    one JSON line with the arm's metric and unit."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "batch512",
                        "--steps", "1", "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["unit"] == "unknowns/s" and rec["value"] > 0
    assert rec["config"]["workload"] == "batch512" and "8 of the 512" in rec["cpu_baseline"]["sample"]


def test_reference_arm_of_the_default_workload_runs_on_every_requested_core():
    """Default workload (the annulus): the oracle on its 1025^2 sample, one copy per host core
    at once (two here, to bound the test's time); the line states the sample and the cores."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3",
                        "--ref-cores", "2"], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    rec = json.loads(lines[0])
    assert rec["config"]["workload"] == "annulus_8193" and rec["config"]["smoother"] == "xline"
    assert rec["cpu_baseline"]["cores"] == 2 and "1025^2" in rec["cpu_baseline"]["sample"]
    assert rec["e2e"]["value"] == rec["value"] > 0
