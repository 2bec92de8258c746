"""Host-side arithmetic of the benchmark's figures (CPU): the algorithmic bytes per fine node
of one multigrid cycle behind the V-cycle bandwidth, the per-workload smoother defaults,
and the profiled-traffic table the roofline lines read."""
import argparse
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_point_cycle_bytes_match_the_three_pass_count():
    """V(2,2) with two sweeps per pass: pre-smoothing pass, residual + restriction pass,
    post-smoothing pass with the coarse correction; each pass reads the five operator arrays
    (C = 5 elements per node); vectors 3 + 2.25 + 3.25 elements: 68 + 3C bytes at FP64 =
    188 B, 94 B at FP32, times 4/3 for the coarser levels."""
    b64, f64 = bench.cycle_model("fp64", "gs4", (2, 2))
    b32, f32 = bench.cycle_model("mixed", "gs4", (2, 2))
    assert b64 == pytest.approx(188.0 * 4 / 3)
    assert b32 == pytest.approx(94.0 * 4 / 3)
    assert f64 == f32 == pytest.approx((4 * 18 + 18 + 8) * 4 / 3)
    # three sweeps a side take two passes a side
    b33, _ = bench.cycle_model("fp64", "gs4", (3, 3))
    assert b33 == pytest.approx((5 * 5 * 8 + 2 * 3 * 8 + 2.25 * 8 + 2 * 3 * 8 + 0.25 * 8) * 4 / 3)


def test_line_cycle_bytes():
    """x-line V(1,1): two sweeps of 14 elements, the even-row residual + restriction pass
    (5.5 + 0.25: x of all rows, b, diag and cE of the even rows, cN, cNE and cNW of all rows)
    and the prolongation pass (2.25): 144 B per fine node at FP32; 5-point finest level:
    two sweeps of 10, 3.5 + 0.25 and 2.25: 104 B.  Without pre-smoothing the residual pass
    reads everything (7.25, 5.25)."""
    b, f = bench.cycle_model("mixed", "xline", (1, 1))
    assert b == pytest.approx(144.0 * 4 / 3)
    assert f == pytest.approx((2 * 24 + 9 + 8) * 4 / 3)
    b64, _ = bench.cycle_model("fp64", "xline", (1, 1))
    assert b64 == pytest.approx(2 * b)
    b5, f5 = bench.cycle_model("mixed", "xline", (1, 1), five=True)
    assert b5 == pytest.approx(104.0 * 4 / 3)
    assert f5 == pytest.approx((2 * 16 + 5 + 8) * 4 / 3)
    b01, _ = bench.cycle_model("mixed", "xline", (0, 1))
    assert b01 == pytest.approx((56 + 29 + 9) * 4 / 3)
    b015, _ = bench.cycle_model("mixed", "xline", (0, 1), five=True)
    assert b015 == pytest.approx((40 + 21 + 9) * 4 / 3)


def _args(workload, smoother=None, nu=None):
    return argparse.Namespace(workload=workload, smoother=smoother, nu=nu)


def test_smoother_defaults_per_workload():
    assert bench.smoother_of(_args("annulus_8193")) == ("xline", (1, 1))
    assert bench.smoother_of(_args("inclusion_1025")) == ("gs4", (2, 2))
    assert bench.smoother_of(_args("batch512")) == ("gs4", (2, 2))
    assert bench.smoother_of(_args("annulus_8193", "gs4", (2, 2))) == ("gs4", (2, 2))
    assert bench.smoother_of(_args("inclusion_1025", None, (2, 1))) == ("gs4", (2, 1))


def test_profiled_traffic_against_the_algorithmic_bytes():
    """Every recorded per-launch DRAM figure (profiles/dram_traffic.json) belongs to a kernel
    the roofline line can name, names its capture command, and lies in the band its capture
    documented: the per-colour kernels re-read most rows of the operator in each of a sweep's
    four launches (2-3.5x their share of a sweep's bytes); the marching and line kernels move
    their algorithmic bytes (0.9-1.2x).  Scaling to another level size goes by node count."""
    band = {"k_gs_colour<double>": (2.0, 3.5), "k_gs_colour<float>": (2.0, 3.5),
            "k_smooth_march<float> w240/2": (0.9, 1.2), "k_line_zebra<float>": (0.9, 1.2),
            "k_line_zebra<float> 5-point": (0.9, 1.2)}
    entries = bench._traffic_table()
    assert entries
    for e in entries:
        kern = e["kernel"]
        assert kern in band, kern
        assert e["command"].startswith("ncu ") and "--clock-control none" in e["command"]
        assert os.path.exists(os.path.join(ROOT, "profiles", e["summary"]))
        nx, rows = e["captured"]
        nodes = float(nx) * rows
        traffic = bench.profiled_traffic(kern, nx, rows)
        algo = {"k_gs_colour<double>": 64.0 * nodes / 4,       # a sweep's 8 FP64 arrays over 4 launches
                "k_gs_colour<float>": 32.0 * nodes / 4,
                "k_smooth_march<float> w240/2": 32.0 * nodes,  # two sweeps, each array once
                "k_line_zebra<float>": 14 * 4.0 * nodes / 2,
                "k_line_zebra<float> 5-point": 10 * 4.0 * nodes / 2}[kern]
        lo, hi = band[kern]
        assert lo <= traffic / algo <= hi, (kern, traffic / algo)
        assert bench.profiled_traffic(kern, 2 * nx, rows) == pytest.approx(2 * traffic)
    assert bench.profiled_traffic("k_not_captured", 1025, 1025) is None


def test_hbm_peak_comes_from_the_measured_file_or_the_fallback():
    peak, src = bench._hbm_peak()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        import json
        assert peak == json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
        assert "of measured" in src
    else:
        assert peak == 6800.0 and "of fallback" in src
