"""The roofline bookkeeping of bench.py (CPU): achieved = the library's algorithmic flop over the
CUDA-event time of the stage-2 launches, frac = achieved / peak, and the DRAM traffic of a captured
launch (profiles/stage2_traffic.txt) scaled by flop to the run's average launch."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _capture(prefix):
    vals = {}
    with open(os.path.join(ROOT, "profiles", "stage2_traffic.txt")) as f:
        for ln in f:
            if ln.startswith(prefix) and "=" in ln:
                k, v = ln.strip().split("=", 1)
                vals[k[len(prefix):]] = float(v)
    return vals


# two calls of 14 and 7 launches: 21 launches, 4.2e12 flop in 210 ms of stage-2 time
STATS = [{"stage2_ms": 140.0, "stage2_launches": 14, "stage2_flops": 2.8e12},
         {"stage2_ms": 70.0, "stage2_launches": 7, "stage2_flops": 1.4e12}]


def test_grid_dft_roofline_and_scaled_traffic():
    import bench
    r = bench.roofline(7, STATS, 0)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(4.2e12 / 0.210 / 1e12)
    assert r["peak"] == pytest.approx(148 * 128 * 2 * 2.032e9 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["algorithmic_flops_per_launch"] == pytest.approx(4.2e12 / 21)
    assert r["avg_launch_ms"] == pytest.approx(10.0)
    cap = _capture("dft_capture_")
    assert r["traffic"] == pytest.approx(cap["bytes"] * (4.2e12 / 21) / cap["flops"])
    # a profiling case (a k subset) reports no traffic: the capture is of the whole-plane batches
    assert bench.roofline(7, STATS, 600)["traffic"] is None


@pytest.mark.parametrize("prec,split,ratio", [(5, 3, 1.0), (1, 6, 1.0), (2, 3, 0.5)])
def test_tensor_core_roofline_against_the_sustained_peak(prec, split, ratio):
    import bench
    peaks, _ = bench._peaks()
    r = bench.roofline(prec, STATS, 0)
    peak = peaks.get("bf16_tflops_sustained", 1400.0) * ratio
    assert r["bound"] == "tensor" and r["peak"] == pytest.approx(peak)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    kpad = (-(-2 * 429 // 64) * 64) / (2 * 429)
    assert r["issued_frac"] == pytest.approx(r["achieved"] * split * kpad / peak)
    if prec == 5:
        cap = _capture("tc_capture_")
        assert r["traffic"] == pytest.approx(cap["bytes"] * (4.2e12 / 21) / cap["flops"])
    else:
        assert r["traffic"] is None


def test_fp64_paths_against_the_nominal_fp64_rate():
    import bench
    for prec in (0, 8):
        r = bench.roofline(prec, STATS, 0)
        assert r["peak"] == 1.25 and r["frac"] == pytest.approx(r["achieved"] / 1.25)
