"""Host-side logic of bench.py that needs no GPU: the roofline object built from
per-class timer totals, the clock summary built from nvidia-smi samples, and
the all-core oracle leg of the CPU baseline."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_roofline_of_a_stored_cost_pass():
    # row_lse dominates: 100 launches of 30 us over a 4096 x 4096 FP32 matrix
    prof = {"row_lse": (3.0, 100), "col_lse": (2.0, 100), "cg": (1.0, 10)}
    roof, dom = bench.roofline(prof, 4096, 4096, 4, cg_iters=500, nnz=8191,
                               peaks={"hbm_gbs": 6800.0}, streamed=False)
    assert dom == "row_lse"
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    want = 4096 * 4096 * 4 / 30e-6 / 1e9
    assert roof["achieved"] == pytest.approx(want, rel=1e-12)
    assert roof["frac"] == pytest.approx(want / 6800.0, rel=1e-12)
    assert roof["peak_source"] == "measured"
    assert roof["avg_launch_us"] == pytest.approx(30.0)


def test_roofline_falls_back_without_measured_peaks():
    roof, _ = bench.roofline({"trial": (1.0, 10)}, 64, 64, 8, 0, 0, peaks={}, streamed=False)
    assert roof["peak"] == 6800.0 and roof["peak_source"] == "fallback"


def test_roofline_of_a_streamed_cost_pass_counts_entries_against_the_ex2_rate():
    # grid cost: 20 launches of 10 us over 4096 x 4096 generated entries
    roof, dom = bench.roofline({"row_lse": (0.2, 20), "cg": (0.1, 5)}, 4096, 4096, 4,
                               cg_iters=0, nnz=0, peaks={"hbm_gbs": 6800.0}, streamed=True)
    assert dom == "row_lse" and roof["bound"] == "alu" and roof["unit"] == "G entries/s"
    want = 4096 * 4096 / 10e-6 / 1e9
    assert roof["achieved"] == pytest.approx(want, rel=1e-12)
    assert roof["peak"] == pytest.approx(152 * 16 * 2.07)
    assert roof["frac"] == pytest.approx(want / (152 * 16 * 2.07), rel=1e-12)


def test_roofline_of_the_cg_counts_the_methods_own_flops():
    """4 nnz + 14 (m + n) per CG iteration (SpMV on both copies, diagonal, three
    inner products, four vector updates) against the FP32 units' rate."""
    m = n = 4096
    nnz, launches, iters_total = 8191, 10, 540
    prof = {"cg": (2.3, launches), "row_lse": (1.0, 100)}
    roof, dom = bench.roofline(prof, m, n, 4, cg_iters=iters_total, nnz=nnz, peaks={},
                               streamed=True)
    assert dom == "cg" and roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    t = 2.3e-3 / launches
    flops = (4.0 * nnz + 14.0 * (m + n)) * (iters_total / launches)
    assert roof["achieved"] == pytest.approx(flops / t / 1e12, rel=1e-12)
    assert roof["peak"] == pytest.approx(bench.FP32_PEAK_TFLOPS)
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"], rel=1e-12)
    assert roof["iters_per_launch"] == pytest.approx(54.0)


def test_roofline_without_launches_is_absent():
    roof, dom = bench.roofline({"cg": (0.0, 0)}, 8, 8, 4, 0, 0, peaks={}, streamed=True)
    assert roof is None and dom == "cg"


def test_certified_counts_only_ok_results_within_the_gap():
    assert bench.certified({"status": 0, "rel_gap": 9e-7})
    assert not bench.certified({"status": 0, "rel_gap": 2e-6})
    assert not bench.certified({"status": 3, "rel_gap": 1e-7})


def test_one_request_per_grid_size():
    sub = bench.one_per_size(1e-3)
    assert [w.grid[0] for w in sub] == [16, 28, 32, 48, 64]


def test_clock_summary_takes_the_median_and_the_active_reasons():
    cs = bench.ClockSampler()
    cs.samples = [
        ["2070", "2070", "900.1", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["1980", "2070", "1400.0", "Not Active", "Not Active", "Not Active", "Active"],
        ["2070", "2070", "1200.5", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["[N/A]", "2070", "1200.5", "Not Active", "Not Active", "Not Active", "Not Active"],
    ]
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 4


def test_clock_summary_without_samples_says_so():
    assert bench.ClockSampler().summary()["reasons"] == ["unsampled"]


def test_all_core_oracle_leg_runs_full_certified_solves():
    """The all-core CPU baseline: one oracle solve per core at a time in a
    spawn-started pool; every solve reaches the certified gap."""
    saved = sys.argv
    sys.argv = ["bench.py"]
    try:
        args = bench.parse()
    finally:
        sys.argv = saved
    done, dt, gmax = bench.oracle_sample_cores(args, 0.0, 2)
    assert done == 2 and dt > 0.0
    assert gmax <= bench.TOL_GAP
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()
