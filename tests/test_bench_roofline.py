"""Host logic of the bench line's rooflines: the work of each kernel split by
the unit that executes it, and each part's fraction of its own peak."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402

P, NF = 19, 12
NH, N1 = NF + 1, 2 * NF + 1
MXP = (N1 + 1) & ~1
STATS = {"n_fout": 100, "n_fin": 300, "incoming_reads": 3000, "local_flops": 9.0e9,
         "near_pairs": 5_000_000, "near_pairs_screened": 2_000_000, "near_pairs_inside": 600_000}
PRM = {"p": P, "nf": NF, "q_degree": 11}


def test_kernel_work_units_and_amounts():
    n = 1000
    w = bench.kernel_work(STATS, PRM, n, n)
    up = dict((name, (a, kind)) for name, a, kind in w["k_upward"])
    # the single-precision anterpolation of p = 19 runs on the CUDA cores
    assert up["anterpolation"] == (2.0 * P ** 3 * n, "fp32")
    assert up["c2p shifts"] == (3.0 * P ** 3 * (P + 1) * (STATS["n_fout"] - 1), "fp32")
    inc = dict((name, (a, kind)) for name, a, kind in w["k_incoming"])
    assert inc["translation"] == (8.0 * N1 * N1 * NH * STATS["incoming_reads"], "fp32")
    assert inc["plane waves to Chebyshev"][1] == "tensor"
    assert inc["plane waves read once, coefficients written"] == (
        8.0 * STATS["n_fout"] * NH * N1 * MXP + 4.0 * STATS["n_fin"] * P ** 3, "hbm")
    loc = dict((name, (a, kind)) for name, a, kind in w["k_local"])
    assert loc["leaf evaluation"] == (2.0 * P ** 3 * n, "tensor")
    assert loc["p2c shifts and sums"][0] == pytest.approx(STATS["local_flops"] - 2.0 * P ** 3 * n)
    # the near field counts the pairs it screens, not every pair of the lists
    (name, amount, kind), = w["k_near"]
    per_inside = bench.near_flops_per_pair(11) - bench.NEAR_SCREEN_FLOPS
    assert kind == "fp32"
    assert amount == STATS["near_pairs_screened"] * bench.NEAR_SCREEN_FLOPS + STATS["near_pairs_inside"] * per_inside


def test_high_orders_anterpolate_on_the_tensor_cores():
    w = bench.kernel_work(STATS, {"p": 28, "nf": 19, "q_degree": 11}, 10, 10)
    assert dict((name, kind) for name, _, kind in w["k_upward"])["anterpolation"] == "tensor"


def test_rooflines_take_the_largest_fraction():
    work = {"k": [("a", 2.0e12, "fp32"), ("b", 6.0e9, "hbm"), ("c", 1.0e12, "tensor")]}
    peaks = {"fp32": 80.0, "hbm": 6000.0, "tensor": 250.0}
    r = bench.rooflines(work, {"k": 100.0}, peaks)["k"]
    # 2e12 flops in 0.1 s = 20 TFLOP/s = 0.25 of 80; 6e9 B in 0.1 s = 60 GB/s = 0.01;
    # 1e12 flops = 10 TFLOP/s = 0.04 of 250
    fr = {c["work"]: c["frac"] for c in r["components"]}
    assert fr == pytest.approx({"a": 0.25, "b": 0.01, "c": 0.04})
    assert r["bound"] == "alu" and r["frac"] == pytest.approx(0.25) and r["unit"] == "TFLOP/s"
    assert r["ms_per_eval"] == 100.0


def test_rooflines_skip_kernels_without_time_or_work():
    work = {"timed": [("x", 1.0e9, "hbm")], "untimed": [("y", 1.0, "fp32")], "idle": [("z", 0.0, "fp32")]}
    r = bench.rooflines(work, {"timed": 1.0, "idle": 1.0}, {"hbm": 1000.0, "fp32": 1.0})
    assert set(r) == {"timed"}
    assert r["timed"]["bound"] == "hbm" and r["timed"]["achieved"] == pytest.approx(1000.0)


def test_fp32_peak_scales_with_the_clock():
    peak, basis = bench.fp32_peak(152, bench.FFMA_MEASURED_MHZ / 2)
    assert peak == pytest.approx(bench.FFMA_MEASURED_TFLOPS / 2)
    assert "FFMA probe" in basis


def test_log2d_near_roofline():
    """The 2D near field's roofline: 24 + 2 (q_degree - 1) FP64 flops per pair
    inside the support against the DFMA probe, or 34 + 3 q_degree_f32 FP32
    flops on the mixed path against the FFMA probe, both at the sampled clock."""
    prm = {"q_degree": 15, "q_degree_f32": 11}
    r = bench.log2d_near_roofline(1_000_000_000, prm, 100.0, bench.FFMA_MEASURED_MHZ, False)
    assert r["bound"] == "fp64" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(1e9 * 52 / 0.1 / 1e12)
    assert r["peak"] == pytest.approx(bench.DFMA_MEASURED_TFLOPS)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    m = bench.log2d_near_roofline(1_000_000_000, prm, 10.0, bench.FFMA_MEASURED_MHZ / 2, True)
    assert m["bound"] == "fp32"
    assert m["achieved"] == pytest.approx(1e9 * (34 + 33) / 0.01 / 1e12)
    assert m["peak"] == pytest.approx(bench.FFMA_MEASURED_TFLOPS / 2)
