"""Host arithmetic of bench.py (no GPU): percentiles, the algorithmic-byte
model of each stage, the HBM fractions and the ALU roofline of the
compositing kernels."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_nearest_rank_percentile():
    assert bench._pct([3.0], 99) == 3.0
    assert bench._pct(list(range(1, 101)), 50) == 50
    assert bench._pct(list(range(1, 101)), 99) == 99
    assert bench._pct(list(range(1, 1001)), 99) == 990
    assert bench._pct([5, 1, 4, 2, 3], 100) == 5


def test_stage_bytes_follow_the_per_unit_model():
    n, keys, P = 200_000, 491_000, 640 * 480
    b = bench.stage_bytes(n, keys, P)
    assert set(b) == {"project_bin_sort", "render_fwd_loss", "render_bwd", "project_bwd_pose_step"}
    assert b["project_bin_sort"] == 124 * n + 28 * keys
    assert b["render_fwd_loss"] == 48 * keys + 56 * P
    assert b["render_bwd"] == 76 * keys + 40 * P
    assert b["project_bwd_pose_step"] == 112 * n
    # linear in each count
    b2 = bench.stage_bytes(2 * n, 2 * keys, 2 * P)
    assert all(b2[k] == 2 * b[k] for k in b)


def test_hbm_fractions_add_up():
    n, keys, P = 1000, 3000, 100
    stage_ms = {"project_bin_sort": 0.01, "render_fwd_loss": 0.02, "render_bwd": 0.03, "project_bwd_pose_step": 0.005}
    h = bench.hbm_fractions(stage_ms, n, keys, P, iter_ms=0.07)
    total = sum(bench.stage_bytes(n, keys, P).values())
    assert h["iteration"]["bytes"] == total
    assert h["iteration"]["gbs"] == pytest.approx(total / 0.07e-3 / 1e9)
    for k, v in h["stages"].items():
        assert v["frac"] == pytest.approx(v["gbs"] / h["peak_gbs"])


def test_alu_roofline_of_the_dominant_compositing_kernel():
    stage_ms = {"project_bin_sort": 0.07, "render_fwd_loss": 0.09, "render_bwd": 0.15, "project_bwd_pose_step": 0.02}
    r = bench.roofline(stage_ms, 200_000, 491_000, 640 * 480, blended=12_570_000, clk=None)
    assert r["bound"] == "alu" and r["kernel"] == "render_bwd" and r["unit"] == "TFLOP/s"
    flops = bench.FLOP_PER_FRAGMENT["render_bwd"] * 12_570_000
    assert r["algorithmic_flops"] == flops
    assert r["achieved"] == pytest.approx(flops / 0.15e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # 152 SMs x 128 lanes x 2 FLOPs x the maximum SM clock
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2070.0e6 / 1e12, rel=1e-6)
