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
    fma = {"tflops": 78.0}
    walked, blended = 54_000_000, 12_570_000
    r = bench.roofline(stage_ms, 200_000, 491_000, 640 * 480, blended, walked, fma)
    assert r["bound"] == "alu" and r["kernel"] == "render_bwd" and r["unit"] == "TFLOP/s"
    # 45 FLOP per evaluated fragment (sum of last_idx) against the measured FMA peak
    assert r["algorithmic_flops"] == 45 * walked
    assert r["achieved"] == pytest.approx(45 * walked / 0.15e-3 / 1e12)
    assert r["peak"] == 78.0
    assert r["frac"] == pytest.approx(r["achieved"] / 78.0)
    # the per-blended view and the forward beside it
    assert r["per_blended"]["achieved"] == pytest.approx(67 * blended / 0.15e-3 / 1e12)
    assert r["render_fwd_loss"]["achieved"] == pytest.approx(15 * walked / 0.09e-3 / 1e12)
    assert r["render_fwd_loss"]["frac"] == pytest.approx(r["render_fwd_loss"]["achieved"] / 78.0)


def test_clock_summary_counts_the_timed_samples():
    import datetime
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0).timestamp()

    def row(dt, mhz, pcap="Not Active", mx=2070, w=500.5):
        ts = datetime.datetime.fromtimestamp(t0 + dt).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, 0, {mhz}, {mx}, {w}, 0x0, Not Active, Not Active, Not Active, {pcap}"

    lines = [row(0.0, 1900, mx=2055, w=300.0), row(0.1, 2070, w=612.25), row(0.2, 2070, "Active"), row(0.3, 2000),
             "garbage line"]
    c = bench.Clocks.parse(lines, timed=[(t0 + 0.15, t0 + 0.25)])
    assert c["samples"] == 4 and c["sm_max_mhz"] == 2070.0 and c["power_w_max"] == 612.25
    assert c["sm_mhz"] == pytest.approx(2035.0)
    assert c["reasons"] == ["sw_power_cap"]
    # the timed region (widened by one sampling interval) holds the samples at 0.1, 0.2 and 0.3 s
    assert c["samples_timed"] == 3 and c["sm_mhz_timed"] == 2070.0


def test_mask_visits_counts_warp_entry_pairs():
    """The bench's count of the masked backward's (warp, entry) visits
    against a plain loop over tiles, warps and entries on random per-pixel
    blend-mask words (garbage past each warp's last run and past each list's
    end must not count).  The words are sparse (a bit set with probability
    1/64), so that their OR over a warp's 32 lanes depends on which words
    are read."""
    import numpy as np
    import torch
    import bench
    rng = np.random.default_rng(5)
    TX, TY, H, W = 3, 2, 29, 45          # ragged: the last tile row/column is partial
    T = TX * TY
    lens = rng.integers(0, 90, T)
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]]) + 7
    ranges = np.stack([starts, starts + lens], 1).astype(np.int32)
    nwords = 256 * (int(starts.max()) // 32 + T) + 256 * 8 + 256
    bits = rng.random((nwords, 32)) < 1 / 64
    bm = (bits * (np.uint64(1) << np.arange(32, dtype=np.uint64))).sum(1).astype(np.uint32).view(np.int32)
    last = np.zeros((H, W), np.int64)
    for t in range(T):
        tx, ty = t % TX, t // TX
        for py in range(16):
            for px in range(16):
                y, x = ty * 16 + py, tx * 16 + px
                if y < H and x < W:
                    last[y, x] = rng.integers(0, lens[t] + 1)
    want = 0
    for t in range(T):
        tx, ty = t % TX, t // TX
        for w in range(8):
            wl = 0
            for lane in range(32):
                y = ty * 16 + (w // 2) * 4 + lane // 8
                x = tx * 16 + (w % 2) * 8 + lane % 8
                if y < H and x < W:
                    wl = max(wl, int(last[y, x]))
            for e in range(wl if wl % 32 == 0 else (wl // 32 + 1) * 32):
                if e >= lens[t]:
                    continue
                r, b = divmod(e, 32)
                base = 256 * (int(starts[t]) // 32 + t) + 256 * r + 32 * w
                if any((int(bm.view(np.uint32)[base + lane]) >> b) & 1 for lane in range(32)):
                    want += 1
    got = bench.mask_visits(torch.from_numpy(bm), torch.from_numpy(ranges), torch.from_numpy(last), TX, TY)
    assert got == want
    assert 0.2 * lens.sum() * 8 < want < 0.9 * lens.sum() * 8   # neither empty nor saturated
