"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/gs.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(gs_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2510_06644_gb300 import build
    return build.build()


def test_header_declares_the_hot_path_entry_points():
    names = declared_functions()
    for need in ("gs_project", "gs_bin_sort", "gs_render_fwd", "gs_render_bwd", "gs_prune", "gs_downsample",
                 "gs_project_bwd", "gs_loss_l1", "gs_status_poll", "gs_last_error"):
        assert need in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_targets_sm_103a_only(built_lib):
    from paper_2510_06644_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_only_entry_points_without_gpu(built_lib):
    """Pure host functions answer without touching a device."""
    from paper_2510_06644_gb300 import gs
    cfg = gs.default_config()
    assert abs(cfg.alpha_min - 1 / 255) < 1e-9 and cfg.k0 == 5 and abs(cfg.lambda_score - 0.8) < 1e-7
    assert b"sm_103a" in gs.lib().gs_version()
    for (n, k, kf, expect) in [(11, 10, False, (4, 4)), (12, 10, False, (4, 2)), (13, 10, False, (2, 2)),
                               (20, 10, False, (2, 2)), (10, 10, True, (1, 1))]:
        sx, sy, _ = gs.gs_downsample(n, k, kf, 2)
        assert (sx, sy) == expect
    with pytest.raises(gs.GsError):
        gs.gs_downsample(12, 10, False, 3)


def test_argument_errors_are_synchronous(built_lib):
    from paper_2510_06644_gb300 import gs
    cam = gs.camera({"R": [1, 0, 0, 0, 1, 0, 0, 0, 1], "t": [0, 0, 0], "fx": 10, "fy": 10, "cx": 5, "cy": 5,
                     "W": 0, "H": 10})
    nb = ctypes.c_size_t(0)
    cfg = gs.default_config()
    rc = gs.lib().gs_bin_sort(ctypes.byref(cfg), ctypes.byref(cam), 0, None, 10, 100, None, ctypes.byref(nb), None,
                              None, None, None, None, None)
    assert rc == gs.GS_ERR_INVALID_ARG
    assert b"camera" in gs.lib().gs_last_error()


def test_workspace_size_queries_need_no_device(built_lib):
    """A NULL workspace only asks for the size: pure host arithmetic."""
    from paper_2510_06644_gb300 import gs
    cam = gs.camera({"R": [1, 0, 0, 0, 1, 0, 0, 0, 1], "t": [0, 0, 0], "fx": 525, "fy": 525, "cx": 320,
                     "cy": 240, "W": 640, "H": 480})
    small = gs.gs_bin_sort_workspace(cam, gs.GS_F32, 1000, 10_000)
    big = gs.gs_bin_sort_workspace(cam, gs.GS_F32, 200_000, 1_000_000)
    assert 0 < small < big and big % 256 == 0
    # the merge buffer for long tile buckets dominates: 8 bytes per key of capacity
    assert big >= 8 * 1_000_000
    with pytest.raises(gs.GsError):
        gs.gs_bin_sort_workspace(cam, gs.GS_F32, 10, 1 << 30)   # capacity limit 2^30


def test_fused_entry_points_reject_bad_arguments_on_the_host(built_lib):
    """The fused forms check their extra arguments before any device work."""
    from paper_2510_06644_gb300 import gs
    cfg = gs.default_config()
    cam = gs.camera({"R": [1, 0, 0, 0, 1, 0, 0, 0, 1], "t": [0, 0, 0], "fx": 10, "fy": 10, "cx": 5, "cy": 5,
                     "W": 10, "H": 10})
    g = gs.gs_gaussians()
    g.n = 10
    step = gs.gs_pose_step(None, None, 1e-3, 1e-3, 0.9, 0.999, 1e-8)
    nb = ctypes.c_size_t(1 << 20)
    # a pose step needs the pose-gradient output
    rc = gs.lib().gs_project_bwd_step(ctypes.byref(cfg), ctypes.byref(cam), ctypes.byref(g), None, None, None,
                                      None, ctypes.byref(step), None, ctypes.byref(nb), None)
    assert rc == gs.GS_ERR_INVALID_ARG and b"pose_grad6" in gs.lib().gs_last_error()
    # ... and a pose and an Adam state
    pg = ctypes.c_double * 6
    rc = gs.lib().gs_project_bwd_step(ctypes.byref(cfg), ctypes.byref(cam), ctypes.byref(g), None, None,
                                      ctypes.cast(pg(), ctypes.c_void_p), None, ctypes.byref(step), None,
                                      ctypes.byref(nb), None)
    assert rc == gs.GS_ERR_INVALID_ARG and b"pose step" in gs.lib().gs_last_error()
    # forward + loss: targets, gradients and the loss word are required
    rc = gs.lib().gs_render_fwd_loss(ctypes.byref(cfg), ctypes.byref(cam), gs.GS_F32, None, 0, None,
                                     ctypes.c_void_p(16), None, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                     ctypes.c_void_p(16), ctypes.c_void_p(16), None, None, None, None, None,
                                     None, None, None)
    assert rc == gs.GS_ERR_INVALID_ARG and b"target" in gs.lib().gs_last_error()


def test_reduction_probe_rejects_bad_arguments_on_the_host(built_lib):
    from paper_2510_06644_gb300 import gs
    L = gs.lib()
    assert L.gs_probe_red_f32(None, 16, 16, 1, None) == gs.GS_ERR_INVALID_ARG
    fake = ctypes.c_void_p(16)  # never dereferenced: the counts are checked first
    for n_dst, n_thr, per in ((0, 16, 1), (16, 0, 1), (16, 16, 0), (16, -5, 1)):
        assert L.gs_probe_red_f32(fake, n_dst, n_thr, per, None) == gs.GS_ERR_INVALID_ARG
    assert L.gs_probe_fma_f32(None, 16, 1, None) == gs.GS_ERR_INVALID_ARG
    for n_thr, iters in ((0, 1), (16, 0), (-3, 4)):
        assert L.gs_probe_fma_f32(fake, n_thr, iters, None) == gs.GS_ERR_INVALID_ARG


def test_blend_mask_words_host_arithmetic(built_lib):
    """256 words per 32 keys of capacity plus 256 per tile (and one spare
    run): enough for every pixel's runs of 32 list entries in tiles of up to
    256 pixels (64 per tile and run for entry-parallel frames)."""
    from paper_2510_06644_gb300 import gs
    cam = gs.camera({"R": [1, 0, 0, 0, 1, 0, 0, 0, 1], "t": [0, 0, 0], "fx": 500, "fy": 500, "cx": 320,
                     "cy": 240, "W": 640, "H": 480})
    T = 40 * 30
    for cap in (0, 31, 32, 491244, 10 ** 7):
        assert gs.gs_blend_mask_words(cam, cap) == 256 * T + 256 * (cap // 32 + 1)
    # entry-parallel frames (both strides >= 2) keep a run per pixel: 64 per tile
    cam2 = gs.camera({"R": [1, 0, 0, 0, 1, 0, 0, 0, 1], "t": [0, 0, 0], "fx": 500, "fy": 500, "cx": 320,
                      "cy": 240, "W": 640, "H": 480, "sx": 2, "sy": 2})
    assert gs.gs_blend_mask_words(cam2, 491244) == 64 * T + 64 * (491244 // 32 + 1)
    bad = gs.camera({"R": [1, 0, 0, 0, 1, 0, 0, 0, 1], "t": [0, 0, 0], "fx": 1, "fy": 1, "cx": 0, "cy": 0,
                     "W": 0, "H": 10})
    assert gs.gs_blend_mask_words(bad, 100) == 0


def test_fused_projection_binning_checks_arguments_on_the_host(built_lib):
    from paper_2510_06644_gb300 import gs
    cfg = gs.default_config()
    cam = gs.camera({"R": [1, 0, 0, 0, 1, 0, 0, 0, 1], "t": [0, 0, 0], "fx": 100, "fy": 100, "cx": 48,
                     "cy": 36, "W": 96, "H": 72})
    nb = ctypes.c_size_t(0)
    L = gs.lib()
    assert L.gs_project_bin_sort(ctypes.byref(cfg), ctypes.byref(cam), None, gs.GS_F32, None, 100, None,
                                 ctypes.byref(nb), None, None, None, None, None, None) == gs.GS_ERR_INVALID_ARG
    g = gs.gs_gaussians()
    g.n = 0
    assert L.gs_project_bin_sort(ctypes.byref(cfg), ctypes.byref(cam), ctypes.byref(g), 7, None, 100, None,
                                 ctypes.byref(nb), None, None, None, None, None, None) == gs.GS_ERR_INVALID_ARG
    # a size query with no Gaussians needs no device
    assert L.gs_project_bin_sort(ctypes.byref(cfg), ctypes.byref(cam), ctypes.byref(g), gs.GS_F32, None, 100,
                                 None, ctypes.byref(nb), None, None, None, None, None, None) == gs.GS_OK
    assert nb.value > 0


def test_track_wave_rejects_bad_arguments_on_the_host(built_lib):
    """gs_track_wave checks every job before it enqueues anything: the
    count of jobs, then each descriptor (the message names the job)."""
    from paper_2510_06644_gb300 import gs
    L = gs.lib()
    cfg = gs.default_config()
    jobs = (gs.gs_track_job * 2)()
    assert L.gs_track_wave(ctypes.byref(cfg), None, 1, None) == gs.GS_ERR_INVALID_ARG
    assert L.gs_track_wave(ctypes.byref(cfg), ctypes.cast(jobs, ctypes.c_void_p), 0, None) == gs.GS_ERR_INVALID_ARG
    assert L.gs_track_wave(ctypes.byref(cfg), ctypes.cast(jobs, ctypes.c_void_p), gs.GS_WAVE_MAX + 1,
                           None) == gs.GS_ERR_INVALID_ARG
    # a camera but no map
    for j in jobs:
        j.cam = gs.camera({"R": [[1, 0, 0], [0, 1, 0], [0, 0, 1]], "t": [0, 0, 0], "fx": 80.0, "fy": 80.0,
                           "cx": 48.0, "cy": 36.0, "W": 96, "H": 72})
    rc = L.gs_track_wave(ctypes.byref(cfg), ctypes.cast(jobs, ctypes.c_void_p), 2, None)
    assert rc == gs.GS_ERR_INVALID_ARG and b"job 0" in L.gs_last_error()
    jobs[0].cam.width = 0
    rc = L.gs_track_wave(ctypes.byref(cfg), ctypes.cast(jobs, ctypes.c_void_p), 2, None)
    assert rc == gs.GS_ERR_INVALID_ARG and b"job 0: bad camera" in L.gs_last_error()


def test_next_interval_follows_the_oracle_rule(built_lib):
    """gs_next_interval (the rule gs_prune applies when an interval ends)
    against the oracle's statement of Sec. 4.1 on scripted change ratios:
    halved above the threshold, doubled below it, capped, never below 1."""
    from oracle import oracle as O
    O.build()
    from paper_2510_06644_gb300 import gs
    cfg = gs.default_config()
    K = int(cfg.k0)
    for r in (0.0, 0.01, 0.2, 0.05, 0.051, 0.3, 0.3, 0.3, 0.3, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0):
        got = gs.gs_next_interval(cfg, K, r)
        assert got == O.next_interval(K, r, K0=int(cfg.k0), thr=float(cfg.change_thr), k_max=int(cfg.k_max)), (K, r)
        K = got
    assert K == 32   # ... 64 at the cap, then one halving
    assert gs.gs_next_interval(cfg, 0, 0.0) == 1
    assert gs.lib().gs_next_interval(None, 5, ctypes.c_float(0.0)) == 1   # no config: the smallest interval


def test_fused_adam_rejects_bad_arguments_on_the_host(built_lib):
    from paper_2510_06644_gb300 import gs
    L = gs.lib()
    cfg = gs.default_config()
    cam = gs.camera({"R": [[1, 0, 0], [0, 1, 0], [0, 0, 1]], "t": [0, 0, 0], "fx": 80.0, "fy": 80.0,
                     "cx": 48.0, "cy": 36.0, "W": 96, "H": 72})
    g = gs.gs_gaussians()
    a = gs.gs_map_adam()
    a.lr, a.beta1, a.beta2, a.eps = 1e-3, 0.9, 0.999, 1e-15
    assert L.gs_project_bwd_adam(ctypes.byref(cfg), ctypes.byref(cam), ctypes.byref(g), None, None, None, None,
                                 None) == gs.GS_ERR_INVALID_ARG
    # no state word
    assert L.gs_project_bwd_adam(ctypes.byref(cfg), ctypes.byref(cam), ctypes.byref(g), None, ctypes.byref(a), None,
                                 None, None) == gs.GS_ERR_INVALID_ARG
    a.state = 16
    a.beta1 = 1.0
    assert L.gs_project_bwd_adam(ctypes.byref(cfg), ctypes.byref(cam), ctypes.byref(g), None, ctypes.byref(a), None,
                                 None, None) == gs.GS_ERR_INVALID_ARG
    assert b"Adam" in L.gs_last_error()


def test_downsample_schedule_follows_the_oracle(built_lib):
    """gs_downsample's strides without a target (host only, Sec. 4.2)
    against the oracle's schedule for frames around several keyframes and
    every m, including the arguments both reject: m not a power of two >= 2,
    a non-keyframe at or before its keyframe."""
    from oracle import oracle as O
    O.build()
    from paper_2510_06644_gb300 import gs
    checked = rejected = 0
    for k in (0, 3, 10):
        for n in range(max(0, k - 2), k + 8):
            for m in (1, 2, 3, 4, 8):
                for kf in (False, True):
                    try:
                        want = O.downsample_schedule(n, k, kf, m=m)
                    except ValueError:
                        want = None
                    try:
                        got = gs.gs_downsample(n, k, kf, m)[:2]
                    except gs.GsError:
                        got = None
                    assert got == want, (n, k, m, kf, got, want)
                    checked += 1
                    rejected += want is None
    assert checked == 280 and 50 < rejected < 200
    # either stride pointer NULL is rejected
    sx = ctypes.c_int32(0)
    for a, b in ((None, ctypes.byref(sx)), (ctypes.byref(sx), None)):
        rc = gs.lib().gs_downsample(6, 5, 0, 2, a, b, None, 0, 0, 0, None, None)
        assert rc == gs.GS_ERR_INVALID_ARG


def test_default_config_holds_the_papers_values_and_the_readings(built_lib):
    """gs_default_config against the paper's fixed hyper-parameters
    (tests/golden/hyperparams.json: Sec. 6.1, Sec. 4.1, Sec. 6.2) and the
    oracle's configuration of the unstated thresholds (near plane,
    dilation, alpha skip and clamp, termination, background, loss weights;
    prune fraction 10 % per interval, K capped at 64)."""
    import json
    from oracle import oracle as O
    from paper_2510_06644_gb300 import gs
    hp = json.load(open(os.path.join(ROOT, "tests", "golden", "hyperparams.json")))
    c = gs.default_config()
    f32 = lambda x: float(ctypes.c_float(x).value)
    assert c.lambda_score == f32(hp["lambda_score"]) and c.k0 == hp["k0"]
    assert c.change_thr == f32(hp["change_ratio_threshold"]) and c.prune_cap == f32(hp["prune_cap"])
    d = O.DEFAULT_CFG
    for k in ("near_z", "dilation", "alpha_min", "alpha_max", "t_eps"):
        assert getattr(c, k) == f32(d[k]), k
    assert list(c.bg) == [f32(v) for v in d["bg"]]
    assert (c.w_rgb, c.w_depth) == (1.0, 0.5)        # reading c10: L1 RGB + 0.5 L1 depth
    assert c.prune_frac == f32(0.1) and c.k_max == 64  # readings c13, c15
