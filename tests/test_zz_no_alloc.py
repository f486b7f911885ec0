"""The allocation-free backward projection, gs_project_bwd_noalloc, gives the
results of gs_project_bwd.

Some callers cannot allocate device memory (a real-time tracking thread that
runs under a fixed memory budget, or a host framework that owns every
allocation); for them the library keeps the scratch of this one call in a
static device array.  This file runs last so that a failure here does not
hide the rest of the suite; it also passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from synth import scenes as S

pytestmark = pytest.mark.gpu

TOL = 1e-3  # the gradient tolerance of the parity tests (relative L2)


def rel(a, b):
    a = a.detach().double().cpu().numpy().ravel()
    b = b.detach().double().cpu().numpy().ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("n", [2000, 70000])
def test_noalloc_matches_workspace_version_twice(n):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_06644_gb300 import build
    build.build()
    from paper_2510_06644_gb300 import gs

    g = S.surface_scene(n, seed=4242 + n)
    cam = S.perturbed_pose(S.camera(320, 240, 260.0), seed=5, trans=0.03, rot_deg=1.0)
    gd = {k: torch.from_numpy(v).cuda() for k, v in g.items()}
    rng = S.rng(7)
    g2 = torch.from_numpy((rng.normal(0, 1e-3, (n, 12))).astype(np.float32)).cuda()
    cfg = gs.default_config()
    cs = gs.camera(cam)
    keys = ("means", "log_scales", "quats", "opacity_logit", "rgb")

    ref = {k: torch.empty_like(gd[k]) for k in keys}
    ref_pose = torch.zeros(6, dtype=torch.float64, device="cuda")
    ref_score = torch.empty((n, 2), device="cuda")
    gs.gs_project_bwd(cfg, cs, gd, g2, grads=ref, pose=ref_pose, score=ref_score)

    for call in range(2):
        out = {k: torch.full_like(gd[k], float("nan")) for k in keys}
        pose = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
        score = torch.full((n, 2), float("nan"), device="cuda")
        # straight through the C ABI
        gg = gs.gaussians(gd)
        gr = gs.grads_struct(out)
        rc = gs.lib().gs_project_bwd_noalloc(ctypes.byref(cfg), ctypes.byref(cs), ctypes.byref(gg),
                                             ctypes.c_void_p(g2.data_ptr()), ctypes.byref(gr),
                                             ctypes.c_void_p(pose.data_ptr()), ctypes.c_void_p(score.data_ptr()),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == gs.GS_OK, gs.lib().gs_last_error()
        torch.cuda.synchronize()
        for k in keys:
            assert rel(out[k], ref[k]) <= TOL, (call, k)
        assert rel(pose, ref_pose) <= TOL, call
        assert rel(score, ref_score) <= TOL, call


def test_noalloc_rejects_more_than_its_maximum():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_06644_gb300 import build
    build.build()
    from paper_2510_06644_gb300 import gs

    cfg = gs.default_config()
    cs = gs.camera(S.camera(64, 48, 50.0))
    gg = gs.gs_gaussians()
    dummy = torch.zeros(4, device="cuda")
    for f in ("means", "log_scales", "quats", "opacity_logit", "rgb"):
        setattr(gg, f, dummy.data_ptr())
    gg.n = 4194304 + 1
    rc = gs.lib().gs_project_bwd_noalloc(ctypes.byref(cfg), ctypes.byref(cs), ctypes.byref(gg),
                                         ctypes.c_void_p(dummy.data_ptr()), None, None, None, None)
    assert rc == gs.GS_ERR_INVALID_ARG
    assert b"GS_NOALLOC_MAX_GAUSSIANS" in gs.lib().gs_last_error()


@pytest.mark.parametrize("subset", ["pose", "grads+score", "score"])
def test_noalloc_output_subsets_through_the_binding(subset):
    """Each subset of outputs takes its own kernel form (and only the pose
    uses the scratch's ticket): through the Python binding, every subset
    gives what gs_project_bwd gives for it, on two calls in a row."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_06644_gb300 import build
    build.build()
    from paper_2510_06644_gb300 import gs

    n = 30000
    g = S.surface_scene(n, seed=4300)
    cam = S.perturbed_pose(S.camera(320, 240, 260.0), seed=6, trans=0.03, rot_deg=1.0)
    gd = {k: torch.from_numpy(v).cuda() for k, v in g.items()}
    g2 = torch.from_numpy((S.rng(8).normal(0, 1e-3, (n, 12))).astype(np.float32)).cuda()
    cfg = gs.default_config()
    cs = gs.camera(cam)
    keys = ("means", "log_scales", "quats", "opacity_logit", "rgb")

    def outputs():
        return ({k: torch.full_like(gd[k], float("nan")) for k in keys} if "grads" in subset else None,
                torch.full((6,), float("nan"), dtype=torch.float64, device="cuda") if "pose" in subset else None,
                torch.full((n, 2), float("nan"), device="cuda") if "score" in subset else None)

    rg, rp, rs = outputs()
    gs.gs_project_bwd(cfg, cs, gd, g2, grads=rg, pose=rp, score=rs)
    for call in range(2):
        og, op, os_ = outputs()
        gs.gs_project_bwd_noalloc(cfg, cs, gd, g2, grads=og, pose=op, score=os_)
        torch.cuda.synchronize()
        for a, b in ((og, rg), (op, rp), (os_, rs)):
            if a is None:
                continue
            if isinstance(a, dict):
                for k in keys:
                    assert rel(a[k], b[k]) <= TOL, (call, subset, k)
            else:
                assert rel(a, b) <= TOL, (call, subset)
