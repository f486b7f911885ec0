"""The fused forms of the tracking iteration against the separate calls:
forward + loss in one launch (gs_render_fwd_loss) and the backward
projection with the pose step in its last block (gs_project_bwd_step)."""
import numpy as np
import pytest
import torch

from synth import scenes as S
from tests.gpu_helpers import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_06644_gb300 import build
    build.build()
    from paper_2510_06644_gb300 import gs
    return gs


def scene_and_cams(seed=40):
    g = S.surface_scene(40000, seed=seed)
    true_cam = S.camera(320, 240, 260.0)
    start = S.perturbed_pose(true_cam, seed=seed + 1, trans=0.02, rot_deg=1.0)
    return g, true_cam, start


@pytest.mark.parametrize("sx,sy,rec", [(1, 1, "f32"), (2, 2, "f32"), (4, 4, "bf16"), (1, 2, "f16")])
def test_forward_with_fused_loss_equals_separate_calls(G, sx, sy, rec):
    from paper_2510_06644_gb300.pipeline import Rasterizer
    dt = {"f32": G.GS_F32, "bf16": G.GS_BF16, "f16": G.GS_F16}[rec]
    g, true_cam, start = scene_and_cams()
    gd = dev(g)
    r = Rasterizer(40000, dict(start, sx=sx, sy=sy), rec_dtype=dt, capacity=400000)
    tgt = Rasterizer(40000, dict(true_cam, sx=sx, sy=sy), rec_dtype=dt, capacity=400000)
    img_t = tgt.forward(gd, dict(true_cam, sx=sx, sy=sy))
    trgb, tdep = img_t["rgb"].clone(), img_t["depth"].clone()
    tdep[::7, ::5] = 0.0  # invalid depths take no depth term
    cs = G.camera(dict(start, sx=sx, sy=sy))
    r.forward(gd, cs)
    sep = {k: v.clone() for k, v in r.img.items()}
    d = G.gs_loss_l1(r.cfg, cs, r.img["rgb"], r.img["depth"], trgb, tdep)
    out, dimg = G.gs_render_fwd_loss(r.cfg, cs, r.splats, r.n, r.vals, r.ranges, trgb, tdep, dt, order=r.order)
    torch.cuda.synchronize()
    for k in sep:
        assert torch.equal(out[k], sep[k]), k
    assert torch.equal(dimg["d_rgb"], d["d_rgb"])
    assert torch.equal(dimg["d_depth"], d["d_depth"])
    a, b = float(dimg["loss"].item()), float(d["loss"].item())
    assert a > 0 and abs(a - b) <= 1e-6 * abs(b)
    r.check()


def test_backward_projection_with_fused_pose_step_equals_separate_calls(G):
    from paper_2510_06644_gb300.pipeline import Rasterizer
    g, true_cam, start = scene_and_cams(seed=50)
    gd = dev(g)
    r = Rasterizer(40000, start, capacity=400000)
    trgb = r.forward(gd, true_cam)["rgb"].clone()
    tdep = r.img["depth"].clone()
    pose = G.pose_tensor(start)
    cs = G.camera(start, pose=pose)
    r.forward(gd, cs)
    r.loss_grad(cs, trgb, tdep)
    r.backward(gd, cs, r.dimg["d_rgb"], r.dimg["d_depth"], want_pose=False, want_score=False)
    grad2d = r.grad2d.clone()  # one backward, shared by both routes
    res = []
    for fused in (False, True):
        p = pose.clone()
        adam = torch.zeros(13, device="cuda")
        pg = torch.zeros(6, dtype=torch.float64, device="cuda")
        c = G.camera(start, pose=p)
        for _ in range(3):
            if fused:
                G.gs_project_bwd_step(r.cfg, c, gd, grad2d, pg, G.pose_step(p, adam, 1e-3, 2e-3))
            else:
                G.gs_project_bwd(r.cfg, c, gd, grad2d, pose=pg)
                G.gs_pose_update(p, pg, adam, 1e-3, 2e-3)
        torch.cuda.synchronize()
        res.append((p.cpu().numpy(), adam.cpu().numpy(), pg.cpu().numpy()))
    (pa, aa, ga), (pb, ab, gb) = res
    assert np.abs(pb - pose.cpu().numpy()).max() > 1e-5  # the pose moved
    assert np.array_equal(ga, gb)
    assert np.array_equal(aa, ab)
    assert np.array_equal(pa, pb)
    r.check()


@pytest.mark.parametrize("sx,sy", [(1, 1), (2, 2)])
def test_fused_tracking_iterations_follow_the_separate_ones(G, sx, sy):
    """Ten iterations of Rasterizer.track_step (as a wave of one session, and
    through the separate fused calls) against step() + gs_pose_update: same
    pose trajectory (to the nondeterministic order of the backward's float
    atomics)."""
    from paper_2510_06644_gb300.pipeline import Rasterizer
    g, true_cam, start = scene_and_cams(seed=60)
    gd = dev(g)
    tgt = Rasterizer(40000, dict(true_cam, sx=sx, sy=sy), capacity=400000)
    img = tgt.forward(gd, dict(true_cam, sx=sx, sy=sy))
    trgb, tdep = img["rgb"].clone(), img["depth"].clone()
    traj = []
    for fused in (False, True, "calls"):
        r = Rasterizer(40000, dict(start, sx=sx, sy=sy), capacity=400000)
        pose = G.pose_tensor(start)
        adam = torch.zeros(13, device="cuda")
        cs = G.camera(dict(start, sx=sx, sy=sy), pose=pose)
        poses = []
        for _ in range(10):
            if fused:
                r.track_step(gd, cs, trgb, tdep, pose, adam, wave=fused is True)
            else:
                r.step(gd, cs, trgb, tdep, G.GS_TRACK)
                G.gs_pose_update(pose, r.pose, adam)
            poses.append(pose.cpu().numpy().copy())
        r.check()
        traj.append(np.array(poses))
    a, b, c = traj
    assert np.abs(a[-1] - a[0]).max() > 1e-4
    assert np.abs(a - b).max() <= 1e-5, np.abs(a - b).max()
    assert np.abs(a - c).max() <= 1e-5, np.abs(a - c).max()


@pytest.mark.parametrize("n,W,H,sx,sy,dt,mask_frac", [
    (40000, 320, 240, 1, 1, 0, 0.0),
    (40000, 320, 240, 2, 2, 1, 0.1),
    (40000, 320, 240, 4, 2, 2, 0.0),
    (30000, 333, 197, 1, 2, 0, 0.3),
    (0, 320, 240, 1, 1, 0, 0.0),            # no Gaussians
    (20000, 2048, 1080, 1, 1, 0, 0.0),      # more than 8192 tiles: the two calls
    (600000, 1920, 1080, 1, 1, 0, 0.0),     # more than 256 Gaussians per tile row
])
def test_project_bin_sort_equals_the_two_calls(G, n, W, H, sx, sy, dt, mask_frac):
    """gs_project_bin_sort (projection counting the binning's tiles, scatter
    from the kept rects) gives the records, keys, values, ranges and order of
    gs_project followed by gs_bin_sort, bit for bit."""
    g = S.surface_scene(max(n, 1), seed=70 + n % 7)
    if n == 0:
        g = {k: v[:0] for k, v in g.items()}
    if mask_frac > 0:
        g["mask"] = (np.random.default_rng(5).random(n) < mask_frac).astype(np.uint8)
    gd = dev(g)
    cam = S.camera(W, H, 0.8 * W, sx=sx, sy=sy)
    cfg = G.default_config()
    cs = G.camera(cam)
    words = G.SPLAT_WORDS[dt]
    rtype = torch.float32 if dt == G.GS_F32 else torch.int32
    rec_a = torch.empty((max(n, 1), words), dtype=rtype, device="cuda")
    rec_b = torch.empty_like(rec_a)
    G.gs_project(cfg, cs, gd, dt, rec_a)
    cap = max(int(G.gs_bin_count(cs, rec_a, n, dt).item()), 1024) if n > 0 else 1024
    ka, va, na, ra, oa = G.gs_bin_sort(cs, rec_a, n, cap, dt, cfg=cfg)
    kb, vb, nb, rb, ob = G.gs_project_bin_sort(cfg, cs, gd, rec_b, cap, dt)
    torch.cuda.synchronize()
    assert int(na.item()) == int(nb.item())
    k = int(na.item())
    assert torch.equal(rec_a[:n], rec_b[:n])
    assert torch.equal(ka[:k], kb[:k]) and torch.equal(va[:k], vb[:k])
    assert torch.equal(ra, rb) and torch.equal(oa, ob)


def test_backward_projection_with_fused_adam_equals_separate_calls(G):
    """A mapping iteration's map update fused into the backward projection
    (gs_project_bwd_adam) against gs_project_bwd followed by gs_adam:
    parameters, moments, step count, gradients and score terms bit for bit,
    over three steps (the second and third project the updated map), with a
    masked Gaussian and Gaussians behind the camera in the map."""
    from paper_2510_06644_gb300.pipeline import Rasterizer
    g, true_cam, start = scene_and_cams(seed=47)
    g["means"][:50, 2] = -1.0                      # behind the camera: zero gradients, still stepped
    mask = np.zeros(40000, np.uint8)
    mask[60:70] = 1
    gd = dev(g)
    r = Rasterizer(40000, start, capacity=400000)
    tgt = Rasterizer(40000, true_cam, capacity=400000)
    img_t = tgt.forward(gd, true_cam)
    trgb, tdep = img_t["rgb"].clone(), img_t["depth"].clone()
    r.forward(gd, start)
    r.loss_grad(start, trgb, tdep)
    r.backward(gd, start, r.dimg["d_rgb"], r.dimg["d_depth"], G.GS_MAP, want_pose=False, want_score=False)
    grad2d = r.grad2d.clone()
    keys = G.PARAM_KEYS
    cs = G.camera(start)
    cfg = G.default_config()
    sides = []
    for fused in (False, True):
        p = {k: gd[k].clone() for k in keys}
        p["mask"] = torch.from_numpy(mask).cuda()
        ms = {k: torch.zeros_like(gd[k]) for k in keys}
        vs = {k: torch.zeros_like(gd[k]) for k in keys}
        state = torch.zeros(2, device="cuda")
        grads = {k: torch.empty_like(gd[k]) for k in keys}
        score = torch.empty((40000, 2), device="cuda")
        for _ in range(3):
            if fused:
                G.gs_project_bwd_adam(cfg, cs, p, grad2d, ms, vs, state, lr=1e-3, grads=grads, score=score)
            else:
                G.gs_project_bwd(cfg, cs, p, grad2d, grads=grads, score=score)
                G.gs_adam([p[k] for k in keys], [grads[k] for k in keys], [ms[k] for k in keys],
                          [vs[k] for k in keys], state, lr=1e-3)
        torch.cuda.synchronize()
        sides.append((p, ms, vs, state, grads, score))
    a, b = sides
    for k in keys:
        assert torch.equal(a[0][k], b[0][k]), ("param", k)
        assert torch.equal(a[1][k], b[1][k]), ("m", k)
        assert torch.equal(a[2][k], b[2][k]), ("v", k)
        assert torch.equal(a[4][k], b[4][k]), ("grad", k)
    assert torch.equal(a[3], b[3]) and float(a[3][0]) == 3.0
    assert torch.equal(a[5], b[5])
    assert not torch.equal(a[0]["means"], gd["means"])   # the map moved
