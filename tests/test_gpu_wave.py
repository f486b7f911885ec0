"""Multi-session waves (gs_track_wave): one launch per stage whose grid spans
every session gives each session exactly the results of its own fused
tracking iteration.  Sessions differ in map size, resolution and stride, so
every compositing form (full tiles, smaller pixel-parallel tiles, strided
tiles of 32 and of 64 pixels) runs in the same wave."""
import numpy as np
import pytest
import torch

from synth import scenes as S

pytestmark = pytest.mark.gpu

# (Gaussians, W, H, f, sx, sy, seed)
SESSIONS = [
    (30000, 320, 240, 262.5, 1, 1, 61),   # full-resolution tiles
    (60000, 640, 480, 525.0, 2, 2, 62),   # strided tiles of 64 pixels
    (20000, 320, 240, 262.5, 4, 2, 63),   # strided tiles of 32 pixels
    (40000, 640, 480, 525.0, 4, 4, 64),   # strided tiles of 16 pixels
    (25000, 200, 120, 160.0, 1, 2, 65),   # pixel-parallel, two tiles per CTA
    (1500, 96, 72, 80.0, 1, 1, 66),       # tiny map
]


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_06644_gb300 import build
    build.build()
    from paper_2510_06644_gb300 import gs
    gs.gs_status_reset()
    return gs


def make_session(G, n, W, H, f, sx, sy, seed):
    from paper_2510_06644_gb300.pipeline import Rasterizer
    scene = S.surface_scene(n, seed)
    gd = {k: torch.from_numpy(v).cuda() for k, v in scene.items()}
    true_cam = S.camera(W, H, f, sx=sx, sy=sy)
    start = S.perturbed_pose(true_cam, seed + 1, trans=0.02, rot_deg=1.0)
    probe = G.gs_project(G.default_config(), G.camera(start), gd)
    cap = int(int(G.gs_bin_count(G.camera(start), probe, n).item()) * 1.5) + 4096
    r0 = Rasterizer(n, start, capacity=cap)
    img = r0.forward(gd, true_cam)
    return {"g": gd, "start": start, "cap": cap, "trgb": img["rgb"].clone(), "tdep": img["depth"].clone()}


def fresh(G, sess):
    from paper_2510_06644_gb300.pipeline import Rasterizer
    r = Rasterizer(sess["g"]["means"].shape[0], sess["start"], capacity=sess["cap"])
    pose = G.pose_tensor(sess["start"])
    adam = torch.zeros(13, device="cuda")
    return r, pose, adam, G.camera(sess["start"], pose=pose)


def outputs(r):
    k = int(r.n_keys.item())
    return {"keys": r.keys[:k].clone(), "vals": r.vals[:k].clone(), "ranges": r.ranges.clone(),
            "order": r.order.clone(), **{n: v.clone() for n, v in r.img.items()},
            "d_rgb": r.dimg["d_rgb"].clone(), "loss": r.dimg["loss"].clone(), "grad2d": r.grad2d.clone(),
            "pose_grad": r.pose.clone(), "score": r.score.clone()}


def test_wave_equals_each_session_alone(G):
    sess = [make_session(G, *p) for p in SESSIONS]
    # every session alone: one fused iteration
    ref = []
    for s in sess:
        r, pose, adam, cs = fresh(G, s)
        r.track_step(s["g"], cs, s["trgb"], s["tdep"], pose, adam, wave=False)   # the separate calls
        torch.cuda.synchronize()
        r.check()
        ref.append((outputs(r), pose.clone()))
    # all sessions in one wave
    state = [fresh(G, s) for s in sess]
    jobs = [r.track_job(s["g"], cs, s["trgb"], s["tdep"], pose, adam) for s, (r, pose, adam, cs) in zip(sess, state)]
    G.gs_track_wave(None, jobs)
    torch.cuda.synchronize()
    state[0][0].check()
    for i, (s, (r, pose, adam, cs)) in enumerate(zip(sess, state)):
        out, pose_ref = ref[i]
        got = outputs(r)
        # binning, sort, ranges, order and the whole forward are the same
        # kernels on the same inputs: bit for bit
        for k in ("keys", "vals", "ranges", "order", "rgb", "depth", "t_final", "last_idx", "n_blended", "d_rgb"):
            assert torch.equal(got[k], out[k]), (i, k)
        assert abs(float(got["loss"]) - float(out["loss"])) <= 1e-6 * abs(float(out["loss"])), i
        # the backward adds with float atomics: equal to summation order
        for k in ("grad2d", "score"):
            a, b = got[k].double(), out[k].double()
            assert float((a - b).norm() / b.norm().clamp_min(1e-30)) <= 1e-5, (i, k)
        e = float((got["pose_grad"] - out["pose_grad"]).norm() / out["pose_grad"].norm())
        assert e <= 1e-5, (i, e)
        assert float((pose - pose_ref).abs().max()) <= 1e-5, i
        assert int(out["keys"].numel()) > 0


def test_waves_track_like_the_plain_loop(G):
    """Ten waves against ten fused iterations per session: the same pose
    trajectories (to the float32 summation order of the backward)."""
    sess = [make_session(G, *p) for p in SESSIONS[:4]]
    iters = 10
    ref = []
    for s in sess:
        r, pose, adam, cs = fresh(G, s)
        for _ in range(iters):
            r.track_step(s["g"], cs, s["trgb"], s["tdep"], pose, adam, wave=False)
        ref.append(pose.clone())
    state = [fresh(G, s) for s in sess]
    jobs = [r.track_job(s["g"], cs, s["trgb"], s["tdep"], pose, adam) for s, (r, pose, adam, cs) in zip(sess, state)]
    arr = (G.gs_track_job * len(jobs))(*jobs)
    for _ in range(iters):
        G.gs_track_wave(None, arr)
    torch.cuda.synchronize()
    for i, (r, pose, adam, cs) in enumerate(state):
        moved = float((ref[i] - G.pose_tensor(sess[i]["start"])).abs().max())
        assert moved > 1e-6, i
        assert float((pose - ref[i]).abs().max()) <= 1e-4 * max(1.0, moved * 1e3), (i, float((pose - ref[i]).abs().max()))


def test_wave_of_one_and_the_capacity_check(G):
    """A wave of one session equals its fused iteration; a wave whose key
    capacity is too small raises the capacity condition on the device."""
    s = make_session(G, *SESSIONS[0])
    r, pose, adam, cs = fresh(G, s)
    G.gs_track_wave(None, [r.track_job(s["g"], cs, s["trgb"], s["tdep"], pose, adam)])
    torch.cuda.synchronize()
    r.check()
    from paper_2510_06644_gb300.pipeline import Rasterizer
    small = Rasterizer(s["g"]["means"].shape[0], s["start"], capacity=1024)
    pose2 = G.pose_tensor(s["start"])
    adam2 = torch.zeros(13, device="cuda")
    G.gs_track_wave(None, [small.track_job(s["g"], G.camera(s["start"], pose=pose2), s["trgb"], s["tdep"], pose2,
                                           adam2)])
    code, _ = G.gs_status_poll(blocking=True)
    assert code == G.GS_ERR_CAPACITY
    G.gs_status_reset()
    torch.cuda.synchronize()
