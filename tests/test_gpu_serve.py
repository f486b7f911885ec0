"""Serving form on the GPU: continuous batching of several SLAM sessions,
by streams (mode "batched") and inside the kernels (mode "wave": launches
whose grids span every session).  Each session's result is the same alone
and in the mix (within the nondeterminism of float atomics in the
backward), every frame is served, and a snapshot restores a session's state
for an identical continuation."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def SV():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_06644_gb300 import build
    build.build()
    from paper_2510_06644_gb300 import serve
    return serve


def small_specs(SV, k=3, frames=6, iters=10):
    specs = SV.make_session_specs(k, seed=900, n_frames=frames, n_range=(20_000, 60_000),
                                  resolutions=((160, 120), (320, 240)), iters=iters, fps=200.0)
    return specs


def build_sessions(SV, specs, use_graphs=True):
    out = []
    for sp in specs:
        scene, cams = SV.session_inputs(sp)
        s = SV.Session(sp, scene, cams, use_graphs=use_graphs)
        s.prepare()
        out.append(s)
    return out


@pytest.mark.parametrize("mode", ["batched", "wave"])
def test_result_same_alone_and_in_the_mix(SV, mode):
    specs = small_specs(SV)
    arr = SV.poisson_arrivals(specs, seed=3)
    alone = build_sessions(SV, specs[:1])
    SV.Server(alone, {0: arr[0]}, mode="plain").run()
    mix = build_sessions(SV, specs)
    st = SV.Server(mix, arr, mode=mode, slots=4).run()
    assert st["frames"] == sum(s.n_frames for s in specs)
    a = np.array(alone[0].poses)
    b = np.array(mix[0].poses)
    assert a.shape == b.shape == (specs[0].n_frames, 12)
    # the pose moved, and it moved the same way alone and in the mix
    assert np.abs(a[-1] - a[0]).max() > 1e-4
    assert np.abs(a - b).max() <= 1e-4, np.abs(a - b).max()
    for k in SV.PARAMS:
        ga, gb = alone[0].g[k].double(), mix[0].g[k].double()
        assert float((ga - gb).norm() / ga.norm()) <= 1e-4, k


def test_plain_loop_serves_every_frame_in_arrival_order(SV):
    specs = small_specs(SV, k=2, frames=4, iters=4)
    arr = SV.poisson_arrivals(specs, seed=4)
    sess = build_sessions(SV, specs)
    srv = SV.Server(sess, arr, mode="plain")
    st = srv.run()
    assert st["frames"] == 8 and st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]
    per = {}
    for sid, fr, lat in srv.latency:
        per.setdefault(sid, []).append(fr)
        assert lat >= 0
    assert all(v == sorted(v) for v in per.values())


def test_admission_waits_for_memory(SV):
    specs = small_specs(SV, k=3, frames=3, iters=4)
    arr = SV.poisson_arrivals(specs, seed=5)
    sess = build_sessions(SV, specs)
    biggest = max(SV.Session.footprint_bytes(s) for s in specs)
    srv = SV.Server(sess, arr, mode="batched", slots=16, budget_bytes=int(biggest * 1.5))
    st = srv.run()
    assert st["frames"] == 9
    assert srv.adm.used == 0 and not srv.adm.active


def test_snapshot_restore_continues_identically(SV):
    specs = small_specs(SV, k=1, frames=6, iters=8)
    (s,) = build_sessions(SV, specs)
    stream = torch.cuda.Stream()
    for fr in range(3):
        s.launch_frame(fr, stream).synchronize()
    snap = s.snapshot()
    for fr in range(3, 6):
        s.launch_frame(fr, stream).synchronize()
    first = s.pose.cpu().numpy().copy()
    s.restore(snap)
    for fr in range(3, 6):
        s.launch_frame(fr, stream).synchronize()
    second = s.pose.cpu().numpy().copy()
    assert np.abs(first - second).max() <= 1e-5


def test_waves_serve_every_frame_with_sessions_joining_and_leaving(SV):
    """Sessions of different sizes, resolutions and frame counts arrive at
    different times: every frame is served once, in order per session, and
    the slots and memory are all released at the end."""
    specs = SV.make_session_specs(4, seed=910, n_frames=5, n_range=(5_000, 40_000),
                                  resolutions=((160, 120), (320, 240), (200, 120)), iters=6, fps=60.0)
    specs[1].n_frames = 3
    arr = SV.poisson_arrivals(specs, seed=6)
    arr[2] = [t + 0.05 for t in arr[2]]   # joins late
    sess = build_sessions(SV, specs, use_graphs=False)
    srv = SV.Server(sess, arr, mode="wave", slots=3)
    st = srv.run()
    assert st["frames"] == sum(s.n_frames for s in specs)
    per = {}
    for sid, fr, lat in srv.latency:
        per.setdefault(sid, []).append(fr)
        assert lat >= 0
    assert all(v == list(range(specs[sid].n_frames)) for sid, v in per.items())
    assert srv.adm.used == 0 and not srv.adm.active
    for s in sess:
        assert np.all(np.isfinite(np.array(s.poses)))
