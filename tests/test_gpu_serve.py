"""Serving form on the GPU: continuous batching of several SLAM sessions.
Each session's result is the same alone and in the mix (within the
nondeterminism of float atomics in the backward), every frame is served, and
a snapshot restores a session's state for an identical continuation."""
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


def test_result_same_alone_and_in_the_mix(SV):
    specs = small_specs(SV)
    arr = SV.poisson_arrivals(specs, seed=3)
    alone = build_sessions(SV, specs[:1])
    SV.Server(alone, {0: arr[0]}, mode="batched", slots=4).run()
    mix = build_sessions(SV, specs)
    st = SV.Server(mix, arr, mode="batched", slots=4).run()
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
