"""Host logic (no GPU) of the serving form -- admission by HBM budget into
slots, the keyframe/stride schedule of frames, Poisson arrivals -- and of
the rasterizer's buffers and list-reuse policy."""
import numpy as np
import pytest


def test_admission_by_budget_and_slots():
    from paper_2510_06644_gb300.serve import Admission
    a = Admission(budget_bytes=100, slots=2)
    assert a.try_admit(0, 60)
    assert not a.try_admit(1, 50)        # over budget
    assert a.try_admit(2, 40)
    assert not a.try_admit(3, 1)         # no slot
    a.release(0)
    assert a.used == 40
    assert a.try_admit(1, 50)
    assert a.used == 90 and set(a.active) == {1, 2}


def test_frame_schedule_follows_keyframes_and_downsampling():
    pytest.importorskip("torch")
    from paper_2510_06644_gb300 import build
    build.build()
    from paper_2510_06644_gb300.serve import stride_of
    got = [stride_of(f, 5) for f in range(11)]
    assert got[0] == (True, 1, 1) and got[5] == (True, 1, 1) and got[10] == (True, 1, 1)
    assert [g[1:] for g in got[1:5]] == [(4, 4), (4, 2), (2, 2), (2, 2)]


def test_poisson_arrivals_and_specs():
    from paper_2510_06644_gb300.serve import make_session_specs, poisson_arrivals
    specs = make_session_specs(16, n_frames=50)
    ns = np.array([s.n for s in specs])
    assert ns.min() >= 50_000 and ns.max() <= 1_500_000
    assert {(s.W, s.H) for s in specs} <= {(320, 240), (640, 480), (1200, 680)}
    arr = poisson_arrivals(specs)
    gaps = np.concatenate([np.diff(arr[s.sid]) for s in specs])
    assert abs(gaps.mean() - 1 / 30) < 0.2 / 30
    assert all(arr[s.sid][0] == 0.0 for s in specs)


def test_footprint_grows_with_map_and_resolution():
    from paper_2510_06644_gb300.serve import Session, SessionSpec
    a = Session.footprint_bytes(SessionSpec(0, 50_000, 320, 240, 262.5, 10, 1))
    b = Session.footprint_bytes(SessionSpec(0, 1_500_000, 320, 240, 262.5, 10, 1))
    c = Session.footprint_bytes(SessionSpec(0, 50_000, 1200, 680, 984.0, 10, 1))
    assert a < b and a < c
    # 16 of the largest sessions fit the 150 GB budget of the serving workload
    assert 16 * Session.footprint_bytes(SessionSpec(0, 1_500_000, 1200, 680, 984.0, 10, 1)) < 150 << 30


def test_rasterizer_result_buffer_holds_pose_gradient_and_loss():
    """The rasterizer's pose gradient and loss are views of one 7-double
    buffer (read back in one copy), also after the grid changes."""
    import torch
    from paper_2510_06644_gb300.pipeline import Rasterizer
    from synth import scenes as S
    cam = S.camera(96, 72, 100.0)
    r = Rasterizer(100, cam, device="cpu")
    for c in (cam, dict(cam, sx=2, sy=2)):
        r.set_grid(c)
        assert r.pose.data_ptr() == r.result.data_ptr() and r.pose.numel() == 6
        assert r.dimg["loss"].data_ptr() == r.result.data_ptr() + 6 * 8 and r.dimg["loss"].numel() == 1
        assert r.result.dtype == torch.float64


def test_list_reuse_rebins_at_each_interval_and_follows_the_interval_rule(monkeypatch):
    """ListReuse (Sec. 4.1, Obs. 6) with its GPU calls replaced by host
    fakes: the first iteration of every interval bins; when an interval of K
    iterations ends, the change ratio compares the records the lists were
    built from with the records at the current pose, and the library's
    gs_next_interval (checked against the oracle's rule elsewhere) sets the
    next K: scripted ratios 0.10, 0.01, 0.01, 0.20 from K0 = 5 give
    intervals 5, 2, 4, 8 and then 4."""
    import torch
    from paper_2510_06644_gb300 import build, gs
    from paper_2510_06644_gb300.pipeline import ListReuse
    build.build()
    cfg = gs.default_config()
    assert int(cfg.k0) == 5 and abs(float(cfg.change_thr) - 0.05) < 1e-7

    class FakeRast:
        def __init__(self):
            self.cfg, self.n, self.rec_dtype, self.device = cfg, 4, gs.GS_F32, torch.device("cpu")
            self.splats = torch.zeros(4, 12)
            self.rebins = []

        def track_step(self, g, cam, trgb, tdep, pose, adam, lr_t, lr_r, rebin=True):
            self.rebins.append(rebin)
            self.splats.fill_(float(len(self.rebins)))   # this iteration's records

    ratios = iter([0.10, 0.01, 0.01, 0.20])
    seen = []

    def fake_project(cfg_, cam, g, rec_dtype, out):
        out.fill_(-1.0)   # the records at the current pose

    def fake_change_ratio(cam, a, b, n, rec_dtype=gs.GS_F32, out=None, stream=None, cfg=None):
        seen.append((float(a[0, 0]), float(b[0, 0])))
        out.fill_(next(ratios))
        return out

    monkeypatch.setattr(gs, "gs_project", fake_project)
    monkeypatch.setattr(gs, "gs_change_ratio", fake_change_ratio)
    r = FakeRast()
    lr = ListReuse(r, g=None)
    for _ in range(5 + 2 + 4 + 8):
        lr.step(gs.gs_camera(), None, None, None, None)
    starts = [0, 5, 7, 11]
    assert r.rebins == [i in starts for i in range(19)]
    assert [k for k, _ in lr.intervals] == [5, 2, 4, 8]
    np.testing.assert_allclose([x for _, x in lr.intervals], [0.10, 0.01, 0.01, 0.20], rtol=1e-6)
    assert lr.K == 4 and lr.i == 0
    # each ratio: the records binned at the interval's first iteration against the current ones
    assert seen == [(s + 1.0, -1.0) for s in starts]


def _fake_server_env(monkeypatch, n_sessions=5, n_frames=3, iters=4, weights=(5, 1, 4, 2, 3), polls=3):
    """Sessions, CUDA streams/events and the clock replaced by host fakes: an
    event completes at its `polls`-th query, the clock advances 0.1 ms per
    read (and by the slept time), gs_track_wave is recorded.  Frames of
    session s arrive at 4 ms s + 20 ms i.  Returns (sessions, arrivals, env)
    with env.log (launch / start / finish entries with the serving clock),
    env.waves ((jobs, stream index, waves pending on that stream)) and
    env.streams (stream indices in creation order)."""
    import types
    import torch
    from paper_2510_06644_gb300 import gs, serve
    from paper_2510_06644_gb300.serve import SessionSpec

    env = types.SimpleNamespace(log=[], waves=[], streams=[], t=1000.0, t0=None, inflight=0, max_inflight=0)

    def perf_counter():
        env.t += 1e-4
        if env.t0 is None:
            env.t0 = env.t
        return env.t

    def sleep(dt):
        env.t += dt

    monkeypatch.setattr(serve, "time", types.SimpleNamespace(perf_counter=perf_counter, sleep=sleep))

    def now():
        return env.t - env.t0

    class FakeStream:
        def __init__(self, device=None):
            self.idx = len(env.streams)
            self.pending = []
            env.streams.append(self.idx)

    class FakeEvent:
        def __init__(self):
            self.left, self.stream = polls, None

        def record(self, stream=None):
            self.stream = stream
            if stream is not None:
                stream.pending.append(self)

        def query(self):
            self.left -= 1
            if self.left == 0:
                if self.stream is not None and self in self.stream.pending:
                    self.stream.pending.remove(self)
                if getattr(self, "frame", False):
                    env.inflight -= 1
            return self.left <= 0

    class FakeSession:
        def __init__(self, sid, n):
            self.spec = SessionSpec(sid=sid, n=n * 1000, W=64, H=48, f=60.0, n_frames=n_frames, seed=sid,
                                    iters=iters, kf_every=2)
            self.cfg = None
            self.pose = torch.zeros(12)
            self.pose_log = torch.zeros(n_frames, 12)
            self.poses = []

        def launch_frame(self, fr, stream):
            env.log.append(("launch", self.spec.sid, fr, now(), stream.idx))
            ev = FakeEvent()
            ev.record(stream)
            ev.frame = True
            env.inflight += 1
            env.max_inflight = max(env.max_inflight, env.inflight)
            return ev

        def start_frame(self, fr, stream):
            env.log.append(("start", self.spec.sid, fr, now(), stream.idx))
            return fr % 2 == 0, 1, 1

        def wave_job(self, sx, sy):
            return self.spec.sid

        def finish_frame(self, fr, keyframe, stream):
            env.log.append(("finish", self.spec.sid, fr, keyframe))
            return FakeEvent()

    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(gs, "gs_track_wave",
                        lambda cfg, jobs, stream=None: env.waves.append((list(jobs), stream.idx, len(stream.pending))))
    sessions = [FakeSession(i, w) for i, w in enumerate(weights[:n_sessions])]
    arrivals = {s.spec.sid: [0.004 * s.spec.sid + 0.020 * i for i in range(n_frames)] for s in sessions}
    return sessions, arrivals, env


def _check_arrivals_and_latency(srv, arrivals, env, kind):
    """No frame starts before it arrives; every latency lies in [0, makespan]
    and the makespan within the serving clock's span."""
    for e in env.log:
        if e[0] == kind:
            assert e[3] >= arrivals[e[1]][e[2]], e
    lat = [x for _, _, x in srv.latency]
    assert min(lat) >= 0 and max(lat) <= srv.makespan <= env.t - env.t0


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_server_loops_complete_every_frame_in_order(monkeypatch, mode):
    """The plain and stream-batched loops with fake sessions: every frame of
    every session completes once, in frame order per session, never before
    it arrives; the plain loop runs one frame at a time on one stream, the
    batched one admits up to `slots` sessions at once (never more), each on
    its own stream, with frames of different sessions in flight together."""
    from paper_2510_06644_gb300.serve import Server
    # batched: a frame takes about 100 polls x 0.12 ms, longer than the 4 ms
    # between sessions' arrivals and shorter than the 20 ms between a
    # session's frames; plain: a few polls
    sessions, arrivals, env = _fake_server_env(monkeypatch, polls=3 if mode == "plain" else 100)
    srv = Server(sessions, arrivals, mode=mode, slots=3, budget_bytes=1 << 50, device="cpu")
    st = srv.run()
    assert st["frames"] == 15
    log = env.log
    for s in sessions:
        assert [e[2] for e in log if e[1] == s.spec.sid] == [0, 1, 2]
        assert [fr for sid, fr, _ in srv.latency if sid == s.spec.sid] == [0, 1, 2]
        assert len(s.poses) == 3
    _check_arrivals_and_latency(srv, arrivals, env, "launch")
    # at most `slots` sessions in progress (one in the plain loop)
    first, last = {}, {}
    for i, e in enumerate(log):
        first.setdefault(e[1], i)
        last[e[1]] = i
    for i in range(len(log)):
        live = sum(1 for sid in first if first[sid] <= i <= last[sid])
        assert live <= (1 if mode == "plain" else 3)
    assert [e[1] for e in log if e[2] == 0] == sorted(first, key=lambda q: arrivals[q][0])
    stream_of = {e[1]: e[4] for e in log}
    if mode == "plain":
        assert env.max_inflight == 1 and len(set(stream_of.values())) == 1
    else:
        assert env.max_inflight >= 2 and len(set(stream_of.values())) == len(sessions)


def test_server_waves_group_sessions_and_run_every_iteration(monkeypatch):
    """The wave loop with fake sessions: sessions are dealt at admission to
    the lightest of two groups by map size; every wave holds sessions of one
    group only, on that group's stream (the groups' streams are created in
    group order), heaviest first, with fewer than `depth` = 3 waves of the
    group pending; each frame starts no earlier than it arrives and is in
    exactly `iters` waves, and a keyframe's mapping step follows its frame's
    last wave."""
    from paper_2510_06644_gb300.serve import Server
    sessions, arrivals, env = _fake_server_env(monkeypatch, weights=(5, 1, 4, 2, 3), polls=6)
    weights = {s.spec.sid: s.spec.n for s in sessions}
    # all five arrive within 16 ms: dealt in arrival order
    srv = Server(sessions, arrivals, mode="wave", slots=8, budget_bytes=1 << 50, device="cpu", groups=2)
    assert srv.run()["frames"] == 15
    load, want = [0, 0], {}
    for sid in sorted(weights, key=lambda q: arrivals[q][0]):
        gi = min(range(2), key=lambda q: load[q])
        want[sid] = gi
        load[gi] += weights[sid]
    group_stream = env.streams[:2]
    assert max(p for _, _, p in env.waves) == 2   # the queue reaches the depth limit
    for jobs, stream, pending in env.waves:
        assert jobs == sorted(jobs, key=lambda q: -weights[q])
        assert pending < 3
        for sid in jobs:
            assert stream == group_stream[want[sid]]
    for e in env.log:
        if e[0] == "start":
            assert e[4] == group_stream[want[e[1]]]
    _check_arrivals_and_latency(srv, arrivals, env, "start")
    for s in sessions:
        sid = s.spec.sid
        assert sum(sid in jobs for jobs, _, _ in env.waves) == 3 * 4
        fin = [e for e in env.log if e[0] == "finish" and e[1] == sid]
        assert [(e[2], e[3]) for e in fin] == [(0, True), (1, False), (2, True)]
