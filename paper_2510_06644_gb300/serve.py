"""Serving form: many concurrent SLAM sessions on one GPU.

Each session owns, on the device, its Gaussian map (the 3D parameters), the
map's Adam state, its camera pose and the pose's Adam state, and a queue of
RGB-D frames that arrive at `fps` Hz (Poisson).  A frame is 40 tracking
iterations (pose-only backward, Sec. 2.2) at the resolution the keyframe
schedule gives it (Sec. 4.2: keyframes at full resolution, the frames after a
keyframe at strides (4,4), (4,2), (2,2), ...), and every `kf_every`-th frame is
a keyframe that also runs one mapping iteration (per-Gaussian backward and an
Adam step of the map).  The work of one frame at one stride is captured once
per session as a CUDA graph ("frame program"): every kernel of the frame runs
back to back on the device with no host synchronisation.

Server(mode="batched") is continuous batching: sessions are admitted into
`slots` while the HBM budget allows (admission by the session's device
footprint), each admitted session gets its own stream, and whenever a
session has an arrived frame and no frame in flight the frame program is
launched on its stream, so frames of different sessions overlap on the GPU;
finished sessions release their slot and memory, which admits the next.
Server(mode="wave") batches inside the kernels: every tracking iteration of
every session with a frame in progress runs in one wave (gs_track_wave), a
set of launches whose grids span all those sessions; a session joins the
wave when its next frame has arrived and leaves it after the frame's 40th
iteration (its keyframe mapping iteration follows on the same stream).
Server(mode="plain") is the per-session sequential loop: one stream, frames
in arrival order, each frame run to completion before the next.

Latency of a frame = completion time (host observes its event) - arrival
time; throughput = frames / makespan.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np
import torch

from . import gs
from .pipeline import Rasterizer

PARAMS = ("means", "log_scales", "quats", "opacity_logit", "rgb")


@dataclasses.dataclass
class SessionSpec:
    sid: int
    n: int               # Gaussians in the map
    W: int
    H: int
    f: float             # focal length (fx = fy)
    n_frames: int
    seed: int
    fps: float = 30.0    # Poisson frame rate
    iters: int = 40      # tracking iterations per frame
    kf_every: int = 5    # keyframe (mapping) period


def stride_of(frame, kf_every, m=2):
    """(is_keyframe, sx, sy) of a frame under the Sec. 4.2 schedule."""
    k = (frame // kf_every) * kf_every
    if frame == k:
        return True, 1, 1
    sx, sy, _ = gs.gs_downsample(frame, k, False, m)
    return False, sx, sy


class Session:
    """Device-resident state and frame programs of one SLAM session."""

    def __init__(self, spec: SessionSpec, scene, true_cams, device="cuda", lr_pose=1e-3, lr_map=1e-4,
                 use_graphs=True):
        self.spec = spec
        self.device = torch.device(device)
        self.cfg = gs.default_config()
        self.g = {k: torch.from_numpy(np.ascontiguousarray(v)).to(self.device) for k, v in scene.items()}
        self.m = {k: torch.zeros_like(v) for k, v in self.g.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.g.items()}
        self.grads = {k: torch.zeros_like(v) for k, v in self.g.items()}
        self.map_state = torch.zeros(2, device=self.device)
        self.cams = true_cams
        c0 = true_cams[0]
        self.pose = gs.pose_tensor(c0, self.device)
        self.pose_adam = torch.zeros(13, device=self.device)
        self.lr_pose, self.lr_map = lr_pose, lr_map
        self.use_graphs = use_graphs
        # observations: full-resolution RGB-D rendered from the true poses
        self.targets = []
        n_keys = int(gs.gs_bin_count(gs.camera(c0), gs.gs_project(self.cfg, gs.camera(c0), self.g), spec.n,
                                     cfg=self.cfg).item())
        self.capacity = int(n_keys * 1.5) + 4096
        probe = Rasterizer(spec.n, c0, self.cfg, capacity=self.capacity, device=self.device)
        for cam in true_cams:
            img = probe.forward(self.g, cam)
            self.targets.append((img["rgb"].clone(), img["depth"].clone()))
        probe.check()
        del probe
        self.rast = {}      # (sx, sy) -> Rasterizer
        self.tgt = {}       # (sx, sy) -> (rgb, depth) work targets at that stride
        self.programs = {}  # (sx, sy, keyframe) -> CUDA graph
        self.frames_done = 0
        self.poses = []
        self.pose_log = torch.empty((spec.n_frames, 12), device=self.device)  # final pose of each frame

    # -- footprint ---------------------------------------------------------
    @staticmethod
    def footprint_bytes(spec: SessionSpec, keys_per_gaussian=4.0):
        """Device bytes of a session: map + Adam (3 x 56 B/G), gradients
        (56 B/G), four rasterizer instances (records, 2D gradients, scores,
        keys, sort scratch, blend masks: a word per pixel and run of 32 list
        entries, 32 B per key of capacity plus 1 KB per tile) and the frames'
        RGB-D targets."""
        n, P = spec.n, spec.W * spec.H
        cap = int(keys_per_gaussian * n * 1.5) + 4096
        per_rast = n * (48 + 48 + 8) + cap * (8 + 4 + 8 + 32) + P * 44
        return n * 56 * 4 + 4 * per_rast + spec.n_frames * P * 16

    # -- frame programs ----------------------------------------------------
    def _rast(self, sx, sy):
        key = (sx, sy)
        if key not in self.rast:
            cam = dict(self.cams[0], sx=sx, sy=sy)
            self.rast[key] = Rasterizer(self.spec.n, cam, self.cfg, capacity=self.capacity, device=self.device)
            Ws, Hs, _, _ = gs.grid(cam)
            self.tgt[key] = (torch.empty((3, Hs, Ws), device=self.device),
                             torch.empty((Hs, Ws), device=self.device))
        return self.rast[key], self.tgt[key]

    def _frame_body(self, sx, sy, keyframe):
        """Enqueue one frame's kernels on the current stream (graph-capturable)."""
        r, (trgb, tdep) = self._rast(sx, sy)
        cam = gs.camera(dict(self.cams[0], sx=sx, sy=sy), pose=self.pose)
        for _ in range(self.spec.iters):
            r.track_step(self.g, cam, trgb, tdep, self.pose, self.pose_adam, self.lr_pose, self.lr_pose)
        if keyframe:
            r.forward(self.g, cam)
            r.loss_grad(cam, trgb, tdep)
            r.backward(self.g, cam, r.dimg["d_rgb"], r.dimg["d_depth"], gs.GS_MAP, grads=self.grads,
                       want_pose=False, want_score=True)
            gs.gs_adam([self.g[k] for k in PARAMS], [self.grads[k] for k in PARAMS], [self.m[k] for k in PARAMS],
                       [self.v[k] for k in PARAMS], self.map_state, lr=self.lr_map)

    def prepare(self):
        """Builds (and captures) the frame programs of every stride used."""
        for fr in range(self.spec.n_frames):
            kf, sx, sy = stride_of(fr, self.spec.kf_every)
            key = (sx, sy, kf)
            if key in self.programs:
                continue
            self._rast(sx, sy)
            if not self.use_graphs:
                self.programs[key] = None
                continue
            # warm up outside capture (static initialisation), then restore state
            snap = self.snapshot()
            s = torch.cuda.Stream(device=self.device)
            s.wait_stream(torch.cuda.current_stream(self.device))
            with torch.cuda.stream(s):
                self._frame_body(sx, sy, kf)
            torch.cuda.current_stream(self.device).wait_stream(s)
            torch.cuda.synchronize(self.device)
            self.restore(snap)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, capture_error_mode="relaxed"):
                self._frame_body(sx, sy, kf)
            self.programs[key] = graph
        torch.cuda.synchronize(self.device)
        for r in self.rast.values():
            r.check()

    def launch_frame(self, fr, stream):
        """Enqueue frame `fr` on `stream`; returns the completion event."""
        kf, sx, sy = stride_of(fr, self.spec.kf_every)
        trgb_full, tdep_full = self.targets[fr]
        with torch.cuda.stream(stream):
            _, (trgb, tdep) = self._rast(sx, sy)
            k = (fr // self.spec.kf_every) * self.spec.kf_every
            # Sec. 4.2: gather the observation at the frame's sampled pixels
            gs.gs_downsample(fr, k, kf, 2, trgb_full, out=trgb, stream=stream)
            gs.gs_downsample(fr, k, kf, 2, tdep_full, out=tdep, stream=stream)
            prog = self.programs.get((sx, sy, kf))
            if prog is not None:
                prog.replay()
            else:
                self._frame_body(sx, sy, kf)
            ev = torch.cuda.Event()
            ev.record(stream)
        return ev

    # -- waves -------------------------------------------------------------
    def wave_job(self, sx, sy):
        """The gs_track_job of one tracking iteration at stride (sx, sy)
        (cached: it points at this session's device buffers)."""
        if not hasattr(self, "_jobs"):
            self._jobs = {}
        key = (sx, sy)
        if key not in self._jobs:
            r, (trgb, tdep) = self._rast(sx, sy)
            cam = gs.camera(dict(self.cams[0], sx=sx, sy=sy), pose=self.pose)
            self._jobs[key] = r.track_job(self.g, cam, trgb, tdep, self.pose, self.pose_adam, self.lr_pose,
                                          self.lr_pose)
        return self._jobs[key]

    def start_frame(self, fr, stream):
        """Gathers frame fr's observation at its stride (Sec. 4.2) on
        `stream`; returns (keyframe, sx, sy)."""
        kf, sx, sy = stride_of(fr, self.spec.kf_every)
        trgb_full, tdep_full = self.targets[fr]
        _, (trgb, tdep) = self._rast(sx, sy)
        k = (fr // self.spec.kf_every) * self.spec.kf_every
        gs.gs_downsample(fr, k, kf, 2, trgb_full, out=trgb, stream=stream)
        gs.gs_downsample(fr, k, kf, 2, tdep_full, out=tdep, stream=stream)
        return kf, sx, sy

    def finish_frame(self, fr, keyframe, stream):
        """The keyframe's mapping iteration (if any) on `stream`, then a copy
        of the frame's final pose (later waves may move the pose before the
        host looks); returns the frame's completion event."""
        with torch.cuda.stream(stream):
            if keyframe:
                r, (trgb, tdep) = self._rast(1, 1)
                cam = gs.camera(dict(self.cams[0], sx=1, sy=1), pose=self.pose)
                r.forward(self.g, cam)
                r.loss_grad(cam, trgb, tdep)
                r.backward(self.g, cam, r.dimg["d_rgb"], r.dimg["d_depth"], gs.GS_MAP, grads=self.grads,
                           want_pose=False, want_score=True)
                gs.gs_adam([self.g[k] for k in PARAMS], [self.grads[k] for k in PARAMS],
                           [self.m[k] for k in PARAMS], [self.v[k] for k in PARAMS], self.map_state, lr=self.lr_map)
            self.pose_log[fr].copy_(self.pose)
            ev = torch.cuda.Event()
            ev.record(stream)
        return ev

    # -- state snapshots (checkpoint / resume) ------------------------------
    def snapshot(self):
        st = {"pose": self.pose.clone(), "pose_adam": self.pose_adam.clone(), "map_state": self.map_state.clone()}
        for k in PARAMS:
            st["g_" + k] = self.g[k].clone()
            st["m_" + k] = self.m[k].clone()
            st["v_" + k] = self.v[k].clone()
        return st

    def restore(self, st):
        self.pose.copy_(st["pose"])
        self.pose_adam.copy_(st["pose_adam"])
        self.map_state.copy_(st["map_state"])
        for k in PARAMS:
            self.g[k].copy_(st["g_" + k])
            self.m[k].copy_(st["m_" + k])
            self.v[k].copy_(st["v_" + k])


def make_session_specs(n_sessions, seed=5000, n_frames=10, n_range=(50_000, 1_500_000),
                       resolutions=((320, 240), (640, 480), (1200, 680)), iters=40, kf_every=5, fps=30.0):
    """Map sizes log-uniform in n_range, resolutions drawn uniformly."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for i in range(n_sessions):
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        W, H = resolutions[int(rng.integers(0, len(resolutions)))]
        specs.append(SessionSpec(i, n, W, H, 525.0 * W / 640.0, n_frames, seed + 17 * i + 1, fps, iters, kf_every))
    return specs


def session_inputs(spec: SessionSpec):
    """Synthetic map and true trajectory of a session: a surface-sampled
    scene and a camera moving ~1 cm and ~0.3 deg per frame."""
    from synth import scenes as S
    scene = S.surface_scene(spec.n, spec.seed)
    rng = np.random.Generator(np.random.PCG64(spec.seed + 1))
    cams = [S.camera(spec.W, spec.H, spec.f)]
    axis = rng.normal(size=3)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    for _ in range(1, spec.n_frames):
        c = S.perturbed_pose(cams[-1], seed=int(rng.integers(1 << 30)), trans=0.01, rot_deg=0.3)
        cams.append(c)
    return scene, cams


class Admission:
    """HBM-budget admission into a bounded number of slots (host logic)."""

    def __init__(self, budget_bytes, slots):
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.used = 0
        self.active = {}

    def try_admit(self, sid, nbytes):
        if len(self.active) >= self.slots or self.used + nbytes > self.budget:
            return False
        self.active[sid] = nbytes
        self.used += nbytes
        return True

    def release(self, sid):
        self.used -= self.active.pop(sid)


class Server:
    def __init__(self, sessions, arrivals, mode="batched", slots=16, budget_bytes=150 << 30, device="cuda",
                 groups=4):
        """sessions: prepared Session objects; arrivals[sid] = frame arrival
        times (seconds from the start); groups: wave groups (mode "wave")."""
        self.sessions = {s.spec.sid: s for s in sessions}
        self.arrivals = arrivals
        self.mode = mode
        self.groups = groups
        self.adm = Admission(budget_bytes, slots if mode in ("batched", "wave") else 1)
        self.device = torch.device(device)
        self.latency = []   # (sid, frame, seconds)

    def run(self):
        if self.mode == "wave":
            return self.run_waves()
        order = sorted(self.sessions, key=lambda sid: self.arrivals[sid][0])
        waiting = list(order)
        done_frames = {sid: 0 for sid in self.sessions}
        inflight = {}       # sid -> (frame, event)
        streams = {}
        plain_stream = torch.cuda.Stream(device=self.device)
        t0 = time.perf_counter()
        total = sum(s.spec.n_frames for s in self.sessions.values())
        completed = 0
        while completed < total:
            now = time.perf_counter() - t0
            # admission
            while waiting:
                sid = waiting[0]
                if self.arrivals[sid][0] > now:
                    break
                nb = Session.footprint_bytes(self.sessions[sid].spec)
                if not self.adm.try_admit(sid, nb):
                    break
                waiting.pop(0)
                streams[sid] = torch.cuda.Stream(device=self.device) if self.mode == "batched" else plain_stream
            # dispatch
            if self.mode == "plain":
                if not inflight:
                    # oldest arrived frame among admitted sessions
                    cand = [(self.arrivals[sid][done_frames[sid]], sid) for sid in self.adm.active
                            if done_frames[sid] < self.sessions[sid].spec.n_frames
                            and self.arrivals[sid][done_frames[sid]] <= now]
                    if cand:
                        _, sid = min(cand)
                        fr = done_frames[sid]
                        inflight[sid] = (fr, self.sessions[sid].launch_frame(fr, streams[sid]))
            else:
                for sid in list(self.adm.active):
                    if sid in inflight:
                        continue
                    fr = done_frames[sid]
                    if fr < self.sessions[sid].spec.n_frames and self.arrivals[sid][fr] <= now:
                        inflight[sid] = (fr, self.sessions[sid].launch_frame(fr, streams[sid]))
            # completion
            progressed = False
            for sid, (fr, ev) in list(inflight.items()):
                if ev.query():
                    t = time.perf_counter() - t0
                    self.latency.append((sid, fr, t - self.arrivals[sid][fr]))
                    self.sessions[sid].poses.append(self.sessions[sid].pose.detach().cpu().numpy().copy())
                    del inflight[sid]
                    done_frames[sid] += 1
                    completed += 1
                    progressed = True
                    if done_frames[sid] == self.sessions[sid].spec.n_frames:
                        self.adm.release(sid)
            if not progressed:
                time.sleep(20e-6)
        self.makespan = time.perf_counter() - t0
        return self.stats()

    def run_waves(self, depth=3):
        """Continuous batching inside the kernels: each wave is one tracking
        iteration of every session of a group with a frame in progress (one
        gs_track_wave call); sessions join at frame boundaries as their frames
        arrive and slots and memory free up.  Sessions are dealt to
        `self.groups` groups (the lightest group by map size at admission),
        each with its own stream, so one group's stage boundaries overlap
        with another's work.  At most `depth` waves per group are queued
        ahead of the GPU, so a frame that arrives joins within a few waves."""
        order = sorted(self.sessions, key=lambda sid: self.arrivals[sid][0])
        waiting = list(order)
        done_frames = {sid: 0 for sid in self.sessions}
        started = {sid: 0 for sid in self.sessions}
        progress = {}      # sid -> [frame, iteration, keyframe, sx, sy]
        pending = []       # (sid, frame, completion event)
        ng = max(1, int(self.groups))
        queued = [[] for _ in range(ng)]   # events of each group's waves in flight
        streams = [torch.cuda.Stream(device=self.device) for _ in range(ng)]
        group = {}         # sid -> group
        load = [0] * ng
        weight = {sid: s.spec.n for sid, s in self.sessions.items()}
        t0 = time.perf_counter()
        total = sum(s.spec.n_frames for s in self.sessions.values())
        completed = 0
        while completed < total:
            now = time.perf_counter() - t0
            while waiting:
                sid = waiting[0]
                if self.arrivals[sid][0] > now:
                    break
                if not self.adm.try_admit(sid, Session.footprint_bytes(self.sessions[sid].spec)):
                    break
                waiting.pop(0)
                gi = min(range(ng), key=lambda q: load[q])
                group[sid] = gi
                load[gi] += weight[sid]
            # sessions whose next frame has arrived join their group's wave
            for sid in self.adm.active:
                s = self.sessions[sid]
                fr = started[sid]
                if sid not in progress and fr < s.spec.n_frames and self.arrivals[sid][fr] <= now:
                    kf, sx, sy = s.start_frame(fr, streams[group[sid]])
                    progress[sid] = [fr, 0, kf, sx, sy]
                    started[sid] += 1
            # completions
            progressed = False
            for item in list(pending):
                sid, fr, ev = item
                if ev.query():
                    self.latency.append((sid, fr, time.perf_counter() - t0 - self.arrivals[sid][fr]))
                    self.sessions[sid].poses.append(self.sessions[sid].pose_log[fr].cpu().numpy().copy())
                    pending.remove(item)
                    done_frames[sid] += 1
                    completed += 1
                    progressed = True
                    if done_frames[sid] == self.sessions[sid].spec.n_frames:
                        self.adm.release(sid)
                        load[group.pop(sid)] -= weight[sid]
            for gi in range(ng):
                queued[gi] = [e for e in queued[gi] if not e.query()]
                sids = sorted((q for q in progress if group[q] == gi), key=lambda q: -weight[q])
                if not sids or len(queued[gi]) >= depth:
                    continue
                st_ = streams[gi]
                jobs = [self.sessions[q].wave_job(progress[q][3], progress[q][4]) for q in sids]
                gs.gs_track_wave(self.sessions[sids[0]].cfg, jobs, stream=st_)
                ev = torch.cuda.Event()
                ev.record(st_)
                queued[gi].append(ev)
                for q in sids:
                    st = progress[q]
                    st[1] += 1
                    if st[1] == self.sessions[q].spec.iters:
                        pending.append((q, st[0], self.sessions[q].finish_frame(st[0], st[2], st_)))
                        del progress[q]
                progressed = True
            if not progressed:
                time.sleep(20e-6)
        self.makespan = time.perf_counter() - t0
        return self.stats()

    def stats(self):
        lat = np.array([x[2] for x in self.latency]) * 1e3
        return {"frames": int(lat.size), "makespan_s": self.makespan, "frames_per_s": lat.size / self.makespan,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean())}


def poisson_arrivals(specs, seed=7):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {}
    for s in specs:
        gaps = rng.exponential(1.0 / s.fps, s.n_frames)
        gaps[0] = 0.0
        out[s.sid] = np.cumsum(gaps).tolist()
    return out
