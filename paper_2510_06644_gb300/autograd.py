"""gs_render as a torch.autograd.Function whose adjoint is the hand-written
backward of the C ABI (gs_render_bwd + gs_project_bwd).

    rgb, depth = gs_render(means, log_scales, quats, opacity_logit, colors,
                           pose_delta, cam, cfg=None, rec_dtype=GS_F32,
                           memory_budget=None)

* means [n,3], log_scales [n,3], quats [n,4], opacity_logit [n], colors [n,3]:
  float32 CUDA tensors (gradients flow to all of them).
* pose_delta [6] (rho, phi): a left perturbation applied to the camera pose,
  T_cw <- exp(pose_delta^) T_cw (exact SE(3) exponential, evaluated on the
  host).  Its gradient is the pose gradient of Sec. 2.2 Step 5, exact at
  pose_delta = 0 (the tracking use: the perturbation is folded into the pose
  after each step); away from 0 it omits the SE(3) left Jacobian.
* Forward intermediates -- 2D records, sorted lists, tile ranges and order,
  T_final and last index -- are stored for the backward when their size fits
  `memory_budget` bytes (None = always store); otherwise only the inputs are
  kept and the forward is recomputed inside the backward.
* Returns the planar image [3, Hs, Ws] and depth [Hs, Ws].

Buffers: rasterizers are pooled per (Gaussian count, sampled grid, record
type, device).  A forward borrows one (a stored one stays lent until its
backward), so renders of several views before one backward do not share
buffers.  The key capacity of a pooled rasterizer follows the key counts it
has seen (with headroom), so a forward launches without reading the count on
the host; only a rasterizer's first use counts its keys first.  The backward
synchronises once (its status check): a capacity overflow in the forward is
raised there (the forward's outputs were truncated) and the capacity grows
for the next call.  A forward whose inputs need no gradient checks itself.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import gs
from .pipeline import Rasterizer

PARAMS = ("means", "log_scales", "quats", "opacity_logit", "rgb")


def _skew(v):
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def apply_pose_delta(cam, delta):
    """Camera dict with T_cw replaced by exp(delta^) T_cw, delta = (rho, phi)."""
    d = np.asarray(delta, dtype=np.float64).reshape(6)
    rho, phi = d[:3], d[3:]
    th = float(np.linalg.norm(phi))
    K = _skew(phi)
    if th < 1e-8:
        Rd = np.eye(3) + K + 0.5 * K @ K
        V = np.eye(3) + 0.5 * K + K @ K / 6.0
    else:
        Rd = np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / th ** 2 * K @ K
        V = np.eye(3) + (1 - math.cos(th)) / th ** 2 * K + (th - math.sin(th)) / th ** 3 * K @ K
    c = dict(cam)
    c["R"] = Rd @ np.asarray(cam["R"], dtype=np.float64).reshape(3, 3)
    c["t"] = Rd @ np.asarray(cam["t"], dtype=np.float64).reshape(3) + V @ rho
    return c


def stored_bytes(n, n_keys, cam, rec_dtype=gs.GS_F32):
    """Device bytes the store mode keeps alive between forward and backward."""
    Ws, Hs, TX, TY = gs.grid(cam)
    rec = 4 * gs.SPLAT_WORDS[rec_dtype]
    return n * rec + 12 * n_keys + 8 * Hs * Ws + 12 * TX * TY


class _Pool:
    """Rasterizers per (n, sampled grid, record type, device), lent one
    caller at a time, each with the key capacity its past counts call for."""

    def __init__(self):
        self.free = {}

    @staticmethod
    def key(n, cam, rec_dtype, device):
        return (n, gs.grid(cam), int(cam.get("sx", 1)), int(cam.get("sy", 1)), rec_dtype, str(device))

    def take(self, n, cam, cfg, rec_dtype, device, g):
        k = self.key(n, cam, rec_dtype, device)
        lst = self.free.setdefault(k, [])
        if lst:
            r = lst.pop()
            r.cfg = cfg
            return r
        # a new rasterizer counts its keys once (one host read)
        cs = gs.camera(cam)
        probe = gs.gs_project(cfg, cs, g, rec_dtype)
        n_keys = int(gs.gs_bin_count(cs, probe, n, rec_dtype, cfg=cfg).item())
        r = Rasterizer(n, cam, cfg, rec_dtype, capacity=_headroom(n_keys), device=device)
        r.pool_key = k
        return r

    def give(self, r):
        self.free.setdefault(r.pool_key, []).append(r)


_POOL = _Pool()


def _headroom(n_keys):
    return int(n_keys * 1.25) + 4096


def _settle(rast):
    """The backward's one synchronisation: raise a capacity overflow of the
    forward (and grow the capacity for the next call), else keep the
    capacity in line with the count just seen."""
    code, _ = gs.gs_status_poll(blocking=True)
    n_keys = int(rast.n_keys.item())
    if code == gs.GS_ERR_CAPACITY or n_keys > rast.capacity:
        gs.gs_status_reset()
        _grow(rast, _headroom(n_keys))
        raise gs.GsError(gs.GS_ERR_CAPACITY, f"{n_keys} keys exceeded the capacity; the forward was truncated "
                                             f"(the capacity is now {rast.capacity}: render again)")
    if code != gs.GS_OK:
        raise gs.GsError(code, f"device status {code}")
    if n_keys > 0.9 * rast.capacity:
        _grow(rast, _headroom(n_keys))


def _grow(rast, cap):
    if cap <= rast.capacity:
        return
    rast.capacity = cap
    rast.keys = torch.empty(cap, dtype=torch.int64, device=rast.device)
    rast.vals = torch.empty(cap, dtype=torch.int32, device=rast.device)
    rast._ws_sort = None
    rast._ws_pb = None
    rast._bm = None


class GsRenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logit, colors, pose_delta, cam, cfg, rec_dtype,
                memory_budget, grad_on=True):
        g = {"means": means.detach().contiguous(), "log_scales": log_scales.detach().contiguous(),
             "quats": quats.detach().contiguous(), "opacity_logit": opacity_logit.detach().contiguous(),
             "rgb": colors.detach().contiguous()}
        cam_p = apply_pose_delta(cam, pose_delta.detach().double().cpu().numpy())
        n = int(g["means"].shape[0])
        cfg = cfg if cfg is not None else gs.default_config()
        cs = gs.camera(cam_p)
        rast = _POOL.take(n, cam_p, cfg, rec_dtype, means.device, g)
        img = rast.forward(g, cs)
        rgb, depth = img["rgb"].clone(), img["depth"].clone()
        # the store-mode footprint, from the capacity (no host read of the count)
        store = memory_budget is None or stored_bytes(n, rast.capacity, cam_p, rec_dtype) <= memory_budget
        ctx.store = store
        ctx.cam_p = cam_p
        ctx.cfg = cfg
        ctx.rec_dtype = rec_dtype
        if not grad_on:
            # no backward will run: check the forward here and lend the buffers out again
            try:
                _settle(rast)
            finally:
                _POOL.give(rast)
            ctx.rast = None
        else:
            ctx.rast = rast if store else None
            if not store:
                _POOL.give(rast)
        ctx.save_for_backward(*[g[k] for k in PARAMS])
        return rgb, depth

    @staticmethod
    def backward(ctx, d_rgb, d_depth):
        vals = ctx.saved_tensors
        g = dict(zip(PARAMS, vals))
        cs = gs.camera(ctx.cam_p)
        rast = ctx.rast
        if rast is None:  # recompute the forward intermediates
            n = int(g["means"].shape[0])
            rast = _POOL.take(n, ctx.cam_p, ctx.cfg, ctx.rec_dtype, g["means"].device, g)
            rast.forward(g, cs)
        ctx.rast = None
        try:
            d_rgb = torch.zeros_like(rast.img["rgb"]) if d_rgb is None else d_rgb.contiguous().float()
            d_depth = torch.zeros_like(rast.img["depth"]) if d_depth is None else d_depth.contiguous().float()
            need = ctx.needs_input_grad
            grads = {k: torch.empty_like(g[k]) for k in PARAMS}
            rast.backward(g, cs, d_rgb, d_depth, mode=gs.GS_MAP, grads=grads, want_pose=need[5], want_score=False)
            _settle(rast)
            pose_grad = rast.pose.float().clone() if need[5] else None
        finally:
            _POOL.give(rast)
        return (grads["means"], grads["log_scales"], grads["quats"], grads["opacity_logit"], grads["rgb"],
                pose_grad, None, None, None, None, None)


def gs_render(means, log_scales, quats, opacity_logit, colors, pose_delta, cam, cfg=None, rec_dtype=gs.GS_F32,
              memory_budget=None):
    grad_on = torch.is_grad_enabled() and any(
        t.requires_grad for t in (means, log_scales, quats, opacity_logit, colors, pose_delta))
    return GsRenderFn.apply(means, log_scales, quats, opacity_logit, colors, pose_delta, cam, cfg, rec_dtype,
                            memory_budget, grad_on)
