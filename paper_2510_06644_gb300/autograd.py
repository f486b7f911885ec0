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


class GsRenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logit, colors, pose_delta, cam, cfg, rec_dtype,
                memory_budget):
        g = {"means": means.detach().contiguous(), "log_scales": log_scales.detach().contiguous(),
             "quats": quats.detach().contiguous(), "opacity_logit": opacity_logit.detach().contiguous(),
             "rgb": colors.detach().contiguous()}
        cam_p = apply_pose_delta(cam, pose_delta.detach().double().cpu().numpy())
        n = int(g["means"].shape[0])
        cfg = cfg if cfg is not None else gs.default_config()
        cs = gs.camera(cam_p)
        probe = gs.gs_project(cfg, cs, g, rec_dtype)
        n_keys = int(gs.gs_bin_count(cs, probe, n, rec_dtype, cfg=cfg).item())
        rast = Rasterizer(n, cam_p, cfg, rec_dtype, capacity=max(n_keys, 1), device=means.device)
        img = rast.forward(g, cs)
        rgb, depth = img["rgb"].clone(), img["depth"].clone()
        store = memory_budget is None or stored_bytes(n, n_keys, cam_p, rec_dtype) <= memory_budget
        ctx.store = store
        ctx.cam_p = cam_p
        ctx.cfg = cfg
        ctx.rec_dtype = rec_dtype
        ctx.rast = rast if store else None
        ctx.n_keys = n_keys
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
            rast = Rasterizer(n, ctx.cam_p, ctx.cfg, ctx.rec_dtype, capacity=max(ctx.n_keys, 1),
                              device=g["means"].device)
            rast.forward(g, cs)
        d_rgb = torch.zeros_like(rast.img["rgb"]) if d_rgb is None else d_rgb.contiguous().float()
        d_depth = torch.zeros_like(rast.img["depth"]) if d_depth is None else d_depth.contiguous().float()
        need = ctx.needs_input_grad
        grads = {k: torch.empty_like(g[k]) for k in PARAMS}
        rast.backward(g, cs, d_rgb, d_depth, mode=gs.GS_MAP, grads=grads, want_pose=need[5], want_score=False)
        rast.check()
        pose_grad = rast.pose.float().clone() if need[5] else None
        ctx.rast = None
        return (grads["means"], grads["log_scales"], grads["quats"], grads["opacity_logit"], grads["rgb"],
                pose_grad, None, None, None, None)


def gs_render(means, log_scales, quats, opacity_logit, colors, pose_delta, cam, cfg=None, rec_dtype=gs.GS_F32,
              memory_budget=None):
    return GsRenderFn.apply(means, log_scales, quats, opacity_logit, colors, pose_delta, cam, cfg, rec_dtype,
                            memory_budget)
