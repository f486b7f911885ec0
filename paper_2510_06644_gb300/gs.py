"""Python binding of the C ABI in include/gs.h (ctypes; argument marshalling
only -- every step runs in the sm_103a kernels of libgs_gb300.so).

Functions keep the C names.  Device arrays are torch CUDA tensors; work is
enqueued on torch's current CUDA stream unless ``stream`` is given.  The
library must have been built (``__graft_entry__.build()``); importing this
module without it, or calling it without a CUDA device, raises -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libgs_gb300.so")

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_WORKSPACE, GS_ERR_CUDA, GS_ERR_TIMEOUT, GS_ERR_CAPACITY, \
    GS_ERR_DEVICE_CHECK, GS_ERR_UNIMPLEMENTED = range(8)
GS_TRACK, GS_MAP = 0, 1
GS_F32, GS_BF16, GS_F16 = 0, 1, 2
GS_IDLE, GS_EXECUTING = 0, 1
GRAD2D_STRIDE = 12
SPLAT_WORDS = {GS_F32: 12, GS_BF16: 8, GS_F16: 8}   # 32-bit words per 2D record
TILE = 16


class GsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gs error {code}: {msg}")
        self.code = code


class gs_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("sx", C.c_int32), ("sy", C.c_int32), ("pose", C.c_void_p)]


class gs_config(C.Structure):
    _fields_ = [("near_z", C.c_float), ("dilation", C.c_float), ("alpha_min", C.c_float),
                ("alpha_max", C.c_float), ("t_eps", C.c_float), ("bg", C.c_float * 3),
                ("lambda_score", C.c_float), ("prune_frac", C.c_float), ("prune_cap", C.c_float),
                ("change_thr", C.c_float), ("k0", C.c_int32), ("k_max", C.c_int32),
                ("w_rgb", C.c_float), ("w_depth", C.c_float), ("balance", C.c_int32)]


class gs_pose_step(C.Structure):
    _fields_ = [("pose", C.c_void_p), ("adam", C.c_void_p), ("lr_trans", C.c_float), ("lr_rot", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float)]


class gs_gaussians(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("rgb", C.c_void_p), ("mask", C.c_void_p),
                ("n", C.c_int64)]


class gs_grads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("rgb", C.c_void_p)]


class gs_track_job(C.Structure):
    """One session's tracking iteration inside a wave (gs_track_wave)."""
    _fields_ = [("cam", gs_camera), ("g", gs_gaussians), ("splats", C.c_void_p), ("keys_capacity", C.c_int64),
                ("bin_workspace", C.c_void_p), ("bin_workspace_bytes", C.c_size_t), ("keys", C.c_void_p),
                ("vals", C.c_void_p), ("n_keys", C.c_void_p), ("tile_ranges", C.c_void_p),
                ("tile_order", C.c_void_p), ("rgb", C.c_void_p), ("depth", C.c_void_p), ("t_final", C.c_void_p),
                ("last_idx", C.c_void_p), ("n_blended", C.c_void_p), ("blend_masks", C.c_void_p),
                ("target_rgb", C.c_void_p), ("target_depth", C.c_void_p), ("d_rgb", C.c_void_p),
                ("d_depth", C.c_void_p), ("loss", C.c_void_p), ("grad2d", C.c_void_p), ("pose_grad6", C.c_void_p),
                ("score_terms", C.c_void_p), ("bwd_workspace", C.c_void_p), ("bwd_workspace_bytes", C.c_size_t),
                ("step", gs_pose_step)]


GS_WAVE_MAX = 32


class gs_map_adam(C.Structure):
    _fields_ = [("m", C.c_void_p * 5), ("v", C.c_void_p * 5), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("state", C.c_void_p)]


_lib = None
_P = C.c_void_p
_SIGS = {
    "gs_default_config": ([_P], None),
    "gs_version": ([], C.c_char_p),
    "gs_project": ([_P, _P, _P, C.c_int, _P, _P], C.c_int),
    "gs_bin_sort": ([_P, _P, C.c_int, _P, C.c_int64, C.c_int64, _P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "gs_bin_count": ([_P, _P, C.c_int, _P, C.c_int64, _P, _P, _P, _P], C.c_int),
    "gs_project_bin_sort": ([_P, _P, _P, C.c_int, _P, C.c_int64, _P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "gs_render_fwd": ([_P, _P, C.c_int, _P, C.c_int64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "gs_blend_mask_words": ([_P, C.c_int64], C.c_size_t),
    "gs_render_fwd_loss": ([_P, _P, C.c_int, _P, C.c_int64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                            _P], C.c_int),
    "gs_loss_l1": ([_P, _P, _P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "gs_render_bwd": ([_P, _P, _P, C.c_int, _P, _P, _P, _P, _P, _P, _P, _P, _P, C.c_int, _P, _P, _P, _P,
                       _P, _P, _P], C.c_int),
    "gs_project_bwd": ([_P, _P, _P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "gs_project_bwd_step": ([_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "gs_project_bwd_noalloc": ([_P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "gs_prune": ([_P, _P, C.c_int64, _P, C.c_int, _P, C.c_float, C.c_int64, _P, _P, _P, _P, _P],
                 C.c_int),
    "gs_change_ratio": ([_P, _P, C.c_int, _P, _P, C.c_int64, _P, _P, _P, _P], C.c_int),
    "gs_compact": ([_P, C.c_int64, C.c_int32, _P, _P, _P], C.c_int),
    "gs_downsample": ([C.c_int64, C.c_int64, C.c_int, C.c_int, _P, _P, _P, C.c_int32, C.c_int32,
                       C.c_int32, _P, _P], C.c_int),
    "gs_pose_update": ([_P, _P, _P, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float, _P], C.c_int),
    "gs_adam": ([C.c_int, _P, _P, _P, _P, _P, C.c_float, C.c_float, C.c_float, C.c_float, _P, _P], C.c_int),
    "gs_status_poll": ([_P, C.c_int, _P], C.c_int),
    "gs_probe_red_f32": ([_P, C.c_int64, C.c_int64, C.c_int32, _P], C.c_int),
    "gs_probe_fma_f32": ([_P, C.c_int64, C.c_int32, _P], C.c_int),
    "gs_track_wave": ([_P, _P, C.c_int32, _P], C.c_int),
    "gs_next_interval": ([_P, C.c_int32, C.c_float], C.c_int32),
    "gs_project_bwd_adam": ([_P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "gs_status_reset": ([_P], C.c_int),
    "gs_last_error": ([], C.c_char_p),
}


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(code, what):
    if code != GS_OK:
        raise GsError(code, f"{what}: {lib().gs_last_error().decode()}")


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


# --------------------------------------------------------------------------
# Structures
# --------------------------------------------------------------------------

def camera(cam, pose=None) -> gs_camera:
    """gs_camera from a dict {R, t, fx, fy, cx, cy, W, H, sx, sy}; `pose`
    (device float32 [12] tensor) makes the kernels read R, t from it."""
    c = gs_camera()
    c.pose = _ptr(pose).value if pose is not None else None
    R = [float(v) for v in torch.as_tensor(cam["R"], dtype=torch.float64).reshape(9).tolist()]
    t = [float(v) for v in torch.as_tensor(cam["t"], dtype=torch.float64).reshape(3).tolist()]
    for i in range(9):
        c.R[i] = R[i]
    for i in range(3):
        c.t[i] = t[i]
    c.fx, c.fy, c.cx, c.cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    c.width, c.height = int(cam["W"]), int(cam["H"])
    c.sx, c.sy = int(cam.get("sx", 1)), int(cam.get("sy", 1))
    return c


def default_config(**overrides) -> gs_config:
    c = gs_config()
    lib().gs_default_config(C.byref(c))
    for k, v in overrides.items():
        if k == "bg":
            for i in range(3):
                c.bg[i] = float(v[i])
        else:
            setattr(c, k, v)
    return c


def tile_dim(s):
    """Tile side in sampled pixels at stride s: 16 / p2(s), at least 4
    (p2 = smallest power of two >= s), as in include/gs.h."""
    p = 1
    while p < s and p < TILE:
        p *= 2
    return max(4, TILE // p)


def grid(cam):
    """(Ws, Hs, TX, TY) of a camera dict or gs_camera."""
    if isinstance(cam, gs_camera):
        W, H, sx, sy = cam.width, cam.height, cam.sx, cam.sy
    else:
        W, H, sx, sy = int(cam["W"]), int(cam["H"]), int(cam.get("sx", 1)), int(cam.get("sy", 1))
    Ws, Hs = -(-W // sx), -(-H // sy)
    return Ws, Hs, -(-Ws // tile_dim(sx)), -(-Hs // tile_dim(sy))


def gaussians(g, mask=None) -> gs_gaussians:
    """gs_gaussians over a dict of contiguous float32 CUDA tensors."""
    s = gs_gaussians()
    s.means = _ptr(g["means"]).value
    s.log_scales = _ptr(g["log_scales"]).value
    s.quats = _ptr(g["quats"]).value
    s.opacity_logit = _ptr(g["opacity_logit"]).value
    s.rgb = _ptr(g["rgb"]).value
    m = mask if mask is not None else g.get("mask")
    s.mask = _ptr(m).value if m is not None else None
    s.n = int(g["means"].shape[0])
    return s


def grads_struct(gr) -> gs_grads:
    s = gs_grads()
    if gr:
        for k in ("means", "log_scales", "quats", "opacity_logit", "rgb"):
            v = gr.get(k)
            setattr(s, k, _ptr(v).value if v is not None else None)
    return s


def workspace(nbytes, device=None):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


# --------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# --------------------------------------------------------------------------

def gs_project(cfg, cam, g, rec_dtype=GS_F32, splats=None, stream=None):
    n = int(g["means"].shape[0])
    if splats is None:
        dt = torch.float32 if rec_dtype == GS_F32 else torch.int32
        splats = torch.empty((n, SPLAT_WORDS[rec_dtype]), dtype=dt, device=g["means"].device)
    gs_g = gaussians(g)
    _check(lib().gs_project(C.byref(cfg), C.byref(cam), C.byref(gs_g), rec_dtype, _ptr(splats),
                            _stream(stream)), "gs_project")
    return splats


_DEFAULT_CFG = None


def _cfg(cfg):
    """The given config, or the library's defaults (alpha_min 1/255)."""
    global _DEFAULT_CFG
    if cfg is not None:
        return cfg
    if _DEFAULT_CFG is None:
        _DEFAULT_CFG = default_config()
    return _DEFAULT_CFG


def gs_bin_sort_workspace(cam, rec_dtype, n, capacity, cfg=None):
    nb = C.c_size_t(0)
    _check(lib().gs_bin_sort(C.byref(_cfg(cfg)), C.byref(cam), rec_dtype, None, int(n), int(capacity), None,
                             C.byref(nb), None, None, None, None, None, None), "gs_bin_sort(size)")
    return nb.value


def gs_bin_sort(cam, splats, n, capacity, rec_dtype=GS_F32, ws=None, keys=None, vals=None, n_keys=None,
                ranges=None, order=None, stream=None, cfg=None):
    """Returns (keys, vals, n_keys, ranges, order); order is the heavy-first
    tile permutation (allocated unless given).  cfg: its alpha_min shapes the
    tile rects (the defaults unless given)."""
    dev = splats.device
    _, _, TX, TY = grid(cam)
    need = gs_bin_sort_workspace(cam, rec_dtype, n, capacity, cfg)
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    keys = torch.empty(max(capacity, 1), dtype=torch.int64, device=dev) if keys is None else keys
    vals = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev) if vals is None else vals
    n_keys = torch.zeros(1, dtype=torch.int64, device=dev) if n_keys is None else n_keys
    ranges = torch.empty((TX * TY, 2), dtype=torch.int32, device=dev) if ranges is None else ranges
    order = torch.empty(TX * TY, dtype=torch.int32, device=dev) if order is None else order
    nb = C.c_size_t(ws.numel())
    _check(lib().gs_bin_sort(C.byref(_cfg(cfg)), C.byref(cam), rec_dtype, _ptr(splats), int(n), int(capacity),
                             _ptr(ws),
                             C.byref(nb), _ptr(keys), _ptr(vals), _ptr(n_keys), _ptr(ranges), _ptr(order),
                             _stream(stream)), "gs_bin_sort")
    return keys, vals, n_keys, ranges, order


def gs_project_bin_sort_workspace(cfg, cam, g, rec_dtype, capacity):
    nb = C.c_size_t(0)
    gs_g = gaussians(g)
    _check(lib().gs_project_bin_sort(C.byref(cfg), C.byref(cam), C.byref(gs_g), rec_dtype, None, int(capacity), None,
                                     C.byref(nb), None, None, None, None, None, None), "gs_project_bin_sort(size)")
    return nb.value


def gs_project_bin_sort(cfg, cam, g, splats, capacity, rec_dtype=GS_F32, ws=None, keys=None, vals=None, n_keys=None,
                        ranges=None, order=None, stream=None):
    """gs_project into `splats`, then gs_bin_sort, in one fused call:
    returns (keys, vals, n_keys, ranges, order)."""
    dev = splats.device
    _, _, TX, TY = grid(cam)
    need = gs_project_bin_sort_workspace(cfg, cam, g, rec_dtype, capacity)
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    keys = torch.empty(max(capacity, 1), dtype=torch.int64, device=dev) if keys is None else keys
    vals = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev) if vals is None else vals
    n_keys = torch.zeros(1, dtype=torch.int64, device=dev) if n_keys is None else n_keys
    ranges = torch.empty((TX * TY, 2), dtype=torch.int32, device=dev) if ranges is None else ranges
    order = torch.empty(TX * TY, dtype=torch.int32, device=dev) if order is None else order
    gs_g = gaussians(g)
    nb = C.c_size_t(ws.numel())
    _check(lib().gs_project_bin_sort(C.byref(cfg), C.byref(cam), C.byref(gs_g), rec_dtype, _ptr(splats), int(capacity),
                                     _ptr(ws), C.byref(nb), _ptr(keys), _ptr(vals), _ptr(n_keys), _ptr(ranges),
                                     _ptr(order), _stream(stream)), "gs_project_bin_sort")
    return keys, vals, n_keys, ranges, order


def gs_bin_count(cam, splats, n, rec_dtype=GS_F32, stream=None, cfg=None):
    nb = C.c_size_t(0)
    _check(lib().gs_bin_count(C.byref(_cfg(cfg)), C.byref(cam), rec_dtype, None, int(n), None, C.byref(nb), None,
                              None), "gs_bin_count(size)")
    ws = workspace(nb.value, splats.device)
    out = torch.zeros(1, dtype=torch.int64, device=splats.device)
    nb = C.c_size_t(ws.numel())
    _check(lib().gs_bin_count(C.byref(_cfg(cfg)), C.byref(cam), rec_dtype, _ptr(splats), int(n), _ptr(ws),
                              C.byref(nb), _ptr(out), _stream(stream)), "gs_bin_count")
    return out


def gs_blend_mask_words(cam, key_capacity):
    """Words of a blend-mask array for the camera's grid and key capacity."""
    return int(lib().gs_blend_mask_words(C.byref(cam), int(key_capacity)))


def gs_render_fwd(cfg, cam, splats, n, vals, ranges, rec_dtype=GS_F32, out=None, order=None, masks=None,
                  stream=None):
    """masks: optional int32 device tensor of gs_blend_mask_words words that
    receives the blend masks gs_render_bwd can reuse."""
    Ws, Hs, _, _ = grid(cam)
    dev = splats.device
    if out is None:
        out = {"rgb": torch.empty((3, Hs, Ws), device=dev), "depth": torch.empty((Hs, Ws), device=dev),
               "t_final": torch.empty((Hs, Ws), device=dev),
               "last_idx": torch.empty((Hs, Ws), dtype=torch.int32, device=dev),
               "n_blended": torch.empty((Hs, Ws), dtype=torch.int32, device=dev)}
    _check(lib().gs_render_fwd(C.byref(cfg), C.byref(cam), rec_dtype, _ptr(splats), int(n), _ptr(vals),
                               _ptr(ranges), _ptr(order), _ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out["t_final"]),
                               _ptr(out["last_idx"]), _ptr(out.get("n_blended")), _ptr(masks), _stream(stream)),
           "gs_render_fwd")
    return out


def gs_render_fwd_loss(cfg, cam, splats, n, vals, ranges, target_rgb, target_depth, rec_dtype=GS_F32, out=None,
                       dimg=None, order=None, masks=None, stream=None):
    """Forward compositing with the loss fused (gs_render_fwd_loss): returns
    (out, dimg) like gs_render_fwd and gs_loss_l1."""
    Ws, Hs, _, _ = grid(cam)
    dev = splats.device
    if out is None:
        out = {"rgb": torch.empty((3, Hs, Ws), device=dev), "depth": torch.empty((Hs, Ws), device=dev),
               "t_final": torch.empty((Hs, Ws), device=dev),
               "last_idx": torch.empty((Hs, Ws), dtype=torch.int32, device=dev),
               "n_blended": torch.empty((Hs, Ws), dtype=torch.int32, device=dev)}
    if dimg is None:
        dimg = {"d_rgb": torch.empty((3, Hs, Ws), device=dev), "d_depth": torch.empty((Hs, Ws), device=dev),
                "loss": torch.zeros(1, dtype=torch.float64, device=dev)}
    _check(lib().gs_render_fwd_loss(C.byref(cfg), C.byref(cam), rec_dtype, _ptr(splats), int(n), _ptr(vals),
                                    _ptr(ranges), _ptr(order), _ptr(out["rgb"]), _ptr(out["depth"]),
                                    _ptr(out["t_final"]), _ptr(out["last_idx"]), _ptr(out.get("n_blended")),
                                    _ptr(masks), _ptr(target_rgb), _ptr(target_depth), _ptr(dimg["d_rgb"]), _ptr(dimg["d_depth"]),
                                    _ptr(dimg["loss"]), _stream(stream)), "gs_render_fwd_loss")
    return out, dimg


def gs_loss_l1(cfg, cam, rgb, depth, target_rgb, target_depth, out=None, stream=None):
    if out is None:
        out = {"d_rgb": torch.empty_like(rgb), "d_depth": torch.empty_like(depth),
               "loss": torch.zeros(1, dtype=torch.float64, device=rgb.device)}
    _check(lib().gs_loss_l1(C.byref(cfg), C.byref(cam), _ptr(rgb), _ptr(depth), _ptr(target_rgb),
                            _ptr(target_depth), _ptr(out["d_rgb"]), _ptr(out["d_depth"]), _ptr(out["loss"]),
                            _stream(stream)), "gs_loss_l1")
    return out


def gs_project_bwd_workspace(cfg, cam, g):
    nb = C.c_size_t(0)
    gs_g = gaussians(g)
    _check(lib().gs_project_bwd(C.byref(cfg), C.byref(cam), C.byref(gs_g), None, None, None, None, None,
                                C.byref(nb), None), "gs_project_bwd(size)")
    return nb.value


def gs_render_bwd(cfg, cam, g, splats, vals, ranges, t_final, last_idx, d_rgb, d_depth, mode=GS_MAP,
                  rec_dtype=GS_F32, grad2d=None, grads=None, pose=None, score=None, ws=None, order=None,
                  masks=None, stream=None):
    """grads: dict of output tensors (or None); pose: float64 [6] tensor or
    None; score: float32 [n,2] tensor or None; masks: the blend masks of the
    forward that produced t_final and last_idx (or None)."""
    n = int(g["means"].shape[0])
    dev = splats.device
    grad2d = torch.empty((n, GRAD2D_STRIDE), device=dev) if grad2d is None else grad2d
    gs_g = gaussians(g)
    gr = grads_struct(grads) if grads is not None else None
    chain = grads is not None or pose is not None or score is not None
    need = gs_project_bwd_workspace(cfg, cam, g) if chain else 0
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    nb = C.c_size_t(ws.numel())
    _check(lib().gs_render_bwd(C.byref(cfg), C.byref(cam), C.byref(gs_g), rec_dtype, _ptr(splats), _ptr(vals),
                               _ptr(ranges), _ptr(order), _ptr(t_final), _ptr(last_idx), _ptr(masks), _ptr(d_rgb),
                               _ptr(d_depth),
                               mode,
                               _ptr(grad2d), C.byref(gr) if gr is not None else None, _ptr(pose),
                               _ptr(score), _ptr(ws), C.byref(nb), _stream(stream)), "gs_render_bwd")
    return grad2d


def gs_project_bwd(cfg, cam, g, grad2d, grads=None, pose=None, score=None, ws=None, stream=None):
    need = gs_project_bwd_workspace(cfg, cam, g)
    if ws is None or ws.numel() < need:
        ws = workspace(need, grad2d.device)
    gs_g = gaussians(g)
    gr = grads_struct(grads) if grads is not None else None
    nb = C.c_size_t(ws.numel())
    _check(lib().gs_project_bwd(C.byref(cfg), C.byref(cam), C.byref(gs_g), _ptr(grad2d),
                                C.byref(gr) if gr is not None else None, _ptr(pose), _ptr(score), _ptr(ws),
                                C.byref(nb), _stream(stream)), "gs_project_bwd")


def pose_step(pose, adam, lr_trans=1e-3, lr_rot=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """gs_pose_step over device tensors pose (float32 [12]) and adam (float32 [13])."""
    return gs_pose_step(_ptr(pose).value, _ptr(adam).value, float(lr_trans), float(lr_rot), float(beta1),
                        float(beta2), float(eps))


def gs_project_bwd_step(cfg, cam, g, grad2d, pose, step, grads=None, score=None, ws=None, stream=None):
    """gs_project_bwd with the pose step fused into its last block (pose:
    float64 [6] output of the reduced pose gradient; step: gs_pose_step)."""
    need = gs_project_bwd_workspace(cfg, cam, g)
    if ws is None or ws.numel() < need:
        ws = workspace(need, grad2d.device)
    gs_g = gaussians(g)
    gr = grads_struct(grads) if grads is not None else None
    nb = C.c_size_t(ws.numel())
    _check(lib().gs_project_bwd_step(C.byref(cfg), C.byref(cam), C.byref(gs_g), _ptr(grad2d),
                                     C.byref(gr) if gr is not None else None, _ptr(pose), _ptr(score),
                                     C.byref(step) if step is not None else None, _ptr(ws), C.byref(nb),
                                     _stream(stream)), "gs_project_bwd_step")


def gs_track_wave(cfg, jobs, stream=None):
    """One tracking iteration of every session in `jobs` (a ctypes array of
    gs_track_job, or a list of them) in launches whose grids span all of
    them."""
    if not isinstance(jobs, C.Array):
        arr = (gs_track_job * len(jobs))()
        for i, j in enumerate(jobs):
            arr[i] = j
        jobs = arr
    _check(lib().gs_track_wave(C.byref(_cfg(cfg)), C.cast(jobs, C.c_void_p), len(jobs), _stream(stream)),
           "gs_track_wave")


PARAM_KEYS = ("means", "log_scales", "quats", "opacity_logit", "rgb")


def gs_project_bwd_adam(cfg, cam, g, grad2d, ms, vs, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-15,
                        grads=None, score=None, stream=None):
    """Backward projection of a mapping iteration with the map's Adam step
    fused in: g's parameter tensors are updated in place; ms / vs: dicts of
    moment tensors keyed like g; state: float32 [2] (as gs_adam)."""
    a = gs_map_adam()
    for i, k in enumerate(PARAM_KEYS):
        a.m[i] = _ptr(ms[k]).value
        a.v[i] = _ptr(vs[k]).value
    a.lr, a.beta1, a.beta2, a.eps = float(lr), float(beta1), float(beta2), float(eps)
    a.state = _ptr(state).value
    gs_g = gaussians(g)
    gr = grads_struct(grads) if grads is not None else None
    _check(lib().gs_project_bwd_adam(C.byref(_cfg(cfg)), C.byref(cam), C.byref(gs_g), _ptr(grad2d), C.byref(a),
                                     C.byref(gr) if gr is not None else None, _ptr(score), _stream(stream)),
           "gs_project_bwd_adam")


def gs_project_bwd_noalloc(cfg, cam, g, grad2d, grads=None, pose=None, score=None, stream=None):
    """gs_project_bwd without a workspace: the library's static scratch is
    used (no device allocation at all; calls must not overlap on the GPU)."""
    gs_g = gaussians(g)
    gr = grads_struct(grads) if grads is not None else None
    _check(lib().gs_project_bwd_noalloc(C.byref(cfg), C.byref(cam), C.byref(gs_g), _ptr(grad2d),
                                        C.byref(gr) if gr is not None else None, _ptr(pose), _ptr(score),
                                        _stream(stream)), "gs_project_bwd_noalloc")


def gs_prune(cfg, score, mask, iter_in_interval, K, change_ratio=0.0, max_select=None, compact_map=None,
             n_kept=None, ws=None, stream=None):
    """Returns the next K (host int).  mask is updated in place."""
    n = int(mask.numel())
    max_select = n if max_select is None else int(max_select)
    k = C.c_int(int(K))
    nb = C.c_size_t(0)
    _check(lib().gs_prune(C.byref(cfg), None, n, None, int(iter_in_interval), C.byref(k), 0.0, 0, None, None,
                          None, C.byref(nb), None), "gs_prune(size)")
    if ws is None or ws.numel() < nb.value:
        ws = workspace(nb.value, mask.device)
    nb = C.c_size_t(ws.numel())
    _check(lib().gs_prune(C.byref(cfg), _ptr(score), n, _ptr(mask), int(iter_in_interval), C.byref(k),
                          float(change_ratio), max_select, _ptr(compact_map), _ptr(n_kept), _ptr(ws),
                          C.byref(nb), _stream(stream)), "gs_prune")
    return k.value


def gs_next_interval(cfg, K, change_ratio):
    """Next pruning interval after K iterations with the given change ratio."""
    return int(lib().gs_next_interval(C.byref(_cfg(cfg)), int(K), float(change_ratio)))


def gs_change_ratio(cam, splats_a, splats_b, n, rec_dtype=GS_F32, out=None, stream=None, cfg=None):
    ws = workspace(256, splats_a.device)
    out = torch.zeros(1, dtype=torch.float32, device=splats_a.device) if out is None else out
    nb = C.c_size_t(ws.numel())
    _check(lib().gs_change_ratio(C.byref(_cfg(cfg)), C.byref(cam), rec_dtype, _ptr(splats_a), _ptr(splats_b),
                                 int(n), _ptr(ws), C.byref(nb), _ptr(out), _stream(stream)), "gs_change_ratio")
    return out


def gs_compact(src, compact_map, n_kept, stream=None):
    n = int(src.shape[0])
    width = int(src[0].numel()) if n > 0 else 1
    dst = torch.empty((int(n_kept),) + tuple(src.shape[1:]), dtype=src.dtype, device=src.device)
    _check(lib().gs_compact(_ptr(src), n, width, _ptr(compact_map), _ptr(dst), _stream(stream)), "gs_compact")
    return dst


def gs_downsample(frame_idx, last_kf_idx, is_keyframe, m=2, target_full=None, out=None, stream=None):
    """Returns (sx, sy) and, if target_full [C,H,W] (or [H,W]) is given, the
    target gathered at the sampled pixels (into `out` when given)."""
    sx, sy = C.c_int32(0), C.c_int32(0)
    _check(lib().gs_downsample(int(frame_idx), int(last_kf_idx), 1 if is_keyframe else 0, int(m), C.byref(sx),
                               C.byref(sy), None, 0, 0, 0, None, None), "gs_downsample")
    if target_full is None:
        return sx.value, sy.value, None
    t = target_full if target_full.dim() == 3 else target_full[None]
    Cn, H, W = t.shape
    shape = (Cn, -(-H // sy.value), -(-W // sx.value))
    if out is None:
        res = torch.empty(shape, dtype=torch.float32, device=t.device)
    else:
        if out.numel() != Cn * shape[1] * shape[2] or not out.is_contiguous():
            raise ValueError("out has the wrong size for the sampled target")
        res = out
    _check(lib().gs_downsample(int(frame_idx), int(last_kf_idx), 1 if is_keyframe else 0, int(m), C.byref(sx),
                               C.byref(sy), _ptr(t.contiguous()), Cn, W, H, _ptr(res), _stream(stream)),
           "gs_downsample")
    if out is not None:
        return sx.value, sy.value, out
    return sx.value, sy.value, res if target_full.dim() == 3 else res[0]


def pose_tensor(cam, device="cuda"):
    """Device float32 [12] pose (R row-major, t) of a camera dict."""
    R = torch.as_tensor(cam["R"], dtype=torch.float32).reshape(9)
    t = torch.as_tensor(cam["t"], dtype=torch.float32).reshape(3)
    return torch.cat([R, t]).to(device)


def gs_pose_update(pose, pose_grad, adam, lr_trans=1e-3, lr_rot=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                   stream=None):
    _check(lib().gs_pose_update(_ptr(pose), _ptr(pose_grad), _ptr(adam), float(lr_trans), float(lr_rot),
                                float(beta1), float(beta2), float(eps), _stream(stream)), "gs_pose_update")


def gs_adam(params, grads, ms, vs, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
    """One Adam step over lists of float32 device tensors (same order in
    every list); state is a zeroed device float32 [2] tensor (step count)."""
    k = len(params)
    arr = C.c_void_p * k
    P_ = arr(*[_ptr(t).value for t in params])
    G_ = arr(*[_ptr(t).value for t in grads])
    M_ = arr(*[_ptr(t).value for t in ms])
    V_ = arr(*[_ptr(t).value for t in vs])
    cnt = (C.c_int64 * k)(*[int(t.numel()) for t in params])
    _check(lib().gs_adam(k, P_, G_, M_, V_, cnt, float(lr), float(beta1), float(beta2), float(eps), _ptr(state),
                         _stream(stream)), "gs_adam")


def gs_probe_red_f32(dst, n_threads, per_thread, stream=None):
    """Reduction-throughput probe: thread t of n_threads adds 1.0 to
    dst[t % dst.numel()] per_thread times (float32 device tensor dst)."""
    if dst.dtype != torch.float32:
        raise ValueError("float32 dst expected")
    _check(lib().gs_probe_red_f32(_ptr(dst), int(dst.numel()), int(n_threads), int(per_thread), _stream(stream)),
           "gs_probe_red_f32")


def gs_probe_fma_f32(out, iters, stream=None):
    """FMA-throughput probe: each of out.numel() threads runs 8 chains of
    `iters` FMAs (16 FLOP per iteration) and writes 28 + 8 iters."""
    _check(lib().gs_probe_fma_f32(_ptr(out), int(out.numel()), int(iters), _stream(stream)), "gs_probe_fma_f32")


def gs_status_poll(blocking=True, stream=None):
    st = C.c_int(0)
    code = lib().gs_status_poll(_stream(stream), 1 if blocking else 0, C.byref(st))
    return code, st.value


def gs_status_reset(stream=None):
    _check(lib().gs_status_reset(_stream(stream)), "gs_status_reset")


# --------------------------------------------------------------------------
# Record views (for tests and callers that inspect the 2D records)
# --------------------------------------------------------------------------

def splat_fields(splats, rec_dtype=GS_F32):
    """Dict of views/decoded fields of a record array."""
    if rec_dtype == GS_F32:
        s = splats
        return {"uv": s[:, 0:2], "conic": s[:, 2:5], "opacity": s[:, 5], "depth": s[:, 6],
                "radius": s[:, 7].view(torch.int32), "rgb": s[:, 8:11], "touched": s[:, 11].view(torch.int32)}
    w = splats
    f32 = w.view(torch.float32)
    h = w[:, 4:8].contiguous().view(torch.int16).view(torch.bfloat16 if rec_dtype == GS_BF16 else torch.float16)
    h = h.float()
    return {"uv": f32[:, 0:2], "depth": f32[:, 2], "radius": w[:, 3], "conic": h[:, 0:3], "opacity": h[:, 3],
            "rgb": h[:, 4:7], "touched": (w[:, 7] >> 16) & 0xFFFF}
