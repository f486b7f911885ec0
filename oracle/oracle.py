"""FP64 CPU oracle of the RTGS rasterizer (arXiv 2510.06644) -- ctypes wrapper.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check of
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import this
module.  It loads ``gs_oracle.c`` (compiled with gcc on first use) and never
touches the CUDA library or its headers; the two implementations share only
the seeded input generators of ``synth/``.

Every function takes and returns numpy arrays.  Camera and configuration are
given as plain dicts:

  cam = {"R": 3x3 world->camera rotation, "t": 3-vector, "fx", "fy", "cx",
         "cy", "W", "H", "sx", "sy"}
  cfg = {"near_z", "dilation", "alpha_min", "alpha_max", "t_eps", "bg"}

Paper sections followed are cited in the C source next to each function.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libgs_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gs_oracle.c into a shared library (plain gcc, no FMA contraction
    so that the float32 score of Eq. 7 rounds exactly as stated)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cam(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3), ("fx", C.c_double),
                ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("W", C.c_int32), ("H", C.c_int32), ("sx", C.c_int32), ("sy", C.c_int32)]


class _Cfg(C.Structure):
    _fields_ = [("near_z", C.c_double), ("dilation", C.c_double), ("alpha_min", C.c_double),
                ("alpha_max", C.c_double), ("t_eps", C.c_double), ("bg", C.c_double * 3)]


class _Splats(C.Structure):
    _fields_ = [("n", C.c_int64), ("uv", C.c_void_p), ("conic", C.c_void_p),
                ("opacity", C.c_void_p), ("rgb", C.c_void_p), ("depth", C.c_void_p),
                ("radius", C.c_void_p)]


DEFAULT_CFG = {"near_z": 0.2, "dilation": 0.3, "alpha_min": 1.0 / 255.0, "alpha_max": 0.99,
               "t_eps": 1e-4, "bg": (0.0, 0.0, 0.0)}


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.or_project.argtypes = [C.c_int64, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P]
            lib.or_project.restype = None
            lib.or_bin_count.argtypes = [C.c_int64, P, P, P, P, C.c_double, P]
            lib.or_bin_count.restype = C.c_int64
            lib.or_bin_sort.argtypes = [C.c_int64, P, P, P, P, P, C.c_double, P, P, P, P]
            lib.or_bin_sort.restype = None
            lib.or_render_fwd.argtypes = [P, P, P, P, P, P, P, P, P, P, P]
            lib.or_render_fwd.restype = C.c_double
            lib.or_loss_l1.argtypes = [C.c_int64, P, P, P, P, C.c_double, C.c_double, P, P]
            lib.or_loss_l1.restype = C.c_double
            lib.or_render_bwd.argtypes = [P, P, P, P, P, P, P, P]
            lib.or_render_bwd.restype = None
            lib.or_project_bwd.argtypes = [C.c_int64] + [P] * 17
            lib.or_project_bwd.restype = None
            lib.or_prune_select.argtypes = [C.c_int64, P, P, C.c_float, C.c_double, C.c_int64, P]
            lib.or_prune_select.restype = C.c_int64
            lib.or_next_interval.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double,
                                             C.c_int32, C.c_int]
            lib.or_next_interval.restype = C.c_int32
            lib.or_change_ratio.argtypes = [C.c_int64, P, C.c_int64, P]
            lib.or_change_ratio.restype = C.c_double
            lib.or_downsample_schedule.argtypes = [C.c_int64, C.c_int64, C.c_int, C.c_int64,
                                                   P, P]
            lib.or_downsample_schedule.restype = C.c_int
            lib.or_gather.argtypes = [P, C.c_int64, C.c_int64, C.c_int64, C.c_int32, C.c_int32, P]
            lib.or_gather.restype = None
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _cam(cam) -> _Cam:
    c = _Cam()
    R = np.asarray(cam["R"], dtype=np.float64).reshape(9)
    for i in range(9):
        c.R[i] = float(R[i])
    t = np.asarray(cam["t"], dtype=np.float64).reshape(3)
    for i in range(3):
        c.t[i] = float(t[i])
    c.fx, c.fy, c.cx, c.cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    c.W, c.H = int(cam["W"]), int(cam["H"])
    c.sx, c.sy = int(cam.get("sx", 1)), int(cam.get("sy", 1))
    return c


def _cfg(cfg=None) -> _Cfg:
    cfg = dict(DEFAULT_CFG, **(cfg or {}))
    c = _Cfg()
    for k in ("near_z", "dilation", "alpha_min", "alpha_max", "t_eps"):
        setattr(c, k, float(cfg[k]))
    for i in range(3):
        c.bg[i] = float(cfg["bg"][i])
    return c


def tile_dim(s):
    """Tile side in sampled pixels at stride s (16 / p2(s), at least 4)."""
    p = 1
    while p < s and p < 16:
        p *= 2
    return max(4, 16 // p)


def grid(cam):
    """Sampled image size and tile grid: (Ws, Hs, TX, TY)."""
    sx, sy = int(cam.get("sx", 1)), int(cam.get("sy", 1))
    Ws = -(-int(cam["W"]) // sx)
    Hs = -(-int(cam["H"]) // sy)
    return Ws, Hs, -(-Ws // tile_dim(sx)), -(-Hs // tile_dim(sy))


# --------------------------------------------------------------------------
# Projection (Sec. 2.1 Step 1)
# --------------------------------------------------------------------------

def project(g, cam, cfg=None):
    """g: dict with means [n,3], log_scales [n,3], quats [n,4] (w,x,y,z),
    opacity_logit [n], rgb [n,3], optional mask [n] (uint8, nonzero = masked).
    Returns a dict of FP64 projected attributes and integer rect/radius."""
    lib = _load()
    n = int(np.asarray(g["means"]).shape[0])
    means = _f64(g["means"], (n, 3))
    ls = _f64(g["log_scales"], (n, 3))
    qs = _f64(g["quats"], (n, 4))
    ol = _f64(g["opacity_logit"], (n,))
    mask = g.get("mask")
    if mask is not None:
        mask = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(n))
    out = {
        "uv": np.zeros((n, 2)), "conic": np.zeros((n, 3)), "depth": np.zeros(n),
        "opacity": np.zeros(n), "radius": np.zeros(n, np.int64), "rect": np.zeros((n, 4), np.int64),
        "touched": np.zeros(n, np.int64), "r3": np.zeros(n),
    }
    c, f = _cam(cam), _cfg(cfg)
    lib.or_project(n, _p(means), _p(ls), _p(qs), _p(ol), _p(mask), C.byref(c), C.byref(f),
                   _p(out["uv"]), _p(out["conic"]), _p(out["depth"]), _p(out["opacity"]),
                   _p(out["radius"]), _p(out["rect"]), _p(out["touched"]), _p(out["r3"]))
    out["rgb"] = _f64(g["rgb"], (n, 3))
    return out


# --------------------------------------------------------------------------
# Binning and sort (Sec. 2.1 Steps 1-2 and 2)
# --------------------------------------------------------------------------

def bin_sort(s, cam, cfg=None):
    """Keys (tile<<32 | f32 depth bits), values (ids) and ranges [T,2] of the
    projected splats s (uv, depth, radius, conic, opacity); the tile rects
    use cfg's alpha_min."""
    lib = _load()
    uv = _f64(s["uv"])
    n = uv.shape[0]
    depth = _f64(s["depth"], (n,))
    radius = np.ascontiguousarray(np.asarray(s["radius"], dtype=np.int64).reshape(n))
    conic = _f64(s["conic"], (n, 3))
    opacity = _f64(s["opacity"], (n,))
    amin = float(_cfg(cfg).alpha_min)
    c = _cam(cam)
    total = lib.or_bin_count(n, _p(uv), _p(radius), _p(conic), _p(opacity), amin, C.byref(c))
    _, _, TX, TY = grid(cam)
    keys = np.zeros(max(total, 1), np.uint64)
    vals = np.zeros(max(total, 1), np.uint32)
    ranges = np.zeros((TX * TY, 2), np.uint32)
    lib.or_bin_sort(n, _p(uv), _p(depth), _p(radius), _p(conic), _p(opacity), amin, C.byref(c), _p(keys),
                    _p(vals), _p(ranges))
    return keys[:total], vals[:total], ranges


# --------------------------------------------------------------------------
# Rendering and its backward (Sec. 2.1 Step 3, Sec. 2.2 Step 4)
# --------------------------------------------------------------------------

def _splats(s):
    n = int(np.asarray(s["uv"]).shape[0])
    keep = {
        "uv": _f64(s["uv"], (n, 2)), "conic": _f64(s["conic"], (n, 3)),
        "opacity": _f64(s["opacity"], (n,)), "rgb": _f64(s["rgb"], (n, 3)),
        "depth": _f64(s["depth"], (n,)),
        "radius": np.ascontiguousarray(np.asarray(s["radius"], dtype=np.int64).reshape(n)),
    }
    st = _Splats(n, _p(keep["uv"]).value, _p(keep["conic"]).value, _p(keep["opacity"]).value,
                 _p(keep["rgb"]).value, _p(keep["depth"]).value, _p(keep["radius"]).value)
    return st, keep


def render_fwd(s, cam, cfg=None, tiled=True, lists=None):
    """Forward render.  s: projected splats (uv, conic, opacity, rgb, depth,
    radius).  tiled=True walks the per-tile sorted lists (computed here, or
    passed as lists=(vals, ranges)); tiled=False is the brute-force per-pixel
    loop over all Gaussians."""
    lib = _load()
    st, keep = _splats(s)
    Ws, Hs, _, _ = grid(cam)
    P = Ws * Hs
    vals = ranges = None
    if tiled:
        if lists is None:
            _, vals, ranges = bin_sort(keep, cam, cfg)
        else:
            vals, ranges = lists
        vals = np.ascontiguousarray(vals, dtype=np.uint32)
        ranges = np.ascontiguousarray(ranges, dtype=np.uint32)
        if vals.size == 0:
            vals = np.zeros(1, np.uint32)
    out = {"rgb": np.zeros((3, Hs, Ws)), "depth": np.zeros((Hs, Ws)), "T": np.zeros((Hs, Ws)),
           "last": np.zeros((Hs, Ws), np.int64), "nfrag": np.zeros((Hs, Ws), np.int64),
           "margin": np.zeros((Hs, Ws), np.uint8)}
    c, f = _cam(cam), _cfg(cfg)
    out["sig"] = lib.or_render_fwd(C.byref(st), C.byref(c), C.byref(f), _p(vals), _p(ranges),
                                   _p(out["rgb"]), _p(out["depth"]), _p(out["T"]), _p(out["last"]),
                                   _p(out["nfrag"]), _p(out["margin"]))
    assert P == out["depth"].size
    return out


def loss_l1(rgb, depth, target_rgb, target_depth, w_rgb=1.0, w_depth=0.5):
    """Eq. 6 with L1 residuals: returns (L, dL/drgb [3,H,W], dL/ddepth [H,W])."""
    lib = _load()
    rgb = _f64(rgb)
    P = rgb.size // 3
    depth = _f64(depth)
    tr = _f64(target_rgb)
    td = _f64(target_depth)
    dr = np.zeros_like(rgb)
    dd = np.zeros_like(depth)
    L = lib.or_loss_l1(P, _p(rgb), _p(depth), _p(tr), _p(td), float(w_rgb), float(w_depth),
                       _p(dr), _p(dd))
    return L, dr, dd


def render_bwd(s, cam, d_rgb, d_depth, cfg=None, tiled=True, lists=None):
    """grad2d [n,12]: du, dv, dA, dB, dC, dopacity, ddepth, 0, dr, dg, db, 0."""
    lib = _load()
    st, keep = _splats(s)
    n = keep["uv"].shape[0]
    vals = ranges = None
    if tiled:
        if lists is None:
            _, vals, ranges = bin_sort(keep, cam, cfg)
        else:
            vals, ranges = lists
        vals = np.ascontiguousarray(vals, dtype=np.uint32)
        ranges = np.ascontiguousarray(ranges, dtype=np.uint32)
        if vals.size == 0:
            vals = np.zeros(1, np.uint32)
    d_rgb = _f64(d_rgb)
    d_depth = _f64(d_depth)
    g = np.zeros((n, 12))
    c, f = _cam(cam), _cfg(cfg)
    lib.or_render_bwd(C.byref(st), C.byref(c), C.byref(f), _p(vals), _p(ranges), _p(d_rgb),
                      _p(d_depth), _p(g))
    return g


# --------------------------------------------------------------------------
# Preprocessing backward and pose (Sec. 2.2 Step 5)
# --------------------------------------------------------------------------

def project_bwd(g, cam, grad2d, cfg=None):
    """3D gradients, camera-pose gradient (rho, phi) and Eq. 7 score terms."""
    lib = _load()
    n = int(np.asarray(g["means"]).shape[0])
    means = _f64(g["means"], (n, 3))
    ls = _f64(g["log_scales"], (n, 3))
    qs = _f64(g["quats"], (n, 4))
    ol = _f64(g["opacity_logit"], (n,))
    mask = g.get("mask")
    if mask is not None:
        mask = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(n))
    g2 = _f64(grad2d, (n, 12))
    out = {"means": np.zeros((n, 3)), "log_scales": np.zeros((n, 3)), "quats": np.zeros((n, 4)),
           "opacity_logit": np.zeros(n), "rgb": np.zeros((n, 3)), "pcam": np.zeros((n, 3)),
           "Sc": np.zeros((n, 9)), "pose": np.zeros(6), "score_terms": np.zeros((n, 2))}
    c, f = _cam(cam), _cfg(cfg)
    lib.or_project_bwd(n, _p(means), _p(ls), _p(qs), _p(ol), _p(mask), C.byref(c), C.byref(f),
                       _p(g2), _p(out["means"]), _p(out["log_scales"]), _p(out["quats"]),
                       _p(out["opacity_logit"]), _p(out["rgb"]), _p(out["pcam"]), _p(out["Sc"]),
                       _p(out["pose"]), _p(out["score_terms"]))
    return out


def forward(g, cam, cfg=None, tiled=True):
    """Project then render (end to end from 3D parameters)."""
    pr = project(g, cam, cfg)
    img = render_fwd(pr, cam, cfg, tiled=tiled)
    return pr, img


def forward_backward(g, cam, d_rgb, d_depth, cfg=None, tiled=True):
    """Full chain: 3D gradients and pose gradient for given image gradients."""
    pr = project(g, cam, cfg)
    g2 = render_bwd(pr, cam, d_rgb, d_depth, cfg, tiled=tiled)
    return pr, g2, project_bwd(g, cam, g2, cfg)


# --------------------------------------------------------------------------
# Pruning (Sec. 4.1) and downsampling (Sec. 4.2)
# --------------------------------------------------------------------------

def prune_select(t_mu, t_sigma, mask, lam=0.8, frac=0.1, max_select=None):
    """Masks the lowest-score unmasked Gaussians; returns (new mask, m)."""
    lib = _load()
    t_mu = np.ascontiguousarray(t_mu, dtype=np.float32)
    t_sigma = np.ascontiguousarray(t_sigma, dtype=np.float32)
    m = np.ascontiguousarray(np.array(mask, dtype=np.uint8, copy=True))
    n = t_mu.size
    if max_select is None:
        max_select = n
    cnt = lib.or_prune_select(n, _p(t_mu), _p(t_sigma), float(lam), float(frac), int(max_select),
                              _p(m))
    return m, int(cnt)


def next_interval(K, r, K0=5, thr=0.05, k_max=64, literal=False):
    return int(_load().or_next_interval(int(K), int(K0), float(r), float(thr), int(k_max),
                                        1 if literal else 0))


def change_ratio(pairs_a, pairs_b):
    a = np.ascontiguousarray(pairs_a, dtype=np.uint64)
    b = np.ascontiguousarray(pairs_b, dtype=np.uint64)
    return float(_load().or_change_ratio(a.size, _p(a) if a.size else None, b.size,
                                         _p(b) if b.size else None))


def downsample_schedule(n, k, is_keyframe, m=2):
    sx = C.c_int32(0)
    sy = C.c_int32(0)
    rc = _load().or_downsample_schedule(int(n), int(k), 1 if is_keyframe else 0, int(m),
                                        C.byref(sx), C.byref(sy))
    if rc != 0:
        raise ValueError("bad downsampling arguments")
    return sx.value, sy.value


def gather(full, sx, sy):
    """full [C,H,W] -> [C, ceil(H/sy), ceil(W/sx)] sampled at (sy*j, sx*i)."""
    full = _f64(full)
    if full.ndim == 2:
        full = full[None]
    Cn, H, W = full.shape
    out = np.zeros((Cn, -(-H // sy), -(-W // sx)))
    _load().or_gather(_p(full), Cn, W, H, int(sx), int(sy), _p(out))
    return out
