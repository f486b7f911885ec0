"""Seeded synthetic scenes and inputs shaped like RGB-D SLAM workloads.

The paper evaluates on TUM-RGBD, Replica, ScanNet and ScanNet++ (Sec. 6.1,
dataset table); none of them is available here, so these generators stand in
for them, keeping only their resolutions and the structure of a SLAM map
(Gaussians sampled on planes and spheres, small log-scales, mostly opaque).

Every generator takes an explicit seed and uses numpy's PCG64.  This module
only draws random numbers and assembles arrays; it holds none of the
rasterizer's arithmetic (projection, binning, compositing, gradients), so the
oracle and the CUDA path can both consume it without sharing method code.
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# --------------------------------------------------------------------------
# Cameras and poses
# --------------------------------------------------------------------------

def camera(W, H, fx, fy=None, R=None, t=None, sx=1, sy=1):
    """Pinhole camera dict; principal point at the image centre."""
    fy = fx if fy is None else fy
    return {
        "R": np.eye(3) if R is None else np.asarray(R, dtype=np.float64).reshape(3, 3),
        "t": np.zeros(3) if t is None else np.asarray(t, dtype=np.float64).reshape(3),
        "fx": float(fx), "fy": float(fy), "cx": W / 2.0, "cy": H / 2.0,
        "W": int(W), "H": int(H), "sx": int(sx), "sy": int(sy),
    }


def axis_angle_matrix(axis, angle):
    """Rotation by `angle` radians about unit `axis` (Rodrigues' formula);
    used only to build test poses."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def perturbed_pose(cam, seed, trans=0.02, rot_deg=1.0):
    """The camera moved by `trans` metres along a random direction and rotated
    by `rot_deg` degrees about a random axis (left-multiplied on T_cw)."""
    g = rng(seed)
    d = g.normal(size=3)
    d /= np.linalg.norm(d)
    ax = g.normal(size=3)
    Rd = axis_angle_matrix(ax, math.radians(rot_deg))
    c = dict(cam)
    c["R"] = Rd @ np.asarray(cam["R"])
    c["t"] = Rd @ np.asarray(cam["t"]) + trans * d
    return c


def look_at(eye, target, up=(0.0, -1.0, 0.0)):
    """World->camera (R, t) for a camera at `eye` looking at `target`
    (camera z forward, y down)."""
    eye = np.asarray(eye, dtype=np.float64)
    z = np.asarray(target, dtype=np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(np.asarray(up, dtype=np.float64), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    return R, -R @ eye


# --------------------------------------------------------------------------
# 3D Gaussian maps
# --------------------------------------------------------------------------

def random_unit_quats(g, n):
    q = g.normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def tiny_scene(seed=1000, n=2000):
    """Plain tiny single view: means uniform in the camera-frame box
    x, y in [-1, 1], z in [2, 5]; log-scales N(-3, 0.3); random unit
    quaternions; opacity logits N(0, 1); RGB uniform [0, 1]."""
    g = rng(seed)
    means = np.stack([g.uniform(-1, 1, n), g.uniform(-1, 1, n), g.uniform(2, 5, n)], 1)
    return {
        "means": means.astype(np.float32),
        "log_scales": g.normal(-3.0, 0.3, (n, 3)).astype(np.float32),
        "quats": random_unit_quats(g, n).astype(np.float32),
        "opacity_logit": g.normal(0.0, 1.0, n).astype(np.float32),
        "rgb": g.uniform(0, 1, (n, 3)).astype(np.float32),
    }


def tiny_camera():
    return camera(96, 72, 80.0)


def surface_scene(n, seed, n_planes=6, n_spheres=4, plane_frac=0.7, log_scale_mu=-4.5,
                  log_scale_sd=0.5, jitter=0.01):
    """SLAM-like map: n Gaussians on `n_planes` 4x4 m planes 1-6 m ahead of
    the identity camera and `n_spheres` spheres (radius 0.2-0.6 m, centres at
    z in [2, 5]); `plane_frac` of the points on planes, split by area inside
    each group; N(0, jitter) surface noise; log-scales N(mu, sd); opacity
    logits N(2, 1); RGB a smooth per-surface colour plus U[-0.1, 0.1]."""
    g = rng(seed)
    n_pl = int(round(n * plane_frac))
    n_sp = n - n_pl
    pts, cols = [], []
    # planes: centre ahead of the camera, normal roughly facing it
    pl_area = np.full(n_planes, 16.0)
    counts = g.multinomial(n_pl, pl_area / pl_area.sum())
    for i in range(n_planes):
        c = np.array([g.uniform(-1.5, 1.5), g.uniform(-1.0, 1.0), g.uniform(1.0, 6.0)])
        nrm = np.array([g.uniform(-0.6, 0.6), g.uniform(-0.6, 0.6), -1.0])
        nrm /= np.linalg.norm(nrm)
        a = np.cross(nrm, [0.0, 1.0, 0.0])
        a /= np.linalg.norm(a)
        b = np.cross(nrm, a)
        s = g.uniform(-2, 2, (counts[i], 2))
        p = c + s[:, :1] * a + s[:, 1:] * b
        base = g.uniform(0.15, 0.85, 3)
        freq = g.uniform(1.0, 4.0, 3)
        col = base + 0.15 * np.sin(freq * s[:, :1] + 2.0 * s[:, 1:] + g.uniform(0, 6, 3))
        pts.append(p)
        cols.append(col)
    radii = g.uniform(0.2, 0.6, n_spheres)
    counts = g.multinomial(n_sp, radii ** 2 / (radii ** 2).sum())
    for i in range(n_spheres):
        c = np.array([g.uniform(-1.2, 1.2), g.uniform(-0.8, 0.8), g.uniform(2.0, 5.0)])
        d = g.normal(size=(counts[i], 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        p = c + radii[i] * d
        base = g.uniform(0.15, 0.85, 3)
        col = base + 0.15 * d[:, [1, 2, 0]]
        pts.append(p)
        cols.append(col)
    means = np.concatenate(pts) + g.normal(0, jitter, (n, 3))
    rgb = np.clip(np.concatenate(cols) + g.uniform(-0.1, 0.1, (n, 3)), 0, 1)
    perm = g.permutation(n)
    return {
        "means": means[perm].astype(np.float32),
        "log_scales": g.normal(log_scale_mu, log_scale_sd, (n, 3)).astype(np.float32),
        "quats": random_unit_quats(g, n).astype(np.float32),
        "opacity_logit": g.normal(2.0, 1.0, n).astype(np.float32),
        "rgb": rgb[perm].astype(np.float32),
    }


def tracking_workload(n=200_000, W=640, H=480, f=525.0, seed=2000):
    """SLAM tracking frame: 640x480, 200k surface-sampled Gaussians; the target
    is rendered from the identity pose, tracking starts 2 cm / 1 deg away."""
    scene = surface_scene(n, seed)
    true_cam = camera(W, H, f)
    start_cam = perturbed_pose(true_cam, seed + 1)
    return scene, true_cam, start_cam


def arc_keyframes(n_kf=8, W=1200, H=680, f=600.0, seed=3000, arc=1.0, centre=(0.0, 0.0, 3.5)):
    """Keyframe cameras with centres on a 1 m circular arc around the origin,
    each looking at the scene centre."""
    g = rng(seed)
    cams = []
    rad = 3.5
    half = arc / rad / 2.0
    for a in np.linspace(-half, half, n_kf):
        eye = np.array([rad * math.sin(a), g.uniform(-0.05, 0.05), 3.5 - rad * math.cos(a)])
        R, t = look_at(eye, centre)
        cams.append(camera(W, H, f, R=R, t=t))
    return cams


# --------------------------------------------------------------------------
# Stage-isolated inputs
# --------------------------------------------------------------------------

def splats(n, W, H, seed, tie_frac=0.05, cull_frac=0.03, sigma_px=(0.6, 12.0), depth=(0.5, 10.0),
           opaque_frac=0.1, aniso=(0.25, 1.0)):
    """Projected 2D Gaussians drawn directly (for stage-isolated binning and
    compositing tests): 2D means uniform over the image plus a 20 px margin,
    random anisotropic 2D covariances given by their inverse (the conic;
    minor / major sigma U(aniso)),
    radius ceil(3 sigma_max) as an input, opacity U(0.05, 0.99) with
    `opaque_frac` at 0.995 (so the alpha clamp is exercised), RGB U[0,1],
    depth U(depth) with `tie_frac` copying another Gaussian's depth exactly
    (equal keys), and `cull_frac` with radius 0.  All float32 / int32."""
    g = rng(seed)
    u = g.uniform(-20, W + 20, n)
    v = g.uniform(-20, H + 20, n)
    s1 = np.exp(g.uniform(math.log(sigma_px[0]), math.log(sigma_px[1]), n))
    s2 = s1 * g.uniform(aniso[0], aniso[1], n)
    th = g.uniform(0, math.pi, n)
    c, s = np.cos(th), np.sin(th)
    i1, i2 = 1.0 / s1 ** 2, 1.0 / s2 ** 2
    A = c * c * i1 + s * s * i2
    B = c * s * (i1 - i2)
    Cc = s * s * i1 + c * c * i2
    op = g.uniform(0.05, 0.99, n)
    op[g.random(n) < opaque_frac] = 0.995
    d = g.uniform(depth[0], depth[1], n).astype(np.float32)
    ties = np.nonzero(g.random(n) < tie_frac)[0]
    if len(ties):
        d[ties] = d[g.integers(0, n, len(ties))]
    rad = np.ceil(3.0 * s1).astype(np.int32)
    rad[g.random(n) < cull_frac] = 0
    return {
        "uv": np.stack([u, v], 1).astype(np.float32),
        "conic": np.stack([A, B, Cc], 1).astype(np.float32),
        "opacity": op.astype(np.float32),
        "rgb": g.uniform(0, 1, (n, 3)).astype(np.float32),
        "depth": d,
        "radius": rad,
    }


def target_image(W, H, seed, depth_range=(2.0, 5.0), invalid_frac=0.1):
    """Uniform random RGB target [3,H,W] and depth target [H,W] with
    `invalid_frac` zero (invalid) depths."""
    g = rng(seed)
    rgb = g.uniform(0, 1, (3, H, W)).astype(np.float32)
    dep = g.uniform(depth_range[0], depth_range[1], (H, W)).astype(np.float32)
    dep[g.random((H, W)) < invalid_frac] = 0
    return rgb, dep


def image_grads(W, H, seed, scale=1.0):
    """Random dL/dimage [3,H,W] and dL/ddepth [H,W] for stage tests."""
    g = rng(seed)
    P = W * H
    return ((g.normal(0, 1, (3, H, W)) * scale / P).astype(np.float32),
            (g.normal(0, 1, (H, W)) * scale / P).astype(np.float32))


def score_terms(n, seed, tie_frac=0.1):
    """Non-negative Eq. 7 score terms with deliberate ties."""
    g = rng(seed)
    t = np.abs(g.standard_cauchy((n, 2))).astype(np.float32) * 1e-3
    ties = np.nonzero(g.random(n) < tie_frac)[0]
    if len(ties):
        t[ties] = t[g.integers(0, n, len(ties))]
    return t
