"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics:
closed forms, invariants, special cases, brute force and finite differences.
None of these tests retypes an oracle formula; each one checks the oracle
against an independent route to the same number."""
import json
import math
import os

import numpy as np
import pytest

from synth import scenes as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def one_gaussian(x, y, z, log_scale, ologit, rgb, quat=(1.0, 0.0, 0.0, 0.0)):
    ls = np.broadcast_to(np.asarray(log_scale, dtype=np.float64), (3,))
    return {
        "means": np.array([[x, y, z]]),
        "log_scales": ls.reshape(1, 3).copy(),
        "quats": np.array([quat], dtype=np.float64),
        "opacity_logit": np.array([ologit]),
        "rgb": np.array([rgb], dtype=np.float64),
    }


def concat(*gs):
    return {k: np.concatenate([g[k] for g in gs]) for k in gs[0]}


# ---------------------------------------------------------------------------
# Closed form: one isotropic Gaussian on the optical axis (Eq. 2, Eq. 3)
# ---------------------------------------------------------------------------

def closed_form_single(W, H, f, z, s, o, c):
    """Image of one isotropic Gaussian at camera (0,0,z): the EWA covariance is
    (f s / z)^2 I + 0.3 I, the radius ceil(3 sqrt(sigma^2 + sqrt(0.1))), and
    each pixel inside the radius box gets alpha = o exp(-d^2 / 2 sigma^2)."""
    sig2 = (f * s / z) ** 2 + 0.3
    r = math.ceil(3 * math.sqrt(sig2 + math.sqrt(0.1)))
    img = np.zeros((3, H, W))
    dep = np.zeros((H, W))
    T = np.ones((H, W))
    cx, cy = W / 2, H / 2
    for py in range(H):
        for px in range(W):
            if abs(px - math.floor(cx)) > r or abs(py - math.floor(cy)) > r:
                continue
            d2 = (px + 0.5 - cx) ** 2 + (py + 0.5 - cy) ** 2
            a = min(0.99, o * math.exp(-d2 / (2 * sig2)))
            if a < 1 / 255:
                continue
            img[:, py, px] = a * np.asarray(c)
            dep[py, px] = a * z
            T[py, px] = 1 - a
    return img, dep, T, r, sig2


@pytest.mark.parametrize("W,H,f,z,s,ol", [(64, 48, 80.0, 3.0, 0.08, 0.3), (32, 32, 50.0, 2.0, 0.2, 1.5)])
def test_single_isotropic_closed_form(oracle_lib, W, H, f, z, s, ol):
    O = oracle_lib
    c = (0.2, 0.5, 0.9)
    g = one_gaussian(0.0, 0.0, z, math.log(s), ol, c)
    cam = S.camera(W, H, f)
    pr, img = O.forward(g, cam)
    o = 1 / (1 + math.exp(-ol))
    ref, dref, Tref, r, sig2 = closed_form_single(W, H, f, z, s, o, c)
    assert pr["radius"][0] == r
    np.testing.assert_allclose(pr["conic"][0], [1 / sig2, 0, 1 / sig2], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(img["rgb"], ref, atol=1e-12)
    np.testing.assert_allclose(img["depth"], dref, atol=1e-12)
    np.testing.assert_allclose(img["T"], Tref, atol=1e-12)
    # even W, H: the image is symmetric under both flips
    np.testing.assert_allclose(img["rgb"], img["rgb"][:, ::-1, :], atol=1e-13)
    np.testing.assert_allclose(img["rgb"], img["rgb"][:, :, ::-1], atol=1e-13)
    # brute force agrees
    _, imgb = O.forward(g, cam, tiled=False)
    np.testing.assert_array_equal(img["rgb"], imgb["rgb"])


def test_single_isotropic_gradients_closed_form(oracle_lib):
    """For L = sum_P w_P C_P (one channel weight per pixel, symmetric weights)
    the derivatives follow from alpha = o exp(-(dx^2/sx2 + dy^2/sy2)/2) with
    sx2 = (f/z)^2 exp(2 ls_x) + 0.3: dL/dc, dL/dlogit, dL/dz, dL/dls_x and
    dL/dls_y in closed form; dL/dx = dL/dy = 0 and dL/dls_z = 0 exactly by
    symmetry and because J has no z column on the axis."""
    O = oracle_lib
    W, H, f, z, s, ol = 40, 40, 60.0, 2.5, 0.1, -0.5
    c = np.array([0.3, 0.6, 0.9])
    g = one_gaussian(0.0, 0.0, z, math.log(s), ol, c)
    cam = S.camera(W, H, f)
    w = np.ones((3, H, W))
    wd = np.full((H, W), 0.7)
    pr, g2, gb = O.forward_backward(g, cam, w, wd)
    o = 1 / (1 + math.exp(-ol))
    sig2 = (f * s / z) ** 2 + 0.3
    r = pr["radius"][0]
    dc = 0.0
    dlogit = 0.0
    dz = 0.0
    dlsx = 0.0
    for py in range(H):
        for px in range(W):
            if abs(px - W // 2) > r or abs(py - H // 2) > r:
                continue
            dx2 = (px + 0.5 - W / 2) ** 2
            dy2 = (py + 0.5 - H / 2) ** 2
            a = o * math.exp(-(dx2 + dy2) / (2 * sig2))
            if a < 1 / 255:
                continue
            dc += a
            # C = a c, D = a z, weights: 1 per colour channel, 0.7 for depth
            dLda = c.sum() + 0.7 * z
            dlogit += dLda * a * (1 - o)
            dsig2_dz = -2 * (f * s) ** 2 / z ** 3
            da_dz = a * (dx2 + dy2) / (2 * sig2 ** 2) * dsig2_dz
            dz += dLda * da_dz + 0.7 * a
            dsx2 = 2 * (f / z) ** 2 * s * s
            dlsx += dLda * a * dx2 / (2 * sig2 ** 2) * dsx2
    np.testing.assert_allclose(gb["rgb"][0], [dc, dc, dc], rtol=1e-10)
    np.testing.assert_allclose(gb["opacity_logit"][0], dlogit, rtol=1e-10)
    np.testing.assert_allclose(gb["means"][0, 2], dz, rtol=1e-9)
    np.testing.assert_allclose(gb["log_scales"][0, 0], dlsx, rtol=1e-9)
    np.testing.assert_allclose(gb["log_scales"][0, 1], dlsx, rtol=1e-9)
    assert abs(gb["means"][0, 0]) < 1e-12 and abs(gb["means"][0, 1]) < 1e-12
    assert abs(gb["log_scales"][0, 2]) < 1e-12
    # Eq. 7 score terms: dL/dmu = (0, 0, dL/dz); Sigma = s^2 I only reaches the
    # 2D covariance through its x-y block ((f/z)^2 times it on the axis), the
    # mirror symmetry of the image zeroes the x-y entry, and Sigma_xx = s_x^2
    # gives dL/dls_x = 2 s^2 dL/dSigma_xx: ||dL/dSigma||_F = sqrt(2) |dls_x| / (2 s^2)
    np.testing.assert_allclose(gb["score_terms"][0, 0], abs(dz), rtol=1e-9)
    np.testing.assert_allclose(gb["score_terms"][0, 1], math.sqrt(2) * abs(dlsx) / (2 * s * s), rtol=1e-9)


# ---------------------------------------------------------------------------
# Occlusion and early termination (Eq. 3 note)
# ---------------------------------------------------------------------------

def test_opaque_front_scales_behind_by_one_hundredth(oracle_lib):
    """A huge front Gaussian with logit 20 has alpha clamped at 0.99 over the
    whole image, so whatever lies behind is weighted by exactly T = 0.01."""
    O = oracle_lib
    W, H, f = 32, 32, 40.0
    front = one_gaussian(0.0, 0.0, 2.0, math.log(50.0), 20.0, (1.0, 0.0, 0.0))
    behind = one_gaussian(0.0, 0.0, 4.0, math.log(0.1), 0.0, (0.0, 1.0, 0.0))
    cam = S.camera(W, H, f)
    _, both = O.forward(concat(front, behind), cam)
    _, only_b = O.forward(behind, cam)
    np.testing.assert_allclose(both["rgb"][0], 0.99, atol=1e-12)
    np.testing.assert_allclose(both["rgb"][1], 0.01 * only_b["rgb"][1], atol=1e-14)


def test_three_opaque_fronts_terminate_before_behind(oracle_lib):
    """After opaque fronts drive T to ~1e-4 the ray stops: the Gaussian behind
    gets exactly zero contribution and exactly zero gradient."""
    O = oracle_lib
    W, H, f = 32, 32, 40.0
    fronts = [one_gaussian(0.0, 0.0, 2.0 + 0.01 * i, math.log(50.0), 20.0, (1.0, 0.0, 0.0))
              for i in range(3)]
    behind = one_gaussian(0.0, 0.0, 4.0, math.log(0.1), 3.0, (0.0, 1.0, 0.0))
    g = concat(*fronts, behind)
    cam = S.camera(W, H, f)
    _, img = O.forward(g, cam)
    assert np.all(img["rgb"][1] == 0.0)
    w = np.ones((3, H, W))
    _, g2, gb = O.forward_backward(g, cam, w, np.ones((H, W)))
    assert np.all(g2[3] == 0.0)
    for k in ("means", "log_scales", "quats", "rgb"):
        assert np.all(gb[k][3] == 0.0)
    # clamped fronts: no gradient through alpha to opacity or shape
    assert np.all(gb["opacity_logit"][:3] == 0.0)
    assert np.all(g2[:3, 0:6] == 0.0)


def test_termination_tests_the_transmittance_after_the_fragment(oracle_lib):
    """The ray stops before fragment k when T (1 - a_k) < t_eps (Eq. 3 note).
    Fronts with a = 0.99 then a ~ 0.5 leave T = 0.005 > t_eps; a third opaque
    layer would bring it to 5e-5 < t_eps, so it is not blended at all, and
    T_final stays 0.005 although T itself never fell below t_eps."""
    O = oracle_lib
    W, H, f = 16, 16, 20.0
    g = concat(one_gaussian(0, 0, 2.0, math.log(80.0), 20.0, (1.0, 0.0, 0.0)),
               one_gaussian(0, 0, 2.5, math.log(80.0), 0.0, (0.0, 1.0, 0.0)),
               one_gaussian(0, 0, 3.0, math.log(80.0), 20.0, (0.0, 0.0, 1.0)))
    _, img = O.forward(g, S.camera(W, H, f))
    assert np.all(img["rgb"][2] == 0.0)
    assert np.all(img["nfrag"] == 2)
    a2 = img["rgb"][1] / 0.01
    np.testing.assert_allclose(a2, 0.5, atol=1e-3)
    np.testing.assert_allclose(img["T"], 0.01 * (1 - a2), rtol=1e-12)


# ---------------------------------------------------------------------------
# Compositing invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.25, 0.5, 0.75)])
def test_transmittance_partition_of_unity(oracle_lib, bg):
    """With every colour 1, C = sum_k T_k a_k + T_final bg and the weights
    T_k a_k sum to 1 - T_final, so C + T_final (1 - bg) = 1 per pixel and
    channel (Eq. 3 with the background behind the last fragment); with every
    depth z0, D = z0 (1 - T_final) (no background depth)."""
    O = oracle_lib
    g = S.tiny_scene(seed=7, n=600)
    cam = S.tiny_camera()
    pr = O.project(g, cam)
    pr["rgb"] = np.ones_like(pr["rgb"])
    pr["depth"] = np.full_like(pr["depth"], 3.25)
    img = O.render_fwd(pr, cam, cfg={"bg": bg})
    for ch in range(3):
        np.testing.assert_allclose(img["rgb"][ch] + img["T"] * (1.0 - bg[ch]), 1.0, atol=1e-12)
    np.testing.assert_allclose(img["depth"], 3.25 * (1 - img["T"]), atol=1e-12)
    assert img["nfrag"].max() > 5
    assert img["T"].min() < 0.5 and img["T"].max() == 1.0


def test_tiled_equals_brute_force(oracle_lib):
    O = oracle_lib
    g = S.tiny_scene(seed=1000)
    cam = S.tiny_camera()
    pr = O.project(g, cam)
    a = O.render_fwd(pr, cam, tiled=True)
    b = O.render_fwd(pr, cam, tiled=False)
    for k in ("rgb", "depth", "T", "nfrag"):
        np.testing.assert_array_equal(a[k], b[k])
    d_rgb, d_dep = S.image_grads(cam["W"], cam["H"], 11)
    ga = O.render_bwd(pr, cam, d_rgb, d_dep, tiled=True)
    gb = O.render_bwd(pr, cam, d_rgb, d_dep, tiled=False)
    np.testing.assert_array_equal(ga, gb)


def one_splat(u, v, op, sig2, radius, depth=3.0):
    """One isotropic 2D Gaussian as projected splats (conic 1 / sig2)."""
    return {"uv": np.array([[u, v]], np.float64), "conic": np.array([[1 / sig2, 0.0, 1 / sig2]]),
            "opacity": np.array([op]), "rgb": np.array([[0.2, 0.5, 0.8]]), "depth": np.array([depth]),
            "radius": np.array([radius])}


@pytest.mark.parametrize("tiled", [True, False])
@pytest.mark.parametrize("u,v,axis,edges", [
    (32.5, 40.0 - 1e-7, "y", (33, 46)),   # floor 39 in float64, 40 in float32
    (32.5, 40.0 + 1e-7, "y", (33, 46)),   # floor 40, 39 a rounding away
    (32.0 + 1e-7, 40.3, "x", (25, 38)),   # floor 32, 31 a rounding away
    (32.0 - 1e-7, 40.3, "x", (25, 38)),   # floor 31, 32 in float32
])
def test_box_edge_decided_by_floor_is_marginal(oracle_lib, tiled, u, v, axis, edges):
    """The integer box of reading new-1 floors the mean (r = 6).  A mean
    within a rounding of an integer puts the box's two edge lines (rows or
    columns) on either side of the decision: exactly those pixels, inside the
    other axis's extent, are marked marginal; the float64 floor decides what
    blends.  A mean far from an integer marks nothing, nor does an ambiguous
    edge where the Gaussian does not reach alpha_min."""
    O = oracle_lib
    cam = S.camera(64, 64, 60.0)
    img = O.render_fwd(one_splat(u, v, 0.9, 16.0, 6), cam, tiled=tiled)
    xi, yi = math.floor(u), math.floor(v)
    want = np.zeros((64, 64), np.uint8)
    if axis == "y":
        want[list(edges), xi - 6:xi + 7] = 1
        inside = [e for e in edges if yi - 6 <= e <= yi + 6]
        outside = [e for e in edges if e not in inside]
        assert len(inside) == 1 and np.all(img["nfrag"][inside[0], xi - 6:xi + 7] == 1)
        assert np.all(img["nfrag"][outside[0], :] == 0)
    else:
        want[yi - 6:yi + 7, list(edges)] = 1
        inside = [e for e in edges if xi - 6 <= e <= xi + 6]
        outside = [e for e in edges if e not in inside]
        assert len(inside) == 1 and np.all(img["nfrag"][yi - 6:yi + 7, inside[0]] == 1)
        assert np.all(img["nfrag"][:, outside[0]] == 0)
    np.testing.assert_array_equal(img["margin"], want)
    # the blended pixels follow Eq. 2 with the float64 box
    a = 0.9 * np.exp(-((np.arange(xi - 6, xi + 7) + 0.5 - u) ** 2 + (yi + 0.5 - v) ** 2) / 32.0)
    np.testing.assert_allclose(img["rgb"][1, yi, xi - 6:xi + 7], 0.5 * a, rtol=1e-12)
    ctrl = O.render_fwd(one_splat(32.5, 40.3, 0.9, 16.0, 6), cam, tiled=tiled)
    assert ctrl["margin"].sum() == 0 and ctrl["nfrag"].sum() == 13 * 13
    # sigma 2: alpha at the edge rows <= 0.5 exp(-6.5^2 / 8) < 1/255
    faint = O.render_fwd(one_splat(u, v, 0.5, 4.0, 6), cam, tiled=tiled)
    assert faint["margin"].sum() == 0


def test_margin_windows(oracle_lib):
    """The oracle marks a pixel marginal where float32 and float64 may take a
    predicate apart: alpha within a relative 1e-4 of alpha_min or alpha_max,
    the exponent within 1e-6 of 0, the transmittance after a fragment within
    a relative 1e-4 of t_eps.  Each case places exactly known pixels inside
    the window (sigma^2 = 16, radius 8, so alpha_min is never approached
    elsewhere) and checks that only they are marked."""
    O = oracle_lib
    cam = S.camera(64, 64, 60.0)
    amin, amax = 1 / 255, 0.99
    def run(sp):
        return O.render_fwd(sp, cam)["margin"]
    def only(*pix):
        m = np.zeros((64, 64), np.uint8)
        for x, y in pix:
            m[y, x] = 1
        return m
    # alpha_min: pixel offsets (3.2, 0.2) and (0.2, 3.2) from (32.3, 32.3)
    op = amin * (1 + 5e-5) / math.exp(-(3.2 ** 2 + 0.2 ** 2) / 32)
    np.testing.assert_array_equal(run(one_splat(32.3, 32.3, op, 16.0, 8)), only((35, 32), (32, 35)))
    # alpha_max: the pixel at offset (0.2, 0.2)
    op = amax * (1 - 5e-5) / math.exp(-0.08 / 32)
    np.testing.assert_array_equal(run(one_splat(32.3, 32.3, op, 16.0, 8)), only((32, 32)))
    # exponent 0: the mean on the centre of pixel (32, 32)
    np.testing.assert_array_equal(run(one_splat(32.5, 32.5, 0.5, 16.0, 8)), only((32, 32)))
    # t_eps: three fronts of alpha a at (32, 32) leave (1 - a)^3 = 1e-4 (1 + 5e-5)
    a = 1 - (1e-4 * (1 + 5e-5)) ** (1 / 3)
    op = a / math.exp(-0.08 / 32)
    three = [one_splat(32.3, 32.3, op, 16.0, 8, depth=d) for d in (2.0, 3.0, 4.0)]
    sp = {k: np.concatenate([t[k] for t in three]) for k in three[0]}
    np.testing.assert_array_equal(run(sp), only((32, 32)))


def test_ewa_jacobian_clamp_closed_form(oracle_lib):
    """An isotropic Gaussian (scale s) at camera point (x, 0, z), R = I: the
    EWA Jacobian is [[f/z, 0, -f t/z], [0, f/z, 0]] with t = x/z clamped to
    1.3 (W/2)/f (reading c5: inside J only), so Sigma2 = s^2 J J^T + 0.3 I =
    diag(s^2 f^2 (1 + t^2)/z^2 + 0.3, s^2 f^2/z^2 + 0.3) and the mean
    projects unclamped to f x/z + W/2.  Likewise on the y axis, with the
    clamp line 1.3 (H/2)/f."""
    O = oracle_lib
    W, H, f, z, s = 64, 48, 80.0, 4.0, 0.05
    limx, limy = 1.3 * (W / 2) / f, 1.3 * (H / 2) / f   # 0.52, 0.39
    cam = S.camera(W, H, f)
    q = s * s * f * f / (z * z)
    for xz in (0.3, 0.8):
        pr = O.project(one_gaussian(xz * z, 0.0, z, math.log(s), 2.0, [0.5, 0.5, 0.5]), cam)
        t = min(xz, limx)
        np.testing.assert_allclose(pr["conic"][0], [1 / (q * (1 + t * t) + 0.3), 0.0, 1 / (q + 0.3)],
                                   rtol=1e-12, atol=1e-15)
        assert math.isclose(pr["uv"][0, 0], f * xz + W / 2, rel_tol=1e-14)
    for yz in (0.3, 0.8):
        pr = O.project(one_gaussian(0.0, yz * z, z, math.log(s), 2.0, [0.5, 0.5, 0.5]), cam)
        t = min(yz, limy)
        np.testing.assert_allclose(pr["conic"][0], [1 / (q + 0.3), 0.0, 1 / (q * (1 + t * t) + 0.3)],
                                   rtol=1e-12, atol=1e-15)
        assert math.isclose(pr["uv"][0, 1], f * yz + H / 2, rel_tol=1e-14)


def test_project_rects_match_the_lists(oracle_lib):
    """or_project's tile rect and count per Gaussian are those of the binning
    (the same alpha-aware rect, reading new-2): counted from the sorted
    lists, Gaussian k appears touched[k] times, and its listed tiles span
    exactly rect[k] = (x0, x1, y0, y1); a Gaussian with no tile (culled, as
    the one behind the near plane, off-screen, or below alpha_min) has an
    all-zero rect."""
    O = oracle_lib
    g = concat(S.tiny_scene(seed=1200, n=600), one_gaussian(0.0, 0.0, 0.1, -3.0, 0.0, [1, 1, 1]))
    cam = S.tiny_camera()
    pr = O.project(g, cam)
    _, vals, ranges = O.bin_sort(pr, cam)
    n = len(pr["radius"])
    assert pr["radius"][-1] == 0
    cnt = np.bincount(vals.astype(np.int64), minlength=n)
    np.testing.assert_array_equal(cnt, pr["touched"])
    _, _, TX, TY = O.grid(cam)
    lo = np.full((n, 2), 1 << 30)
    hi = np.full((n, 2), -1)
    for t in range(TX * TY):
        b, e = ranges[t]
        ids = vals[b:e].astype(np.int64)
        np.minimum.at(lo, ids, [t % TX, t // TX])
        np.maximum.at(hi, ids, [t % TX, t // TX])
    listed = cnt > 0
    assert listed.sum() > 100
    np.testing.assert_array_equal(pr["rect"][listed], np.stack([lo[listed, 0], hi[listed, 0] + 1,
                                                                lo[listed, 1], hi[listed, 1] + 1], 1))
    assert not pr["rect"][~listed].any() and not pr["touched"][~listed].any()


def test_alpha_aware_tiles_lose_no_fragment(oracle_lib):
    """The tile lists leave out a Gaussian only where it cannot reach
    alpha_min (reading new-2): every (pixel, Gaussian) pair whose float64
    alpha is at least alpha_min inside the integer box sits in the pixel's
    tile list, at strides 1 and 2, on faint and anisotropic Gaussians."""
    O = oracle_lib
    s = S.splats(1500, 96, 64, seed=31, sigma_px=(0.6, 10.0))
    # the alpha extent does shrink rects here: about a quarter fewer keys than
    # with the integer boxes alone (opaque, very wide conics)
    wide = dict(s, opacity=np.ones(1500), conic=s["conic"] * 1e-6)
    assert len(O.bin_sort(s, S.camera(96, 64, 80.0))[0]) < 0.85 * len(O.bin_sort(wide, S.camera(96, 64, 80.0))[0])
    for sx in (1, 2):
        cam = S.camera(96, 64, 80.0, sx=sx, sy=sx)
        keys, vals, ranges = O.bin_sort(s, cam)
        Ws, Hs, TX, TY = O.grid(cam)
        td = O.tile_dim(sx)
        lists = [set(vals[b:e].tolist()) for b, e in ranges]
        a, bq, c = s["conic"][:, 0], s["conic"][:, 1], s["conic"][:, 2]
        for j in range(Hs):
            for i in range(Ws):
                px, py = i * sx, j * sx
                dx = px + 0.5 - s["uv"][:, 0].astype(np.float64)
                dy = py + 0.5 - s["uv"][:, 1].astype(np.float64)
                power = -0.5 * (a * dx * dx + c * dy * dy) - bq * dx * dy
                alpha = np.minimum(0.99, s["opacity"] * np.exp(np.minimum(power, 0)))
                xi = np.floor(s["uv"][:, 0]).astype(np.int64)
                yi = np.floor(s["uv"][:, 1]).astype(np.int64)
                r = s["radius"]
                inbox = (r > 0) & (np.abs(px - xi) <= r) & (np.abs(py - yi) <= r)
                need = np.nonzero(inbox & (power <= 0) & (alpha >= 1 / 255))[0]
                have = lists[(j // td) * TX + i // td]
                assert set(need.tolist()) <= have, (sx, i, j)


def test_alpha_aware_rects_are_tight(oracle_lib):
    """How loose the binning's alpha-aware tile rect may be (reading new-2):
    per Gaussian it contains the tile rect of the exact set of pixels that
    can reach alpha_min in float64 (inside the integer box), and over the
    scene it holds at most 8 % more (tile, Gaussian) keys than those exact
    rects (6.4 % on this scene of small, faint and anisotropic Gaussians: the
    float32 bound's slack -- the 1.002 factor, 2e-3 px, the 1e-3 added to the
    log bound, and the bounding box of the ellipse rather than the pixels that
    reach alpha_min -- costs few keys).  Against the integer 3-sigma boxes
    alone the rects save about a fifth of the keys."""
    O = oracle_lib
    W, H = 96, 64
    s = S.splats(1500, W, H, seed=31, sigma_px=(0.6, 10.0))
    cam = S.camera(W, H, 80.0)
    keys, vals, ranges = O.bin_sort(s, cam)
    Ws, Hs, TX, TY = O.grid(cam)
    td = O.tile_dim(1)
    have = {}
    for t, (b, e) in enumerate(ranges):
        for k in vals[b:e].tolist():
            have.setdefault(k, set()).add(t)
    ys, xs = np.mgrid[0:H, 0:W]
    exact_keys = 0
    box_keys = 0
    for k in range(1500):
        r = int(s["radius"][k])
        if r <= 0:
            continue
        u, v = float(s["uv"][k, 0]), float(s["uv"][k, 1])
        xi, yi = math.floor(u), math.floor(v)
        inbox = (np.abs(xs - xi) <= r) & (np.abs(ys - yi) <= r)
        if inbox.any():
            bx = xs[inbox]; by = ys[inbox]
            box_keys += (bx.max() // td - bx.min() // td + 1) * (by.max() // td - by.min() // td + 1)
        a, b, c = (float(x) for x in s["conic"][k])
        dx = xs + 0.5 - u
        dy = ys + 0.5 - v
        power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
        alpha = np.minimum(0.99, float(s["opacity"][k]) * np.exp(np.minimum(power, 0)))
        need = inbox & (power <= 0) & (alpha >= 1 / 255)
        if not need.any():
            continue
        px, py = xs[need], ys[need]
        rect = {(j * TX + i) for j in range(py.min() // td, py.max() // td + 1)
                for i in range(px.min() // td, px.max() // td + 1)}
        assert rect <= have.get(k, set()), k
        exact_keys += len(rect)
    assert exact_keys <= len(keys) <= 1.08 * exact_keys, (len(keys), exact_keys)
    assert len(keys) < 0.85 * box_keys


def test_tiled_equals_brute_force_on_stage_splats(oracle_lib):
    O = oracle_lib
    s = S.splats(400, 70, 50, seed=3)
    cam = S.camera(70, 50, 60.0)
    a = O.render_fwd(s, cam, tiled=True)
    b = O.render_fwd(s, cam, tiled=False)
    for k in ("rgb", "depth", "T", "nfrag"):
        np.testing.assert_array_equal(a[k], b[k])


# ---------------------------------------------------------------------------
# Binning and sort
# ---------------------------------------------------------------------------

def test_binning_hand_cases(oracle_lib):
    O = oracle_lib
    cam = S.camera(64, 48, 50.0)   # 4 x 3 tiles
    uv = np.array([[20.5, 5.2], [16.0, 40.0], [-3.5, 10.0], [63.9, 47.9]])
    depth = np.array([2.0, 1.5, 3.0, 2.5])
    radius = np.array([4, 1, 2, 1])
    # nearly opaque isotropic Gaussians with sigma = r / 3: alpha >= 1/255
    # reaches 3.4 sigma > r, so the integer boxes decide these rects
    sig2 = (radius / 3.0) ** 2
    conic = np.stack([1.0 / sig2, np.zeros(4), 1.0 / sig2], 1)
    opac = np.full(4, 0.99)
    spl = lambda sl: {"uv": uv[sl], "depth": depth[sl], "radius": radius[sl], "conic": conic[sl],
                      "opacity": opac[sl]}
    keys, vals, ranges = O.bin_sort(spl(slice(None)), cam)
    bits = lambda d: int(np.array(d, np.float32).view(np.uint32))
    # G0: box x [16,24] -> tile col 1, y [1,9] -> row 0 -> tile 1
    # G1: box x [15,17] -> cols 0,1; y [39,41] -> row 2 -> tiles 8, 9
    # G2: box x [-6,-2] -> no pixel -> no key
    # G3: box x [62,64] -> col 3 (64 is off-image), y [46,48] -> row 2 -> tile 11
    expect = sorted([(1 << 32 | bits(2.0), 0), (8 << 32 | bits(1.5), 1), (9 << 32 | bits(1.5), 1),
                     (11 << 32 | bits(2.5), 3)])
    assert [(int(k), int(v)) for k, v in zip(keys, vals)] == expect
    assert ranges[1].tolist() == [0, 1]
    assert ranges[8].tolist() == [1, 2] and ranges[9].tolist() == [2, 3]
    assert ranges[11].tolist() == [3, 4]
    assert ranges[0].tolist() == [0, 0]
    # stride 2: tiles are 8x8 sampled pixels; the sampled columns of G0 are
    # 8..12 -> tile column 1, rows 1..4 -> tile row 0; TX = ceil(32/8) = 4
    cam2 = dict(cam, sx=2, sy=2)
    k2, v2, r2 = O.bin_sort(spl(slice(0, 1)), cam2)
    assert [int(k) >> 32 for k in k2] == [1]
    # a faint Gaussian: r = 9 (sigma 3) at (31.0, 24.0), opacity 0.02.  Its
    # integer box x [22, 40], y [15, 33] spans tile columns 1-2 and rows 0-2,
    # but alpha reaches 1/255 only within |d| <= ex = sqrt(2 (B + 1e-3) 9)
    # 1.002 + 2e-3 = 5.4645 (B = 64 (5.1^(1/64) - 1) = 1.6501 >= ln 5.1 =
    # 1.6292): pixels x 26..35, y 19..28 -> row 1 only: tiles 5 and 6
    faint = {"uv": np.array([[31.0, 24.0]]), "depth": np.array([4.0]), "radius": np.array([9]),
             "conic": np.array([[1 / 9.0, 0.0, 1 / 9.0]]), "opacity": np.array([0.02])}
    k3, _, _ = O.bin_sort(faint, cam)
    assert [int(k) >> 32 for k in k3] == [5, 6]
    # below alpha_min it touches no tile at all
    k4, _, _ = O.bin_sort(dict(faint, opacity=np.array([0.003])), cam)
    assert len(k4) == 0
    assert O.tile_dim(1) == 16 and O.tile_dim(2) == 8 and O.tile_dim(3) == 4 and O.tile_dim(4) == 4
    assert O.tile_dim(100) == 4


def test_sort_invariants_and_stability(oracle_lib):
    O = oracle_lib
    cam = S.camera(200, 120, 100.0)
    s = S.splats(3000, 200, 120, seed=5, tie_frac=0.2)
    keys, vals, ranges = O.bin_sort(s, cam)
    # permutation of the expected multiset and non-decreasing keys
    assert np.all(np.diff(keys.astype(np.float64)) >= 0) or np.all(keys[1:] >= keys[:-1])
    _, _, TX, TY = O.grid(cam)
    # brute-force rect: tiles with a pixel p in the integer box whose centre
    # also lies within the alpha extent, |p + 0.5 - u| <= ex, the extent
    # evaluated in numpy float32 from its definition (reading new-2)
    f32 = np.float32
    amin = f32(1.0) / f32(255.0)
    pr_rect = []
    total = 0
    for k in range(3000):
        r = int(s["radius"][k])
        ca, cb, cc = (f32(v) for v in s["conic"][k])
        op = f32(s["opacity"][k])
        if r <= 0 or not op >= amin:
            pr_rect.append(None)
            continue
        det = f32(ca * cc) - f32(cb * cb)
        q = f32(op / amin)
        for _ in range(6):
            q = np.sqrt(q)
        B = f32(f32(64.0) * f32(q - f32(1.0)))
        t2 = f32(f32(2.0) * f32(max(B, f32(0.0)) + f32(1e-3)))
        ex = f32(f32(np.sqrt(f32(f32(t2 * cc) / det)) * f32(1.002)) + f32(2e-3))
        ey = f32(f32(np.sqrt(f32(f32(t2 * ca) / det)) * f32(1.002)) + f32(2e-3))
        u, v = f32(s["uv"][k, 0]), f32(s["uv"][k, 1])
        xi, yi = math.floor(u), math.floor(v)
        okx = lambda p: abs(p - xi) <= r and abs(f32(f32(p) + f32(0.5)) - u) <= ex
        oky = lambda p: abs(p - yi) <= r and abs(f32(f32(p) + f32(0.5)) - v) <= ey
        tx = [t for t in range(TX) if any(okx(p) for p in range(16 * t, min(16 * t + 16, 200)))]
        ty = [t for t in range(TY) if any(oky(p) for p in range(16 * t, min(16 * t + 16, 120)))]
        pr_rect.append((tx, ty))
        total += len(tx) * len(ty)
    assert len(keys) == total
    # every value in tile t's range has t in its rect (brute-force rect)
    for t in range(TX * TY):
        b, e = ranges[t]
        for i in range(b, e):
            k = int(vals[i])
            tx, ty = pr_rect[k]
            assert (t % TX) in tx and (t // TX) in ty
            assert int(keys[i]) >> 32 == t
    # equal keys keep id order
    same = keys[1:] == keys[:-1]
    assert same.sum() > 0
    assert np.all(vals[1:][same] > vals[:-1][same])


# ---------------------------------------------------------------------------
# Projection against independent routes
# ---------------------------------------------------------------------------

def test_projection_matches_numerical_jacobian(oracle_lib):
    """Sigma2 - 0.3 I equals J_num Sigma_c J_num^T, with J_num the numerical
    Jacobian of the pinhole map and Sigma_c built with scipy's rotation."""
    from scipy.spatial.transform import Rotation
    O = oracle_lib
    g = S.rng(9)
    n = 40
    q = S.random_unit_quats(g, n)
    means = np.stack([g.uniform(-0.5, 0.5, n), g.uniform(-0.4, 0.4, n), g.uniform(1.0, 4.0, n)], 1)
    ls = g.normal(-2.5, 0.5, (n, 3))
    gs = {"means": means, "log_scales": ls, "quats": q, "opacity_logit": np.zeros(n),
          "rgb": np.zeros((n, 3))}
    ang = 0.2
    Rcw = S.axis_angle_matrix([0.3, 1.0, -0.2], ang)
    t = np.array([0.05, -0.02, 0.3])
    cam = S.camera(160, 120, 140.0, R=Rcw, t=t)
    pr = O.project(gs, cam)
    for k in range(n):
        assert pr["radius"][k] > 0
        Rq = Rotation.from_quat([q[k, 1], q[k, 2], q[k, 3], q[k, 0]]).as_matrix()
        Sig = Rq @ np.diag(np.exp(2 * ls[k])) @ Rq.T
        Sc = Rcw @ Sig @ Rcw.T
        p = Rcw @ means[k] + t

        def pin(pp):
            return np.array([140.0 * pp[0] / pp[2] + 80.0, 140.0 * pp[1] / pp[2] + 60.0])

        J = np.zeros((2, 3))
        h = 1e-6
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            J[:, j] = (pin(p + e) - pin(p - e)) / (2 * h)
        S2 = J @ Sc @ J.T + 0.3 * np.eye(2)
        A, B, Cc = pr["conic"][k]
        S2o = np.linalg.inv(np.array([[A, B], [B, Cc]]))
        np.testing.assert_allclose(S2o, S2, rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(pr["uv"][k], pin(p), rtol=1e-12)
        lmax = np.linalg.eigvalsh(S2).max()
        mid = 0.5 * (S2[0, 0] + S2[1, 1])
        if mid * mid - np.linalg.det(S2) > 0.1:
            r3 = 3 * math.sqrt(lmax)
            if abs(r3 - round(r3)) > 1e-6:
                assert pr["radius"][k] == math.ceil(r3)


def test_near_plane_and_mask_cull(oracle_lib):
    O = oracle_lib
    g = concat(one_gaussian(0, 0, 0.19, -3, 0, (1, 1, 1)), one_gaussian(0, 0, 0.21, -3, 0, (1, 1, 1)),
               one_gaussian(0, 0, 1.0, -3, 0, (1, 1, 1)))
    g["mask"] = np.array([0, 0, 1], np.uint8)
    pr = O.project(g, S.camera(32, 32, 30.0))
    assert pr["radius"].tolist()[0] == 0 and pr["radius"][1] > 0 and pr["radius"][2] == 0


# ---------------------------------------------------------------------------
# Finite differences (Sec. 2.2 backward, Step 4 and Step 5)
# ---------------------------------------------------------------------------

def small_fd_scene(seed):
    g = S.rng(seed)
    n = 14
    means = np.stack([g.uniform(-0.6, 0.6, n), g.uniform(-0.45, 0.45, n), g.uniform(1.5, 3.0, n)], 1)
    # one Gaussian beyond each Jacobian clamp line whose footprint still
    # reaches the 40x30 image at f = 36 (clamp lines x/z = 1.3 * 20/36 = 0.72,
    # y/z = 1.3 * 15/36 = 0.54)
    means[0] = [0.8 * 2.6, 0.1, 2.6]
    means[1] = [0.1, 0.65 * 2.6, 2.6]
    gs = {"means": means, "log_scales": g.normal(-2.2, 0.25, (n, 3)),
          "quats": S.random_unit_quats(g, n) * g.uniform(0.7, 1.4, (n, 1)),
          "opacity_logit": g.normal(0.5, 1.0, n), "rgb": g.uniform(0, 1, (n, 3))}
    gs["log_scales"][0] = [-0.7, -0.7, -0.7]
    gs["log_scales"][1] = [-0.7, -0.7, -0.7]
    return gs


def assert_beyond_clamp_lines(gs, cam):
    """Gaussians 0 and 1 of small_fd_scene lie beyond the x and the y clamp
    line in this camera's frame."""
    p = gs["means"][:2] @ np.asarray(cam["R"]).T + np.asarray(cam["t"])
    assert p[0, 0] / p[0, 2] > 1.3 * (cam["W"] / 2) / cam["fx"]
    assert p[1, 1] / p[1, 2] > 1.3 * (cam["H"] / 2) / cam["fy"]


def fd_loss(O, gs, cam, w, wd, cfg=None):
    pr, img = O.forward(gs, cam, cfg)
    return float((w * img["rgb"]).sum() + (wd * img["depth"]).sum()), img["sig"], tuple(pr["radius"])


BGS = [(0.0, 0.0, 0.0), (0.25, 0.5, 0.75)]


@pytest.mark.parametrize("bg", BGS)
def test_gradients_match_central_differences(oracle_lib, bg):
    """Every parameter kind against central differences of the forward; with
    a non-black background the alpha gradients also carry the background seen
    through the transmittance, -T_final bg / (1 - a_k) (Eq. 3 differentiated)."""
    O = oracle_lib
    W, H = 40, 30
    gs = small_fd_scene(21)
    R = S.axis_angle_matrix([0.2, -0.5, 1.0], 0.05)
    cam = S.camera(W, H, 36.0, R=R, t=[0.01, -0.02, 0.05])
    assert_beyond_clamp_lines(gs, cam)
    cfg = {"bg": bg}
    g = S.rng(22)
    w = g.normal(0, 1, (3, H, W))
    wd = g.normal(0, 1, (H, W))
    _, _, an = O.forward_backward(gs, cam, w, wd, cfg)
    h = 1e-5
    checked = 0
    for key, width in (("means", 3), ("log_scales", 3), ("quats", 4), ("opacity_logit", 1),
                       ("rgb", 3)):
        for k in range(len(gs["means"])):
            for j in range(width):
                gp = {kk: np.array(v, dtype=np.float64, copy=True) for kk, v in gs.items()}
                gm = {kk: np.array(v, dtype=np.float64, copy=True) for kk, v in gs.items()}
                if width == 1:
                    gp[key][k] += h
                    gm[key][k] -= h
                else:
                    gp[key][k, j] += h
                    gm[key][k, j] -= h
                Lp, sp, rp = fd_loss(O, gp, cam, w, wd, cfg)
                Lm, sm, rm = fd_loss(O, gm, cam, w, wd, cfg)
                L0, s0, r0 = fd_loss(O, gs, cam, w, wd, cfg)
                if not (sp == s0 == sm and rp == r0 == rm):
                    continue  # the stencil crosses a predicate; not differentiable here
                fd = (Lp - Lm) / (2 * h)
                a = an[key][k] if width == 1 else an[key][k, j]
                assert abs(fd - a) <= 2e-5 * max(1.0, abs(a)), (key, k, j, fd, a)
                checked += 1
    assert checked > 150
    # the clamped-Jacobian Gaussians 0 (x) and 1 (y) were exercised
    assert abs(an["means"][0]).sum() > 0 and abs(an["means"][1]).sum() > 0


def pose_perturb(cam, xi):
    """Left perturbation T_cw <- exp(xi^) T_cw to first order along xi, with
    the rotation part exact (Rodrigues) -- a smooth curve whose tangent at
    zero is xi^."""
    rho, phi = np.asarray(xi[:3]), np.asarray(xi[3:])
    ang = np.linalg.norm(phi)
    Rd = np.eye(3) if ang == 0 else S.axis_angle_matrix(phi / ang, ang)
    c = dict(cam)
    c["R"] = Rd @ np.asarray(cam["R"])
    c["t"] = Rd @ np.asarray(cam["t"]) + rho
    return c


@pytest.mark.parametrize("bg", BGS)
def test_pose_gradient_matches_central_differences(oracle_lib, bg):
    O = oracle_lib
    W, H = 40, 30
    gs = small_fd_scene(31)
    cam = S.camera(W, H, 36.0, R=S.axis_angle_matrix([1, 0.3, 0.1], 0.04), t=[0.02, 0.01, -0.03])
    assert_beyond_clamp_lines(gs, cam)
    cfg = {"bg": bg}
    g = S.rng(32)
    w = g.normal(0, 1, (3, H, W))
    wd = g.normal(0, 1, (H, W))
    _, _, an = O.forward_backward(gs, cam, w, wd, cfg)
    h = 1e-6
    for i in range(6):
        e = np.zeros(6)
        e[i] = h
        Lp, sp, rp = fd_loss(O, gs, pose_perturb(cam, e), w, wd, cfg)
        Lm, sm, rm = fd_loss(O, gs, pose_perturb(cam, -e), w, wd, cfg)
        assert sp == sm and rp == rm
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - an["pose"][i]) <= 1e-5 * max(1.0, abs(fd)), (i, fd, an["pose"][i])


def sigma_to_params(Sig):
    """Log-scales and a (w, x, y, z) unit quaternion whose
    R(q) diag(exp(2 ls)) R(q)^T is the symmetric positive definite Sig (its
    eigendecomposition, with the eigenvector basis made a proper rotation)."""
    from scipy.spatial.transform import Rotation
    lam, V = np.linalg.eigh(Sig)
    if np.linalg.det(V) < 0:
        V[:, 2] = -V[:, 2]
    x, y, z, w = Rotation.from_matrix(V).as_quat()
    return 0.5 * np.log(lam), np.array([w, x, y, z])


def test_score_terms_match_differences_in_mean_and_covariance(oracle_lib):
    """Both terms of the Eq. 7 score against central differences of the
    forward alone (reading c12: the 3D mean's 2-norm and the Frobenius norm,
    over all nine entries, of the 3D covariance's gradient).  The covariance
    is moved directly: Sigma + h E for the six symmetric directions
    E = e_i e_i^T and e_i e_j^T + e_j e_i^T, each turned back into log-scales
    and a quaternion by an eigendecomposition, so dL/dh = <dL/dSigma, E>
    needs neither the projection's chain rule nor its parameterisation.  The
    camera-frame gradient dL/dSigma_c = R dL/dSigma R^T is checked entrywise."""
    from scipy.spatial.transform import Rotation
    O = oracle_lib
    W, H = 40, 30
    gs = small_fd_scene(21)
    R = S.axis_angle_matrix([0.2, -0.5, 1.0], 0.05)
    cam = S.camera(W, H, 36.0, R=R, t=[0.01, -0.02, 0.05])
    g = S.rng(23)
    w = g.normal(0, 1, (3, H, W))
    wd = g.normal(0, 1, (H, W))
    _, _, an = O.forward_backward(gs, cam, w, wd)
    n = gs["means"].shape[0]
    checked = 0
    offdiag = 0.0
    for k in range(n):
        qk = gs["quats"][k] / np.linalg.norm(gs["quats"][k])
        Rq = Rotation.from_quat([qk[1], qk[2], qk[3], qk[0]]).as_matrix()
        Sig = Rq @ np.diag(np.exp(2 * gs["log_scales"][k])) @ Rq.T
        h = 1e-5 * np.trace(Sig) / 3
        Gfd = np.zeros((3, 3))
        ok = True
        for i in range(3):
            for j in range(i, 3):
                E = np.zeros((3, 3))
                E[i, j] += 1.0
                E[j, i] += 1.0 if i != j else 0.0
                Ls = []
                for sgn in (1.0, -1.0):
                    ls, q = sigma_to_params(Sig + sgn * h * E)
                    gg = {kk: np.array(v, dtype=np.float64, copy=True) for kk, v in gs.items()}
                    gg["log_scales"][k] = ls
                    gg["quats"][k] = q
                    Ls.append(fd_loss(O, gg, cam, w, wd))
                L0 = fd_loss(O, gs, cam, w, wd)
                if not (Ls[0][1:] == L0[1:] == Ls[1][1:]):
                    ok = False   # the stencil crosses a predicate
                    break
                d = (Ls[0][0] - Ls[1][0]) / (2 * h)
                Gfd[i, j] = Gfd[j, i] = d if i == j else 0.5 * d
            if not ok:
                break
        gmu = np.zeros(3)
        hm = 1e-6
        for i in range(3):
            Ls = []
            for sgn in (1.0, -1.0):
                gg = {kk: np.array(v, dtype=np.float64, copy=True) for kk, v in gs.items()}
                gg["means"][k, i] += sgn * hm
                Ls.append(fd_loss(O, gg, cam, w, wd))
            if not (Ls[0][1:] == Ls[1][1:]):
                ok = False
            gmu[i] = (Ls[0][0] - Ls[1][0]) / (2 * hm)
        if not ok:
            continue
        fro = np.linalg.norm(Gfd)
        st = an["score_terms"][k]
        assert abs(st[1] - fro) <= 1e-5 * max(1.0, fro), (k, st[1], fro)
        assert abs(st[0] - np.linalg.norm(gmu)) <= 1e-5 * max(1.0, np.linalg.norm(gmu)), (k, st[0], gmu)
        Gc = np.asarray(cam["R"]) @ Gfd @ np.asarray(cam["R"]).T
        np.testing.assert_allclose(an["Sc"][k].reshape(3, 3), Gc, rtol=0, atol=1e-5 * max(1.0, fro))
        offdiag = max(offdiag, np.abs(Gfd - np.diag(np.diag(Gfd))).max() / max(fro, 1e-30))
        checked += fro > 0
    assert checked >= 8
    # the off-diagonal entries carry weight: a norm over the diagonal alone is far off
    assert offdiag > 0.1


def test_pose_gradient_zero_at_target_and_descent_when_perturbed(oracle_lib):
    """At the exact target pose every L1 residual is 0 and sign(0) = 0, so the
    pose gradient is exactly 0.  From a pose 2 cm / 1 deg away, a small step
    along -grad lowers the loss (Eq. 6)."""
    O = oracle_lib
    gs = S.tiny_scene(seed=44, n=500)
    cam = S.tiny_camera()
    _, tgt = O.forward(gs, cam)
    _, img = O.forward(gs, cam)
    L, dr, dd = O.loss_l1(img["rgb"], img["depth"], tgt["rgb"], tgt["depth"])
    assert L == 0.0
    _, _, gb = O.forward_backward(gs, cam, dr, dd)
    assert np.all(gb["pose"] == 0.0)
    start = S.perturbed_pose(cam, seed=45, trans=0.02, rot_deg=1.0)
    _, img = O.forward(gs, start)
    L0, dr, dd = O.loss_l1(img["rgb"], img["depth"], tgt["rgb"], tgt["depth"])
    _, _, gb = O.forward_backward(gs, start, dr, dd)
    step = -gb["pose"] / np.linalg.norm(gb["pose"]) * 2e-3
    _, img1 = O.forward(gs, pose_perturb(start, step))
    L1, _, _ = O.loss_l1(img1["rgb"], img1["depth"], tgt["rgb"], tgt["depth"])
    assert L1 < L0


# ---------------------------------------------------------------------------
# Loss (Eq. 6)
# ---------------------------------------------------------------------------

def test_loss_hand_values(oracle_lib):
    O = oracle_lib
    rgb = np.array([[[0.5, 0.2]], [[0.1, 0.1]], [[1.0, 0.0]]])      # [3,1,2]
    tr = np.array([[[0.25, 0.2]], [[0.3, 0.0]], [[0.5, 0.5]]])
    dep = np.array([[2.0, 3.0]])
    td = np.array([[1.5, 0.0]])                                      # second invalid
    L, dr, dd = O.loss_l1(rgb, dep, tr, td, w_rgb=0.9, w_depth=0.1)
    # |res| = .25,0,.2,.1,.5,.5 -> sum 1.55 ; depth |.5| on the valid pixel
    assert math.isclose(L, 0.9 * 1.55 / 6 + 0.1 * 0.5 / 2, rel_tol=1e-14)
    np.testing.assert_array_equal(np.sign(dr).ravel(), [1, 0, -1, 1, 1, -1])
    np.testing.assert_allclose(np.abs(dr[dr != 0]), 0.9 / 6)
    np.testing.assert_allclose(dd, [[0.1 / 2, 0.0]])
    # a negative depth residual, an invalid target and a zero residual: the
    # gradient is sign(r) w / P with P every sampled pixel, sign(0) = 0
    z = np.zeros((3, 1, 3))
    L2, dr2, dd2 = O.loss_l1(z, np.array([[0.5, 2.0, 1.0]]), z, np.array([[0.5, 0.0, 1.5]]), w_rgb=0.9,
                             w_depth=0.1)
    assert math.isclose(L2, 0.1 * 0.5 / 3, rel_tol=1e-14)
    assert not dr2.any()
    np.testing.assert_allclose(dd2, [[0.0, 0.0, -0.1 / 3]], rtol=1e-14)


# ---------------------------------------------------------------------------
# Pruning (Sec. 4.1, Eq. 7) and interval schedule
# ---------------------------------------------------------------------------

def test_prune_select_hand_case(oracle_lib):
    O = oracle_lib
    t_mu = np.array([3, 1, 2, 1, 0, 5, 1], np.float32)
    t_sig = np.array([0, 0, 0, 0, 0, 0, 0], np.float32)
    mask = np.array([0, 0, 0, 0, 0, 0, 1], np.uint8)     # id 6 already masked
    m, cnt = O.prune_select(t_mu, t_sig, mask, lam=0.8, frac=0.5)
    # 6 active -> mask 3: scores 0 (id 4), 1 (id 1), 1 (id 3); id 6 untouched
    assert cnt == 3
    assert m.tolist() == [0, 1, 0, 1, 1, 0, 1]
    # lambda weights the covariance term: (0,10) scores 8 > (7,0)
    m2, _ = O.prune_select(np.array([0, 7], np.float32), np.array([10, 0], np.float32),
                           np.zeros(2, np.uint8), lam=0.8, frac=0.5)
    assert m2.tolist() == [0, 1]
    # cap on the number selected
    m3, c3 = O.prune_select(t_mu, t_sig, np.zeros(7, np.uint8), frac=0.5, max_select=1)
    assert c3 == 1 and m3.tolist() == [0, 0, 0, 0, 1, 0, 0]
    # the weight multiplies the covariance term: at lambda = 0.5, (0, 5)
    # scores 2.5, below (3, 0); and both terms add: (9, 6) scores 13.8, above
    # (5, 0) (all scores non-negative, so their bit patterns order them)
    m5, _ = O.prune_select(np.array([0, 3], np.float32), np.array([5, 0], np.float32), np.zeros(2, np.uint8),
                           lam=0.5, frac=0.5)
    assert m5.tolist() == [1, 0]
    m6, _ = O.prune_select(np.array([5, 9], np.float32), np.array([0, 6], np.float32), np.zeros(2, np.uint8),
                           lam=0.8, frac=0.5)
    assert m6.tolist() == [1, 0]
    # all equal: ids decide
    m4, c4 = O.prune_select(np.ones(10, np.float32), np.ones(10, np.float32), np.zeros(10, np.uint8),
                            frac=0.3)
    assert c4 == 3 and m4.tolist() == [1, 1, 1, 0, 0, 0, 0, 0, 0, 0]


def test_interval_schedule(oracle_lib):
    O = oracle_lib
    hp = json.load(open(os.path.join(GOLD, "hyperparams.json")))
    K0, thr = hp["k0"], hp["change_ratio_threshold"]
    K = K0
    seq = []
    for r in [0.10, 0.01, 0.01, 0.20, 0.05, 0.0]:
        K = O.next_interval(K, r, K0=K0, thr=thr)
        seq.append(K)
    assert seq == [2, 4, 8, 4, 8, 16]
    assert O.next_interval(1, 0.9) == 1
    assert O.next_interval(64, 0.0) == 64
    # the paper's literal constants: K0/2 or 2 K0
    assert O.next_interval(7, 0.10, K0=5, literal=True) == 2
    assert O.next_interval(7, 0.01, K0=5, literal=True) == 10
    # a ratio equal to the threshold does not exceed it: the interval grows
    assert O.next_interval(8, thr, thr=thr) == 16
    assert O.next_interval(7, thr, K0=5, thr=thr, literal=True) == 10


def test_change_ratio_hand_case(oracle_lib):
    O = oracle_lib
    A = [(0 << 32) | 1, (0 << 32) | 2, (1 << 32) | 3]
    B = [(0 << 32) | 1, (1 << 32) | 3, (2 << 32) | 5, (2 << 32) | 6]
    assert O.change_ratio(A, B) == pytest.approx(3 / 3)
    assert O.change_ratio(A, A) == 0.0
    assert O.change_ratio([], B) == 4.0


# ---------------------------------------------------------------------------
# Downsampling (Sec. 4.2)
# ---------------------------------------------------------------------------

def test_downsample_schedule_table(oracle_lib):
    O = oracle_lib
    tab = json.load(open(os.path.join(GOLD, "downsample_schedule.json")))
    k = 10
    for row in tab["rows"]:
        sx, sy = O.downsample_schedule(k + 1 + row["e"], k, False, m=tab["m"])
        assert (sx, sy) == (row["sx"], row["sy"])
        assert 1.0 / (sx * sy) == row["fraction"]
    assert O.downsample_schedule(k, k, True) == (1, 1)
    with pytest.raises(ValueError):
        O.downsample_schedule(12, 10, False, m=3)
    # a non-keyframe comes after its keyframe
    for n in (k, k - 1):
        with pytest.raises(ValueError):
            O.downsample_schedule(n, k, False)


@pytest.mark.parametrize("sx,sy", [(2, 2), (4, 2), (4, 4), (3, 1)])
def test_strided_render_equals_subsampled_full_render(oracle_lib, sx, sy):
    O = oracle_lib
    g = S.tiny_scene(seed=77)
    cam = S.tiny_camera()
    pr = O.project(g, cam)
    full = O.render_fwd(pr, cam)
    cs = dict(cam, sx=sx, sy=sy)
    sub = O.render_fwd(pr, cs)
    np.testing.assert_array_equal(sub["rgb"], full["rgb"][:, ::sy, ::sx])
    np.testing.assert_array_equal(sub["depth"], full["depth"][::sy, ::sx])
    np.testing.assert_array_equal(O.gather(full["rgb"], sx, sy), full["rgb"][:, ::sy, ::sx])
    noise = S.rng(78).normal(0, 1, (3, 37, 29))   # every sample distinct: a shifted index shows
    np.testing.assert_array_equal(O.gather(noise, sx, sy), noise[:, ::sy, ::sx])
