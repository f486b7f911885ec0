"""Precision form (16-bit record storage): conic, opacity and colour stored as
bf16 or fp16, means, depths and radii in float32, all compositing and
accumulation in float32; the pose-gradient sum over all Gaussians is carried
as float32 pairs (error-free two-sums) inside each block and across blocks,
and returned as float64.  Each output's error against the FP64 oracle is measured and printed
(`pytest -s`), and bounded by a figure derived from the storage precision:

  u = unit roundoff of the storage type (bf16 2^-8, fp16 2^-11).  Colour and
  opacity carry a relative error <= u; a conic entry <= u, so the exponent
  -(a dx^2 + 2 b dx dy + c dy^2)/2 carries <= u |power| with |power| <=
  ln(255 o) < 5.6 where alpha >= 1/255.  alpha = o exp(power) then has a
  relative error <= u (1 + 5.6) and a blended colour <= ~8u, which the test
  rounds up to 16u for maxima (and also covers the rare alpha-threshold flips)
  and 2u for means.  Gradients sum per-pixel terms of both signs, so their
  relative error is the storage error times the cancellation of that sum;
  the quaternion gradient cancels most (rotating a nearly isotropic Gaussian
  hardly changes it: ~37u measured on 3M Gaussians at 1920x1080), so
  gradients are held to 64u relative L2 against full-precision FP64.
  Against the FP64 oracle fed the same 16-bit-rounded records the float32
  bars hold (1e-4 image away from marginal pixels, 1e-3 gradients).

Binning reads only the float32 fields, so keys, order and ranges are
identical to the float32 path.
"""
import numpy as np
import pytest
import torch

from synth import scenes as S
from tests.gpu_helpers import dev, np_of, rel_l2, stored_splats

pytestmark = pytest.mark.gpu

U = {"bf16": 2.0 ** -8, "fp16": 2.0 ** -11}


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_06644_gb300 import build
    build.build()
    from paper_2510_06644_gb300 import gs
    return gs


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


def dt_of(G, name):
    return {"bf16": G.GS_BF16, "fp16": G.GS_F16}[name]


@pytest.mark.parametrize("name", ["bf16", "fp16"])
def test_records_round_the_float32_fields(G, name):
    g = S.surface_scene(20000, seed=71)
    cam = S.camera(320, 240, 260.0)
    cfg = G.default_config()
    gd = dev(g)
    r32 = G.gs_project(cfg, G.camera(cam), gd, G.GS_F32)
    r16 = G.gs_project(cfg, G.camera(cam), gd, dt_of(G, name))
    f32 = G.splat_fields(r32, G.GS_F32)
    f16 = G.splat_fields(r16, dt_of(G, name))
    for k in ("uv", "depth", "radius"):
        assert torch.equal(f16[k], f32[k]), k
    tt = torch.bfloat16 if name == "bf16" else torch.float16
    for k in ("conic", "opacity", "rgb"):
        assert torch.equal(f16[k], f32[k].to(tt).float()), k
    # the tile count follows the stored (rounded) conic and opacity
    t32 = f32["touched"].long()
    t16 = f16["touched"].long()
    assert (t16 != torch.clamp(t32, max=65535)).float().mean().item() <= 0.02


@pytest.mark.parametrize("name", ["bf16", "fp16"])
def test_binning_of_16bit_records_bit_exact(G, O, name):
    """The binning reads the 16-bit records' conic and opacity (the tile
    rects' alpha extent): bit-exact against the oracle on the same rounded
    values, and within a few percent of the float32 keys."""
    g = S.surface_scene(30000, seed=72)
    cam = S.camera(333, 197, 260.0)
    cfg = G.default_config()
    gd = dev(g)
    cs = G.camera(cam)
    out = {}
    for dtn, dt in (("f32", G.GS_F32), (name, dt_of(G, name))):
        rec = G.gs_project(cfg, cs, gd, dt)
        keys, vals, nk, ranges, _ = G.gs_bin_sort(cs, rec, 30000, 400000, dt)
        k = int(nk.item())
        out[dtn] = (np_of(keys[:k]), np_of(vals[:k]), np_of(ranges))
        if dtn == name:
            f = {kk: np_of(v) for kk, v in G.splat_fields(rec, dt).items()}
            ok_, ov_, or_ = O.bin_sort(f, cam)
            assert np.array_equal(out[dtn][0], ok_) and np.array_equal(out[dtn][1], ov_)
            assert np.array_equal(out[dtn][2], or_)
    assert abs(len(out[name][0]) - len(out["f32"][0])) <= 0.02 * len(out["f32"][0])


@pytest.mark.parametrize("name", ["bf16", "fp16"])
@pytest.mark.parametrize("scene", ["tiny", "slam"])
def test_errors_against_fp64_oracle(G, O, name, scene):
    from paper_2510_06644_gb300.pipeline import Rasterizer
    if scene == "tiny":
        g = S.tiny_scene(seed=1000)
        cam = S.tiny_camera()
        trgb, tdep = S.target_image(96, 72, seed=1001)
    else:
        g = S.surface_scene(60000, seed=73)
        cam = S.perturbed_pose(S.camera(320, 240, 260.0), seed=74, trans=0.02, rot_deg=1.0)
        trgb, tdep = S.target_image(320, 240, seed=75, depth_range=(1.0, 6.0))
    u = U[name]
    n = g["means"].shape[0]
    gd = dev(g)
    r = Rasterizer(n, cam, rec_dtype=dt_of(G, name))
    grads = {k: torch.empty_like(gd[k]) for k in ("means", "log_scales", "quats", "opacity_logit", "rgb")}
    pr, img = O.forward(g, cam)
    L, dr, dd = O.loss_l1(img["rgb"], img["depth"], trgb, tdep)
    _, _, ref = O.forward_backward(g, cam, dr, dd)
    r.forward(gd, cam)
    # both sides differentiate the oracle's image gradient, so the comparison
    # isolates the renderer from sign flips of near-zero L1 residuals
    r.backward(gd, cam, torch.from_numpy(dr.astype(np.float32)).cuda(),
               torch.from_numpy(dd.astype(np.float32)).cuda(), mode=G.GS_MAP, grads=grads)
    r.check()
    errs = {}
    e_rgb = np.abs(np_of(r.img["rgb"]) - img["rgb"])
    errs["rgb_max"], errs["rgb_mean"] = float(e_rgb.max()), float(e_rgb.mean())
    zmax = float(np.abs(img["depth"]).max())
    e_d = np.abs(np_of(r.img["depth"]) - img["depth"]) / max(zmax, 1.0)
    errs["depth_max_rel"], errs["depth_mean_rel"] = float(e_d.max()), float(e_d.mean())
    e_t = np.abs(np_of(r.img["t_final"]) - img["T"])
    errs["T_max"] = float(e_t.max())
    for k in grads:
        errs["d_" + k] = rel_l2(np_of(grads[k]), ref[k])
    errs["pose"] = rel_l2(np_of(r.pose), ref["pose"])
    print(f"\n[{name} {scene}] u={u:.2e} " + " ".join(f"{k}={v:.2e}" for k, v in errs.items()))
    assert errs["rgb_max"] <= 16 * u and errs["rgb_mean"] <= 2 * u
    assert errs["depth_max_rel"] <= 16 * u and errs["depth_mean_rel"] <= 2 * u
    assert errs["T_max"] <= 16 * u
    for k in list(grads) + ["pose"]:
        key = "d_" + k if k != "pose" else "pose"
        assert errs[key] <= 64 * u, (key, errs[key])
    # the same definition on the stored (rounded) records: float32 bars
    sq = stored_splats(pr, name)
    imq = O.render_fwd(sq, cam)
    good = imq["margin"] == 0
    assert good.mean() > 0.97
    assert np.abs(np_of(r.img["rgb"]) - imq["rgb"]).max(0)[good].max() <= 1e-4
    g2q = O.render_bwd(sq, cam, dr, dd)
    g2 = np_of(r.grad2d)
    for cols in ([0, 1], [2, 3, 4], [5], [6], [8, 9, 10]):
        assert rel_l2(g2[:, cols], g2q[:, cols]) <= 1e-3, cols


def test_pose_reduction_holds_under_cancellation(G):
    """The pose gradient is a sum over every Gaussian.  3M Gaussians on the
    optical axis at z = 1 with fx = fy = 1 and only dL/du set make each term
    exactly dL/du_k (rho_x and phi_y components), so the exact sum is known:
    +-a pairs spread over 8 decades (|a| from 1e-4 to 1e4, shuffled across
    warps and blocks) cancel to a residual of about 1e3 out of ~1.6e9 of
    absolute mass.  The kernel's compensated reduction meets 1e-6 relative
    against the exactly rounded host sum (math.fsum); a plain float32 sum of
    the same terms (numpy's pairwise one) does not."""
    import math
    n = 3_000_000
    rng = np.random.Generator(np.random.PCG64(77))
    half = (n - 1000) // 2
    a = (10.0 ** rng.uniform(-4, 4, half)).astype(np.float32)
    terms = np.concatenate([a, -a, rng.uniform(0.5, 1.5, n - 2 * half).astype(np.float32)])
    terms = terms[rng.permutation(n)]
    exact = math.fsum(terms.astype(np.float64).tolist())
    plain = float(np.sum(terms, dtype=np.float32))
    assert abs(plain - exact) / abs(exact) > 1e-6        # the case defeats a float32 sum
    g = {"means": np.tile(np.array([[0.0, 0.0, 1.0]], np.float32), (n, 1)),
         "log_scales": np.full((n, 3), -6.0, np.float32),
         "quats": np.tile(np.array([[1.0, 0.0, 0.0, 0.0]], np.float32), (n, 1)),
         "opacity_logit": np.zeros(n, np.float32), "rgb": np.zeros((n, 3), np.float32)}
    cam = S.camera(64, 64, 1.0)
    g2 = np.zeros((n, 12), np.float32)
    g2[:, 0] = terms
    gd = dev(g)
    pose = torch.zeros(6, dtype=torch.float64, device="cuda")
    G.gs_project_bwd(G.default_config(), G.camera(cam), gd, torch.from_numpy(g2).cuda(), pose=pose)
    torch.cuda.synchronize()
    p = np_of(pose)
    # dL/drho_x = sum dL/dx_c = sum dL/du (fx / z = 1); dL/dphi_y = z dL/dx_c
    assert abs(p[0] - exact) / abs(exact) <= 1e-6, (p[0], exact, plain)
    assert abs(p[4] - exact) / abs(exact) <= 1e-6, (p[4], exact)
    assert p[1] == 0 and p[2] == 0 and p[3] == 0 and p[5] == 0
    print(f"\npose reduction under cancellation: exact {exact:.9g}, kernel {p[0]:.9g} "
          f"(rel {abs(p[0] - exact) / abs(exact):.2e}), float32 sum {plain:.9g} "
          f"(rel {abs(plain - exact) / abs(exact):.2e})")
