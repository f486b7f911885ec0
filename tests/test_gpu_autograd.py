"""gs_render as a torch.autograd.Function: its hand-written adjoint against
the FP64 oracle's analytic gradient, against central finite differences of
its own forward (h = 1e-3, 64 random parameters), and store == recompute."""
import numpy as np
import pytest
import torch

from synth import scenes as S
from tests.gpu_helpers import np_of, rel_l2

pytestmark = pytest.mark.gpu

KEYS = ("means", "log_scales", "quats", "opacity_logit", "rgb")


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_06644_gb300 import build
    build.build()
    from paper_2510_06644_gb300 import autograd
    return autograd


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


def leaf_params(g):
    return {k: torch.from_numpy(np.ascontiguousarray(g[k])).cuda().requires_grad_(True) for k in KEYS}


def weights(W, H, seed):
    r = S.rng(seed)
    return r.normal(0, 1, (3, H, W)).astype(np.float32), r.normal(0, 1, (H, W)).astype(np.float32)


def run(A, p, delta, cam, w, wd, **kw):
    rgb, depth = A.gs_render(p["means"], p["log_scales"], p["quats"], p["opacity_logit"], p["rgb"], delta, cam, **kw)
    return (rgb.double() * torch.from_numpy(w).cuda().double()).sum() + \
        (depth.double() * torch.from_numpy(wd).cuda().double()).sum()


@pytest.mark.parametrize("budget", [None, 0])
def test_adjoint_matches_oracle(A, O, budget):
    g = S.tiny_scene(seed=1000)
    cam = S.perturbed_pose(S.tiny_camera(), seed=3, trans=0.01, rot_deg=0.5)
    w, wd = weights(96, 72, 9)
    p = leaf_params(g)
    delta = torch.zeros(6, device="cuda", requires_grad=True)
    L = run(A, p, delta, cam, w, wd, memory_budget=budget)
    L.backward()
    _, _, ref = O.forward_backward(g, cam, w, wd)
    for k in KEYS:
        assert rel_l2(np_of(p[k].grad), ref[k]) <= 1e-3, k
    assert rel_l2(np_of(delta.grad), ref["pose"]) <= 1e-3


def test_store_and_recompute_agree(A):
    g = S.surface_scene(30000, seed=12)
    cam = S.camera(200, 150, 160.0)
    w, wd = weights(200, 150, 13)
    out = []
    for budget in (None, 0):
        p = leaf_params(g)
        delta = torch.zeros(6, device="cuda", requires_grad=True)
        run(A, p, delta, cam, w, wd, memory_budget=budget).backward()
        out.append({**{k: np_of(p[k].grad) for k in KEYS}, "pose": np_of(delta.grad)})
    for k in out[0]:
        # same kernels on the same inputs; only the order of float atomics may differ
        assert rel_l2(out[1][k], out[0][k]) <= 1e-5, k


def test_central_differences_on_64_parameters(A, O):
    """h = 1e-3 on 64 random scalar parameters (and the 6 pose components);
    picks whose stencil changes the set of blended fragments (checked with the
    oracle's fragment signature) are replaced by new picks."""
    g = S.tiny_scene(seed=1000)
    cam = S.tiny_camera()
    w, wd = weights(96, 72, 21)
    p = leaf_params(g)
    delta = torch.zeros(6, device="cuda", requires_grad=True)
    run(A, p, delta, cam, w, wd).backward()
    an = {k: np_of(p[k].grad) for k in KEYS}
    rng = S.rng(22)
    h = 1e-3

    def sig(gg, cc):
        pr, img = O.forward(gg, cc)
        return img["sig"], tuple(pr["radius"])

    base_sig = sig(g, cam)
    checked, tries = 0, 0
    errs = []
    while checked < 64 and tries < 400:
        tries += 1
        k = KEYS[rng.integers(0, len(KEYS))]
        shape = g[k].shape
        idx = tuple(int(rng.integers(0, s)) for s in shape)
        gp = {kk: np.array(v, copy=True) for kk, v in g.items()}
        gm = {kk: np.array(v, copy=True) for kk, v in g.items()}
        gp[k][idx] += h
        gm[k][idx] -= h
        if not (sig(gp, cam) == base_sig == sig(gm, cam)):
            continue
        with torch.no_grad():
            Lp = float(run(A, leaf_params(gp), delta.detach(), cam, w, wd))
            Lm = float(run(A, leaf_params(gm), delta.detach(), cam, w, wd))
        fd = (Lp - Lm) / (2 * h)
        a = float(an[k][idx])
        errs.append(abs(fd - a))
        assert abs(fd - a) <= 2e-2 * max(abs(a), 1.0), (k, idx, fd, a)
        checked += 1
    assert checked == 64


def test_pose_central_differences(A, O):
    """The 6 pose components by central differences of the GPU forward on a
    sparse scene (any pose step moves every Gaussian, so a dense scene always
    changes some blended fragment); h = 3e-4 (the camera reaches the kernels
    in float32, so a smaller step is dominated by the rounding of R and t),
    stencils that change the oracle's fragment signature are skipped, at
    least 4 of 6 must be checked."""
    g = S.tiny_scene(seed=1114, n=6)
    cam = S.tiny_camera()
    w, wd = weights(96, 72, 23)
    p = leaf_params(g)
    delta = torch.zeros(6, device="cuda", requires_grad=True)
    run(A, p, delta, cam, w, wd).backward()
    h = 3e-4

    def sig(cc):
        pr, img = O.forward(g, cc)
        return img["sig"], tuple(pr["radius"])

    base = sig(cam)
    pose_checked = 0
    for i in range(6):
        e = np.zeros(6)
        e[i] = h
        if not (sig(A.apply_pose_delta(cam, e)) == base == sig(A.apply_pose_delta(cam, -e))):
            continue
        pose_checked += 1
        with torch.no_grad():
            Lp = float(run(A, leaf_params(g), torch.tensor(e, device="cuda").float(), cam, w, wd))
            Lm = float(run(A, leaf_params(g), torch.tensor(-e, device="cuda").float(), cam, w, wd))
        fd = (Lp - Lm) / (2 * h)
        a = float(delta.grad[i])
        assert abs(fd - a) <= 2e-2 * max(abs(a), 1.0), (i, fd, a)
    assert pose_checked >= 4


def test_two_views_before_one_backward(A):
    """Two renders of the same map (the same pooled buffer shape) before one
    backward: each keeps its own intermediates, so the gradient of the sum
    is the sum of the two single-view gradients."""
    g = S.surface_scene(30000, seed=14)
    c1 = S.camera(200, 150, 160.0)
    c2 = S.perturbed_pose(c1, seed=15, trans=0.03, rot_deg=2.0)
    w1, wd1 = weights(200, 150, 16)
    w2, wd2 = weights(200, 150, 17)
    single = []
    for cam, w, wd in ((c1, w1, wd1), (c2, w2, wd2)):
        p = leaf_params(g)
        delta = torch.zeros(6, device="cuda", requires_grad=True)
        run(A, p, delta, cam, w, wd).backward()
        single.append({k: np_of(p[k].grad) for k in KEYS})
    p = leaf_params(g)
    delta = torch.zeros(6, device="cuda", requires_grad=True)
    (run(A, p, delta, c1, w1, wd1) + run(A, p, delta, c2, w2, wd2)).backward()
    for k in KEYS:
        assert rel_l2(np_of(p[k].grad), single[0][k] + single[1][k]) <= 1e-5, k


def test_capacity_overflow_is_raised_then_grown(A):
    """A pooled rasterizer sized by a sparse view overflows on a dense one of
    the same grid: the backward raises, the capacity grows, and the render
    that follows is complete."""
    g = S.surface_scene(30000, seed=18)
    away = S.camera(200, 150, 160.0, R=S.axis_angle_matrix([0, 1, 0], 2.5))   # turned away: no keys
    near = S.camera(200, 150, 160.0)
    w, wd = weights(200, 150, 19)
    A._POOL.free.clear()                                       # (earlier tests pooled this shape)
    p = leaf_params(g)
    delta = torch.zeros(6, device="cuda", requires_grad=True)
    run(A, p, delta, away, w, wd).backward()                   # sizes the pooled buffers
    with pytest.raises(RuntimeError, match="exceeded the capacity"):
        run(A, leaf_params(g), delta, near, w, wd).backward()
    p = leaf_params(g)
    run(A, p, delta, near, w, wd).backward()
    fresh = leaf_params(g)
    A._POOL.free.clear()
    run(A, fresh, delta, near, w, wd).backward()
    for k in KEYS:
        assert rel_l2(np_of(p[k].grad), np_of(fresh[k].grad)) <= 1e-5, k


def test_autograd_3M_1920x1080_bf16(A, O):
    """The precision workload through gs_render: 3M Gaussians at 1920x1080
    with bf16 records, loss weights on a 256x256 crop; gradients within the
    64u bound of the precision form against the FP64 oracle on the crop, and
    recompute (memory budget 0) equal to store."""
    import torch as T
    from tests.test_gpu_scale import oracle_crop
    g = S.surface_scene(3_000_000, seed=4000)
    cam = S.perturbed_pose(S.camera(1920, 1080, 1000.0), seed=4001, trans=0.02, rot_deg=1.0)
    x0, y0, w, h = 832, 412, 256, 256
    rng = S.rng(4005)
    W = np.zeros((3, 1080, 1920), np.float32)
    Wd = np.zeros((1080, 1920), np.float32)
    W[:, y0:y0 + h, x0:x0 + w] = rng.normal(0, 1, (3, h, w)) / (w * h)
    Wd[y0:y0 + h, x0:x0 + w] = rng.normal(0, 1, (h, w)) / (w * h)
    from paper_2510_06644_gb300 import gs
    out = []
    for budget in (None, 0):
        p = leaf_params(g)
        delta = T.zeros(6, device="cuda", requires_grad=True)
        run(A, p, delta, cam, W, Wd, rec_dtype=gs.GS_BF16, memory_budget=budget).backward()
        out.append({**{k: np_of(p[k].grad) for k in KEYS}, "pose": np_of(delta.grad)})
    for k in out[0]:
        assert rel_l2(out[1][k], out[0][k]) <= 1e-5, k
    pr = O.project(g, cam)
    sp, ccam = oracle_crop(O, pr, cam, x0, y0, w, h)
    g2 = O.render_bwd(sp, ccam, W[:, y0:y0 + h, x0:x0 + w], Wd[y0:y0 + h, x0:x0 + w])
    ref = O.project_bwd(g, cam, g2)
    u = 2.0 ** -8
    errs = {k: rel_l2(out[0][k], ref[k]) for k in KEYS}
    errs["pose"] = rel_l2(out[0]["pose"], ref["pose"])
    print("\n[autograd bf16 3M 1920x1080 crop] " + " ".join(f"{k}={v:.2e}" for k, v in errs.items()))
    for k, v in errs.items():
        assert v <= 64 * u, (k, v)
