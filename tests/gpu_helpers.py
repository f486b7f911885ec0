"""Helpers shared by the GPU parity tests: moving synthetic inputs to the
device, packing stage-isolated 2D records, comparison metrics and the
predicate-margin bookkeeping of the parity policy."""
import numpy as np
import torch


def dev(g, device="cuda"):
    return {k: torch.as_tensor(np.ascontiguousarray(v)).to(device) for k, v in g.items()}


def pack_splats(s, device="cuda"):
    """float32 [n, 12] gs_splat records from drawn 2D Gaussians (the record
    layout of include/gs.h: x, y, conic a, b, c, opacity, depth, radius bits,
    r, g, b, tiles_touched bits)."""
    n = s["uv"].shape[0]
    rec = np.zeros((n, 12), np.float32)
    rec[:, 0:2] = s["uv"]
    rec[:, 2:5] = s["conic"]
    rec[:, 5] = s["opacity"]
    rec[:, 6] = s["depth"]
    rec[:, 7] = np.asarray(s["radius"], np.int32).view(np.float32)
    rec[:, 8:11] = s["rgb"]
    return torch.from_numpy(rec).to(device)


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def dilate(mask, r=0):
    if r <= 0:
        return mask
    out = mask.copy()
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            out |= np.roll(np.roll(mask, dy, 0), dx, 1)
    return out


def np_of(t):
    return t.detach().cpu().numpy()


def round_storage(x, name):
    """Round float64 values the way the 16-bit records store them: to float32
    first (the kernels compute in float32), then to bf16 (round to nearest
    even on the top 16 bits) or fp16."""
    x32 = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    if name == "fp16":
        return x32.astype(np.float16).astype(np.float64)
    b = x32.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def stored_splats(pr, name):
    """Projected splats with conic, opacity and colour as the 16-bit records hold them."""
    sp = dict(pr)
    for k in ("conic", "opacity", "rgb"):
        sp[k] = round_storage(pr[k], name)
    return sp
