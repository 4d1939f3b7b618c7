"""Shared helpers of the GPU parity tests (test infrastructure)."""
import numpy as np
import torch

import oracle
import synth
from paper_2301_01719_gb300 import api

ORACLE_FMT = {api.RT_F32: oracle.F32, api.RT_F16: oracle.F16, api.RT_BF16: oracle.BF16,
              api.RT_E4M3_BUCKET_SCALE: oracle.E4M3}
FILTERS = [api.RT_NEAREST, api.RT_ANGULAR_BILINEAR, api.RT_QUADRILINEAR]
COLOUR_TOL = 1e-5  # absolute, FP32 kernel vs FP64 oracle, colours in [0, 1]


def dev():
    return torch.device("cuda", 0)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def gbuffer_to_dev(g):
    return to_dev(g.uv), to_dev(g.dir), to_dev(g.obj)


def planes_to_atlas(t: np.ndarray, W: int, H: int, n: int) -> np.ndarray:
    """(n, n, h, w, 4) [t, s, j, i] -> (h n, w n, 4)."""
    return t.reshape(n, n, H, W, 4).transpose(2, 0, 3, 1, 4).reshape(H * n, W * n, 4)


def atlas_to_planes(a: np.ndarray, W: int, H: int, n: int) -> np.ndarray:
    return a.reshape(H, n, W, n, 4).transpose(1, 3, 0, 2, 4).copy()


# RT_LAYOUT_QUADS, written out from its definition: a plane holds
# wq hq quads, wq = ceil(w / 2), hq = ceil(h / 2) (an odd side padded), and
# texel (i, j, s, t) lies at (t n + s) 4 wq hq + 4 ((j // 2) wq + i // 2) +
# 2 (j % 2) + i % 2, i.e. the C-order array (t, s, j // 2, i // 2, j % 2, i % 2, channel).

def quads_to_atlas(t: np.ndarray, W: int, H: int, n: int) -> np.ndarray:
    """(n, n, hq, wq, 2, 2, k) -> (h n, w n, k): row j n + t = (2 jq + jr) n + t,
    column (2 iq + ir) n + s; the padding is dropped."""
    wq, hq = (W + 1) // 2, (H + 1) // 2
    k = t.size // (4 * wq * hq * n * n)
    a = t.reshape(n, n, hq, wq, 2, 2, k).transpose(2, 4, 0, 3, 5, 1, 6).reshape(2 * hq * n, 2 * wq * n, k)
    return a[: H * n, : W * n]


def atlas_to_quads(a: np.ndarray, W: int, H: int, n: int) -> np.ndarray:
    """(h n, w n, k) -> (n, n, hq, wq, 2, 2, k), the padding zero."""
    wq, hq = (W + 1) // 2, (H + 1) // 2
    k = a.size // (W * H * n * n)
    p = np.zeros((2 * hq * n, 2 * wq * n, k), a.dtype)
    p[: H * n, : W * n] = a.reshape(H * n, W * n, k)
    return p.reshape(hq, 2, n, wq, 2, n, k).transpose(2, 5, 0, 3, 1, 4, 6).copy()


def storage_to_atlas(t: np.ndarray, layout: int, W: int, H: int, n: int) -> np.ndarray:
    """A PLANES or QUADS buffer (any shape, 4 channels) as the (h n, w n, 4) atlas."""
    if layout == api.RT_LAYOUT_QUADS:
        return quads_to_atlas(t, W, H, n)
    return planes_to_atlas(t, W, H, n)


def atlas_to_storage(a: np.ndarray, layout: int, W: int, H: int, n: int) -> np.ndarray:
    if layout == api.RT_LAYOUT_QUADS:
        return atlas_to_quads(a, W, H, n)
    return atlas_to_planes(a, W, H, n)


def storage_index(layout: int, W: int, H: int, n: int, i, j, s, t):
    """Flat texel index of (i, j, s, t) in a PLANES or QUADS buffer (numpy arrays or ints)."""
    if layout == api.RT_LAYOUT_QUADS:
        wq, hq = (W + 1) // 2, (H + 1) // 2
        i, j = np.asarray(i, np.int64), np.asarray(j, np.int64)
        return (np.asarray(t, np.int64) * n + s) * (4 * wq * hq) + 4 * ((j // 2) * wq + i // 2) + 2 * (j % 2) + i % 2
    return (np.asarray(t, np.int64) * n + s) * (W * H) + np.asarray(j, np.int64) * W + i


def grad_to_atlas(ctx, oid: int, t) -> np.ndarray:
    """The texel-gradient buffer of object oid (its storage layout) as an atlas."""
    info = api.rt_texture_info(ctx, oid)
    a = t.detach().cpu().numpy() if isinstance(t, torch.Tensor) else np.asarray(t)
    return storage_to_atlas(a, info["layout"], info["w"], info["h"], info["n"])


def index_taus(W: int, H: int, n: int):
    """Band half-widths (in coordinate units) within which FP32 and FP64 floors may differ:
    8 W 2^-24 for the spatial coordinates and 64 n 2^-24 for the in-bucket ones."""
    return np.array([8 * W, 8 * H, 64 * n, 64 * n], dtype=np.float64) * 2.0 ** -24


def compare_indices(g_idx, g_coord, o_idx, o_coord, taus, mask=None):
    """Floors must match bit-exactly outside the band; inside it they may differ by one.

    Returns (fragments whose floors differ -- all inside the band --, number of
    shaded fragments whose oracle coordinate lies inside the band).  A coordinate
    that sits exactly on an integer on both sides (a clamped one) is no mismatch."""
    g_idx = np.asarray(g_idx)
    o_idx = np.asarray(o_idx)
    mask = np.ones(len(o_idx), bool) if mask is None else mask
    dist = np.abs(o_coord - np.round(o_coord))
    taus = np.broadcast_to(taus, o_coord.shape)
    in_band = (dist < taus) & mask[:, None]
    diff = (g_idx != o_idx) & mask[:, None]
    bad = diff & ~in_band
    assert not bad.any(), f"{bad.sum()} index mismatches outside the band, first at {np.argwhere(bad)[:5]}"
    assert np.all(np.abs(g_idx[diff].astype(np.int64) - o_idx[diff]) == 1)
    # continuous coordinates agree to the band as well
    ok = ~in_band & mask[:, None]
    assert np.all(np.abs(g_coord - o_coord)[ok] <= taus[ok])
    near_integer = in_band & (dist > 0)
    return diff.any(axis=1), int(near_integer.any(axis=1).sum())


def floor_mismatch(ctx, g, obj_np, filt, table):
    """Fragments whose GPU floors differ from the oracle's (checked to lie in the band)."""
    uv, d, _ = gbuffer_to_dev(g)
    idx, coord = api.rt_locate(ctx, uv, d, to_dev(obj_np.astype(np.int32)), filt)
    oi, oc, _ = oracle.locate(table, g.uv, g.dir, obj_np, filt)
    taus = np.stack([index_taus(T.W, T.H, T.n) if T is not None else np.zeros(4) for T in table])
    per_frag = taus[np.maximum(obj_np, 0)]
    mism, _ = compare_indices(idx.cpu().numpy(), coord.cpu().numpy().astype(np.float64), oi, oc, per_frag,
                              mask=obj_np >= 0)
    return mism


def quad_workload(fmt=api.RT_F32, W=64, H=64, n=8, seed=1001, width=256, height=256):
    """The tiny quad workload: 256^2 pinhole frame of the quad, W x H buckets of n^2 texels
    from the multi-lobe field."""
    lobes = synth.field_lobes(seed)
    atlas = oracle.fill_field(W, H, n, lobes)
    g = synth.quad_scene(seed, width, height)
    T = oracle.Texture.from_f32(atlas, W, H, n, ORACLE_FMT[fmt])
    return atlas, g, T
