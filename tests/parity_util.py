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
