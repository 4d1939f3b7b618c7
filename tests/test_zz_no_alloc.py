"""rt_footprint_noalloc: the footprint counter for callers that cannot allocate
device memory (their device memory belongs to another allocator or budget, or
a cudaMalloc / cudaFree would stall their frame loop).  Its scratch lives in
static device arrays; here it is called through the C ABI, and its counts are
checked against the distinct taps that the oracle's floors give (on fragments
whose coordinates lie outside the FP32/FP64 rounding band, so the count must be
exact) and against rt_footprint, which allocates, on two calls in a row (the
second smaller than the first, so bits the first call left behind would show).

This file is collected last on purpose: it needs nothing from the other test
files and passes alone in a fresh process as well as after them."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2301_01719_gb300 import _lib, api

pytestmark = pytest.mark.gpu

ORACLE_FMT = {api.RT_F32: oracle.F32, api.RT_F16: oracle.F16}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_01719_gb300 import build

    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _noalloc(ctx, uv, d, o, filt, n_counts):
    """Calls rt_footprint_noalloc through ctypes; the counts buffer starts with junk."""
    counts = torch.full((max(n_counts, 1),), 987654321, dtype=torch.int64, device=uv.device)
    stream = torch.cuda.current_stream(uv.device).cuda_stream
    rc = _lib.lib().rt_footprint_noalloc(ctx.handle, ctypes.c_void_p(uv.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                         ctypes.c_void_p(o.data_ptr()), o.numel(), filt,
                                         ctypes.c_void_p(counts.data_ptr()), n_counts, ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    return rc, counts.cpu().numpy()[:n_counts]


def _band_free(table, g_uv, g_dir, obj, filt):
    """Fragments whose oracle coordinates all lie farther than the rounding band
    (8 w 2^-24 spatial, 64 n 2^-24 in-bucket coordinate units) from an integer:
    the GPU's floors must equal the oracle's on them."""
    _, oc, _ = oracle.locate(table, g_uv, g_dir, obj, filt)
    taus = np.zeros((len(obj), 4))
    for k, T in enumerate(table):
        if T is not None:
            taus[obj == k] = np.array([8 * T.W, 8 * T.H, 64 * T.n, 64 * T.n], np.float64) * 2.0 ** -24
    near = (np.abs(oc - np.round(oc)) < taus) & (np.abs(oc - np.round(oc)) > 0)
    return ~near.any(axis=1)


def _oracle_counts(table, g_uv, g_dir, obj, filt):
    """Distinct texels of every object: the oracle's floors and their +1
    neighbours (per filter), clamped to the texture, gathered in a set."""
    oi, _, _ = oracle.locate(table, g_uv, g_dir, obj, filt)
    out = []
    offs = [0, 1] if filt == api.RT_QUADRILINEAR else [0]
    aoffs = [0, 1] if filt != api.RT_NEAREST else [0]
    for k, T in enumerate(table):
        sel = obj == k
        if T is None or not sel.any():
            out.append(0)
            continue
        idx = oi[sel].astype(np.int64)
        dims = np.array([T.W, T.H, T.n, T.n])
        keys = set()
        for a in offs:
            for b in offs:
                for p in aoffs:
                    for q in aoffs:
                        keys.update(map(tuple, np.clip(idx + np.array([a, b, p, q]), 0, dims - 1)))
        out.append(len(keys))
    return np.array(out, np.int64)


def test_noalloc_counts_match_oracle_and_rt_footprint_twice(ctx):
    dev = torch.device("cuda", 0)
    oids, textures = [], []
    for k, (W, H, n, fmt) in enumerate(((64, 64, 8, api.RT_F16), (48, 40, 6, api.RT_F32))):
        atlas = oracle.fill_field(W, H, n, synth.field_lobes(900 + k))
        oids.append(api.rt_create_texture(ctx, W, H, n, fmt, api.RT_LAYOUT_ATLAS, torch.from_numpy(atlas).to(dev)))
        textures.append(oracle.Texture.from_f32(atlas, W, H, n, ORACLE_FMT[fmt]))
    table = [None] * (max(oids) + 1)
    for o, T in zip(oids, textures):
        table[o] = T
    g = synth.quad_scene(1001)
    rng = np.random.default_rng(0)
    obj_a = np.where(g.obj >= 0, np.array(oids, np.int32)[rng.integers(0, 2, g.F)], -1).astype(np.int32)
    hit = np.nonzero(g.obj >= 0)[0][:5000]  # the second call: 5000 fragments that hit the quad
    obj_b = np.full(len(hit), oids[1], np.int32)
    calls = [(g.uv, g.dir, obj_a, api.RT_QUADRILINEAR), (g.uv[hit], g.dir[hit], obj_b, api.RT_NEAREST)]
    n_counts = max(oids) + 1
    for k, (u_np, d_np, o_np, filt) in enumerate(calls):
        keep = _band_free(table, u_np, d_np, o_np, filt)
        assert keep.mean() > 0.9
        u_np, d_np, o_np = (np.ascontiguousarray(a[keep]) for a in (u_np, d_np, o_np))
        u, dd, o = (torch.from_numpy(a).to(dev) for a in (u_np, d_np, o_np))
        want = _oracle_counts(table, u_np, d_np, o_np, filt)
        assert want.sum() > 0
        ref = api.rt_footprint(ctx, u, dd, o, filt, n_counts)
        rc, got = _noalloc(ctx, u, dd, o, filt, n_counts)
        assert rc == api.RT_OK, api.rt_status_string(rc)
        np.testing.assert_array_equal(got, want, err_msg=f"call {k}: against the oracle's distinct taps")
        np.testing.assert_array_equal(got, np.array(ref, dtype=np.int64), err_msg=f"call {k}: against rt_footprint")
    assert api.rt_get_error(ctx) == api.RT_OK
    for o in oids:
        api.rt_destroy_texture(ctx, o)


def test_noalloc_counts_longer_and_shorter_than_the_object_table(ctx):
    dev = torch.device("cuda", 0)
    W, H, n = 32, 24, 4
    atlas = oracle.fill_field(W, H, n, synth.field_lobes(950))
    a = api.rt_create_texture(ctx, W, H, n, api.RT_F16, api.RT_LAYOUT_ATLAS, torch.from_numpy(atlas).to(dev))
    b = api.rt_create_texture(ctx, W, H, n, api.RT_F32, api.RT_LAYOUT_ATLAS, torch.from_numpy(atlas).to(dev))
    g = synth.quad_scene(1001, 128, 128)
    obj = np.where(g.obj >= 0, np.where(np.arange(g.F) % 2 == 0, a, b), -1).astype(np.int32)
    uv, d, o = (torch.from_numpy(x).to(dev) for x in (g.uv, g.dir, obj))
    n_obj = max(a, b) + 1
    ref = np.array(api.rt_footprint(ctx, uv, d, o, api.RT_QUADRILINEAR, n_obj), np.int64)
    rc, got = _noalloc(ctx, uv, d, o, api.RT_QUADRILINEAR, n_obj + 5)  # entries past the last object: zero
    assert rc == api.RT_OK
    np.testing.assert_array_equal(got[:n_obj], ref)
    np.testing.assert_array_equal(got[n_obj:], np.zeros(5, np.int64))
    rc, got = _noalloc(ctx, uv, d, o, api.RT_QUADRILINEAR, a + 1)  # only the objects up to a
    assert rc == api.RT_OK
    np.testing.assert_array_equal(got, ref[: a + 1])
    rc, _ = _noalloc(ctx, uv, d, o, api.RT_QUADRILINEAR, 0)  # no counts at all
    assert rc == api.RT_OK
    assert api.rt_get_error(ctx) == api.RT_OK
    api.rt_destroy_texture(ctx, a)
    api.rt_destroy_texture(ctx, b)


def test_noalloc_rejects_textures_beyond_its_bitmap():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_01719_gb300 import build

    build.build()
    c = api.Context(0)
    try:
        # 1024 x 1024 buckets of 9 x 9 texels: 84.9 M texels > 2^26
        big = api.rt_create_texture(c, 1024, 1024, 9, api.RT_E4M3_BUCKET_SCALE)
        dev = torch.device("cuda", 0)
        uv = torch.full((4, 2), 0.5, device=dev)
        d = torch.tensor([[0.0, 0.0, 1.0]] * 4, device=dev)
        o = torch.full((4,), big, dtype=torch.int32, device=dev)
        rc, _ = _noalloc(c, uv, d, o, api.RT_QUADRILINEAR, big + 1)
        assert rc == api.RT_ERR_INVALID_ARG
    finally:
        c.close()
