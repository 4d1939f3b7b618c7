"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars: bit-exact codes for the encoders; floors bit-exact outside the FP32/FP64
band (parity_util.index_taus); colours within 1e-5 absolute; texel gradients
within the FP32 summation bound 1e-5 * sum_f w |g|; UV and direction
gradients within 1e-3 relative away from the kinks of the lookup.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2301_01719_gb300 import api, autograd
from parity_util import (COLOUR_TOL, FILTERS, ORACLE_FMT, atlas_to_planes, atlas_to_storage, compare_indices, dev,
                         floor_mismatch, gbuffer_to_dev, grad_to_atlas, index_taus, planes_to_atlas, quad_workload,
                         quads_to_atlas, to_dev)

pytestmark = pytest.mark.gpu

FORMATS = [api.RT_F32, api.RT_F16, api.RT_BF16, api.RT_E4M3_BUCKET_SCALE]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_01719_gb300 import build

    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _new_texture(ctx, atlas, W, H, n, fmt, layout=api.RT_LAYOUT_ATLAS, flags=0):
    src = to_dev(atlas if layout == api.RT_LAYOUT_ATLAS else atlas_to_storage(atlas, layout, W, H, n))
    oid = api.rt_create_texture(ctx, W, H, n, fmt, layout, src, flags)
    return oid, src


@pytest.mark.parametrize("fmt", FORMATS)
def test_encoders_bit_exact(ctx, fmt):
    W, H, n = 64, 64, 8
    atlas, _, T = quad_workload(fmt, W, H, n)
    # include values that exercise rounding: scale some buckets up, some to zero
    atlas = atlas.copy()
    atlas[: 2 * n] *= 37.0
    atlas[2 * n: 3 * n, : 5 * n] = 0.0
    T = oracle.Texture.from_f32(atlas, W, H, n, ORACLE_FMT[fmt])
    oid, _ = _new_texture(ctx, atlas, W, H, n, fmt)
    codes, scales = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_ATLAS)
    got = codes.cpu().numpy()
    if fmt == api.RT_F32:
        np.testing.assert_array_equal(got.view(np.uint32), T.codes.view(np.uint32))
    else:
        np.testing.assert_array_equal(got.view(T.codes.dtype), T.codes)
    if fmt == api.RT_E4M3_BUCKET_SCALE:
        np.testing.assert_array_equal(scales.cpu().numpy().view(np.uint32), T.scales.view(np.uint32))
    # stored in 2 x 2 bucket quads; planes and quads read-backs are the same codes, permuted
    assert api.rt_texture_info(ctx, oid)["layout"] == api.RT_LAYOUT_QUADS
    pc, _ = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_PLANES)
    np.testing.assert_array_equal(planes_to_atlas(pc.cpu().numpy(), W, H, n), got)
    qc, _ = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_QUADS)
    assert tuple(qc.shape) == (n, n, H // 2, W // 2, 2, 2, 4)
    np.testing.assert_array_equal(quads_to_atlas(qc.cpu().numpy(), W, H, n), got)
    api.rt_destroy_texture(ctx, oid)


def test_owned_textures_are_stored_in_quads(ctx):
    """Owned dense textures are stored in 2 x 2 bucket quads, an odd side padded
    (zero codes there), bit textures in planes; read-backs and conversions agree
    with the definition of each layout at even and odd sides; a borrowed quads
    buffer shades like the owned texture."""
    W, H, n = 5, 3, 4
    a = np.random.default_rng(4).normal(size=(H * n, W * n, 4)).astype(np.float32)
    oid, _ = _new_texture(ctx, a, W, H, n, api.RT_F32)
    info = api.rt_texture_info(ctx, oid)
    assert info["layout"] == api.RT_LAYOUT_QUADS
    assert info["bytes"] == 16 * 4 * 3 * 2 * n * n  # 3 x 2 quads of 4 buckets per plane
    qc, _ = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_QUADS)
    want = atlas_to_storage(a, api.RT_LAYOUT_QUADS, W, H, n)  # zero padding
    np.testing.assert_array_equal(qc.cpu().numpy(), want)
    bits = api.rt_create_texture(ctx, 8, 8, 2, api.RT_BIT1)  # bit textures keep the planes bit numbering
    assert api.rt_texture_info(ctx, bits)["layout"] == api.RT_LAYOUT_PLANES
    api.rt_destroy_texture(ctx, bits)
    for W2, H2 in ((10, 6), (5, 3), (1, 1)):
        b = np.random.default_rng(W2).normal(size=(H2 * n, W2 * n, 4)).astype(np.float32)
        for src_l in (api.RT_LAYOUT_ATLAS, api.RT_LAYOUT_PLANES, api.RT_LAYOUT_QUADS):
            for dst_l in (api.RT_LAYOUT_ATLAS, api.RT_LAYOUT_PLANES, api.RT_LAYOUT_QUADS):
                src = to_dev(b if src_l == api.RT_LAYOUT_ATLAS else atlas_to_storage(b, src_l, W2, H2, n))
                out = api.rt_convert_layout(src, src_l, dst_l, W2, H2, n).cpu().numpy()
                want = b if dst_l == api.RT_LAYOUT_ATLAS else atlas_to_storage(b, dst_l, W2, H2, n)
                np.testing.assert_array_equal(out.reshape(-1), want.reshape(-1))
    # the same texels borrowed as a padded quads buffer shade bit for bit like the owned texture
    g = synth.quad_scene(1009, 64, 64)
    uv, d, o = gbuffer_to_dev(g)
    bid, keep = _new_texture(ctx, a, W, H, n, api.RT_F32, api.RT_LAYOUT_QUADS, api.RT_BORROW)
    for filt in FILTERS:
        own = api.rt_shade(ctx, uv, d, torch.where(o >= 0, torch.full_like(o, oid), o), filt)
        bor = api.rt_shade(ctx, uv, d, torch.where(o >= 0, torch.full_like(o, bid), o), filt)
        assert torch.equal(own, bor)
    assert api.rt_get_error(ctx) == api.RT_OK
    api.rt_destroy_texture(ctx, bid)
    api.rt_destroy_texture(ctx, oid)


@pytest.mark.parametrize("filt", FILTERS)
def test_locate_indices(ctx, filt):
    W, H, n = 64, 64, 8
    atlas, g, T = quad_workload(api.RT_F32, W, H, n)
    oid, _ = _new_texture(ctx, atlas, W, H, n, api.RT_F32)
    uv, d, o = gbuffer_to_dev(g)
    obj = torch.where(o >= 0, torch.full_like(o, oid), o)
    idx, coord = api.rt_locate(ctx, uv, d, obj, filt)
    textures = [None] * (oid + 1)
    textures[oid] = T
    oi, oc, flags = oracle.locate(textures, g.uv, g.dir, np.where(g.obj >= 0, oid, -1), filt)
    assert flags == 0
    _, band = compare_indices(idx.cpu().numpy(), coord.cpu().numpy().astype(np.float64), oi, oc,
                              index_taus(W, H, n), mask=g.obj >= 0)
    assert band <= 8, band
    assert api.rt_get_error(ctx) == api.RT_OK
    api.rt_destroy_texture(ctx, oid)


def _shade_both(ctx, textures_np, oids, g, filt, obj_np=None):
    obj_np = g.obj if obj_np is None else obj_np
    uv, d, _ = gbuffer_to_dev(g)
    o = to_dev(obj_np.astype(np.int32))
    out = api.rt_shade(ctx, uv, d, o, filt).cpu().numpy()
    status = api.rt_get_error(ctx)
    table = [None] * (max(oids) + 1)
    for T, k in zip(textures_np, oids):
        table[k] = T
    ref, flags = oracle.shade(table, g.uv, g.dir, obj_np, filt)
    return out, ref, status, flags


def _nearest_band(ctx, g, obj_np, filt, W, H, n, T, oid):
    """Fragments whose FP32 floors differ from the FP64 ones (all inside the band)."""
    table = [None] * (oid + 1)
    table[oid] = T
    return floor_mismatch(ctx, g, obj_np, filt, table)


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("filt", FILTERS)
def test_shade_matches_oracle(ctx, fmt, filt):
    W, H, n = 64, 64, 8
    atlas, g, T = quad_workload(fmt, W, H, n)
    oid, _ = _new_texture(ctx, atlas, W, H, n, fmt)
    obj_np = np.where(g.obj >= 0, oid, -1).astype(np.int32)
    out, ref, status, flags = _shade_both(ctx, [T], [oid], g, filt, obj_np)
    assert status == api.RT_OK and flags == 0
    keep = np.ones(g.F, bool)
    if filt != api.RT_QUADRILINEAR:  # a nearest axis may flip inside the band: colour jumps there
        keep = ~_nearest_band(ctx, g, obj_np, filt, W, H, n, T, oid)
    err = np.abs(out - ref)[keep]
    assert err.max() <= COLOUR_TOL, err.max()
    assert np.all(out[obj_np < 0] == 0)
    api.rt_destroy_texture(ctx, oid)


@pytest.mark.parametrize("filt", FILTERS)
def test_borrowed_layouts_match_owned(ctx, filt):
    W, H, n = 48, 40, 6
    atlas, g, T = quad_workload(api.RT_F32, W, H, n)
    uv, d, o = gbuffer_to_dev(g)
    outs, keep, oids = [], [], []
    for layout, flags in ((api.RT_LAYOUT_ATLAS, 0), (api.RT_LAYOUT_ATLAS, api.RT_BORROW),
                          (api.RT_LAYOUT_PLANES, api.RT_BORROW), (api.RT_LAYOUT_QUADS, api.RT_BORROW)):
        oid, src = _new_texture(ctx, atlas, W, H, n, api.RT_F32, layout, flags)
        obj = torch.where(o >= 0, torch.full_like(o, oid), o)
        outs.append(api.rt_shade(ctx, uv, d, obj, filt).cpu().numpy())
        keep.append(src)
        oids.append(oid)
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])
    np.testing.assert_array_equal(outs[0], outs[3])
    obj_np = np.where(g.obj >= 0, oids[0], -1).astype(np.int32)
    table = [None] * (oids[0] + 1)
    table[oids[0]] = T
    ref, _ = oracle.shade(table, g.uv, g.dir, obj_np, filt)
    ok = np.ones(g.F, bool)
    if filt != api.RT_QUADRILINEAR:
        ok = ~_nearest_band(ctx, g, obj_np, filt, W, H, n, T, oids[0])
    assert np.abs(outs[0] - ref)[ok].max() <= COLOUR_TOL
    for oid in oids:
        api.rt_destroy_texture(ctx, oid)


@pytest.mark.parametrize("F", [0, 1, 3, 4, 255, 256, 257, 1003, 65533])
def test_ragged_sizes(ctx, F):
    W, H, n = 64, 64, 8
    atlas, g, T = quad_workload(api.RT_F16, W, H, n)
    oid, _ = _new_texture(ctx, atlas, W, H, n, api.RT_F16)
    sel = np.random.default_rng(F).permutation(g.F)[:F]
    sub = synth.GBuffer(g.uv[sel].copy(), g.dir[sel].copy(), np.where(g.obj[sel] >= 0, oid, -1).astype(np.int32),
                        F, 1, 1)
    if F == 0:
        uv = torch.empty((0, 2), device=dev())
        d = torch.empty((0, 3), device=dev())
        o = torch.empty((0,), dtype=torch.int32, device=dev())
        out = api.rt_shade(ctx, uv, d, o, api.RT_QUADRILINEAR)
        assert out.shape == (0, 4)
        api.rt_shade_backward(ctx, uv, d, o, api.RT_QUADRILINEAR, torch.empty((0, 4), device=dev()))
    else:
        table = [None] * (oid + 1)
        table[oid] = T
        uv, d, o = gbuffer_to_dev(sub)
        out = api.rt_shade(ctx, uv, d, o, api.RT_QUADRILINEAR).cpu().numpy()
        ref, _ = oracle.shade(table, sub.uv, sub.dir, sub.obj, oracle.QUADRILINEAR)
        assert np.abs(out - ref).max() <= COLOUR_TOL
    assert api.rt_get_error(ctx) == api.RT_OK
    api.rt_destroy_texture(ctx, oid)


def _edge_gbuffer(rng, F, oid):
    uv = rng.uniform(-0.3, 1.3, (F, 2))
    z = rng.uniform(-1, 1, F)
    phi = rng.uniform(0, 2 * np.pi, F)
    r = np.sqrt(1 - z * z)
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], 1)
    specials_d = [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0.7071068, 0.7071068, 0],
                  [0.5, 0.5, 0.7071068], [3.0, 0.0, 4.0], [0.1, 0.2, 0.3], [1e-20, 0, 1], [0, 1e-35, 1],
                  [-0.6, 0.0, -0.8], [2e-8, -3e-8, -1.0]]
    specials_uv = [[0, 0], [1, 1], [0.5, 0.5], [1, 0], [0, 1], [-5, 7], [0.999999, 1e-7], [0.25, 0.75]]
    d[: len(specials_d)] = specials_d
    uv[: len(specials_uv)] = specials_uv
    return synth.GBuffer(uv.astype(np.float32), d.astype(np.float32), np.full(F, oid, np.int32), F, 1, 1)


@pytest.mark.parametrize("W,H,n", [(1, 1, 1), (1, 1, 2), (3, 2, 3), (5, 7, 5), (33, 17, 12), (2, 3, 64),
                                   (4096, 3, 2)])
@pytest.mark.parametrize("filt", FILTERS)
def test_edge_cases(ctx, W, H, n, filt):
    rng = np.random.default_rng(W * 1000 + H * 10 + n)
    atlas = rng.uniform(0, 1, (H * n, W * n, 4)).astype(np.float32)
    oid, _ = _new_texture(ctx, atlas, W, H, n, api.RT_F32)
    T = oracle.Texture.from_f32(atlas, W, H, n, oracle.F32)
    g = _edge_gbuffer(rng, 3001, oid)
    table = [None] * (oid + 1)
    table[oid] = T
    uv, d, o = gbuffer_to_dev(g)
    idx, coord = api.rt_locate(ctx, uv, d, o, filt)
    oi, oc, flags = oracle.locate(table, g.uv, g.dir, g.obj, filt)
    assert flags == 0
    mism, _ = compare_indices(idx.cpu().numpy(), coord.cpu().numpy().astype(np.float64), oi, oc,
                              index_taus(W, H, n))
    out = api.rt_shade(ctx, uv, d, o, filt).cpu().numpy()
    ref, _ = oracle.shade(table, g.uv, g.dir, g.obj, filt)
    keep = ~mism if filt != api.RT_QUADRILINEAR else np.ones(g.F, bool)
    assert np.abs(out - ref)[keep].max() <= COLOUR_TOL
    assert api.rt_get_error(ctx) == api.RT_OK
    api.rt_destroy_texture(ctx, oid)


def test_errors_and_status(ctx):
    W, H, n = 4, 4, 4
    atlas = np.ones((H * n, W * n, 4), np.float32)
    oid, _ = _new_texture(ctx, atlas, W, H, n, api.RT_F32)
    uv = to_dev(np.full((8, 2), 0.5, np.float32))
    d = to_dev(np.tile(np.float32([[0, 0, 1]]), (8, 1)))
    obj = to_dev(np.array([oid, -1, oid + 5, 1000, oid, oid, -3, oid], np.int32))
    out = api.rt_shade(ctx, uv, d, obj, api.RT_QUADRILINEAR).cpu().numpy()
    np.testing.assert_array_equal(out[:, 0], [1, 0, 0, 0, 1, 1, 0, 1])
    assert api.rt_get_error(ctx) == api.RT_ERR_BAD_OBJ_ID
    assert api.rt_get_error(ctx) == api.RT_OK  # cleared
    d2 = d.clone()
    d2[4, 1] = float("nan")
    uv2 = uv.clone()
    uv2[5, 0] = float("inf")
    out = api.rt_shade(ctx, uv2, d2, to_dev(np.full(8, oid, np.int32)), api.RT_QUADRILINEAR).cpu().numpy()
    np.testing.assert_array_equal(out[:, 0], [1, 1, 1, 1, 0, 0, 1, 1])
    assert api.rt_get_error(ctx) == api.RT_ERR_NONFINITE
    # host-side validation
    big = torch.zeros(64, device=dev())
    with pytest.raises(api.RadtexError) as e:
        api._lib.call("rt_shade", ctx.handle, api._ptr(big[1:]), api._ptr(d), api._ptr(obj), 8,
                      api.RT_QUADRILINEAR, api._ptr(big), None)
    assert e.value.status == api._lib.RT_ERR_INVALID_ARG
    with pytest.raises(api.RadtexError):
        api.rt_shade(ctx, uv, d, obj, 7)
    with pytest.raises(api.RadtexError):
        api.rt_create_texture(ctx, 0, 4, 4, api.RT_F32)
    with pytest.raises(api.RadtexError):
        api.rt_create_texture(ctx, 4, 4, 4, api.RT_F16, api.RT_LAYOUT_ATLAS, to_dev(atlas), api.RT_BORROW)
    # a destroyed texture: its fragments read nothing and raise BAD_OBJ_ID
    api.rt_destroy_texture(ctx, oid)
    out = api.rt_shade(ctx, uv, d, to_dev(np.full(8, oid, np.int32)), api.RT_QUADRILINEAR).cpu().numpy()
    assert np.all(out == 0)
    assert api.rt_get_error(ctx) == api.RT_ERR_BAD_OBJ_ID


def test_many_objects_mixed(ctx):
    """Objects of different bucket matrices, direction resolutions and formats in one launch."""
    rng = np.random.default_rng(77)
    specs = [(64, 64, 8, api.RT_F16), (17, 9, 12, api.RT_F32), (128, 32, 4, api.RT_BF16),
             (24, 24, 16, api.RT_E4M3_BUCKET_SCALE), (5, 3, 32, api.RT_F16)]
    oids, Ts = [], []
    for k, (W, H, n, fmt) in enumerate(specs):
        atlas = oracle.fill_field(W, H, n, synth.field_lobes(500 + k))
        oid, _ = _new_texture(ctx, atlas, W, H, n, fmt)
        oids.append(oid)
        Ts.append(oracle.Texture.from_f32(atlas, W, H, n, ORACLE_FMT[fmt]))
    F = 50000
    g = _edge_gbuffer(rng, F, 0)
    g.uv[:] = rng.uniform(0, 1, (F, 2))
    obj = np.array(oids, np.int32)[rng.integers(0, len(oids), F)]
    obj[rng.uniform(size=F) < 0.1] = -1
    out, ref, status, flags = _shade_both(ctx, Ts, oids, g, api.RT_QUADRILINEAR, obj)
    assert status == api.RT_OK and flags == 0
    assert np.abs(out - ref).max() <= COLOUR_TOL
    for o in oids:
        api.rt_destroy_texture(ctx, o)


def test_texel_centres_reproduced(ctx):
    """A texture filled from an analytic field returns the field at bucket and texel centres."""
    W, H, n = 9, 7, 8
    lobes = synth.field_lobes(33)
    atlas = oracle.fill_field(W, H, n, lobes)
    oid, _ = _new_texture(ctx, atlas, W, H, n, api.RT_F32)
    jj, ii, tt, ss = np.meshgrid(np.arange(H), np.arange(W), np.arange(n), np.arange(n), indexing="ij")
    ii, jj, ss, tt = (x.reshape(-1) for x in (ii, jj, ss, tt))
    dirs = oracle.texel_directions(n)[tt, ss]
    uv = np.stack([(ii + 0.5) / W, (jj + 0.5) / H], 1).astype(np.float32)
    g = synth.GBuffer(uv, dirs.astype(np.float32), np.full(len(ii), oid, np.int32), len(ii), 1, 1)
    stored = atlas[jj * n + tt, ii * n + ss]
    for filt in FILTERS:
        out = api.rt_shade(ctx, *gbuffer_to_dev(g), filt).cpu().numpy()
        if filt == api.RT_NEAREST:
            np.testing.assert_array_equal(out, stored)
        else:
            assert np.abs(out - stored).max() <= COLOUR_TOL
    api.rt_destroy_texture(ctx, oid)


def test_constant_texture_exact(ctx):
    W, H, n = 8, 8, 8
    c = np.float32([0.1, 0.7, 0.3, 1.0])
    atlas = np.broadcast_to(c, (H * n, W * n, 4)).copy()
    rng = np.random.default_rng(5)
    for fmt in FORMATS:
        oid, _ = _new_texture(ctx, atlas, W, H, n, fmt)
        g = _edge_gbuffer(rng, 5000, oid)
        T = oracle.Texture.from_f32(atlas, W, H, n, ORACLE_FMT[fmt])
        expect = np.float32(T.values()[0, 0])
        for filt in FILTERS:
            out = api.rt_shade(ctx, *gbuffer_to_dev(g), filt).cpu().numpy()
            np.testing.assert_array_equal(out, np.broadcast_to(expect, out.shape))
        api.rt_destroy_texture(ctx, oid)


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("W,H", [(37, 23), (38, 24)])  # stored in planes / in quads
def test_fill_bucket_lobes(ctx, fmt, W, H):
    n = 16
    params = synth.bucket_lobe_params(9, W, H)
    oid = api.rt_create_texture(ctx, W, H, n, fmt)
    api.rt_fill_bucket_lobes(ctx, oid, to_dev(params))
    codes, scales = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_ATLAS)
    ref = oracle.fill_bucket_lobes(W, H, n, params).astype(np.float64)
    ofmt = ORACLE_FMT[fmt]
    c = codes.cpu().numpy()
    if ofmt in (oracle.F16, oracle.BF16):
        c = c.view(np.uint16)
    got = oracle.decode(ofmt, c)
    if fmt == api.RT_E4M3_BUCKET_SCALE:
        s = np.repeat(np.repeat(scales.cpu().numpy().astype(np.float64), n, 0), n, 1)[..., None]
        got = got * s
        tol = 2.0 ** -4 * np.abs(ref) + 2.0 ** -10 * s + 1e-4
    else:
        rel = {api.RT_F32: 0.0, api.RT_F16: 2.0 ** -11, api.RT_BF16: 2.0 ** -8}[fmt]
        # FP32 evaluation of max(0, I.d)^p with p <= 200: relative error ~ p * 8 ulp
        tol = rel * np.abs(ref) + 2e-4 * np.abs(ref) + 1e-6
    assert np.all(np.abs(got - ref) <= tol)
    api.rt_destroy_texture(ctx, oid)


def _kink_mask(table, g, obj, filt, W, H, n, margin=1e-3):
    """Fragments away from the kinks of the lookup, where FP32 and FP64 may take
    different one-sided derivatives: integer coordinates (floor changes) and the
    clamp bounds of B.  (The Eq. 3 branch is decided on the same FP32 inputs on
    both sides, so its diagonal needs no margin.)"""
    _, oc, _ = oracle.locate(table, g.uv, g.dir, obj, filt)
    far = (np.abs(oc - np.round(oc)) > margin).all(axis=1)
    B = oracle.squarify(oracle.equisolid(g.dir.astype(np.float64)))
    lo = 1.0 / n - 1.0
    far &= (np.abs(np.abs(B) - abs(lo)) > margin).all(axis=1)
    return far


@pytest.mark.parametrize("fmt", [api.RT_F32, api.RT_F16, api.RT_E4M3_BUCKET_SCALE])
@pytest.mark.parametrize("filt", FILTERS)
@pytest.mark.parametrize("W,H", [(64, 64), (37, 23)])  # quads, and quads with padded odd sides
def test_backward_matches_oracle(ctx, fmt, filt, W, H):
    n = 8
    atlas, g, T = quad_workload(fmt, W, H, n)
    oid, _ = _new_texture(ctx, atlas, W, H, n, fmt)
    obj_np = np.where(g.obj >= 0, oid, -1).astype(np.int32)
    table = [None] * (oid + 1)
    table[oid] = T
    rng = np.random.default_rng(3)
    gout = rng.normal(size=(g.F, 4)).astype(np.float32)
    uv, d, _ = gbuffer_to_dev(g)
    o = to_dev(obj_np)
    dtex = torch.empty(api.layout_shape(api.rt_texture_info(ctx, oid)["layout"], W, H, n), dtype=torch.float32,
                       device=dev())
    duv = torch.empty_like(uv)
    ddir = torch.empty_like(d)
    api.rt_shade_backward(ctx, uv, d, o, filt, to_dev(gout), {oid: dtex}, duv, ddir)
    assert api.rt_get_error(ctx) == api.RT_OK
    gt, guv, gdir, flags = oracle.shade_backward(table, g.uv, g.dir, obj_np, filt, gout)
    gabs, _, _, _ = oracle.shade_backward(table, g.uv, g.dir, obj_np, filt, np.abs(gout), want_uv=False,
                                          want_dir=False)
    got = grad_to_atlas(ctx, oid, dtex)
    # FP32 summation (1e-4 relative to sum w|g|) plus FP32 weights, whose
    # coordinates carry up to ~8 n 2^-24 of rounding per contributing fragment
    tol = 1e-4 * gabs[oid] + 2e-5 * np.abs(gout).max()
    assert np.all(np.abs(got - gt[oid]) <= tol)
    far = _kink_mask(table, g, obj_np, filt, W, H, n) & (obj_np >= 0)
    assert far.sum() > 1000
    for got_c, ref_c in ((duv.cpu().numpy(), guv), (ddir.cpu().numpy(), gdir)):
        scale = np.abs(ref_c[far]).max() + 1e-30
        assert np.all(np.abs(got_c[far] - ref_c[far]) <= 1e-3 * np.abs(ref_c[far]) + 1e-5 * scale)
        assert np.all(got_c[obj_np < 0] == 0)
    # accumulate adds to what is there
    duv2 = duv.clone()
    api.rt_shade_backward(ctx, uv, d, o, filt, to_dev(gout), {oid: dtex}, duv2, None, api.RT_ACCUMULATE)
    np.testing.assert_allclose(duv2.cpu().numpy(), 2 * duv.cpu().numpy(), rtol=1e-6, atol=0)
    got2 = grad_to_atlas(ctx, oid, dtex)
    assert np.all(np.abs(got2 - 2 * gt[oid]) <= 2 * tol)
    api.rt_destroy_texture(ctx, oid)


def test_autograd_function(ctx):
    W, H, n = 32, 32, 8
    atlas, g, T = quad_workload(api.RT_F32, W, H, n)
    tex = to_dev(atlas_to_planes(atlas, W, H, n)).requires_grad_(True)
    oid = api.rt_create_texture(ctx, W, H, n, api.RT_F32, api.RT_LAYOUT_PLANES, tex.detach(), api.RT_BORROW)
    uv, d, o = gbuffer_to_dev(g)
    o = torch.where(o >= 0, torch.full_like(o, oid), o)
    uv.requires_grad_(True)
    d.requires_grad_(True)
    out = autograd.shade(ctx, uv, d, o, api.RT_QUADRILINEAR, {oid: tex})
    target = torch.zeros_like(out)
    loss = 0.5 * ((out - target) ** 2).sum()
    loss.backward()
    table = [None] * (oid + 1)
    table[oid] = T
    obj_np = o.cpu().numpy()
    ref, _ = oracle.shade(table, g.uv, g.dir, obj_np, oracle.QUADRILINEAR)
    gt, guv, gdir, _ = oracle.shade_backward(table, g.uv, g.dir, obj_np, oracle.QUADRILINEAR, ref)
    got = planes_to_atlas(tex.grad.cpu().numpy(), W, H, n)
    assert np.abs(got - gt[oid]).max() <= 1e-4 * max(1.0, np.abs(gt[oid]).max())
    far = _kink_mask(table, g, obj_np, oracle.QUADRILINEAR, W, H, n) & (obj_np >= 0)
    np.testing.assert_allclose(uv.grad.cpu().numpy()[far], guv[far], rtol=1e-3, atol=1e-4)
    api.rt_destroy_texture(ctx, oid)


@pytest.mark.parametrize("filt", FILTERS)
def test_footprint_counts(ctx, filt):
    W, H, n = 64, 64, 8
    atlas, g, T = quad_workload(api.RT_F16, W, H, n)
    oid, _ = _new_texture(ctx, atlas, W, H, n, api.RT_F16)
    obj_np = np.where(g.obj >= 0, oid, -1).astype(np.int32)
    uv, d, _ = gbuffer_to_dev(g)
    counts = api.rt_footprint(ctx, uv, d, to_dev(obj_np), filt, oid + 1)
    # distinct taps from the oracle's floors, clamped to the texture
    table = [None] * (oid + 1)
    table[oid] = T
    oi, oc, _ = oracle.locate(table, g.uv, g.dir, obj_np, filt)
    band = (np.abs(oc - np.round(oc)) < index_taus(W, H, n)).any(axis=1)[obj_np >= 0]
    idx = oi[obj_np >= 0].astype(np.int64)
    dims = np.array([W, H, n, n])
    keys = set()
    offs = [0, 1] if filt == api.RT_QUADRILINEAR else [0]
    aoffs = [0, 1] if filt != api.RT_NEAREST else [0]
    for a in offs:
        for b in offs:
            for p in aoffs:
                for q in aoffs:
                    t = idx + np.array([a, b, p, q])
                    t = np.clip(t, 0, dims - 1)
                    keys.update(map(tuple, t))
    assert abs(counts[oid] - len(keys)) <= 16 * int(band.sum())
    api.rt_destroy_texture(ctx, oid)


@pytest.mark.parametrize("filt", [api.RT_ANGULAR_BILINEAR, api.RT_QUADRILINEAR])
def test_direction_gradient_at_eq3_ties(ctx, filt):
    """Directions with |I_x| = |I_y| exactly (so |A_x| = |A_y| in FP32 and FP64
    alike) sit on Eq. 3's kink; the kernel takes the x branch as the oracle does
    (reading R6)."""
    W, H, n = 6, 5, 8
    rng = np.random.default_rng(77)
    atlas = rng.uniform(0, 1, (H * n, W * n, 4)).astype(np.float32)
    oid = api.rt_create_texture(ctx, W, H, n, api.RT_F32, api.RT_LAYOUT_ATLAS, to_dev(atlas))
    F = 512
    a = rng.uniform(0.15, 0.6, F).astype(np.float32)
    sx, sy = rng.choice([-1.0, 1.0], F).astype(np.float32), rng.choice([-1.0, 1.0], F).astype(np.float32)
    d = np.stack([sx * a, sy * a, np.sqrt(1 - 2 * a * a)], 1).astype(np.float32)
    assert np.all(np.abs(d[:, 0]) == np.abs(d[:, 1]))
    uv = rng.uniform(0.1, 0.9, (F, 2)).astype(np.float32)
    obj = np.full(F, oid, np.int32)
    g = rng.normal(size=(F, 4)).astype(np.float32)
    ddir = torch.empty((F, 3), device="cuda")
    api.rt_shade_backward(ctx, to_dev(uv), to_dev(d), to_dev(obj), filt, to_dev(g), None, None, ddir)
    assert api.rt_get_error(ctx) == api.RT_OK
    T = oracle.Texture.from_f32(atlas, W, H, n, oracle.F32)
    table = [None] * oid + [T]
    _, _, gdir, flags = oracle.shade_backward(table, uv, d, obj, filt, g.astype(np.float64), want_tex=False)
    assert flags == 0
    _, oc, _ = oracle.locate(table, uv, d, obj, filt)
    far = (np.abs(oc - np.round(oc)) > 1e-3).all(axis=1)
    assert far.sum() > F // 2
    got = ddir.cpu().numpy()
    scale = np.abs(gdir[far]).max()
    assert np.all(np.abs(got[far] - gdir[far]) <= 1e-3 * np.abs(gdir[far]) + 1e-5 * scale)
    api.rt_destroy_texture(ctx, oid)


def test_zero_texture_grads(ctx):
    """rt_zero_texture_grads clears exactly each listed object's gradient extent on
    the stream, leaves unlisted buffers alone, and rejects dead objects; with it,
    clear + RT_ACCUMULATE equals the backward's own clear (no RT_ACCUMULATE)."""
    W, H, n = 24, 16, 4
    atlas, g, T = quad_workload(api.RT_F16, W, H, n, width=64, height=64)
    a, _ = _new_texture(ctx, atlas, W, H, n, api.RT_F16)
    b, _ = _new_texture(ctx, atlas, W, H, n, api.RT_F32)
    size = n * n * H * W * 4
    ga = torch.full((size + 4,), 7.0, device="cuda")  # 4 guard floats past the extent
    gb = torch.full((size,), 3.0, device="cuda")
    api.rt_zero_texture_grads(ctx, {a: ga[:size]})
    torch.cuda.synchronize()
    assert float(ga[:size].abs().max()) == 0.0 and bool((ga[size:] == 7.0).all())
    assert bool((gb == 3.0).all())
    obj_np = np.where(g.obj >= 0, a, -1).astype(np.int32)
    uv, d, _ = gbuffer_to_dev(g)
    o = to_dev(obj_np)
    gout = torch.rand((g.F, 4), device="cuda")
    own = torch.full((size,), 5.0, device="cuda")
    api.rt_shade_backward(ctx, uv, d, o, api.RT_NEAREST, gout, {a: own})  # the backward's own clear
    gb.fill_(9.0)
    api.rt_zero_texture_grads(ctx, {a: gb})
    api.rt_shade_backward(ctx, uv, d, o, api.RT_NEAREST, gout, {a: gb}, flags=api.RT_ACCUMULATE)
    torch.cuda.synchronize()
    assert float(own.abs().sum()) > 0
    torch.testing.assert_close(gb, own, rtol=1e-5, atol=1e-6)  # equal up to the order of the atomic sums
    # RT_ACCUMULATE_TEXELS: texel gradients add to the cleared buffer, per-fragment outputs are overwritten
    filt = api.RT_QUADRILINEAR
    duv0, ddir0 = torch.empty_like(uv), torch.empty_like(d)
    g0 = torch.empty((size,), device="cuda")
    api.rt_shade_backward(ctx, uv, d, o, filt, gout, {a: g0}, duv0, ddir0)
    duv1, ddir1 = torch.full_like(uv, float("nan")), torch.full_like(d, float("nan"))
    g1 = torch.full((size,), 4.0, device="cuda")
    api.rt_zero_texture_grads(ctx, {a: g1})
    api.rt_shade_backward(ctx, uv, d, o, filt, gout, {a: g1}, duv1, ddir1, flags=api.RT_ACCUMULATE_TEXELS)
    torch.cuda.synchronize()
    assert torch.equal(duv1, duv0) and torch.equal(ddir1, ddir0)
    torch.testing.assert_close(g1, g0, rtol=1e-5, atol=1e-6)
    api.rt_shade_backward(ctx, uv, d, o, filt, gout, {a: g1}, duv1, ddir1, flags=api.RT_ACCUMULATE_TEXELS)
    torch.testing.assert_close(g1, 2 * g0, rtol=1e-5, atol=1e-6)  # no clear: the second call adds
    assert torch.equal(duv1, duv0) and torch.equal(ddir1, ddir0)  # overwritten, not summed
    api.rt_destroy_texture(ctx, b)
    with pytest.raises(api.RadtexError):
        api.rt_zero_texture_grads(ctx, {b: torch.zeros(size, device="cuda")})
    api.rt_destroy_texture(ctx, a)
