"""GPU: 1-bit shadow textures (Section 5, "Shadowing"; reading R13) against the
oracle.

- The shadow bake must reproduce the oracle's visibility bits.  Only texels
  whose bit flips under the oracle's perturbed rays, where the ray grazes an
  occluder and either bit is correct, may differ, and those stay rare.
- Bits encoded from FP32 are bit-exact.
- Filtered bits and averaged multi-sample lookups (area shadows) agree with
  the oracle within 1e-5, outside the FP32 floor band."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2301_01719_gb300 import api
from parity_util import COLOUR_TOL, FILTERS, floor_mismatch, gbuffer_to_dev, to_dev

pytestmark = pytest.mark.gpu
SURFACES = {api.RT_SURFACE_SPHERE: oracle.SURFACE_SPHERE, api.RT_SURFACE_PLANE: oracle.SURFACE_PLANE}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_01719_gb300 import build

    build.build()
    c = api.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("surface", [api.RT_SURFACE_SPHERE, api.RT_SURFACE_PLANE])
@pytest.mark.parametrize("shape", [(37, 13, 5), (24, 24, 8)])
def test_shadow_bake_matches_oracle(ctx, surface, shape):
    W, H, n = shape  # 37 x 13 = 481 bits per plane: 32-bit words straddle planes
    scene = synth.bake_scene(41)
    oid = api.rt_create_texture(ctx, W, H, n, api.RT_BIT1)
    assert api.rt_texture_info(ctx, oid)["bytes"] == (W * H * n * n + 31) // 32 * 4
    api.rt_bake_shadow(ctx, oid, surface, scene)
    bits, _ = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_ATLAS)
    got = bits.cpu().numpy()
    vis, band = oracle.bake_shadow(W, H, n, SURFACES[surface], scene)
    assert got.shape == vis.shape
    np.testing.assert_array_equal(got[~band], vis[~band])
    assert band.mean() < 0.02
    assert 0 < vis.mean() < 1
    assert api.rt_get_error(ctx) == api.RT_OK
    api.rt_destroy_texture(ctx, oid)


def test_bits_from_fp32_and_filtering(ctx):
    W, H, n = 29, 17, 6
    rng = np.random.default_rng(3)
    src = rng.uniform(0, 1, (H * n, W * n, 4)).astype(np.float32)
    oid = api.rt_create_texture(ctx, W, H, n, api.RT_BIT1, api.RT_LAYOUT_ATLAS, to_dev(src))
    bits = (src[..., 0] >= 0.5).astype(np.uint8)
    got, _ = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_ATLAS)
    np.testing.assert_array_equal(got.cpu().numpy(), bits)
    T = oracle.bit_texture(bits, W, H, n)
    g = synth.quad_scene(1021, 160, 128)
    obj = np.where(g.obj >= 0, oid, -1).astype(np.int32)
    table = [None] * oid + [T]
    uv, d, _ = gbuffer_to_dev(g)
    for filt in FILTERS:
        out = api.rt_shade(ctx, uv, d, to_dev(obj), filt).cpu().numpy()
        ref, _ = oracle.shade(table, g.uv, g.dir, obj, filt)
        ok = ~floor_mismatch(ctx, g, obj, filt, table)
        assert np.abs(out - ref)[ok].max() <= COLOUR_TOL
        assert (out[:, 0] == out[:, 3]).all()
    # bits carry no texel gradient; coordinate gradients are available
    gout = to_dev(rng.normal(size=(g.F, 4)).astype(np.float32))
    with pytest.raises(api.RadtexError) as e:
        api.rt_shade_backward(ctx, uv, d, to_dev(obj), api.RT_QUADRILINEAR, gout,
                              {oid: torch.empty((n, n, H, W, 4), device=uv.device)})
    assert e.value.status == api.RT_ERR_UNSUPPORTED
    duv = torch.empty_like(uv)
    api.rt_shade_backward(ctx, uv, d, to_dev(obj), api.RT_QUADRILINEAR, gout, None, duv, None)
    assert api.rt_get_error(ctx) == api.RT_OK
    api.rt_destroy_texture(ctx, oid)


def jittered(d, S, spread, seed):
    """S unit directions per fragment around d (a cone of half-angle ~spread)."""
    rng = np.random.default_rng(seed)
    out = d[:, None, :] + rng.normal(scale=spread, size=(d.shape[0], S, 3))
    out[..., 2] = np.abs(out[..., 2])
    return (out / np.linalg.norm(out, axis=2, keepdims=True)).astype(np.float32)


def test_area_shadow_multi_sample(ctx):
    W, H, n, S = 32, 24, 8, 6
    scene = synth.bake_scene(42)
    oid = api.rt_create_texture(ctx, W, H, n, api.RT_BIT1)
    api.rt_bake_shadow(ctx, oid, api.RT_SURFACE_PLANE, scene)
    bits, _ = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_ATLAS)
    T = oracle.bit_texture(bits.cpu().numpy(), W, H, n)
    g = synth.quad_scene(1022, 96, 80)
    obj = np.where(g.obj >= 0, oid, -1).astype(np.int32)
    L = jittered(g.dir, S, 0.1, 5)  # F x S x 3 light samples
    uv, _, _ = gbuffer_to_dev(g)
    for filt in FILTERS:
        out = api.rt_shade_multi(ctx, uv, to_dev(L), to_dev(obj), filt).cpu().numpy()
        # oracle: the mean of S single lookups; fragments with a sample in the floor band are skipped
        uvS = np.repeat(g.uv, S, axis=0)
        objS = np.repeat(obj, S)
        refS, _ = oracle.shade([None] * oid + [T], uvS, L.reshape(-1, 3), objS, filt)
        ref = refS.reshape(-1, S, 4).mean(axis=1)
        gS = synth.GBuffer(uv=uvS, dir=L.reshape(-1, 3), obj=objS, width=0, height=0, views=1)
        mism = floor_mismatch(ctx, gS, objS, filt, [None] * oid + [T]).reshape(-1, S).any(axis=1)
        assert (~mism).mean() > 0.95
        assert np.abs(out - ref)[~mism].max() <= COLOUR_TOL
    assert api.rt_get_error(ctx) == api.RT_OK
    api.rt_destroy_texture(ctx, oid)


@pytest.mark.parametrize("surface", [api.RT_SURFACE_SPHERE, api.RT_SURFACE_PLANE])
def test_shadow_bake_full_size_sampled(ctx, surface):
    """The 1024^2 x 16^2 shadow texture (32 MiB of bits), 20000 sampled texels."""
    W = H = 1024
    n = 16
    scene = synth.bake_scene(2001)
    oid = api.rt_create_texture(ctx, W, H, n, api.RT_BIT1)
    api.rt_bake_shadow(ctx, oid, surface, scene)
    bits, _ = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_PLANES)  # (n, n, H, W) uint8
    api.rt_destroy_texture(ctx, oid)
    rng = np.random.default_rng(12)
    K = 20000
    q = np.stack([rng.integers(0, W, K), rng.integers(0, H, K), rng.integers(0, n, K), rng.integers(0, n, K)], 1)
    qt = torch.from_numpy(q).to(bits.device)
    got = bits.reshape(n, n, H, W)[qt[:, 3], qt[:, 2], qt[:, 1], qt[:, 0]].cpu().numpy()
    vis, band = oracle.bake_shadow_texels(W, H, n, SURFACES[surface], scene, q)
    np.testing.assert_array_equal(got[~band], vis[~band])
    assert band.mean() < 0.02
