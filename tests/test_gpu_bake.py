"""GPU: rt_bake against the oracle's bake (Section 2.2, Eq. 4a, Eq. 4b; reading R10).

Tolerance per texel.  The kernel computes in FP32, so its inputs to every hit
decision and every smooth function are one rounding chain (~1e-6) away from
the oracle's.  The oracle therefore also returns the range [lo, hi] of each
texel over rays perturbed by delta = 2^-17 (origin along T, B; direction
along T, B, N).  With spread M = max(hi - val, val - lo), each texel must lie
within 1e-5 + M/4 of the exact value, plus the storage format's rounding
bound.  Where M > 1e-3 the ray grazes a hit decision (a silhouette or the
ray offset), so either side is correct; there the texel must lie inside
[lo, hi] widened by the same bounds, and such texels must stay rare (< 2%)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2301_01719_gb300 import api
from parity_util import storage_to_atlas

pytestmark = pytest.mark.gpu

DELTA = 2.0 ** -17
TOL = 1e-5
JUMP = 1e-3
BAND_MAX = 0.02
ORACLE_FMT = {api.RT_F32: oracle.F32, api.RT_F16: oracle.F16, api.RT_BF16: oracle.BF16,
              api.RT_E4M3_BUCKET_SCALE: oracle.E4M3}
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


def quant_bound(fmt, val, scale):
    """Half an ulp of the storage format at |val| (P-quant bounds)."""
    a = np.abs(val)
    if fmt == api.RT_F32:
        return np.zeros_like(a)
    if fmt == api.RT_F16:
        return 2.0 ** -11 * a + 2.0 ** -25
    if fmt == api.RT_BF16:
        return 2.0 ** -8 * a
    return 2.0 ** -4 * a + 2.0 ** -10 * scale


def decode(fmt, codes, scales, n):
    """Atlas-layout codes read back from the device -> FP64 values."""
    codes = codes.cpu().numpy()
    if fmt == api.RT_F32:
        return codes.astype(np.float64), None
    if fmt in (api.RT_F16, api.RT_BF16):
        return oracle.decode(ORACLE_FMT[fmt], codes.view(np.uint16)), None
    s = np.repeat(np.repeat(scales.cpu().numpy().astype(np.float64), n, 0), n, 1)[..., None]
    return oracle.decode(oracle.E4M3, codes) * s, s


def check(gpu, val, lo, hi, fmt, scale=None, jump=JUMP, band_max=BAND_MAX):
    """Returns the fraction of band texels; asserts the per-texel bounds."""
    if scale is None:
        scale = np.zeros_like(val)
    M = np.maximum(hi - val, val - lo).max(axis=-1, keepdims=True)
    band = (M > jump)[..., 0]
    q = quant_bound(fmt, np.maximum(np.abs(lo), np.abs(hi)), scale)
    tol = TOL + M / 4 + q * (1 + TOL)
    err = np.abs(gpu - val)
    smooth = ~band
    bad = smooth[..., None] & (err > tol)
    assert not bad.any(), (f"{bad.sum()} texels off; worst excess {(err - tol)[bad].max():.3e}, "
                           f"at {np.argwhere(bad)[:3].tolist()}")
    widened = TOL + q
    inside = (gpu >= lo - widened) & (gpu <= hi + widened)
    assert inside[band].all(), f"{(~inside[band]).sum()} band texels outside their perturbed range"
    assert band.mean() < band_max, band.mean()
    return float(band.mean())


@pytest.mark.parametrize("surface", [api.RT_SURFACE_SPHERE, api.RT_SURFACE_PLANE])
@pytest.mark.parametrize("fmt", [api.RT_F32, api.RT_F16, api.RT_BF16, api.RT_E4M3_BUCKET_SCALE])
@pytest.mark.parametrize("shape", [(24, 24, 8), (37, 13, 5)])
def test_bake_matches_oracle(ctx, surface, fmt, shape):
    W, H, n = shape
    scene = synth.bake_scene(31)
    oid = api.rt_create_texture(ctx, W, H, n, fmt)
    api.rt_bake(ctx, oid, surface, scene)
    codes, scales = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_ATLAS)
    gpu, s = decode(fmt, codes, scales, n)
    val, lo, hi = oracle.bake(W, H, n, SURFACES[surface], scene, DELTA)
    check(gpu, val, lo, hi, fmt, s)
    if fmt == api.RT_E4M3_BUCKET_SCALE:
        # the scale is the bucket's amax / 448 (amax of the FP32 values)
        amax = np.abs(val).reshape(H, n, W, n, 4).max(axis=(1, 3, 4))
        M = np.maximum(hi - val, val - lo).reshape(H, n, W, n, 4).max(axis=(1, 3, 4))
        got = scales.cpu().numpy().astype(np.float64)
        assert (np.abs(got * 448 - amax) <= 2e-6 * amax + TOL + M).all()
    assert api.rt_get_error(ctx) == api.RT_OK
    api.rt_destroy_texture(ctx, oid)


@pytest.mark.parametrize("layout,W,H", [(api.RT_LAYOUT_ATLAS, 19, 11), (api.RT_LAYOUT_PLANES, 19, 11),
                                        (api.RT_LAYOUT_QUADS, 20, 12)])
def test_bake_into_borrowed_fp32(ctx, layout, W, H):
    n = 6
    scene = synth.bake_scene(32)
    dev = torch.device("cuda", 0)
    buf = torch.full(api.layout_shape(layout, W, H, n), -7.0, device=dev)
    oid = api.rt_create_texture(ctx, W, H, n, api.RT_F32, layout, buf, api.RT_BORROW)
    api.rt_bake(ctx, oid, api.RT_SURFACE_PLANE, scene)
    got = buf.cpu().numpy().astype(np.float64)
    if layout != api.RT_LAYOUT_ATLAS:
        got = storage_to_atlas(got, layout, W, H, n)
    val, lo, hi = oracle.bake(W, H, n, oracle.SURFACE_PLANE, scene, DELTA)
    check(got, val, lo, hi, api.RT_F32)
    api.rt_destroy_texture(ctx, oid)


def test_baked_texel_comes_back_at_its_centre(ctx):
    """Shading a fragment at a bucket centre whose direction is a texel's own
    Eq. 2c incidence (NEAREST) returns exactly that baked texel."""
    W, H, n = 16, 12, 8
    scene = synth.bake_scene(33)
    oid = api.rt_create_texture(ctx, W, H, n, api.RT_F32)
    api.rt_bake(ctx, oid, api.RT_SURFACE_SPHERE, scene)
    atlas = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_ATLAS)[0].cpu().numpy()
    dirs_ts = oracle.texel_directions(n)  # [t, s]
    rng = np.random.default_rng(5)
    q = np.stack([rng.integers(0, W, 500), rng.integers(0, H, 500), rng.integers(0, n, 500),
                  rng.integers(0, n, 500)], 1)
    uv = np.stack([(q[:, 0] + 0.5) / W, (q[:, 1] + 0.5) / H], 1).astype(np.float32)
    d = dirs_ts[q[:, 3], q[:, 2]].astype(np.float32)
    dev = torch.device("cuda", 0)
    out = api.rt_shade(ctx, torch.from_numpy(uv).to(dev), torch.from_numpy(d).to(dev),
                       torch.full((500,), oid, dtype=torch.int32, device=dev), api.RT_NEAREST).cpu().numpy()
    want = atlas[q[:, 1] * n + q[:, 3], q[:, 0] * n + q[:, 2]]
    np.testing.assert_array_equal(out, want)
    api.rt_destroy_texture(ctx, oid)


def test_bake_rejects_bad_arguments(ctx):
    scene = synth.bake_scene(34)
    oid = api.rt_create_texture(ctx, 4, 4, 4, api.RT_F16)
    for bad in (dict(scene, sphere_radius=0.0), dict(scene, fog=-1.0), dict(scene, ambient=float("nan")),
                dict(scene, plane_half_extent=0.0), dict(scene, sun_exponent=-2.0), dict(scene, ray_offset=-1.0)):
        with pytest.raises(api.RadtexError) as e:
            api.rt_bake(ctx, oid, api.RT_SURFACE_PLANE, bad)
        assert e.value.status == api.RT_ERR_INVALID_ARG
    with pytest.raises(api.RadtexError):
        api.rt_bake(ctx, oid, 7, scene)
    with pytest.raises(api.RadtexError):
        api.rt_bake(ctx, oid + 100, api.RT_SURFACE_PLANE, scene)
    assert api.rt_get_error(ctx) == api.RT_OK
    api.rt_destroy_texture(ctx, oid)


@pytest.mark.parametrize("surface", [api.RT_SURFACE_SPHERE, api.RT_SURFACE_PLANE])
def test_bake_full_size_sampled(ctx, surface):
    """The 1024^2-bucket x 16^2 FP16 texture of the sphere-plane workload, in the
    launch configuration the benchmark times; 20000 sampled texels against the
    oracle texel by texel."""
    W = H = 1024
    n = 16
    scene = synth.bake_scene(2001)
    oid = api.rt_create_texture(ctx, W, H, n, api.RT_F16)
    api.rt_bake(ctx, oid, surface, scene)
    codes, _ = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_PLANES)  # (n, n, H, W, 4)
    api.rt_destroy_texture(ctx, oid)
    rng = np.random.default_rng(6)
    K = 20000
    q = np.stack([rng.integers(0, W, K), rng.integers(0, H, K), rng.integers(0, n, K), rng.integers(0, n, K)], 1)
    qt = torch.from_numpy(q).to(codes.device)
    got = codes[qt[:, 3], qt[:, 2], qt[:, 1], qt[:, 0]].cpu().numpy()
    del codes
    gpu = oracle.decode(oracle.F16, got.view(np.uint16))
    val, lo, hi = oracle.bake_texels(W, H, n, SURFACES[surface], scene, q, DELTA)
    check(gpu, val, lo, hi, api.RT_F16)
