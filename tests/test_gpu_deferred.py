"""GPU: rt_bake_deferred against the oracle's deferred payload (Section 1:
deferred ambient occlusion and reflections; reading R15).

The tolerance rule is the radiance bake's (test_gpu_bake.check): FP32 against
FP64, with the oracle's range [lo, hi] over perturbed rays.  For the payload
that range also spans every AO direction whose test flips when the hit point
moves or the direction tilts by 2^-17 (a direction grazing an occluder), and
the other basis choice when a sphere hit's normal has z within 2^-16 of zero.
A texel whose range exceeds 1e-3, or half an AO step 1/(2K), is a band texel:
it must lie inside its range.  Band texels stay under 5 %: more than the
radiance bake's 2 %, because the unlit albedo of a far, grazing hit on the
plane's pattern is not damped by fog and changes fast along the ray."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2301_01719_gb300 import api
from test_gpu_bake import DELTA, JUMP, SURFACES, check, decode

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_01719_gb300 import build

    build.build()
    c = api.Context(0)
    yield c
    c.close()


def check_deferred(gpu, val, lo, hi, fmt, K, scale=None, scene=None):
    """The bake's check with the payload's AO step; with the scene, also counts
    (prints, and bounds below 1 %) the texels whose albedo range is the plane
    pattern's whole range [albedo / 2, albedo] -- the far, grazing plane hits
    that FP32 cannot place on the pattern (reading R15's widened range)."""
    frac = check(gpu, val, lo, hi, fmt, scale, jump=min(JUMP, 0.5 / K), band_max=0.05)
    if scene is not None:
        alb = np.asarray(scene["plane_albedo"])
        widened = ((lo[..., :3] <= 0.5 * alb + 1e-12) & (hi[..., :3] >= alb - 1e-12)).all(axis=-1)
        print(f"deferred: {int(widened.sum())} of {widened.size} texels take the widened grazing-plane range "
              f"({widened.mean():.4%}); band texels {frac:.4%}")
        assert widened.mean() < 0.01, widened.mean()
    return frac


def dev_dirs(K, seed):
    d = synth.ao_directions(seed, K)
    return d, torch.from_numpy(d).to(torch.device("cuda", 0))


@pytest.mark.parametrize("surface", [api.RT_SURFACE_SPHERE, api.RT_SURFACE_PLANE])
@pytest.mark.parametrize("fmt", [api.RT_F32, api.RT_F16, api.RT_BF16, api.RT_E4M3_BUCKET_SCALE])
@pytest.mark.parametrize("shape,K", [((24, 24, 8), 16), ((37, 13, 5), 7)])
def test_deferred_matches_oracle(ctx, surface, fmt, shape, K):
    W, H, n = shape
    scene = synth.bake_scene(51)
    dirs, ddirs = dev_dirs(K, 52)
    oid = api.rt_create_texture(ctx, W, H, n, fmt)
    api.rt_bake_deferred(ctx, oid, surface, scene, ddirs)
    codes, scales = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_ATLAS)
    gpu, s = decode(fmt, codes, scales, n)
    val, lo, hi = oracle.bake_deferred(W, H, n, SURFACES[surface], scene, dirs, DELTA)
    check_deferred(gpu, val, lo, hi, fmt, K, s, scene)
    # both payload kinds occur: sky texels and hits with partial occlusion
    sky = (val == [0, 0, 0, 1]).all(axis=-1)
    assert 0 < sky.mean() < 1 and (val[..., 3] < 1).any()
    assert api.rt_get_error(ctx) == api.RT_OK
    api.rt_destroy_texture(ctx, oid)


def test_deferred_single_direction_and_lifted_scene(ctx):
    """K = 1 along the hit normal, and a scene whose plane lies two radii below
    the sphere: the occlusion is a 0/1 visibility bit along the normal."""
    W, H, n = 20, 20, 6
    scene = synth.bake_scene(53, plane_height=-3.0)
    dirs = np.array([[0.0, 0.0, 1.0]], np.float32)
    for surface in (api.RT_SURFACE_SPHERE, api.RT_SURFACE_PLANE):
        oid = api.rt_create_texture(ctx, W, H, n, api.RT_F32)
        api.rt_bake_deferred(ctx, oid, surface, scene, torch.from_numpy(dirs).cuda())
        gpu = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_ATLAS)[0].cpu().numpy().astype(np.float64)
        val, lo, hi = oracle.bake_deferred(W, H, n, SURFACES[surface], scene, dirs, DELTA)
        check_deferred(gpu, val, lo, hi, api.RT_F32, 1)
        assert set(np.unique(gpu[..., 3])) <= {0.0, 1.0}
        api.rt_destroy_texture(ctx, oid)


def test_deferred_into_borrowed_planes(ctx):
    W, H, n, K = 19, 11, 6, 12
    scene = synth.bake_scene(54)
    dirs, ddirs = dev_dirs(K, 55)
    buf = torch.full((n, n, H, W, 4), -7.0, device="cuda")
    oid = api.rt_create_texture(ctx, W, H, n, api.RT_F32, api.RT_LAYOUT_PLANES, buf, api.RT_BORROW)
    api.rt_bake_deferred(ctx, oid, api.RT_SURFACE_SPHERE, scene, ddirs)
    got = buf.cpu().numpy().astype(np.float64).transpose(2, 0, 3, 1, 4).reshape(H * n, W * n, 4)
    val, lo, hi = oracle.bake_deferred(W, H, n, oracle.SURFACE_SPHERE, scene, dirs, DELTA)
    check_deferred(got, val, lo, hi, api.RT_F32, K)
    api.rt_destroy_texture(ctx, oid)


def test_deferred_rejects_bad_arguments(ctx):
    scene = synth.bake_scene(56)
    _, ddirs = dev_dirs(8, 57)
    oid = api.rt_create_texture(ctx, 4, 4, 4, api.RT_F16)
    for bad_dirs in (ddirs[:0], torch.zeros((api.RT_MAX_AO_DIRECTIONS + 1, 3), device="cuda")):
        with pytest.raises(api.RadtexError) as e:
            api.rt_bake_deferred(ctx, oid, api.RT_SURFACE_PLANE, scene, bad_dirs)
        assert e.value.status == api.RT_ERR_INVALID_ARG
    with pytest.raises(api.RadtexError) as e:
        api.rt_bake_deferred(ctx, oid, api.RT_SURFACE_PLANE, dict(scene, fog=-1.0), ddirs)
    assert e.value.status == api.RT_ERR_INVALID_ARG
    with pytest.raises(api.RadtexError):
        api.rt_bake_deferred(ctx, oid, 7, scene, ddirs)
    bits = api.rt_create_texture(ctx, 4, 4, 4, api.RT_BIT1)
    with pytest.raises(api.RadtexError) as e:
        api.rt_bake_deferred(ctx, bits, api.RT_SURFACE_PLANE, scene, ddirs)
    assert e.value.status == api.RT_ERR_UNSUPPORTED
    # the most directions the call takes (their table staged in shared memory next to n^2 vectors)
    big = torch.from_numpy(synth.ao_directions(58, api.RT_MAX_AO_DIRECTIONS)).cuda()
    api.rt_bake_deferred(ctx, oid, api.RT_SURFACE_SPHERE, scene, big)
    assert api.rt_get_error(ctx) == api.RT_OK
    api.rt_destroy_texture(ctx, oid)
    api.rt_destroy_texture(ctx, bits)


def test_deferred_max_n_and_directions(ctx):
    """n = 64 (48 KiB of reflection vectors) with 1024 directions: 64 KiB of
    shared memory, above the default per-block limit."""
    W, H, n = 3, 2, 64
    scene = synth.bake_scene(59)
    dirs, ddirs = dev_dirs(api.RT_MAX_AO_DIRECTIONS, 60)
    oid = api.rt_create_texture(ctx, W, H, n, api.RT_F32)
    api.rt_bake_deferred(ctx, oid, api.RT_SURFACE_PLANE, scene, ddirs)
    gpu = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_ATLAS)[0].cpu().numpy().astype(np.float64)
    val, lo, hi = oracle.bake_deferred(W, H, n, oracle.SURFACE_PLANE, scene, dirs, DELTA)
    check_deferred(gpu, val, lo, hi, api.RT_F32, api.RT_MAX_AO_DIRECTIONS)
    api.rt_destroy_texture(ctx, oid)


@pytest.mark.parametrize("surface", [api.RT_SURFACE_SPHERE, api.RT_SURFACE_PLANE])
def test_deferred_full_size_sampled(ctx, surface):
    """The 1024^2 x 16^2 FP16 texture with 32 directions, as the benchmark's
    deferred bake runs it; 20000 sampled texels against the oracle."""
    W = H = 1024
    n, K = 16, 32
    scene = synth.bake_scene(2001)
    dirs, ddirs = dev_dirs(K, 4242)
    oid = api.rt_create_texture(ctx, W, H, n, api.RT_F16)
    api.rt_bake_deferred(ctx, oid, surface, scene, ddirs)
    codes, _ = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_PLANES)
    api.rt_destroy_texture(ctx, oid)
    rng = np.random.default_rng(61)
    S = 20000
    q = np.stack([rng.integers(0, W, S), rng.integers(0, H, S), rng.integers(0, n, S), rng.integers(0, n, S)], 1)
    qt = torch.from_numpy(q).to(codes.device)
    got = codes[qt[:, 3], qt[:, 2], qt[:, 1], qt[:, 0]].cpu().numpy()
    del codes
    gpu = oracle.decode(oracle.F16, got.view(np.uint16))
    val, lo, hi = oracle.bake_deferred_texels(W, H, n, SURFACES[surface], scene, dirs, q, DELTA)
    check_deferred(gpu, val, lo, hi, api.RT_F16, K, scene=scene)
