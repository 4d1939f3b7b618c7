"""GPU: the fused forward + L2 loss + backward step (rt_shade_batched_l2_step)
against the same three calls made one after the other (rt_shade_batched,
rt_l2_loss_grad, rt_shade_batched_backward) and against the oracle.

The fused kernel runs the very arithmetic of the three calls, so colours and
UV / direction gradients must agree bit for bit, texel gradients up to the
order of FP32 atomic additions (bit for bit in the deterministic mode), and the
loss sums up to the order of FP64 additions."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2301_01719_gb300 import api
from parity_util import COLOUR_TOL, ORACLE_FMT, floor_mismatch, to_dev

pytestmark = pytest.mark.gpu
FILTERS = (api.RT_NEAREST, api.RT_ANGULAR_BILINEAR, api.RT_QUADRILINEAR)


@pytest.fixture(scope="module")
def scene():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_01719_gb300 import build

    build.build()
    ctx = api.Context(0)
    W = H = 40
    n = 8
    texs, oids = [], []
    for k, fmt in enumerate((api.RT_F16, api.RT_F32)):
        atlas = oracle.fill_field(W, H, n, synth.field_lobes(800 + k))
        oids.append(api.rt_create_texture(ctx, W, H, n, fmt, api.RT_LAYOUT_ATLAS, to_dev(atlas)))
        texs.append(oracle.Texture.from_f32(atlas, W, H, n, ORACLE_FMT[fmt]))
    yield ctx, oids, texs, (W, H, n)
    ctx.close()


def frames(views, height, width, oids, seed=1002):
    g = synth.sphere_plane_scene(seed, views=views, width=width, height=height)
    obj = np.where(g.obj >= 0, np.array(oids, np.int32)[np.maximum(g.obj, 0)], -1).astype(np.int32)
    return (g, obj, to_dev(g.uv).reshape(views, height, width, 2), to_dev(g.dir).reshape(views, height, width, 3),
            to_dev(obj).reshape(views, height, width))


def unfused(ctx, uv, d, o, filt, target, scale, dt, flags):
    out = api.rt_shade_batched(ctx, uv, d, o, filt)
    g = torch.empty_like(out)
    sums = torch.zeros(2, dtype=torch.float64, device=out.device)
    api.rt_l2_loss_grad(out, target, o, scale, g, sums)
    duv, ddir = torch.zeros_like(uv), torch.zeros_like(d)  # RT_ACCUMULATE adds to them
    api.rt_shade_batched_backward(ctx, uv, d, o, filt, g, dt, duv, ddir, flags)
    return out, sums, duv, ddir


@pytest.mark.parametrize("filt", FILTERS)
@pytest.mark.parametrize("shape", [(3, 72, 96), (2, 37, 61)])
def test_fused_equals_the_three_calls(scene, filt, shape):
    ctx, oids, texs, (W, H, n) = scene
    V, Hh, Ww = shape
    g, obj, uv, d, o = frames(V, Hh, Ww, oids)
    rng = np.random.default_rng(3)
    target = to_dev(rng.uniform(0, 1, (V, Hh, Ww, 4)).astype(np.float32))
    scale = 0.75
    for t in ((8, 4, 2, 2), (32, 1, 4, 1)):
        api.rt_set_tile(ctx, filt, *t)
        dt_a = {k: torch.zeros((n, n, H, W, 4), device=uv.device) for k in oids}
        out_a, sums_a, duv_a, ddir_a = unfused(ctx, uv, d, o, filt, target, scale, dt_a, api.RT_ACCUMULATE)
        dt_b = {k: torch.zeros((n, n, H, W, 4), device=uv.device) for k in oids}
        out_b = torch.empty_like(out_a)
        sums_b = torch.zeros(2, dtype=torch.float64, device=uv.device)
        duv_b, ddir_b = torch.zeros_like(uv), torch.zeros_like(d)
        api.rt_shade_batched_l2_step(ctx, uv, d, o, filt, target, scale, out_b, sums_b, dt_b, duv_b, ddir_b,
                                     api.RT_ACCUMULATE)
        assert api.rt_get_error(ctx) == api.RT_OK
        assert torch.equal(out_a, out_b)
        assert torch.equal(duv_a, duv_b) and torch.equal(ddir_a, ddir_b)
        for k in oids:
            scale_k = dt_a[k].abs().max().item()
            assert (dt_a[k] - dt_b[k]).abs().max().item() <= 1e-5 * max(scale_k, 1.0)
        assert sums_a[1].item() == sums_b[1].item()
        assert abs(sums_a[0].item() - sums_b[0].item()) <= 1e-12 * abs(sums_a[0].item())
    # against the oracle: colours and the loss, outside the FP32 floor band of the nearest axes
    ref, _ = oracle.shade(texs, g.uv, g.dir, obj, filt)
    ok = ~floor_mismatch(ctx, g, obj, filt, texs)
    got = out_b.reshape(-1, 4).cpu().numpy()
    assert np.abs(got - ref)[ok].max() <= COLOUR_TOL
    tv = target.reshape(-1, 4).cpu().numpy().astype(np.float64)
    shaded = obj >= 0
    ref_se = ((np.where(ok[:, None], ref, got) - tv) ** 2)[shaded].sum()
    assert abs(sums_b[0].item() - ref_se) <= 1e-5 * shaded.sum()
    assert sums_b[1].item() == shaded.sum()


def test_fused_deterministic_is_bitwise_the_unfused(scene):
    ctx, oids, _, (W, H, n) = scene
    api.rt_prepare_deterministic(ctx)
    g, obj, uv, d, o = frames(2, 64, 80, oids, seed=1003)
    target = torch.full((2, 64, 80, 4), 0.25, device=uv.device)
    flags = api.RT_DETERMINISTIC
    dt_a = {k: torch.empty((n, n, H, W, 4), device=uv.device) for k in oids}
    unfused(ctx, uv, d, o, api.RT_QUADRILINEAR, target, 1.0, dt_a, flags)
    dt_b = {k: torch.empty((n, n, H, W, 4), device=uv.device) for k in oids}
    api.rt_shade_batched_l2_step(ctx, uv, d, o, api.RT_QUADRILINEAR, target, 1.0, None, None, dt_b, None, None, flags)
    for k in oids:
        assert torch.equal(dt_a[k], dt_b[k])
    assert api.rt_get_error(ctx) == api.RT_OK


def test_fused_arguments_and_edge_cases(scene):
    ctx, oids, _, (W, H, n) = scene
    g, obj, uv, d, o = frames(1, 16, 24, oids)
    target = torch.zeros((1, 16, 24, 4), device=uv.device)
    with pytest.raises(api.RadtexError) as e:  # target required
        api._lib.call("rt_shade_batched_l2_step", ctx.handle, api._ptr(uv), api._ptr(d), api._ptr(o), 1, 16, 24,
                      api.RT_QUADRILINEAR, None, 1.0, None, None, None, 0, None, None, 0, None)
    assert e.value.status == api.RT_ERR_INVALID_ARG
    with pytest.raises(api.RadtexError) as e:  # non-finite scale
        api.rt_shade_batched_l2_step(ctx, uv, d, o, api.RT_QUADRILINEAR, target, float("inf"))
    assert e.value.status == api.RT_ERR_INVALID_ARG
    # nothing requested but the loss
    sums = torch.zeros(2, dtype=torch.float64, device=uv.device)
    api.rt_shade_batched_l2_step(ctx, uv, d, o, api.RT_QUADRILINEAR, target, 1.0, None, sums)
    out = api.rt_shade_batched(ctx, uv, d, o, api.RT_QUADRILINEAR)
    shaded = (o >= 0).unsqueeze(-1)
    assert abs(sums[0].item() - (out.double() ** 2 * shaded).sum().item()) <= 1e-9 * max(sums[0].item(), 1.0)
    # empty batches are no-ops
    e3 = torch.empty((0, 4, 4, 3), device=uv.device)
    api.rt_shade_batched_l2_step(ctx, torch.empty((0, 4, 4, 2), device=uv.device), e3,
                                 torch.empty((0, 4, 4), dtype=torch.int32, device=uv.device), api.RT_QUADRILINEAR,
                                 torch.empty((0, 4, 4, 4), device=uv.device))
    # an unknown object id: zero colour, counted in the loss like rt_l2_loss_grad, status raised
    bad = o.clone()
    bad[0, 0, 0] = 999
    api.rt_shade_batched_l2_step(ctx, uv, d, bad, api.RT_QUADRILINEAR, target, 1.0, torch.empty_like(target))
    assert api.rt_get_error(ctx) == api.RT_ERR_BAD_OBJ_ID
    assert api.rt_get_error(ctx) == api.RT_OK


@pytest.mark.parametrize("fmt", [api.RT_F16, api.RT_BF16, api.RT_E4M3_BUCKET_SCALE, api.RT_F32])
@pytest.mark.parametrize("filt", FILTERS)
def test_fused_single_format_kernels(fmt, filt):
    """A context whose objects share one format runs that format's own kernel
    instantiation (the benchmark's case); it must match the three calls too."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_01719_gb300 import build

    build.build()
    ctx = api.Context(0)
    W = H = 32
    n = 6
    atlas = oracle.fill_field(W, H, n, synth.field_lobes(810))
    oids = [api.rt_create_texture(ctx, W, H, n, fmt, api.RT_LAYOUT_ATLAS, to_dev(atlas)) for _ in range(2)]
    g, obj, uv, d, o = frames(2, 45, 70, oids, seed=1004)
    target = to_dev(np.random.default_rng(4).uniform(0, 1, (2, 45, 70, 4)).astype(np.float32))
    dt_a = {k: torch.zeros((n, n, H, W, 4), device=uv.device) for k in oids}
    out_a, sums_a, duv_a, ddir_a = unfused(ctx, uv, d, o, filt, target, 0.5, dt_a, api.RT_ACCUMULATE)
    dt_b = {k: torch.zeros((n, n, H, W, 4), device=uv.device) for k in oids}
    out_b = torch.empty_like(out_a)
    sums_b = torch.zeros(2, dtype=torch.float64, device=uv.device)
    duv_b, ddir_b = torch.zeros_like(uv), torch.zeros_like(d)
    api.rt_shade_batched_l2_step(ctx, uv, d, o, filt, target, 0.5, out_b, sums_b, dt_b, duv_b, ddir_b,
                                 api.RT_ACCUMULATE)
    assert api.rt_get_error(ctx) == api.RT_OK
    assert torch.equal(out_a, out_b)
    assert torch.equal(duv_a, duv_b) and torch.equal(ddir_a, ddir_b)
    for k in oids:
        assert (dt_a[k] - dt_b[k]).abs().max().item() <= 1e-5 * max(dt_a[k].abs().max().item(), 1.0)
    assert sums_a[1].item() == sums_b[1].item()
    assert abs(sums_a[0].item() - sums_b[0].item()) <= 1e-12 * abs(sums_a[0].item())
    ctx.close()


def test_fused_palette_and_bits(scene):
    """A palette texture (texel gradients per palette bucket) and a 1-bit texture
    (no texel gradient; colours and coordinate gradients only) through the fused
    step, against the three calls."""
    ctx, _, _, _ = scene
    from test_gpu_palette import palette_case

    K, n, W, H = 9, 6, 30, 22
    pal_atlas, index = palette_case(K, n, W, H, seed=61)
    pid = api.rt_create_palette_texture(ctx, W, H, n, K, api.RT_F16, api.RT_LAYOUT_ATLAS, to_dev(pal_atlas),
                                        to_dev(index.view(np.int32)))
    rng = np.random.default_rng(62)
    bid = api.rt_create_texture(ctx, W, H, n, api.RT_BIT1, api.RT_LAYOUT_ATLAS,
                                to_dev(rng.uniform(0, 1, (H * n, W * n, 4)).astype(np.float32)))
    g, obj, uv, d, o = frames(2, 40, 56, [pid, bid], seed=1005)
    target = to_dev(rng.uniform(0, 1, (2, 40, 56, 4)).astype(np.float32))
    dt_a = {pid: torch.zeros((n, n, K, 4), device=uv.device)}
    out_a, sums_a, duv_a, ddir_a = unfused(ctx, uv, d, o, api.RT_QUADRILINEAR, target, 1.0, dt_a, api.RT_ACCUMULATE)
    dt_b = {pid: torch.zeros((n, n, K, 4), device=uv.device)}
    out_b = torch.empty_like(out_a)
    duv_b, ddir_b = torch.zeros_like(uv), torch.zeros_like(d)
    api.rt_shade_batched_l2_step(ctx, uv, d, o, api.RT_QUADRILINEAR, target, 1.0, out_b, None, dt_b, duv_b, ddir_b,
                                 api.RT_ACCUMULATE)
    assert api.rt_get_error(ctx) == api.RT_OK
    assert torch.equal(out_a, out_b)
    assert torch.equal(duv_a, duv_b) and torch.equal(ddir_a, ddir_b)
    assert (dt_a[pid] - dt_b[pid]).abs().max().item() <= 1e-5 * max(dt_a[pid].abs().max().item(), 1.0)
    # a texel gradient for the bit texture is refused, as by the backward
    with pytest.raises(api.RadtexError) as e:
        api.rt_shade_batched_l2_step(ctx, uv, d, o, api.RT_QUADRILINEAR, target, 1.0, None, None,
                                     {bid: torch.zeros((n, n, H, W, 4), device=uv.device)})
    assert e.value.status == api.RT_ERR_UNSUPPORTED
    api.rt_destroy_texture(ctx, pid)
    api.rt_destroy_texture(ctx, bid)
