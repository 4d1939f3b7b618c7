"""GPU: the batched (screen-tiled) entry points against the flat ones and the oracle.

Every tile shape walks the same per-fragment arithmetic, so colours, UV and
direction gradients must be bit-identical to rt_shade / rt_shade_backward;
texel gradients differ only in the order of FP32 atomic additions."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2301_01719_gb300 import api
from parity_util import COLOUR_TOL, ORACLE_FMT, to_dev

pytestmark = pytest.mark.gpu

TILES = [(32, 1, 4, 1), (32, 1, 2, 2), (32, 1, 1, 4), (16, 2, 4, 1), (16, 2, 2, 2), (16, 2, 1, 4), (8, 4, 4, 1),
         (8, 4, 2, 2), (8, 4, 1, 4), (4, 8, 4, 1), (4, 8, 2, 2), (4, 8, 1, 4)]


@pytest.fixture(scope="module")
def scene():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_01719_gb300 import build

    build.build()
    ctx = api.Context(0)
    W = H = 48
    n = 8
    texs, oids = [], []
    for k, fmt in enumerate((api.RT_F16, api.RT_F32)):
        atlas = oracle.fill_field(W, H, n, synth.field_lobes(700 + k))
        oids.append(api.rt_create_texture(ctx, W, H, n, fmt, api.RT_LAYOUT_ATLAS, to_dev(atlas)))
        texs.append(oracle.Texture.from_f32(atlas, W, H, n, ORACLE_FMT[fmt]))
    yield ctx, oids, texs, (W, H, n)
    ctx.close()


def frames(views, height, width, oids):
    g = synth.sphere_plane_scene(1002, views=views, width=width, height=height)
    obj = np.where(g.obj >= 0, np.array(oids, np.int32)[np.maximum(g.obj, 0)], -1).astype(np.int32)
    uv = to_dev(g.uv).reshape(views, height, width, 2)
    d = to_dev(g.dir).reshape(views, height, width, 3)
    o = to_dev(obj).reshape(views, height, width)
    return g, obj, uv, d, o


@pytest.mark.parametrize("shape", [(3, 72, 96), (2, 50, 60), (1, 33, 201), (2, 1, 4), (1, 7, 3)])
def test_batched_equals_flat_every_tile(scene, shape):
    ctx, oids, texs, _ = scene
    V, Hh, Ww = shape
    g, obj, uv, d, o = frames(V, Hh, Ww, oids)
    for filt in (api.RT_NEAREST, api.RT_ANGULAR_BILINEAR, api.RT_QUADRILINEAR):
        flat = api.rt_shade(ctx, uv.reshape(-1, 2), d.reshape(-1, 3), o.reshape(-1), filt).cpu().numpy()
        for t in TILES:
            api.rt_set_tile(ctx, filt, *t)
            assert api.rt_get_tile(ctx, filt) == t
            out = api.rt_shade_batched(ctx, uv, d, o, filt).reshape(-1, 4).cpu().numpy()
            np.testing.assert_array_equal(out, flat, err_msg=f"tile {t} filter {filt}")
    assert api.rt_get_error(ctx) == api.RT_OK
    # against the oracle on the quadrilinear colours
    ref, _ = oracle.shade(texs, g.uv, g.dir, obj, oracle.QUADRILINEAR)
    assert np.abs(flat - ref).max() <= COLOUR_TOL


def test_batched_backward_equals_flat(scene):
    ctx, oids, texs, (W, H, n) = scene
    V, Hh, Ww = 2, 64, 80
    g, obj, uv, d, o = frames(V, Hh, Ww, oids)
    rng = np.random.default_rng(1)
    gout = to_dev(rng.normal(size=(V, Hh, Ww, 4)).astype(np.float32))
    filt = api.RT_QUADRILINEAR

    def run(batched):
        duv = torch.empty_like(uv)
        ddir = torch.empty_like(d)
        dt = {o_: torch.empty((n, n, H, W, 4), device=uv.device) for o_ in oids}
        if batched:
            api.rt_shade_batched_backward(ctx, uv, d, o, filt, gout, dt, duv, ddir)
        else:
            api.rt_shade_backward(ctx, uv.reshape(-1, 2), d.reshape(-1, 3), o.reshape(-1), filt, gout.reshape(-1, 4),
                                  dt, duv.reshape(-1, 2), ddir.reshape(-1, 3))
        return duv.cpu().numpy(), ddir.cpu().numpy(), {k: v.cpu().numpy() for k, v in dt.items()}

    a = run(False)
    for t, fwd_only in (((8, 4, 2, 2), False), ((32, 1, 4, 1), False), ((4, 8, 1, 4), False), ((16, 2, 1, 4), True)):
        if fwd_only:  # the backward's own tile; the forward keeps its tile
            api.rt_set_tile(ctx, filt, 8, 4, 2, 2)
            api.rt_set_backward_tile(ctx, filt, *t)
            assert api.rt_get_tile(ctx, filt) == (8, 4, 2, 2)
        else:
            api.rt_set_tile(ctx, filt, *t)
            assert api.rt_get_tile(ctx, filt) == t
        assert api.rt_get_backward_tile(ctx, filt) == t
        b = run(True)
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])
        for k in a[2]:
            scale = np.abs(a[2][k]).max()
            assert np.abs(a[2][k] - b[2][k]).max() <= 1e-5 * max(scale, 1.0)
    assert api.rt_get_error(ctx) == api.RT_OK


def test_autotune_and_invalid_tiles(scene):
    ctx, oids, _, _ = scene
    g, obj, uv, d, o = frames(2, 90, 128, oids)
    tile, ms = api.rt_autotune(ctx, uv, d, o, api.RT_QUADRILINEAR, reps=2)
    assert tile in TILES and ms > 0
    assert api.rt_get_tile(ctx, api.RT_QUADRILINEAR) == tile
    flat = api.rt_shade(ctx, uv.reshape(-1, 2), d.reshape(-1, 3), o.reshape(-1), api.RT_QUADRILINEAR)
    out = api.rt_shade_batched(ctx, uv, d, o, api.RT_QUADRILINEAR)
    assert torch.equal(out.reshape(-1, 4), flat)
    for bad in ((32, 2, 4, 1), (6, 5, 4, 1), (2, 16, 4, 1), (8, 4, 2, 1), (8, 4, 4, 4)):
        with pytest.raises(api.RadtexError):
            api.rt_set_tile(ctx, api.RT_QUADRILINEAR, *bad)
        with pytest.raises(api.RadtexError):
            api.rt_set_backward_tile(ctx, api.RT_QUADRILINEAR, *bad)
    # the backward's autotuner sets the backward tile only; every tile gives the same coordinate gradients
    W, H, n = scene[3]
    gout = torch.ones((*o.shape, 4), device=uv.device)
    dt = {o_: torch.zeros((n, n, H, W, 4), device=uv.device) for o_ in oids}
    duv, ddir = torch.empty_like(uv), torch.empty_like(d)
    api.rt_shade_batched_backward(ctx, uv, d, o, api.RT_QUADRILINEAR, gout, None, duv, ddir)
    before = api.rt_get_tile(ctx, api.RT_QUADRILINEAR)
    btile, bms = api.rt_autotune_backward(ctx, uv, d, o, api.RT_QUADRILINEAR, gout, dt, None, None,
                                          api.RT_ACCUMULATE, reps=2)
    assert btile in TILES and bms > 0
    assert api.rt_get_backward_tile(ctx, api.RT_QUADRILINEAR) == btile
    assert api.rt_get_tile(ctx, api.RT_QUADRILINEAR) == before
    duv2, ddir2 = torch.empty_like(uv), torch.empty_like(d)
    api.rt_shade_batched_backward(ctx, uv, d, o, api.RT_QUADRILINEAR, gout, None, duv2, ddir2)
    assert torch.equal(duv, duv2) and torch.equal(ddir, ddir2)
    # empty batches are no-ops
    e3 = torch.empty((0, 4, 4, 3), device=uv.device)
    api.rt_shade_batched(ctx, torch.empty((0, 4, 4, 2), device=uv.device), e3,
                         torch.empty((0, 4, 4), dtype=torch.int32, device=uv.device), api.RT_QUADRILINEAR)


def test_cuda_graph_capture_replays_identically(scene):
    """A step (forward, backward with zeroed texel gradients) captured in a CUDA graph
    replays to the same results as eager launches: the entry points neither allocate
    nor synchronise."""
    ctx, oids, _, (W, H, n) = scene
    g, obj, uv, d, o = frames(2, 72, 96, oids)
    filt = api.RT_QUADRILINEAR
    out = torch.empty((2, 72, 96, 4), device=uv.device)
    duv = torch.empty_like(uv)
    ddir = torch.empty_like(d)
    dt = {k: torch.empty((n, n, H, W, 4), device=uv.device) for k in oids}

    def step(stream=None):
        api.rt_shade_batched(ctx, uv, d, o, filt, out, stream=stream)
        api.rt_shade_batched_backward(ctx, uv, d, o, filt, out, dt, duv, ddir, 0, stream=stream)

    step()
    torch.cuda.synchronize()
    eager = [out.clone(), duv.clone(), ddir.clone()]
    eager_dt = {k: v.clone() for k, v in dt.items()}
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            step(s)
    for t in (out, duv, ddir, *dt.values()):
        t.zero_()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    for a_, b_ in zip(eager, (out, duv, ddir)):
        assert torch.equal(a_, b_)
    for k in dt:
        assert torch.allclose(eager_dt[k], dt[k], rtol=1e-5, atol=1e-6)
    assert api.rt_get_error(ctx) == api.RT_OK


def bumpy(V, Hh, Ww, seed):
    rng = np.random.default_rng(seed)
    N = np.concatenate([rng.normal(scale=0.3, size=(V * Hh * Ww, 2)), np.ones((V * Hh * Ww, 1))], 1)
    return to_dev((N / np.linalg.norm(N, axis=1, keepdims=True)).astype(np.float32)).reshape(V, Hh, Ww, 3)


@pytest.mark.parametrize("shape", [(2, 50, 60), (1, 33, 201), (1, 7, 3)])
def test_world_batched_equals_flat(scene, shape):
    """rt_shade_world_batched / rt_shade_world_batched_backward against the flat
    world-space calls: colours and UV, direction and normal gradients bit for
    bit for every tile shape, texel gradients up to the order of atomic
    additions (bit for bit in the deterministic mode)."""
    ctx, oids, texs, (W, H, n) = scene
    V, Hh, Ww = shape
    g, obj, uv, d, o = frames(V, Hh, Ww, oids)
    N = bumpy(V, Hh, Ww, 3)
    flat_args = (uv.reshape(-1, 2), d.reshape(-1, 3), N.reshape(-1, 3), o.reshape(-1))
    for filt in (api.RT_NEAREST, api.RT_ANGULAR_BILINEAR, api.RT_QUADRILINEAR):
        flat = api.rt_shade_world(ctx, *flat_args, filt).cpu().numpy()
        for t in TILES[::3]:
            api.rt_set_tile(ctx, filt, *t)
            out = api.rt_shade_world_batched(ctx, uv, d, N, o, filt).reshape(-1, 4).cpu().numpy()
            np.testing.assert_array_equal(out, flat, err_msg=f"tile {t} filter {filt}")
    ref, _ = oracle.shade_world(texs, g.uv, g.dir, N.reshape(-1, 3).cpu().numpy(), obj, oracle.QUADRILINEAR)
    assert np.abs(flat - ref).max() <= COLOUR_TOL
    gout = to_dev(np.random.default_rng(2).normal(size=(V, Hh, Ww, 4)).astype(np.float32))
    filt = api.RT_QUADRILINEAR
    api.rt_prepare_deterministic(ctx)

    def run(batched, flags):
        duv, ddir, dnrm = torch.empty_like(uv), torch.empty_like(d), torch.empty_like(d)
        dt = {o_: torch.empty((n, n, H, W, 4), device=uv.device) for o_ in oids}
        if batched:
            api.rt_shade_world_batched_backward(ctx, uv, d, N, o, filt, gout, dt, duv, ddir, dnrm, flags)
        else:
            api.rt_shade_world_backward(ctx, *flat_args, filt, gout.reshape(-1, 4), dt, duv.reshape(-1, 2),
                                        ddir.reshape(-1, 3), dnrm.reshape(-1, 3), flags)
        return [x.cpu().numpy() for x in (duv, ddir, dnrm)], {k: v.cpu().numpy() for k, v in dt.items()}

    for flags in (0, api.RT_DETERMINISTIC):
        a = run(False, flags)
        for t in ((8, 4, 2, 2), (32, 1, 4, 1), (4, 8, 1, 4)):
            api.rt_set_backward_tile(ctx, filt, *t)
            b = run(True, flags)
            for x, y in zip(a[0], b[0]):
                np.testing.assert_array_equal(x, y)
            for k in a[1]:
                if flags:
                    np.testing.assert_array_equal(a[1][k], b[1][k])
                else:
                    assert np.abs(a[1][k] - b[1][k]).max() <= 1e-5 * max(np.abs(a[1][k]).max(), 1.0)
    assert api.rt_get_error(ctx) == api.RT_OK


def test_world_batched_rejects_bad_shapes(scene):
    ctx, oids, _, _ = scene
    g, obj, uv, d, o = frames(1, 8, 8, oids)
    N = bumpy(1, 8, 8, 4)
    with pytest.raises(ValueError):
        api.rt_shade_world_batched(ctx, uv.reshape(-1, 2), d.reshape(-1, 3), N.reshape(-1, 3), o.reshape(-1))
    with pytest.raises(ValueError):
        api.rt_shade_world_batched(ctx, uv, d, N[:, :4], o)
