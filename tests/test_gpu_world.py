"""GPU: the world-space lookup (Eq. 1a with a per-fragment normal) and the
repeat address mode (reading R12), against the oracle.

The parity bars are those of the tangent-space path:
- floors match the oracle outside the FP32 band;
- colours agree within 1e-5;
- texel gradients agree within 1e-4 of sum w |g|;
- UV, direction and normal gradients agree within 1e-3 relative away from
  kinks."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2301_01719_gb300 import api
from parity_util import (COLOUR_TOL, FILTERS, ORACLE_FMT, compare_indices, gbuffer_to_dev, grad_to_atlas, index_taus,
                         quad_workload, to_dev)

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


def bumpy_normals(F, seed, amount=0.35):
    """Unit normals tilted from +z by seeded noise (a normal-mapped surface)."""
    rng = np.random.default_rng(seed)
    N = np.concatenate([rng.normal(scale=amount, size=(F, 2)), np.ones((F, 1))], 1)
    return (N / np.linalg.norm(N, axis=1, keepdims=True)).astype(np.float32)


def world_case(ctx, fmt, wrap=0, W=48, H=40, n=8):
    atlas, g, T = quad_workload(fmt, W, H, n, seed=1011, width=192, height=160)
    T.wrap = wrap
    flags = (api.RT_WRAP_U if wrap & 1 else 0) | (api.RT_WRAP_V if wrap & 2 else 0)
    oid = api.rt_create_texture(ctx, W, H, n, fmt, api.RT_LAYOUT_ATLAS, to_dev(atlas), flags)
    obj = np.where(g.obj >= 0, oid, -1).astype(np.int32)
    table = [None] * oid + [T]
    return oid, g, obj, table


def world_mismatch(ctx, g, N, obj, filt, table):
    uv, d, _ = gbuffer_to_dev(g)
    idx, coord = api.rt_locate_world(ctx, uv, d, to_dev(N), to_dev(obj), filt)
    oi, oc, _ = oracle.locate_world(table, g.uv, g.dir, N, obj, filt)
    T = table[-1]
    mism, _ = compare_indices(idx.cpu().numpy(), coord.cpu().numpy().astype(np.float64), oi, oc,
                              index_taus(T.W, T.H, T.n), mask=obj >= 0)
    return mism


@pytest.mark.parametrize("fmt", [api.RT_F32, api.RT_F16, api.RT_E4M3_BUCKET_SCALE])
def test_world_forward_matches_oracle(ctx, fmt):
    oid, g, obj, table = world_case(ctx, fmt)
    N = bumpy_normals(g.F, 3)
    uv, d, _ = gbuffer_to_dev(g)
    for filt in FILTERS:
        out = api.rt_shade_world(ctx, uv, d, to_dev(N), to_dev(obj), filt).cpu().numpy()
        ref, flags = oracle.shade_world(table, g.uv, g.dir, N, obj, filt)
        assert flags == 0
        ok = ~world_mismatch(ctx, g, N, obj, filt, table)
        assert ok.mean() > 0.99
        assert np.abs(out - ref)[ok].max() <= COLOUR_TOL
    assert api.rt_get_error(ctx) == api.RT_OK
    api.rt_destroy_texture(ctx, oid)


def test_world_with_z_normal_is_rt_shade(ctx):
    oid, g, obj, _ = world_case(ctx, api.RT_F16)
    uv, d, o = gbuffer_to_dev(g)
    o = to_dev(obj)
    N = torch.zeros_like(d)
    N[:, 2] = 1.0
    for filt in FILTERS:
        assert torch.equal(api.rt_shade_world(ctx, uv, d, N, o, filt), api.rt_shade(ctx, uv, d, o, filt))
    api.rt_destroy_texture(ctx, oid)


def test_world_backward_matches_oracle(ctx):
    oid, g, obj, table = world_case(ctx, api.RT_F32)
    N = bumpy_normals(g.F, 4)
    T = table[-1]
    rng = np.random.default_rng(5)
    gout = rng.normal(size=(g.F, 4)).astype(np.float32)
    uv, d, _ = gbuffer_to_dev(g)
    dtex = torch.empty((T.n, T.n, T.H, T.W, 4), device=uv.device)
    duv, ddir, dnrm = torch.empty_like(uv), torch.empty_like(d), torch.empty_like(d)
    api.rt_shade_world_backward(ctx, uv, d, to_dev(N), to_dev(obj), api.RT_QUADRILINEAR, to_dev(gout), {oid: dtex},
                                duv, ddir, dnrm)
    assert api.rt_get_error(ctx) == api.RT_OK
    gt, guv, gdir, gnrm, _ = oracle.shade_world_backward(table, g.uv, g.dir, N, obj, api.RT_QUADRILINEAR, gout)
    gabs, _, _, _, _ = oracle.shade_world_backward(table, g.uv, g.dir, N, obj, api.RT_QUADRILINEAR, np.abs(gout))
    got = grad_to_atlas(ctx, oid, dtex)
    assert np.all(np.abs(got - gt[oid]) <= 1e-4 * gabs[oid] + 2e-5 * np.abs(gout).max())
    np.testing.assert_array_equal(ddir.cpu().numpy(), dnrm.cpu().numpy())
    # away from the kinks: integer coordinates and the clamp bounds of B
    _, oc, _ = oracle.locate_world(table, g.uv, g.dir, N, obj, api.RT_QUADRILINEAR)
    far = (np.abs(oc - np.round(oc)) > 1e-3).all(axis=1) & (obj >= 0)
    lo = 1.0 / T.n - 1.0
    far &= (np.abs(np.abs((oc[:, 2:] + 0.5) * 2 / T.n - 1) - abs(lo)) > 1e-3).all(axis=1)
    assert far.sum() > 1000
    for got_c, ref_c in ((duv.cpu().numpy(), guv), (ddir.cpu().numpy(), gdir), (dnrm.cpu().numpy(), gnrm)):
        scale = np.abs(ref_c[far]).max() + 1e-30
        assert np.all(np.abs(got_c[far] - ref_c[far]) <= 1e-3 * np.abs(ref_c[far]) + 1e-5 * scale)
    api.rt_destroy_texture(ctx, oid)


@pytest.mark.parametrize("wrap", [1, 2, 3])
@pytest.mark.parametrize("W,H", [(48, 40), (37, 23)])  # quads, and quads with padded odd sides
def test_wrap_forward_and_backward(ctx, wrap, W, H):
    """Repeat mode on a UV range that crosses the texture's edges: forward
    colours of the flat and the batched entry points, UV gradients, and the texel
    gradients of taps that wrap from the last bucket to the first."""
    oid, g, obj, table = world_case(ctx, api.RT_F16, wrap=wrap, W=W, H=H)
    rng = np.random.default_rng(6)
    g.uv[:] = (g.uv * 2.0 - 0.5 + rng.uniform(-0.01, 0.01, g.uv.shape)).astype(np.float32)
    uv, d, _ = gbuffer_to_dev(g)
    o = to_dev(obj)
    T = table[-1]
    for filt in FILTERS:
        out = api.rt_shade(ctx, uv, d, o, filt).cpu().numpy()
        ref, _ = oracle.shade(table, g.uv, g.dir, obj, filt)
        idx, coord = api.rt_locate(ctx, uv, d, o, filt)
        oi, oc, _ = oracle.locate(table, g.uv, g.dir, obj, filt)
        mism, _ = compare_indices(idx.cpu().numpy(), coord.cpu().numpy().astype(np.float64), oi, oc,
                                  index_taus(T.W, T.H, T.n), mask=obj >= 0)
        assert np.abs(out - ref)[~mism].max() <= COLOUR_TOL
    gout = rng.normal(size=(g.F, 4)).astype(np.float32)
    duv = torch.empty_like(uv)
    dtex = torch.empty(api.storage_numel(ctx, oid), device=uv.device)
    api.rt_shade_backward(ctx, uv, d, o, api.RT_QUADRILINEAR, to_dev(gout), {oid: dtex}, duv, None)
    gt, guv, _, _ = oracle.shade_backward(table, g.uv, g.dir, obj, api.RT_QUADRILINEAR, gout, want_dir=False)
    gabs, _, _, _ = oracle.shade_backward(table, g.uv, g.dir, obj, api.RT_QUADRILINEAR, np.abs(gout),
                                          want_uv=False, want_dir=False)
    got_t = grad_to_atlas(ctx, oid, dtex)
    assert np.all(np.abs(got_t - gt[oid]) <= 1e-4 * gabs[oid] + 2e-5 * np.abs(gout).max())
    _, oc, _ = oracle.locate(table, g.uv, g.dir, obj, api.RT_QUADRILINEAR)
    far = (np.abs(oc - np.round(oc)) > 1e-3).all(axis=1) & (obj >= 0)
    got = duv.cpu().numpy()
    scale = np.abs(guv[far]).max()
    assert np.all(np.abs(got[far] - guv[far]) <= 1e-3 * np.abs(guv[far]) + 1e-5 * scale)
    assert api.rt_get_error(ctx) == api.RT_OK
    api.rt_destroy_texture(ctx, oid)


def test_world_bad_normal_flags_nonfinite(ctx):
    oid, g, obj, _ = world_case(ctx, api.RT_F16)
    N = bumpy_normals(g.F, 7)
    hit = np.flatnonzero(obj >= 0)[:3]
    N[hit[0], 1] = np.nan
    uv, d, _ = gbuffer_to_dev(g)
    out = api.rt_shade_world(ctx, uv, d, to_dev(N), to_dev(obj), api.RT_QUADRILINEAR).cpu().numpy()
    assert (out[hit[0]] == 0).all() and (out[hit[1]] != 0).any()
    assert api.rt_get_error(ctx) == api.RT_ERR_NONFINITE
    api.rt_destroy_texture(ctx, oid)
