"""GPU: palette textures (bucket compression, Section 2; reading R11) and the
k-means encoder, against the oracle.

A palette texture must shade exactly like the dense texture its palette and
index map stand for, so the oracle shades the expanded texture.  Texel
gradients of a palette texture are the dense gradients summed over the
buckets that share a palette bucket.  The k-means steps are checked one at a
time, on the GPU's own inputs:
- an assignment must be a nearest centroid in FP64, up to the FP32 rounding
  of |c|^2 - 2 x.c (2^-14 (|x|^2 + |c|^2));
- an update must be the FP64 mean rounded to FP32."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2301_01719_gb300 import api
from parity_util import COLOUR_TOL, FILTERS, ORACLE_FMT, floor_mismatch, gbuffer_to_dev, planes_to_atlas, to_dev

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


def palette_case(K=9, n=8, W=40, H=28, seed=50):
    pal_atlas = oracle.fill_field(K, 1, n, synth.field_lobes(seed))  # n x K n x 4
    index = np.random.default_rng(seed).integers(0, K, (H, W)).astype(np.uint32)
    return pal_atlas, index


@pytest.mark.parametrize("fmt", [api.RT_F32, api.RT_F16, api.RT_BF16, api.RT_E4M3_BUCKET_SCALE])
def test_palette_shading_matches_expanded_texture(ctx, fmt):
    K, n, W, H = 9, 8, 40, 28
    pal_atlas, index = palette_case(K, n, W, H)
    oid = api.rt_create_palette_texture(ctx, W, H, n, K, fmt, api.RT_LAYOUT_ATLAS, to_dev(pal_atlas),
                                        to_dev(index.view(np.int32)))
    assert api.rt_palette_size(ctx, oid) == K
    assert api.rt_texture_info(ctx, oid)["layout"] == api.RT_LAYOUT_PALETTE
    pal = oracle.Texture.from_f32(pal_atlas, K, 1, n, ORACLE_FMT[fmt])
    # the stored palette is the oracle's encoding, code for code
    codes, scales = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_ATLAS)
    np.testing.assert_array_equal(codes.cpu().numpy().view(pal.codes.dtype), pal.codes)
    if fmt == api.RT_E4M3_BUCKET_SCALE:
        np.testing.assert_array_equal(scales.cpu().numpy().reshape(-1), pal.scales.reshape(-1))
    dense = oracle.palette_expand(pal, index, W, H)
    g = synth.quad_scene(1001, 200, 180)
    obj_np = np.where(g.obj >= 0, oid, -1).astype(np.int32)
    table = [None] * oid + [dense]
    uv, d, _ = gbuffer_to_dev(g)
    for filt in FILTERS:
        out = api.rt_shade(ctx, uv, d, to_dev(obj_np), filt).cpu().numpy()
        ref, flags = oracle.shade(table, g.uv, g.dir, obj_np, filt)
        assert flags == 0
        ok = ~floor_mismatch(ctx, g, obj_np, filt, table)
        assert ok.mean() > 0.99
        assert np.abs(out - ref)[ok].max() <= COLOUR_TOL, filt
    assert api.rt_get_error(ctx) == api.RT_OK
    api.rt_destroy_texture(ctx, oid)


def test_palette_backward_sums_over_shared_buckets(ctx):
    K, n, W, H = 7, 6, 33, 21
    pal_atlas, index = palette_case(K, n, W, H, seed=51)
    # a borrowed FP32 palette in PLANES order (n, n, K, 4): the form a fit updates
    pal_planes = pal_atlas.reshape(n, K, n, 4).transpose(0, 2, 1, 3).copy()
    buf = to_dev(pal_planes)
    oid = api.rt_create_palette_texture(ctx, W, H, n, K, api.RT_F32, api.RT_LAYOUT_PLANES, buf,
                                        to_dev(index.view(np.int32)), api.RT_BORROW)
    pal = oracle.Texture.from_f32(pal_atlas, K, 1, n, oracle.F32)
    dense = oracle.palette_expand(pal, index, W, H)
    g = synth.quad_scene(1003, 160, 160)
    obj_np = np.where(g.obj >= 0, oid, -1).astype(np.int32)
    table = [None] * oid + [dense]
    gout = np.random.default_rng(7).normal(size=(g.F, 4)).astype(np.float32)
    uv, d, _ = gbuffer_to_dev(g)
    dtex = torch.empty((n, n, K, 4), device=uv.device)
    duv = torch.empty_like(uv)
    ddir = torch.empty_like(d)
    api.rt_shade_backward(ctx, uv, d, to_dev(obj_np), api.RT_QUADRILINEAR, to_dev(gout), {oid: dtex}, duv, ddir)
    assert api.rt_get_error(ctx) == api.RT_OK
    gt, guv, gdir, _ = oracle.shade_backward(table, g.uv, g.dir, obj_np, api.RT_QUADRILINEAR, gout)
    gabs, _, _, _ = oracle.shade_backward(table, g.uv, g.dir, obj_np, api.RT_QUADRILINEAR, np.abs(gout),
                                          want_uv=False, want_dir=False)
    # dense gradient (H n, W n, 4) -> per palette bucket: sum over the buckets that use it
    dv = gt[oid].reshape(H, n, W, n, 4)
    av = gabs[oid].reshape(H, n, W, n, 4)
    want = np.zeros((n, K, n, 4))
    wabs = np.zeros((n, K, n, 4))
    for j in range(H):
        for i in range(W):
            want[:, index[j, i]] += dv[j, :, i]
            wabs[:, index[j, i]] += av[j, :, i]
    got = planes_to_atlas(dtex.cpu().numpy(), K, 1, n).reshape(n, K, n, 4)
    tol = 1e-4 * wabs + 2e-5 * np.abs(gout).max()
    assert np.all(np.abs(got - want) <= tol)
    # UV and direction gradients are those of the expanded texture (same values, same lerps)
    ok = ~floor_mismatch(ctx, g, obj_np, api.RT_QUADRILINEAR, table) & (obj_np >= 0)
    for got_c, ref_c in ((duv.cpu().numpy(), guv), (ddir.cpu().numpy(), gdir)):
        scale = np.abs(ref_c[ok]).max() + 1e-30
        err = np.abs(got_c[ok] - ref_c[ok])
        assert np.quantile(err / (1e-3 * np.abs(ref_c[ok]) + 1e-5 * scale), 0.999) <= 1.0
    api.rt_destroy_texture(ctx, oid)


def dense_texture(ctx, W, H, n, fmt, seed):
    atlas = oracle.fill_field(W, H, n, synth.field_lobes(seed))
    oid = api.rt_create_texture(ctx, W, H, n, fmt, api.RT_LAYOUT_ATLAS, to_dev(atlas))
    T = oracle.Texture.from_f32(atlas, W, H, n, ORACLE_FMT[fmt])
    # the kernels see the texels decoded to FP32 (an E4M3 code times its scale is rounded once)
    return oid, oracle.bucket_vectors(T.values().astype(np.float32), W, H, n)


def centroid_rows(C: torch.Tensor, K: int, n: int) -> np.ndarray:
    """(n, n, K, 4) device centroids -> K x (n^2 4) rows in bucket-vector order."""
    return C.cpu().numpy().astype(np.float64).reshape(n * n, K, 4).transpose(1, 0, 2).reshape(K, n * n * 4)


@pytest.mark.parametrize("fmt", [api.RT_F16, api.RT_E4M3_BUCKET_SCALE, api.RT_F32])
def test_kmeans_steps_match_oracle(ctx, fmt):
    W, H, n, K = 53, 37, 4, 70  # several blocks of buckets, a ragged last one, two centroid sweeps
    oid, X = dense_texture(ctx, W, H, n, fmt, 60)
    B = W * H
    pick = np.random.default_rng(8).choice(B, K - 1, replace=False).astype(np.int32)
    pick = np.concatenate([pick, pick[:1]])  # centroid K-1 duplicates centroid 0: never nearest, stays empty
    C = api.rt_kmeans_init(ctx, oid, K, to_dev(pick))
    np.testing.assert_array_equal(centroid_rows(C, K, n), X[pick])
    index, dist = api.rt_kmeans_assign(ctx, oid, K, C, want_dist=True)
    gi = index.cpu().numpy().reshape(-1).astype(np.int64)
    gd = dist.cpu().numpy().reshape(-1).astype(np.float64)
    Cr = centroid_rows(C, K, n)
    oi, od, dall = oracle.kmeans_assign(X, Cr, all_distances=True)
    tau = 2.0 ** -14 * ((X ** 2).sum(1) + (Cr ** 2).sum(1)[gi])
    assert np.all(dall[np.arange(B), gi] <= od + tau)
    assert (gi == oi).mean() > 0.99
    assert np.all(np.abs(gd - dall[np.arange(B), gi]) <= tau)
    assert not (gi == K - 1).any()
    # update from the GPU's assignment
    prev = Cr.copy()
    api.rt_kmeans_update(ctx, oid, K, index, C)
    Cu = centroid_rows(C, K, n)
    want, counts = oracle.kmeans_update(X, gi.astype(np.uint32), prev)
    assert counts[K - 1] == 0
    np.testing.assert_array_equal(Cu[K - 1], prev[K - 1])
    np.testing.assert_allclose(Cu, want, rtol=2.0 ** -23, atol=1e-30)
    assert api.rt_get_error(ctx) == api.RT_OK
    api.rt_destroy_texture(ctx, oid)


def test_duplicate_buckets_round_trip(ctx):
    """Buckets copied from m prototypes: k-means seeded at one copy of each has zero
    error, and the palette texture built from its centroids and assignment shades
    bit-identically to the dense texture."""
    W, H, n, m = 30, 22, 6, 5
    protos = oracle.fill_field(m, 1, n, synth.field_lobes(61)).reshape(n, m, n, 4)
    which = np.random.default_rng(9).integers(0, m, (H, W))
    which.flat[:m] = np.arange(m)
    atlas = np.empty((H, n, W, n, 4), np.float32)
    for j in range(H):
        for i in range(W):
            atlas[j, :, i] = protos[:, which[j, i]]
    atlas = atlas.reshape(H * n, W * n, 4)
    oid = api.rt_create_texture(ctx, W, H, n, api.RT_F32, api.RT_LAYOUT_ATLAS, to_dev(atlas))
    C = api.rt_kmeans_init(ctx, oid, m, to_dev(np.arange(m, dtype=np.int32)))
    index, dist = api.rt_kmeans_assign(ctx, oid, m, C, want_dist=True)
    assert float(dist.abs().max()) == 0.0
    np.testing.assert_array_equal(index.cpu().numpy(), which)
    api.rt_kmeans_update(ctx, oid, m, index, C)
    pid = api.rt_create_palette_texture(ctx, W, H, n, m, api.RT_F32, api.RT_LAYOUT_PLANES, C, index)
    g = synth.quad_scene(1004, 128, 128)
    uv, d, _ = gbuffer_to_dev(g)
    for filt in FILTERS:
        a = api.rt_shade(ctx, uv, d, to_dev(np.where(g.obj >= 0, oid, -1).astype(np.int32)), filt)
        b = api.rt_shade(ctx, uv, d, to_dev(np.where(g.obj >= 0, pid, -1).astype(np.int32)), filt)
        assert torch.equal(a, b)
    api.rt_destroy_texture(ctx, oid)
    api.rt_destroy_texture(ctx, pid)


def test_palette_rejects_bad_index(ctx):
    K, n, W, H = 4, 4, 8, 8
    pal_atlas, index = palette_case(K, n, W, H, seed=52)
    bad = index.copy()
    bad[3, 5] = K
    with pytest.raises(api.RadtexError) as e:
        api.rt_create_palette_texture(ctx, W, H, n, K, api.RT_F16, api.RT_LAYOUT_ATLAS, to_dev(pal_atlas),
                                      to_dev(bad.view(np.int32)))
    assert e.value.status == api.RT_ERR_INVALID_ARG
    oid = api.rt_create_palette_texture(ctx, W, H, n, K, api.RT_F16, api.RT_LAYOUT_ATLAS, to_dev(pal_atlas),
                                        to_dev(index.view(np.int32)))
    with pytest.raises(api.RadtexError) as e:
        api.rt_bake(ctx, oid, api.RT_SURFACE_PLANE, synth.bake_scene(1))
    assert e.value.status == api.RT_ERR_UNSUPPORTED
    api.rt_destroy_texture(ctx, oid)


def test_palette_encode_full_size_sampled(ctx):
    """k-means on the 1024^2 x 16^2 FP16 lobe texture of the sphere-plane workload
    (K = 256, 3 Lloyd steps, assignments on the tensor cores): the error falls,
    and 1500 sampled buckets are assigned to a nearest centroid in FP64 up to
    the FP16 operand bound."""
    W = H = 1024
    n, K = 16, 256
    oid = api.rt_create_texture(ctx, W, H, n, api.RT_F16)
    api.rt_fill_bucket_lobes(ctx, oid, to_dev(synth.bucket_lobe_params(2001, W, H)))
    C, index, sse = api.palette_encode(ctx, oid, K, 3, seed=1)
    assert all(b <= a * (1 + 1e-6) for a, b in zip(sse, sse[1:])) and sse[-1] < sse[0]
    rng = np.random.default_rng(10)
    sample = rng.choice(W * H, 1500, replace=False)
    codes, _ = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_PLANES)  # (n, n, H, W, 4) int16
    st = torch.from_numpy(sample).to(codes.device)
    rows = codes.reshape(n * n, W * H, 4)[:, st].permute(1, 0, 2).cpu().numpy()
    X = oracle.decode(oracle.F16, rows.view(np.uint16)).reshape(len(sample), n * n * 4)
    Cr = centroid_rows(C, K, n)
    gi = index.reshape(-1)[st].cpu().numpy().astype(np.int64)
    _, od, dall = oracle.kmeans_assign(X, Cr, all_distances=True)
    tau = 2.0 ** -9 * ((X ** 2).sum(1) + (Cr ** 2).sum(1)[gi])
    assert np.all(dall[np.arange(len(sample)), gi] <= od + tau)
    api.rt_destroy_texture(ctx, oid)


@pytest.mark.parametrize("shape", [(53, 37, 4, 300), (40, 20, 16, 70), (17, 9, 3, 5), (10, 10, 4, 3),
                                   (160, 161, 4, 300)])
def test_kmeans_tensor_core_assign_matches_oracle(ctx, shape):
    """The tcgen05 assignment (FP16 operands, FP32 accumulation in tensor memory):
    every choice is a nearest centroid in FP64 up to the FP16 rounding of the
    operands, 2^-9 (|x|^2 + |c|^2); it agrees with the FP32 kernel on almost
    every bucket.  Shapes: two 256-centroid tiles with a ragged bucket tile; 16
    K-chunks over 7 bucket tiles; a vector length (3^2 x 4 = 36) padded to 64; a
    single bucket tile; 202 bucket tiles, more than the persistent grid's one CTA
    per SM, so CTAs walk several tiles with the accumulators alternating across
    them."""
    W, H, n, K = shape
    oid, X = dense_texture(ctx, W, H, n, api.RT_F16, 62)
    B = W * H
    pick = np.random.default_rng(9).choice(B, K, replace=False).astype(np.int32)
    C = api.rt_kmeans_init(ctx, oid, K, to_dev(pick))
    ti, td = api.rt_kmeans_assign_tc(ctx, oid, K, C, want_dist=True)
    assert api.rt_get_error(ctx) == api.RT_OK
    fi = api.rt_kmeans_assign(ctx, oid, K, C)
    gi = ti.cpu().numpy().reshape(-1).astype(np.int64)
    gd = td.cpu().numpy().reshape(-1).astype(np.float64)
    Cr = centroid_rows(C, K, n)
    _, od, dall = oracle.kmeans_assign(X, Cr, all_distances=True)
    assert gi.min() >= 0 and gi.max() < K
    tau = 2.0 ** -9 * ((X ** 2).sum(1) + (Cr ** 2).sum(1)[gi])
    assert np.all(dall[np.arange(B), gi] <= od + tau)
    assert np.all(np.abs(gd - dall[np.arange(B), gi]) <= tau)
    assert (gi == fi.cpu().numpy().reshape(-1)).mean() > 0.95
    api.rt_destroy_texture(ctx, oid)


def test_kmeans_tensor_core_wait_timeout_is_reported_and_recoverable(ctx):
    """Failure detection without a GPU fault: with the context's wait limit at one
    poll, the tensor-core assignment's pipeline waits run out (the TMA copies
    cannot land within one poll), so the kernel raises RT_ERR_TIMEOUT, drains
    what it issued and returns; the context stays usable -- with the default
    limit the same assignment passes and matches the FP32 kernel, and shading
    still works."""
    W, H, n, K = 160, 161, 4, 300
    oid, X = dense_texture(ctx, W, H, n, api.RT_F16, 63)
    pick = np.random.default_rng(10).choice(W * H, K, replace=False).astype(np.int32)
    C = api.rt_kmeans_init(ctx, oid, K, to_dev(pick))
    assert api.rt_get_error(ctx) == api.RT_OK
    api.rt_set_wait_limit(ctx, 1)
    try:
        api.rt_kmeans_assign_tc(ctx, oid, K, C)
        assert api.rt_get_error(ctx) == api.RT_ERR_TIMEOUT
    finally:
        api.rt_set_wait_limit(ctx, 0)
    assert api.rt_get_error(ctx) == api.RT_OK  # the sticky word was read and cleared
    ti = api.rt_kmeans_assign_tc(ctx, oid, K, C)
    assert api.rt_get_error(ctx) == api.RT_OK
    fi = api.rt_kmeans_assign(ctx, oid, K, C)
    assert (ti.cpu().numpy() == fi.cpu().numpy()).mean() > 0.95
    uv = torch.full((64, 2), 0.5, device="cuda")
    d = torch.tensor([[0.0, 0.0, 1.0]] * 64, device="cuda")
    o = torch.full((64,), oid, dtype=torch.int32, device="cuda")
    out = api.rt_shade(ctx, uv, d, o, api.RT_QUADRILINEAR)
    assert api.rt_get_error(ctx) == api.RT_OK and bool(torch.isfinite(out).all())
    api.rt_destroy_texture(ctx, oid)
