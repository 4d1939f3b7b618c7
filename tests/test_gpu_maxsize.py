"""GPU parity on textures of 2^32 texels -- beyond 32-bit texel indices and
16-bit bucket counts per axis -- and on the widest and tallest bucket matrices
the API takes (w or h = 65536).

The textures hold synth.pattern_values (values j / 2048, exact in FP16), which
the oracle evaluates per texel (oracle.PatternTexture), so no host-side atlas of
the 34 GB texture is needed.  Per case, on 512 x 512 random fragments:

* rt_locate's floors against the oracle's (equal outside the FP32 band);
* colours of every filter from the owned FP16 texture (the single-format
  kernels; for a nearest axis, away from fragments whose floor flipped inside
  the band) and, quadrilinear, from the FP32 source atlas borrowed in place (the
  format-dispatching kernels on 16-byte texels) against the oracle;
* the backward's UV and direction gradients against the oracle away from kinks;
* its texel gradients, sparse: the oracle's taps and weights (oracle.taps) give
  the expected gradient of every texel a fragment touches, compared at those
  texels, and the absolute gradient mass anywhere else in the 64 GiB gradient
  buffer must be negligible (no stray writes)."""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2301_01719_gb300 import api
from parity_util import COLOUR_TOL, floor_mismatch, storage_index

pytestmark = pytest.mark.gpu

SIDE = 512
CASES = [(2048, 2048, 32), (1024, 1024, 64), (65536, 2, 16), (3, 65536, 8)]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_01719_gb300 import build

    build.build()
    c = api.Context(0)
    yield c
    c.close()


def fragments(seed):
    rng = np.random.default_rng(seed)
    F = SIDE * SIDE
    uv = rng.uniform(0, 1, (F, 2))
    uv[:64] = rng.choice([0.0, 1.0], (64, 2))  # corners and edges of the bucket matrix
    z = rng.uniform(0, 1, F)
    phi = rng.uniform(0, 2 * np.pi, F)
    r = np.sqrt(1 - z * z)
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], 1)
    d[64:96] = [[1.0, 0.0, 0.0], [0.0, -1.0, 0.0]] * 16  # grazing: clamped in-bucket coordinate
    obj = np.zeros(F, np.int32)
    obj[rng.random(F) < 0.03] = -1
    return uv.astype(np.float32), d.astype(np.float32), obj


def pattern_atlas(W, H, n, dev):
    """The FP32 source atlas of the pattern, generated on the device in row blocks."""
    atlas = torch.empty((H * n, W * n, 4), dtype=torch.float32, device=dev)
    X = torch.arange(W * n, dtype=torch.int64, device=dev)[None, :]
    rows = max(1, (1 << 26) // (W * n))
    for y0 in range(0, H * n, rows):
        Y = torch.arange(y0, min(H * n, y0 + rows), dtype=torch.int64, device=dev)[:, None]
        for c in range(4):
            atlas[y0:y0 + Y.shape[0], :, c] = synth.pattern_values(X, Y, c)
    return atlas


@pytest.mark.parametrize("W,H,n", CASES)
def test_max_size_texture(ctx, W, H, n):
    dev = torch.device("cuda", 0)
    texels = W * H * n * n
    if torch.cuda.mem_get_info(dev)[0] < 24 * texels + (8 << 30):
        pytest.skip("not enough free device memory for the texture and its gradient")
    P = oracle.PatternTexture(W, H, n, synth.PATTERN_A, synth.PATTERN_B, synth.PATTERN_K, synth.PATTERN_M)
    uv, d, obj = fragments(W + 7 * H + 31 * n)
    shape = (1, SIDE, SIDE)
    t_uv = torch.from_numpy(uv).to(dev).view(*shape, 2)
    t_d = torch.from_numpy(d).to(dev).view(*shape, 3)
    atlas = pattern_atlas(W, H, n, dev)
    oid = api.rt_create_texture(ctx, W, H, n, api.RT_F16, api.RT_LAYOUT_ATLAS, atlas)
    t_o = torch.from_numpy(np.where(obj >= 0, oid, -1).astype(np.int32)).to(dev).view(*shape)
    o_ref = np.where(obj >= 0, 0, -1).astype(np.int32)
    refs = {}
    table = [None] * oid + [P]
    gb = SimpleNamespace(uv=uv, dir=d, obj=np.where(obj >= 0, oid, -1).astype(np.int32))
    for filt in (api.RT_NEAREST, api.RT_ANGULAR_BILINEAR, api.RT_QUADRILINEAR):
        out = api.rt_shade_batched(ctx, t_uv, t_d, t_o, filt)
        assert api.rt_get_error(ctx) == api.RT_OK
        refs[filt], flags = oracle.shade([P], uv, d, o_ref, filt)
        assert flags == 0
        # rt_locate's floors equal the oracle's outside the FP32 band; a nearest axis may flip
        # inside it, where the colour jumps by a texel step
        mism = floor_mismatch(ctx, gb, gb.obj, filt, table)
        keep = ~mism if filt != api.RT_QUADRILINEAR else np.ones(len(obj), bool)
        assert np.abs(out.view(-1, 4).cpu().numpy() - refs[filt])[keep].max() <= COLOUR_TOL
    # the same texels borrowed in place as an FP32 atlas
    bid = api.rt_create_texture(ctx, W, H, n, api.RT_F32, api.RT_LAYOUT_ATLAS, atlas, api.RT_BORROW)
    t_ob = torch.where(t_o >= 0, bid, -1).to(torch.int32)
    out = api.rt_shade_batched(ctx, t_uv, t_d, t_ob, api.RT_QUADRILINEAR)
    assert api.rt_get_error(ctx) == api.RT_OK
    assert np.abs(out.view(-1, 4).cpu().numpy() - refs[api.RT_QUADRILINEAR]).max() <= COLOUR_TOL
    api.rt_destroy_texture(ctx, bid)
    del atlas
    torch.cuda.empty_cache()

    # backward from the FP16 texture
    rng = np.random.default_rng(5)
    g = rng.normal(size=(SIDE * SIDE, 4)).astype(np.float32)
    t_g = torch.from_numpy(g).to(dev).view(*shape, 4)
    dtex = torch.empty(api.layout_shape(api.rt_texture_info(ctx, oid)["layout"], W, H, n), dtype=torch.float32,
                       device=dev)
    duv = torch.empty_like(t_uv)
    ddir = torch.empty_like(t_d)
    api.rt_shade_batched_backward(ctx, t_uv, t_d, t_o, api.RT_QUADRILINEAR, t_g, {oid: dtex}, duv, ddir)
    assert api.rt_get_error(ctx) == api.RT_OK
    # UV and direction gradients away from kinks
    _, guv, gdir, _ = oracle.shade_backward([P], uv, d, o_ref, oracle.QUADRILINEAR, g.astype(np.float64),
                                            want_tex=False)
    _, oc, _ = oracle.locate([P], uv, d, o_ref, oracle.QUADRILINEAR)
    far = (np.abs(oc - np.round(oc)) > 1e-3).all(axis=1) & (obj >= 0)
    B = oracle.squarify(oracle.equisolid(d.astype(np.float64)))
    far &= (np.abs(np.abs(B) - (1 - 1.0 / n)) > 1e-3).all(axis=1)
    assert far.sum() > SIDE * SIDE // 4
    # The pattern changes by 1/2048 per texel, so an in-bucket derivative is a difference of two
    # projected texels g . T (each up to sum |g|) far smaller than either: in FP32 it carries an
    # absolute error of a few ulps of sum |g|, scaled by dB-coordinate / dB = n / 2 and by the
    # Jacobian of Eq. 3 and Eq. 1b (below 2): 8 n 2^-24 sum |g| bounds it.
    gsum = np.abs(g).sum(axis=1)[far]
    extra = {2: 0.0, 3: 8 * n * 2.0 ** -24 * gsum}
    for got, ref_c in ((duv.view(-1, 2).cpu().numpy(), guv), (ddir.view(-1, 3).cpu().numpy(), gdir)):
        scale = np.abs(ref_c[far]).max()
        tol = 1e-3 * np.abs(ref_c[far]) + 1e-5 * scale + np.reshape(extra[got.shape[1]], (-1, 1))
        assert np.all(np.abs(got[far] - ref_c[far]) <= tol)
    # texel gradients at every touched texel, from the oracle's taps
    idx, w, flags = oracle.taps([P], uv, d, o_ref, oracle.QUADRILINEAR)
    assert flags == 0
    keep = idx >= 0
    touched, inv = np.unique(idx[keep], return_inverse=True)
    expect = np.zeros((touched.shape[0], 4))
    np.add.at(expect, inv, (w[..., None] * g[:, None, :].astype(np.float64))[keep])
    X, Y = touched % (W * n), touched // (W * n)
    i, s, j, t = X // n, X % n, Y // n, Y % n
    flat = storage_index(api.rt_texture_info(ctx, oid)["layout"], W, H, n, i, j, s, t)
    got = dtex.view(-1, 4)[torch.from_numpy(flat).to(dev)].double().cpu().numpy()
    # the texel-gradient bar of the other backward parity tests: FP32 weights of FP32 coordinates
    assert np.all(np.abs(got - expect) <= 1e-4 * np.abs(expect) + 2e-5 * np.abs(g).max())
    total = sum(float(dtex[tt].abs().sum(dtype=torch.float64)) for tt in range(n))
    inside = float(np.abs(got).sum())
    assert total - inside <= 1e-6 * total
    del dtex
    api.rt_destroy_texture(ctx, oid)
    torch.cuda.empty_cache()
