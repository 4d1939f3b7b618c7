"""The oracle's procedural pattern texture (test infrastructure for textures too
large to hold as a host-side atlas) reads like a stored texture of the same
texels: shading it gives bit for bit what shading the stored atlas of
synth.pattern_values gives, in FP64 and FP16 storage, for every filter, with
forward colours and UV / direction gradients, including fragments on the
edges of the bucket matrix and of the in-bucket square.  A mistake in its
texel addressing (rows and columns exchanged, bucket and in-bucket index
confused, a channel's parameters misread) changes the colours.

oracle.taps, the per-fragment list of taps and weights the large-texture GPU
tests use for sparse texel-gradient parity, is checked against the oracle's
colour and texel gradient."""
import numpy as np
import pytest

import synth
from test_oracle_pins import unit_dirs


def pattern_atlas(W, H, n):
    Y = np.arange(H * n, dtype=np.int64)[:, None]
    X = np.arange(W * n, dtype=np.int64)[None, :]
    return np.stack([synth.pattern_values(X, Y, c) for c in range(4)], axis=-1)


def pattern(orc, W, H, n):
    return orc.PatternTexture(W, H, n, synth.PATTERN_A, synth.PATTERN_B, synth.PATTERN_K, synth.PATTERN_M)


def fragments(seed, F):
    rng = np.random.default_rng(seed)
    uv = rng.uniform(0, 1, (F, 2))
    uv[:40] = rng.choice([0.0, 1.0, 0.5], (40, 2))  # edges and centre of the bucket matrix
    d = unit_dirs(rng, F)
    d[40:60] = [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0]] * 5  # grazing: clamped B
    d[60:64] = [0.0, 0.0, 1.0]  # normal incidence: B = 0
    obj = np.zeros(F, np.int32)
    obj[64:80] = -1
    return uv.astype(np.float32), d.astype(np.float32), obj


@pytest.mark.parametrize("W,H,n", [(5, 3, 4), (2, 7, 8), (1, 1, 3)])
@pytest.mark.parametrize("filt", [0, 1, 2])
def test_pattern_reads_like_the_stored_atlas(orc, W, H, n, filt):
    atlas = pattern_atlas(W, H, n)
    # the pattern's values j / 2048 are exact in FP16: both stored forms hold the same texels
    stored64 = orc.Texture(W, H, n, orc.F64, atlas)
    stored16 = orc.Texture.from_f32(atlas.astype(np.float32), W, H, n, orc.F16)
    np.testing.assert_array_equal(stored16.values(), atlas)
    P = pattern(orc, W, H, n)
    uv, d, obj = fragments(10 * W + H + n, 3000)
    ref, f0 = orc.shade([stored64], uv, d, obj, filt)
    got, f1 = orc.shade([P], uv, d, obj, filt)
    assert f0 == f1 == 0
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(orc.shade([stored16], uv, d, obj, filt)[0], ref)
    g = np.random.default_rng(3).normal(size=(len(obj), 4))
    _, ruv, rdir, _ = orc.shade_backward([stored64], uv, d, obj, filt, g, want_tex=False)
    _, guv, gdir, _ = orc.shade_backward([P], uv, d, obj, filt, g, want_tex=False)
    np.testing.assert_array_equal(guv, ruv)
    np.testing.assert_array_equal(gdir, rdir)


def test_pattern_texels_differ_between_neighbours():
    """Every channel changes between horizontally and vertically adjacent texels
    and between adjacent buckets, so a texel read from a neighbouring address
    shows in the colour (by at least 1/2048 per unit weight)."""
    W, H, n = 64, 64, 8
    atlas = pattern_atlas(W, H, n)
    for axis in (0, 1):
        for step in (1, n):
            diff = np.abs(np.diff(atlas[::step, ::step] if step > 1 else atlas, axis=axis))
            assert (diff > 0).mean() > 0.99
            assert diff[diff > 0].min() >= 1.0 / 2048


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_taps_reproduce_colour_and_texel_gradient(orc, filt):
    """oracle.taps lists what the colour sums: the weighted sum of its texels is
    the colour, its weights sum to one, and weight x dL/dout accumulated per
    texel is the oracle's texel gradient."""
    W, H, n = 6, 5, 4
    rng = np.random.default_rng(11)
    vals = rng.uniform(0, 1, (H * n, W * n, 4))
    T = orc.Texture(W, H, n, orc.F64, vals)
    uv, d, obj = fragments(12, 2000)
    idx, w, flags = orc.taps([T], uv, d, obj, filt)
    assert flags == 0
    assert np.all((idx >= 0) == (w > 0))
    shaded = obj >= 0
    np.testing.assert_allclose(w[shaded].sum(axis=1), 1.0, rtol=0, atol=1e-15)
    assert not (idx[~shaded] >= 0).any()
    flat = vals.reshape(-1, 4)
    col = (w[..., None] * np.where(idx[..., None] >= 0, flat[np.maximum(idx, 0)], 0.0)).sum(axis=1)
    ref, _ = orc.shade([T], uv, d, obj, filt)
    np.testing.assert_allclose(col, ref, rtol=0, atol=1e-14)
    g = rng.normal(size=(len(obj), 4))
    gtex = np.zeros((H * n * W * n, 4))
    keep = idx >= 0
    np.add.at(gtex, idx[keep], (w[..., None] * g[:, None, :])[keep])
    rtex, _, _, _ = orc.shade_backward([T], uv, d, obj, filt, g, want_uv=False, want_dir=False)
    np.testing.assert_allclose(gtex.reshape(H * n, W * n, 4), rtex[0], rtol=0, atol=1e-13)
