"""Pins of the oracle's bucket compression (Section 2; reading R11): palette
expansion and the two k-means steps, against brute force on tiny inputs,
identities and invariants."""
import numpy as np

import oracle
import synth


def palette_texture(K, n, seed, fmt=oracle.F32):
    atlas = oracle.fill_field(K, 1, n, synth.field_lobes(seed))
    return oracle.Texture.from_f32(atlas, K, 1, n, fmt)


def test_expand_matches_direct_slicing():
    K, n, W, H = 5, 3, 7, 4
    for fmt in (oracle.F32, oracle.F16, oracle.E4M3):
        pal = palette_texture(K, n, 40, fmt)
        index = np.random.default_rng(1).integers(0, K, (H, W)).astype(np.uint32)
        dense = oracle.palette_expand(pal, index, W, H)
        pv = pal.values().reshape(n, K, n, 4)  # [t, k, s, c]
        dv = dense.values().reshape(H, n, W, n, 4)  # [j, t, i, s, c]
        for j in range(H):
            for i in range(W):
                np.testing.assert_array_equal(dv[j, :, i], pv[:, index[j, i]])


def test_identity_palette_reproduces_the_texture():
    """K = w h with index = bucket number: the palette is the texture itself."""
    W, H, n = 4, 3, 4
    atlas = oracle.fill_field(W, H, n, synth.field_lobes(41))
    dense = oracle.Texture.from_f32(atlas, W, H, n, oracle.F16)
    # the same texels as a K x 1 palette: bucket b = j W + i becomes palette bucket b
    pal_atlas = atlas.reshape(H, n, W, n, 4).transpose(1, 0, 2, 3, 4).reshape(n, H * W * n, 4)
    pal = oracle.Texture.from_f32(pal_atlas, W * H, 1, n, oracle.F16)
    back = oracle.palette_expand(pal, np.arange(W * H, dtype=np.uint32).reshape(H, W), W, H)
    np.testing.assert_array_equal(back.codes, dense.codes)


def test_bucket_vectors_layout():
    W, H, n = 3, 2, 2
    vals = np.arange(H * n * W * n * 4, dtype=np.float64).reshape(H * n, W * n, 4)
    X = oracle.bucket_vectors(vals, W, H, n)
    for j in range(H):
        for i in range(W):
            for t in range(n):
                for s in range(n):
                    np.testing.assert_array_equal(X[j * W + i, (t * n + s) * 4:(t * n + s) * 4 + 4],
                                                  vals[j * n + t, i * n + s])


def test_assign_brute_force_and_ties():
    rng = np.random.default_rng(2)
    X = rng.normal(size=(30, 6))
    C = rng.normal(size=(5, 6))
    C[3] = C[1]  # a tie between 1 and 3 resolves to 1
    idx, dist, dall = oracle.kmeans_assign(X, C, all_distances=True)
    for b in range(30):
        d = [float(np.sum((X[b] - C[k]) ** 2)) for k in range(5)]
        np.testing.assert_allclose(dall[b], d, rtol=1e-14)
        k = int(np.argmin(d))
        assert idx[b] == k and idx[b] != 3
        assert dist[b] == dall[b, k]
    # centroids equal to the rows: each row is its own nearest, at distance 0
    idx, dist = oracle.kmeans_assign(X[:5], X[:5])
    np.testing.assert_array_equal(idx, np.arange(5))
    assert (dist == 0).all()


def test_update_means_empty_and_mass():
    rng = np.random.default_rng(3)
    X = rng.uniform(size=(40, 8))
    index = rng.integers(0, 4, 40).astype(np.uint32)
    index[index == 2] = 0  # cluster 2 is empty
    prev = rng.normal(size=(4, 8))
    C, counts = oracle.kmeans_update(X, index, prev)
    for k in range(4):
        members = X[index == k]
        assert counts[k] == len(members)
        if len(members):
            np.testing.assert_allclose(C[k], members.mean(axis=0), rtol=1e-14)
        else:
            np.testing.assert_array_equal(C[k], prev[k])
    np.testing.assert_allclose((counts[:, None] * C)[counts > 0].sum(0), X.sum(0), rtol=1e-13)


def test_lloyd_is_monotone():
    rng = np.random.default_rng(4)
    X = np.concatenate([rng.normal(loc=m, size=(50, 4)) for m in (0.0, 3.0, -2.0, 5.0)])
    C = X[rng.choice(len(X), 6, replace=False)]
    sse = []
    for _ in range(8):
        idx, dist = oracle.kmeans_assign(X, C)
        sse.append(dist.sum())
        C, _ = oracle.kmeans_update(X, idx, C)
    assert all(b <= a + 1e-9 for a, b in zip(sse, sse[1:]))


def test_duplicate_buckets_compress_exactly():
    """A texture made of m distinct buckets, encoded with K = m seeded at one copy
    of each: one Lloyd step reaches zero error and the palette texture expands
    to the original codes."""
    W, H, n, m = 6, 5, 3, 4
    protos = oracle.fill_field(m, 1, n, synth.field_lobes(42)).reshape(n, m, n, 4)
    which = np.random.default_rng(5).integers(0, m, (H, W))
    which.flat[:m] = np.arange(m)
    atlas = np.empty((H, n, W, n, 4), np.float32)
    for j in range(H):
        for i in range(W):
            atlas[j, :, i] = protos[:, which[j, i]]
    atlas = atlas.reshape(H * n, W * n, 4)
    X = oracle.bucket_vectors(atlas, W, H, n)
    C = X[:m][::-1].copy()  # one copy of each prototype, in another order
    idx, dist = oracle.kmeans_assign(X, C)
    assert (dist == 0).all()
    C2, _ = oracle.kmeans_update(X, idx, C)
    np.testing.assert_array_equal(C2, C)
    pal_atlas = C.reshape(m, n, n, 4).transpose(1, 0, 2, 3).reshape(n, m * n, 4).astype(np.float32)
    pal = oracle.Texture.from_f32(pal_atlas, m, 1, n, oracle.F32)
    back = oracle.palette_expand(pal, idx.reshape(H, W), W, H)
    np.testing.assert_array_equal(back.codes, atlas)
