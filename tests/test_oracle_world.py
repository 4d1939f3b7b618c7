"""Pins of the oracle's world-space lookup (Eq. 1a with a per-fragment normal)
and of the repeat address mode (reading R12).

- Eq. 1a reduces to Eq. 1b when N = +z.
- Closed forms of the equisolid coordinate of a tilted normal.
- Central differences of the FP64 world-space synthesis.
- Repeat mode: periodicity, brute force against periodic tent kernels,
  equality with clamp-to-edge away from the edges, and central differences
  across the seam."""
import numpy as np
import pytest

from test_oracle_pins import brute_shade, tent, unit_dirs


def textures(orc, W, H, n, seed, wrap=0):
    rng = np.random.default_rng(seed)
    vals = rng.uniform(0, 1, (H * n, W * n, 4))
    return orc.Texture(W, H, n, orc.F64, vals, wrap=wrap), vals


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_world_with_z_normal_is_tangent_space(orc, filt):
    T, _ = textures(orc, 5, 4, 4, 1)
    rng = np.random.default_rng(2)
    F = 400
    uv = rng.uniform(0, 1, (F, 2)).astype(np.float32)
    d = unit_dirs(rng, F).astype(np.float32)
    N = np.tile(np.array([0, 0, 1], np.float32), (F, 1))
    obj = np.zeros(F, np.int32)
    a, fa = orc.shade([T], uv, d, obj, filt)
    b, fb = orc.shade_world([T], uv, d, N, obj, filt)
    assert fa == fb == 0
    np.testing.assert_array_equal(a, b)
    ia, ca, _ = orc.locate([T], uv, d, obj, filt)
    ib, cb, _ = orc.locate_world([T], uv, d, N, obj, filt)
    np.testing.assert_array_equal(ia, ib)
    np.testing.assert_array_equal(ca, cb)


def test_world_tilted_normal_closed_forms(orc):
    """N = (sin a, 0, cos a).  With I = N, A = sqrt(2) N_xy = (sqrt(2) sin a, 0).
    With I = +z, A = (sqrt(2) sin(a/2), 0).  In both cases B = A, since A has
    one nonzero axis, and the bilinear in-bucket coordinates are
    c = (B + 1) n/2 - 1/2."""
    n = 8
    T, _ = textures(orc, 2, 2, n, 3)
    for a in (0.05, 0.2, 0.4):
        N = np.array([np.sin(a), 0.0, np.cos(a)])
        for I, Ax in ((N, np.sqrt(2) * np.sin(a)), (np.array([0.0, 0.0, 1.0]), np.sqrt(2) * np.sin(a / 2))):
            _, c, _ = orc.locate_world([T], [[0.5, 0.5]], [I], [N], [0], 1)
            # locate_world takes FP32 inputs: compare at FP32 input precision
            assert abs(c[0, 2] - ((Ax + 1) * n / 2 - 0.5)) < 64 * n * 2.0 ** -24
            assert abs(c[0, 3] - ((0 + 1) * n / 2 - 0.5)) < 64 * n * 2.0 ** -24


def test_world_gradients_central_differences(orc):
    W, H, n = 6, 5, 6
    T, _ = textures(orc, W, H, n, 4)
    rng = np.random.default_rng(5)
    F = 60
    uv = rng.uniform(0.1, 0.9, (F, 2))
    I = unit_dirs(rng, F)
    N = unit_dirs(rng, F)
    N[:, 2] = np.abs(N[:, 2]) + 1.0
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    obj = np.zeros(F, np.int32)
    g = rng.normal(size=(F, 4))
    _, guv, gdir, gnrm, flags = orc.shade_world_backward([T], uv, I, N, obj, 2, g, want_tex=False,
                                                         precise_inputs=True)
    assert flags == 0
    np.testing.assert_array_equal(gdir, gnrm)  # A depends on I + N only
    _, c, _ = orc.locate_world([T], uv, I, N, obj, 2)
    far = (np.abs(c - np.round(c)) > 1e-3).all(axis=1)
    assert far.sum() > 30
    eps = 1e-7

    def L(uv_, I_, N_):
        out, _ = orc.shade_world([T], uv_, I_, N_, obj, 2, precise_inputs=True)
        return (out * g).sum(axis=1)

    for k in range(3):
        e = np.zeros((F, 3))
        e[:, k] = eps
        fd_I = (L(uv, I + e, N) - L(uv, I - e, N)) / (2 * eps)
        fd_N = (L(uv, I, N + e) - L(uv, I, N - e)) / (2 * eps)
        np.testing.assert_allclose(gdir[far, k], fd_I[far], rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(gnrm[far, k], fd_N[far], rtol=1e-5, atol=1e-6)
    for k in range(2):
        e = np.zeros((F, 2))
        e[:, k] = eps
        fd = (L(uv + e, I, N) - L(uv - e, I, N)) / (2 * eps)
        np.testing.assert_allclose(guv[far, k], fd[far], rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_wrap_is_periodic(orc, filt):
    T, _ = textures(orc, 8, 4, 4, 6, wrap=3)
    rng = np.random.default_rng(7)
    F = 300
    uv = np.round(rng.uniform(0, 1, (F, 2)) * 1024) / 1024  # dyadic: u + 1 is exact
    d = unit_dirs(rng, F)
    obj = np.zeros(F, np.int32)
    a, _ = orc.shade([T], uv, d, obj, filt, precise_inputs=True)
    for shift in ([1, 0], [0, 1], [-1, 2], [3, -2]):
        b, _ = orc.shade([T], uv + np.array(shift, float), d, obj, filt, precise_inputs=True)
        np.testing.assert_array_equal(a, b)


def brute_wrap(vals, W, H, n, u, v, I, filt):
    """brute_shade with periodic spatial kernels: bucket i collects the tents of
    every unwrapped position p with p mod size = i (nearest: the bucket whose
    repeated cell contains u)."""
    def spatial_w(x, size):
        w = np.zeros(size)
        if filt == 2:
            c = x * size - 0.5
            for p in range(int(np.floor(c)) - 3 * size, int(np.floor(c)) + 3 * size):
                w[p % size] += tent(c - p)
        else:
            w[int(np.floor(x * size)) % size] = 1.0
        return w

    # reuse the angular part of the clamp-mode brute force on a single-bucket slice
    wu, wv = spatial_w(u, W), spatial_w(v, H)
    Tv = vals.reshape(H, n, W, n, 4)
    out = np.zeros(4)
    for j in range(H):
        for i in range(W):
            if wu[i] == 0 or wv[j] == 0:
                continue
            bucket = Tv[j, :, i, :, :].reshape(n, n, 4)  # [t, s, c] as a 1 x 1 matrix
            out += wu[i] * wv[j] * brute_shade(bucket.reshape(n, n, 4), 1, 1, n, 0.5, 0.5, I, filt)
    return out


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_wrap_brute_force_tiny(orc, filt):
    rng = np.random.default_rng(20 + filt)
    for W, H, n in [(1, 1, 2), (2, 1, 3), (3, 2, 2), (2, 3, 4), (4, 4, 3)]:
        T, vals = textures(orc, W, H, n, 30 + W, wrap=3)
        F = 150
        uv = rng.uniform(-1.5, 2.5, (F, 2))
        uv[:4] = [[0, 0], [1, 1], [-0.5, 0.5], [0.125, 1.875]]
        d = unit_dirs(rng, F)
        out, flags = orc.shade([T], uv, d, np.zeros(F, np.int32), filt, precise_inputs=True)
        assert flags == 0
        for f in range(F):
            ref = brute_wrap(vals, W, H, n, uv[f, 0], uv[f, 1], d[f], filt)
            np.testing.assert_allclose(out[f], ref, atol=1e-13, err_msg=f"W{W} H{H} n{n} f{f}")


def test_wrap_equals_clamp_inside(orc):
    W, H, n = 8, 6, 4
    Tc, vals = textures(orc, W, H, n, 8)
    Tw = orc.Texture(W, H, n, orc.F64, vals, wrap=3)
    rng = np.random.default_rng(9)
    F = 300
    uv = np.stack([rng.uniform(0.5 / W, 1 - 0.5 / W, F), rng.uniform(0.5 / H, 1 - 0.5 / H, F)], 1)
    d = unit_dirs(rng, F)
    obj = np.zeros(F, np.int32)
    for filt in (0, 1, 2):
        a, _ = orc.shade([Tc], uv, d, obj, filt, precise_inputs=True)
        b, _ = orc.shade([Tw], uv, d, obj, filt, precise_inputs=True)
        np.testing.assert_array_equal(a, b)


def test_wrap_gradient_across_the_seam(orc):
    W, H, n = 8, 8, 4
    T, _ = textures(orc, W, H, n, 10, wrap=3)
    rng = np.random.default_rng(11)
    F = 40
    uv = np.stack([rng.uniform(-0.06, 0.06, F), rng.uniform(0.94, 1.06, F)], 1)  # around both seams
    d = unit_dirs(rng, F)
    obj = np.zeros(F, np.int32)
    g = rng.normal(size=(F, 4))
    _, guv, _, _ = orc.shade_backward([T], uv, d, obj, 2, g, want_tex=False, want_dir=False, precise_inputs=True)
    _, c, _ = orc.locate([T], uv.astype(np.float32), d.astype(np.float32), obj, 2)
    far = (np.abs(c[:, :2] - np.round(c[:, :2])) > 1e-3).all(axis=1)
    eps = 1e-7
    for k in range(2):
        e = np.zeros((F, 2))
        e[:, k] = eps
        lp, _ = orc.shade([T], uv + e, d, obj, 2, precise_inputs=True)
        lm, _ = orc.shade([T], uv - e, d, obj, 2, precise_inputs=True)
        fd = ((lp - lm) * g).sum(1) / (2 * eps)
        np.testing.assert_allclose(guv[far, k], fd[far], rtol=1e-5, atol=1e-6)
    assert (np.abs(guv[:, 0]) > 0).any()


@pytest.mark.parametrize("wrap", [1, 2])
def test_wrap_one_axis_only(orc, wrap):
    """Each repeat flag acts on its own axis (reading R12): with u repeating
    and v clamped (wrap = 1) a shift of u by a whole period leaves the colour
    unchanged while v beyond the edge reads the edge row; wrap = 2 the other
    way round."""
    W, H, n = 5, 3, 4
    T, _ = textures(orc, W, H, n, 60 + wrap, wrap=wrap)
    rng = np.random.default_rng(61)
    F = 300
    uv = rng.uniform(0.05, 0.95, (F, 2))
    d = unit_dirs(rng, F)
    obj = np.zeros(F, np.int32)
    rep, clamp = (0, 1) if wrap == 1 else (1, 0)
    base, _ = orc.shade([T], uv, d, obj, 2, precise_inputs=True)
    shifted = uv.copy()
    shifted[:, rep] += 3.0
    got, _ = orc.shade([T], shifted, d, obj, 2, precise_inputs=True)
    np.testing.assert_allclose(got, base, rtol=0, atol=1e-12)
    # the clamped axis: every coordinate beyond the far edge reads the edge
    far1, far2 = uv.copy(), uv.copy()
    far1[:, clamp] = 1.5
    far2[:, clamp] = 7.0
    a, _ = orc.shade([T], far1, d, obj, 2, precise_inputs=True)
    b, _ = orc.shade([T], far2, d, obj, 2, precise_inputs=True)
    np.testing.assert_array_equal(a, b)
    near = uv.copy()
    near[:, clamp] = uv[:, clamp] + 3.0 / [W, H][clamp]
    c, _ = orc.shade([T], near, d, obj, 2, precise_inputs=True)
    assert np.abs(c - base).max() > 1e-3  # not periodic along the clamped axis
