"""Pins of the oracle's shadow textures (Section 5, "Shadowing"; reading R13):
1-bit visibility towards each texel direction, keyed like a radiance texture by
a direction (the light's instead of the view's).

- The geometric occlusion test agrees with the radiance tracer: a ray is
  visible exactly when the tracer returns the sky (zero transmittance).
- Closed forms under the sphere and far from it.
- A constant bit texture filters to its constant, and filtered bits stay in
  [0, 1]."""
import numpy as np

import oracle
import synth

SPHERE, PLANE = oracle.SURFACE_SPHERE, oracle.SURFACE_PLANE


def test_visibility_agrees_with_the_tracer():
    scene = synth.bake_scene(21)
    W, H, n = 12, 10, 6
    I_ts = oracle.texel_directions(n)  # [t, s]
    for surface in (SPHERE, PLANE):
        vis, band = oracle.bake_shadow(W, H, n, surface, scene)
        rays_P, rays_d, want = [], [], []
        for j in range(H):
            for i in range(W):
                P, _, F = oracle.bake_ray(n, surface, scene, (i + 0.5) / W, (j + 0.5) / H, 0, 0)
                for t in range(n):
                    for s in range(n):
                        rays_P.append(P)
                        rays_d.append(I_ts[t, s] @ F)
                        want.append((vis[j * n + t, i * n + s], band[j * n + t, i * n + s]))
        alpha = oracle.trace(scene, np.array(rays_P), np.array(rays_d))[:, 3]
        want = np.array(want)
        ok = ~want[:, 1].astype(bool)
        assert ok.mean() > 0.97
        np.testing.assert_array_equal(want[ok, 0], (alpha[ok] == 0).astype(np.uint8))
        assert 0 < want[:, 0].mean() < 1  # both bits occur


def test_shadow_closed_forms():
    """Odd n: the centre texel points along N.  On the plane y = -2 (the sphere's
    bottom is at y = -1) a vertical ray from under the sphere is blocked, one
    from a far corner is not.  On the sphere the outward ray is free above the
    equator and hits the plane from the bottom cap."""
    scene = dict(synth.bake_scene(22), plane_height=-2.0)
    n, W, H = 5, 16, 16
    c = n // 2
    vis, _ = oracle.bake_shadow(W, H, n, PLANE, scene)
    # bucket under the sphere centre: x, z = 2 e u - e near 0
    i0 = W // 2
    assert vis[i0 * n + c, i0 * n + c] == 0
    assert vis[0 * n + c, 0 * n + c] == 1 and vis[(H - 1) * n + c, (W - 1) * n + c] == 1
    vis, _ = oracle.bake_shadow(W, H, n, SPHERE, scene)
    # rows j: theta = pi (j + 1/2) / H; upper rows see the sky, the bottom row sees the plane
    assert (vis[0 * n + c, c::n] == 1).all()
    assert (vis[(H - 1) * n + c, c::n] == 0).all()


def test_bit_texture_filters():
    rng = np.random.default_rng(3)
    W, H, n = 6, 5, 4
    ones = oracle.bit_texture(np.ones((H * n, W * n), np.uint8), W, H, n)
    bits = rng.integers(0, 2, (H * n, W * n)).astype(np.uint8)
    T = oracle.bit_texture(bits, W, H, n)
    F = 500
    uv = rng.uniform(-0.1, 1.1, (F, 2))
    z = rng.uniform(0, 1, F)
    phi = rng.uniform(0, 2 * np.pi, F)
    d = np.stack([np.sqrt(1 - z * z) * np.cos(phi), np.sqrt(1 - z * z) * np.sin(phi), z], 1)
    obj = np.zeros(F, np.int32)
    for filt in (0, 1, 2):
        out, flags = oracle.shade([ones], uv, d, obj, filt, precise_inputs=True)
        assert flags == 0
        np.testing.assert_allclose(out, 1.0, rtol=0, atol=1e-15)  # the plain weighted sum: weights add to 1
        out, _ = oracle.shade([T], uv, d, obj, filt, precise_inputs=True)
        assert (out >= -1e-15).all() and (out <= 1 + 1e-15).all()
        assert (out[:, 0] == out[:, 3]).all()
    # nearest returns the bit of the selected texel
    idx, _, _ = oracle.locate([T], uv.astype(np.float32), d.astype(np.float32), obj, 0)
    out, _ = oracle.shade([T], uv.astype(np.float32), d.astype(np.float32), obj, 0)
    i = np.clip(idx[:, 0], 0, W - 1)
    j = np.clip(idx[:, 1], 0, H - 1)
    s = np.clip(idx[:, 2], 0, n - 1)
    t = np.clip(idx[:, 3], 0, n - 1)
    np.testing.assert_array_equal(out[:, 0], bits[j * n + t, i * n + s])
