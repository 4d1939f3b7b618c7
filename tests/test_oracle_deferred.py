"""Pins of the oracle's deferred payloads (Section 1: a texel may hold data for
deferred rendering, such as ambient occlusion or reflections; reading R15):
the unlit albedo of the reflected ray's first hit and the ambient occlusion at
that hit over K given local directions.

- The basis around the hit normal is orthonormal and right-handed, at the poles
  and at the equator of the normal's sphere.
- Ambient occlusion at a point of the plane under the sphere tends to one minus
  the configuration factor of a sphere seen from a differential area,
  (r/d)^2 cos(theta) (a textbook closed form), under cosine-distributed
  directions; single directions along the normal give exact 0 / 1 cases.
- With ambient 1 and no fog, the radiance bake traces the hit's albedo, so the
  deferred albedo equals (radiance - own colour) / reflectance on every texel
  whose ray hits a surface.
- Texels whose ray misses everything hold (0, 0, 0, 1); texels whose ray hits
  the sphere (from plane buckets) or the plane (from sphere buckets) hold that
  surface's albedo and the occlusion at an independently solved hit point with
  the normal facing the ray."""
import numpy as np

import oracle
import synth

SPHERE, PLANE = oracle.SURFACE_SPHERE, oracle.SURFACE_PLANE


def test_basis_orthonormal_right_handed():
    rng = np.random.default_rng(1)
    N = rng.normal(size=(500, 3))
    N = np.concatenate([N, [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1, 0], [0, -1, 0], [0.6, 0.8, 0.0],
                            [0.6, 0.8, 1e-12], [0.6, 0.8, -1e-12], [1e-9, 0, -1.0]]])
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    b1, b2 = oracle.onb(N)
    for v in (b1, b2):
        np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-12)
        np.testing.assert_allclose(np.einsum("ij,ij->i", v, N), 0.0, atol=1e-12)
    np.testing.assert_allclose(np.einsum("ij,ij->i", b1, b2), 0.0, atol=1e-12)
    np.testing.assert_allclose(np.cross(b1, b2), N, atol=1e-12)


def test_ao_tends_to_one_minus_sphere_configuration_factor():
    dirs = synth.ao_directions(3, 40000)
    for h in (-1.0, -3.0):  # the plane touches the sphere, or lies two radii below it
        scene = synth.bake_scene(4, plane_height=h)
        for rho in (0.0, 0.5, 1.0, 2.0, 4.0):
            if h == -1.0 and rho == 0.0:
                continue  # the contact point itself
            X = np.array([rho, h, 0.0])
            D = -X  # towards the centre (the origin)
            d = np.linalg.norm(D)
            cos_t = D[1] / d
            F = cos_t / d ** 2  # r = 1: the whole sphere lies above the point's horizon
            ao = oracle.ambient_occlusion(scene, X, [0.0, 1.0, 0.0], dirs)[0]
            assert abs(ao - (1.0 - F)) < 4e-3, (h, rho, ao, 1.0 - F)


def test_ao_single_directions_exact():
    scene = synth.bake_scene(5, plane_height=-3.0)
    up = [[0.0, 0.0, 1.0]]
    # plane points: straight up from under the sphere is blocked, from far away it is free
    assert oracle.ambient_occlusion(scene, [0.0, -3.0, 0.0], [0, 1, 0], up)[0] == 0.0
    assert oracle.ambient_occlusion(scene, [2.5, -3.0, 0.0], [0, 1, 0], up)[0] == 1.0
    # sphere points: the outward normal reaches the plane from the bottom, the sky from the top
    assert oracle.ambient_occlusion(scene, [0.0, -1.0, 0.0], [0, -1, 0], up)[0] == 0.0
    assert oracle.ambient_occlusion(scene, [0.0, 1.0, 0.0], [0, 1, 0], up)[0] == 1.0
    # an equator point of the touching scene: every downward direction meets the plane
    scene = synth.bake_scene(5)
    dirs = synth.ao_directions(6, 256).astype(np.float64)
    N = np.array([1.0, 0.0, 0.0])
    b1, b2 = oracle.onb(N)
    world = dirs[:, :1] * b1 + dirs[:, 1:2] * b2 + dirs[:, 2:] * N
    ao = oracle.ambient_occlusion(scene, N, N, dirs)[0]
    assert ao == np.mean(world[:, 1] >= 0.0)


def test_deferred_albedo_is_the_traced_albedo_without_light_or_fog():
    scene = dict(synth.bake_scene(7), ambient=1.0, fog=0.0)
    dirs = synth.ao_directions(8, 16)
    W, H, n = 10, 8, 6
    for surface in (SPHERE, PLANE):
        val = oracle.bake_deferred(W, H, n, surface, scene, dirs, None)
        rad = oracle.bake(W, H, n, surface, scene, None)
        refl = scene["sphere_reflectance"] if surface == SPHERE else scene["plane_reflectance"]
        own = np.zeros((H * n, W * n, 3))
        for j in range(H):
            for i in range(W):
                u, v = (i + 0.5) / W, (j + 0.5) / H
                if surface == SPHERE:
                    own[j * n:(j + 1) * n, i * n:(i + 1) * n] = scene["sphere_albedo"]
                else:
                    e, w = scene["plane_half_extent"], scene["plane_frequency"]
                    x, z = 2 * e * u - e, 2 * e * v - e
                    own[j * n:(j + 1) * n, i * n:(i + 1) * n] = (np.array(scene["plane_albedo"])
                                                                 * (0.75 + 0.25 * np.cos(w * x) * np.cos(w * z)))
        hit = rad[..., 3] > 0.5  # transmittance 1 on a hit, 0 on the sky
        assert 0 < hit.mean() < 1
        want = (rad[..., :3] - own) / refl
        np.testing.assert_allclose(val[..., :3][hit], want[hit], atol=1e-12)
        assert (val[~hit] == [0.0, 0.0, 0.0, 1.0]).all()
        assert ((val[..., 3] >= 0) & (val[..., 3] <= 1)).all()


def test_deferred_texels_against_independent_hits():
    scene = synth.bake_scene(9)
    dirs = synth.ao_directions(10, 64)
    W, H, n = 16, 16, 8
    val, lo, hi = oracle.bake_deferred(W, H, n, PLANE, scene, dirs)
    checked = 0
    for j in range(H):
        for i in range(W):
            for t in range(n):
                for s in range(n):
                    P, d, _ = oracle.bake_ray(n, PLANE, scene, (i + 0.5) / W, (j + 0.5) / H, s, t)
                    b = P @ d  # sphere at the origin, r = 1
                    disc = b * b - (P @ P - 1.0)
                    v = val[j * n + t, i * n + s]
                    if disc <= 0:  # misses the sphere; upward rays leave the plane: the sky
                        assert (v == [0, 0, 0, 1]).all()
                        continue
                    X = P + (-b - np.sqrt(disc)) * d
                    np.testing.assert_array_equal(v[:3], scene["sphere_albedo"])
                    ao = oracle.ambient_occlusion(scene, X, X, dirs)[0]
                    assert lo[j * n + t, i * n + s, 3] - 1e-12 <= ao <= hi[j * n + t, i * n + s, 3] + 1e-12
                    assert abs(ao - v[3]) < 1e-9 or hi[j * n + t, i * n + s, 3] > lo[j * n + t, i * n + s, 3]
                    checked += 1
    assert checked > 100
    # sphere buckets: a reflected ray leaves the convex sphere and either meets the plane or the sky
    val_s, lo_s, hi_s = oracle.bake_deferred(W, H, n, SPHERE, scene, dirs)
    e, w, yp = scene["plane_half_extent"], scene["plane_frequency"], scene["plane_height"]
    aos = []
    for j in range(H):
        for i in range(W):
            for t in range(n):
                for s in range(n):
                    P, d, _ = oracle.bake_ray(n, SPHERE, scene, (i + 0.5) / W, (j + 0.5) / H, s, t)
                    v, a, z = (x[j * n + t, i * n + s] for x in (val_s, lo_s, hi_s))
                    if d[1] >= 0 or (yp - P[1]) / d[1] <= scene["ray_offset"]:
                        assert (v == [0, 0, 0, 1]).all()
                        continue
                    X = P + (yp - P[1]) / d[1] * d
                    m = 0.75 + 0.25 * np.cos(w * X[0]) * np.cos(w * X[2])
                    np.testing.assert_allclose(v[:3], np.array(scene["plane_albedo"]) * m, atol=1e-12)
                    ao = oracle.ambient_occlusion(scene, X, [0.0, 1.0, 0.0], dirs)[0]
                    assert a[3] - 1e-12 <= ao <= z[3] + 1e-12
                    aos.append(ao)
    assert len(aos) > 100 and min(aos) < 0.9  # hits near the sphere are partly occluded
    # the ranges hold the value, and texels whose range is wide stay rare
    assert ((lo <= val + 1e-15) & (val <= hi + 1e-15)).all()
    assert (np.max(hi - lo, axis=-1) > 1e-3).mean() < 0.02
