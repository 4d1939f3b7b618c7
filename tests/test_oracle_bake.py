"""Pins of the oracle's bake (Section 2.2, Eq. 4a and Eq. 4b; reading R10).

Each pin checks the oracle against something other than its own formulas:
the mirror law applied to the incidence direction of Eq. 2c (a different
route than Eq. 4b), finite differences of the surface parametrisation, closed
forms of single rays, the scene's mirror symmetry, and constant colours."""
import numpy as np
import pytest

import oracle
import synth

SPHERE, PLANE = oracle.SURFACE_SPHERE, oracle.SURFACE_PLANE


@pytest.fixture(scope="module")
def scene():
    return synth.bake_scene(11)


def sky_closed(sc, d):
    d = np.asarray(d, float)
    L = np.asarray(sc["sun_direction"])
    c = max(float(d @ L), 0.0)
    Kz, Kh, S = (np.asarray(sc[k]) for k in ("sky_zenith", "sky_horizon", "sun_rgb"))
    return Kh + (Kz - Kh) * (0.5 + 0.5 * d[1]) + S * c ** sc["sun_exponent"]


def lit_closed(sc, N):
    a = sc["ambient"]
    return a + (1 - a) * max(float(np.asarray(N) @ np.asarray(sc["sun_direction"])), 0.0)


def plane_albedo_closed(sc, x):
    w = sc["plane_frequency"]
    return np.asarray(sc["plane_albedo"]) * (0.75 + 0.25 * np.cos(w * x[0]) * np.cos(w * x[2]))


@pytest.mark.parametrize("surface", [SPHERE, PLANE])
def test_reflection_ray_is_mirror_of_incidence(scene, surface):
    """Eq. 4b's vector, taken to world space, is the mirror image about N of the
    Eq. 2c incidence direction of the same texel centre: d = 2 (N . I) N - I."""
    n = 7
    I_ts = oracle.texel_directions(n).reshape(n, n, 3)  # [t, s]
    rng = np.random.default_rng(3)
    for _ in range(40):
        u, v = rng.uniform(0.02, 0.98, 2)
        s, t = rng.integers(0, n, 2)
        P, d, F = oracle.bake_ray(n, surface, scene, u, v, s, t)
        I = I_ts[t, s] @ F  # world incidence
        N = F[2]
        np.testing.assert_allclose(d, 2 * (N @ I) * N - I, atol=1e-14)
        assert abs(np.linalg.norm(d) - 1) < 1e-14 and d @ N >= -1e-15


@pytest.mark.parametrize("surface", [SPHERE, PLANE])
def test_frame_follows_surface_derivatives(scene, surface):
    """T and B point along dP/du and dP/dv (central differences), N is the unit
    outward normal, and the frame is orthonormal."""
    h = 1e-6
    rng = np.random.default_rng(4)
    for _ in range(20):
        u, v = rng.uniform(0.05, 0.95, 2)
        P, _, F = oracle.bake_ray(4, surface, scene, u, v, 0, 0)
        np.testing.assert_allclose(F @ F.T, np.eye(3), atol=1e-14)
        du = oracle.bake_ray(4, surface, scene, u + h, v, 0, 0)[0] - oracle.bake_ray(4, surface, scene, u - h, v, 0, 0)[0]
        dv = oracle.bake_ray(4, surface, scene, u, v + h, 0, 0)[0] - oracle.bake_ray(4, surface, scene, u, v - h, 0, 0)[0]
        np.testing.assert_allclose(du / np.linalg.norm(du), F[0], atol=1e-8)
        np.testing.assert_allclose(dv / np.linalg.norm(dv), F[1], atol=1e-8)
        if surface == SPHERE:
            np.testing.assert_allclose(F[2], (P - np.asarray(scene["sphere_centre"])) / scene["sphere_radius"],
                                       atol=1e-14)
            assert abs(np.linalg.norm(P) - scene["sphere_radius"]) < 1e-14
        else:
            np.testing.assert_array_equal(F[2], [0.0, 1.0, 0.0])
            assert P[1] == scene["plane_height"]


def test_trace_closed_forms(scene):
    sc = dict(scene, plane_height=-2.0)
    fog = sc["fog"]
    up = np.array([0.0, 1.0, 0.0])
    # escapes to the sky
    out = oracle.trace(sc, [[0.0, 10.0, 0.0]], [up])[0]
    np.testing.assert_allclose(out[:3], sky_closed(sc, up), atol=1e-15)
    assert out[3] == 0.0
    # straight down onto the plane, clear of the sphere
    P = np.array([2.5, 3.0, -1.5])
    out = oracle.trace(sc, [P], [-up])[0]
    t = 3.0 - (-2.0)
    f = np.exp(-fog * t)
    C = plane_albedo_closed(sc, [2.5, -2.0, -1.5]) * lit_closed(sc, up)
    np.testing.assert_allclose(out[:3], f * C + (1 - f) * sky_closed(sc, -up), atol=1e-15)
    np.testing.assert_allclose(out[3], f, rtol=1e-15)
    # along -x onto the sphere's +x pole
    x = np.array([1.0, 0.0, 0.0])
    out = oracle.trace(sc, [[3.0, 0.0, 0.0]], [-x])[0]
    f = np.exp(-fog * 2.0)
    C = np.asarray(sc["sphere_albedo"]) * lit_closed(sc, x)
    np.testing.assert_allclose(out[:3], f * C + (1 - f) * sky_closed(sc, -x), atol=1e-15)
    # from the plane straight up: the sphere's bottom (t = 1) is nearer than anything else
    out = oracle.trace(sc, [[0.0, -2.0, 0.0]], [up])[0]
    f = np.exp(-fog * 1.0)
    C = np.asarray(sc["sphere_albedo"]) * lit_closed(sc, -up)
    np.testing.assert_allclose(out[:3], f * C + (1 - f) * sky_closed(sc, up), atol=1e-15)


def test_centre_texel_closed_form(scene):
    """Odd n: the centre texel has B = 0, so A = 0 and R = N (Eq. 4a, 4b).  On the
    plane a vertical ray clear of the sphere sees the zenith; on the sphere's
    upper half the outward ray sees the sky in direction N."""
    n, W, H = 5, 8, 8
    c = n // 2
    val = oracle.bake(W, H, n, PLANE, scene)
    e = scene["plane_half_extent"]
    for i, j in ((0, 0), (7, 2), (1, 6)):
        u, v = (i + 0.5) / W, (j + 0.5) / H
        x = np.array([2 * e * u - e, scene["plane_height"], 2 * e * v - e])
        assert np.hypot(x[0], x[2]) > scene["sphere_radius"]  # the vertical ray misses the sphere
        base = plane_albedo_closed(scene, x) * lit_closed(scene, [0, 1, 0])
        want = base + scene["plane_reflectance"] * sky_closed(scene, [0, 1, 0])
        np.testing.assert_allclose(val[j * n + c, i * n + c, :3], want, atol=1e-14)
        assert val[j * n + c, i * n + c, 3] == 0.0
    val = oracle.bake(W, H, n, SPHERE, scene)
    for i, j in ((0, 0), (5, 1), (3, 3)):
        u, v = (i + 0.5) / W, (j + 0.5) / H
        phi, theta = 2 * np.pi * u - np.pi, np.pi * v
        N = np.array([np.sin(theta) * np.cos(phi), np.cos(theta), np.sin(theta) * np.sin(phi)])
        base = np.asarray(scene["sphere_albedo"]) * lit_closed(scene, N)
        want = base + scene["sphere_reflectance"] * sky_closed(scene, N)
        np.testing.assert_allclose(val[j * n + c, i * n + c, :3], want, atol=1e-14)


@pytest.mark.parametrize("surface", [SPHERE, PLANE])
def test_zero_reflectance_gives_the_surface_colour(scene, surface):
    """With no reflection every texel of a bucket holds the surface's own lit
    colour, whatever its direction."""
    sc = dict(scene, sphere_reflectance=0.0, plane_reflectance=0.0)
    n, W, H = 4, 6, 5
    val = oracle.bake(W, H, n, surface, sc).reshape(H, n, W, n, 4)
    for j in range(H):
        for i in range(W):
            b = val[j, :, i, :, :3]
            assert np.ptp(b.reshape(-1, 3), axis=0).max() == 0.0
            P, _, F = oracle.bake_ray(n, surface, sc, (i + 0.5) / W, (j + 0.5) / H, 0, 0)
            alb = np.asarray(sc["sphere_albedo"]) if surface == SPHERE else plane_albedo_closed(sc, P)
            np.testing.assert_allclose(b[0, 0], alb * lit_closed(sc, F[2]), atol=1e-15)


def test_mirror_symmetry(scene):
    """With the sun in the x-y plane the scene is symmetric under z -> -z.  On the
    plane that maps bucket row j to H-1-j and in-bucket row t to n-1-t (the
    frame's y axis is +z), so the baked atlas is symmetric under both flips."""
    L = np.array(scene["sun_direction"])
    L[2] = 0.0
    sc = dict(scene, sun_direction=(L / np.linalg.norm(L)).tolist())
    n, W, H = 6, 10, 10
    val = oracle.bake(W, H, n, PLANE, sc).reshape(H, n, W, n, 4)
    np.testing.assert_allclose(val, val[::-1, ::-1], atol=1e-12)


def test_perturbation_range_brackets_value(scene):
    n, W, H = 8, 12, 12
    for surface in (SPHERE, PLANE):
        val, lo, hi = oracle.bake(W, H, n, surface, scene, 2.0 ** -17)
        assert (lo <= val).all() and (val <= hi).all()
        np.testing.assert_array_equal(val, oracle.bake(W, H, n, surface, scene))
