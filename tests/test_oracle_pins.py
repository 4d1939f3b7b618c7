"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here re-types the oracle's formulas: every expected value comes from a
closed form the paper states (Section 2: |A| = sqrt(2) sin(theta/2), the
azimuthal and radial nature of Eq. 1b and Eq. 3), from an identity derived
from them, from an independent library routine (numpy / torch format
conversions), from brute force over all texels, or from finite differences.
"""
import math
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def unit_dirs(rng, k, lower=False):
    """Unit vectors, uniform on the upper hemisphere (or on the whole sphere)."""
    z = rng.uniform(-1.0 if lower else 0.0, 1.0, k)
    phi = rng.uniform(0, 2 * np.pi, k)
    r = np.sqrt(1 - z * z)
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], 1)


# ----------------------------------------------------------------------------
# Golden special values (hand-derived, tests/golden/mapping_special_values.txt)
# ----------------------------------------------------------------------------

def _golden_rows():
    env = {k: getattr(math, k) for k in ("sqrt", "sin", "cos", "tan", "pi")}
    rows = []
    with open(os.path.join(GOLDEN, "mapping_special_values.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = [p.split() for p in line.split("|")]
            vals = [[eval(x, {"__builtins__": {}}, env) for x in p] for p in parts]
            rows.append(vals)
    return rows


def test_golden_special_values(orc):
    rows = _golden_rows()
    assert len(rows) >= 8
    I = np.array([r[0] for r in rows])
    A = orc.equisolid(I)
    B = orc.squarify(A)
    np.testing.assert_allclose(A, np.array([r[1] for r in rows]), atol=1e-15)
    np.testing.assert_allclose(B, np.array([r[2] for r in rows]), atol=1e-15)


# ----------------------------------------------------------------------------
# Eq. 1b, Eq. 3 and their inverses
# ----------------------------------------------------------------------------

def test_eq1b_trig_form(orc):
    """Section 2: the projection radius is sqrt(2) sin(theta/2) along the azimuth phi."""
    rng = np.random.default_rng(1)
    theta = rng.uniform(0, np.pi / 2, 5000)
    phi = rng.uniform(-np.pi, np.pi, 5000)
    I = np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], 1)
    A = orc.equisolid(I)
    expect = np.sqrt(2) * np.sin(theta / 2)[:, None] * np.stack([np.cos(phi), np.sin(phi)], 1)
    np.testing.assert_allclose(A, expect, atol=2e-15)


def test_eq3_closed_form_and_ring_identity(orc):
    """For unit I: |A|^2 = 1 - I_z, so Eq. 3 gives B = sqrt(1 - I_z) I_xy / max(|I_x|, |I_y|)
    and max(|B_x|, |B_y|)^2 = 1 - I_z (rings of equal incidence map to squares)."""
    rng = np.random.default_rng(2)
    I = unit_dirs(rng, 20000, lower=True)
    B = orc.squarify(orc.equisolid(I))
    expect = np.sqrt(1 - I[:, 2])[:, None] * I[:, :2] / np.max(np.abs(I[:, :2]), 1, keepdims=True)
    np.testing.assert_allclose(B, expect, atol=1e-14)
    np.testing.assert_allclose(np.max(np.abs(B), 1) ** 2, 1 - I[:, 2], atol=1e-14)
    # B is along A (radial): cross product zero, same direction
    A = orc.equisolid(I)
    np.testing.assert_allclose(A[:, 0] * B[:, 1] - A[:, 1] * B[:, 0], 0, atol=1e-15)
    assert np.all(A[:, 0] * B[:, 0] + A[:, 1] * B[:, 1] >= 0)


def test_eq3_eq4a_mutual_inverses(orc):
    rng = np.random.default_rng(3)
    B = rng.uniform(-1, 1, (20000, 2))
    B[:5] = [[0, 0], [1, 0], [0, -1], [1, 1], [-1, 0.25]]
    np.testing.assert_allclose(orc.squarify(orc.unsquarify(B)), B, atol=1e-15)
    A = orc.unsquarify(B)
    assert np.all(np.hypot(A[:, 0], A[:, 1]) <= 1 + 1e-15)  # square [-1,1]^2 onto the unit disc
    np.testing.assert_allclose(orc.unsquarify(orc.squarify(A)), A, atol=1e-15)
    # a circle of radius r maps onto the boundary of the square of half-side r
    r = 0.37
    ang = np.linspace(0, 2 * np.pi, 1000)
    C = r * np.stack([np.cos(ang), np.sin(ang)], 1)
    np.testing.assert_allclose(np.max(np.abs(orc.squarify(C)), 1), r, atol=1e-15)


def test_eq2c_inverts_eq1b(orc):
    rng = np.random.default_rng(4)
    I = unit_dirs(rng, 20000)
    np.testing.assert_allclose(orc.equisolid_inverse(orc.equisolid(I)), I, atol=2e-15)
    A = orc.unsquarify(rng.uniform(-1, 1, (5000, 2)))
    I2 = orc.equisolid_inverse(A)
    np.testing.assert_allclose(np.linalg.norm(I2, axis=1), 1, atol=1e-15)  # unit directions
    assert np.all(I2[:, 2] >= -1e-15)  # the unit disc is the upper hemisphere
    np.testing.assert_allclose(orc.equisolid(I2), A, atol=2e-15)


def test_eq1a_general_normal(orc):
    """With N = z, Eq. 1a's first two entries are Eq. 1b and the third is sqrt(2) cos(theta/2)."""
    rng = np.random.default_rng(5)
    I = unit_dirs(rng, 5000)
    A3 = orc.equisolid_normal(I, [0, 0, 1])
    np.testing.assert_allclose(A3[:, :2], orc.equisolid(I), atol=2e-15)
    theta = np.arccos(np.clip(I[:, 2], -1, 1))
    np.testing.assert_allclose(A3[:, 2], np.sqrt(2) * np.cos(theta / 2), atol=2e-15)
    # for any unit normal, the result is sqrt(2) times the unit bisector of I and N
    N = unit_dirs(rng, 5000, lower=True)
    A3 = orc.equisolid_normal(I, N)
    np.testing.assert_allclose(np.linalg.norm(A3, axis=1), np.sqrt(2), atol=1e-14)
    cosI = np.sum(A3 * I, 1)
    cosN = np.sum(A3 * N, 1)
    np.testing.assert_allclose(cosI, cosN, atol=1e-13)


def test_eq2ab_general_normal(orc):
    """Eq. 2a-2b reflect N about the half vector A': with N = z they equal Eq. 2c;
    for any unit N the result is a unit vector making equal angles with A'."""
    rng = np.random.default_rng(6)
    A = orc.unsquarify(rng.uniform(-1, 1, (5000, 2)))
    np.testing.assert_allclose(orc.equisolid_inverse_normal(A, [0, 0, 1]), orc.equisolid_inverse(A), atol=2e-15)
    N = unit_dirs(rng, 5000, lower=True)
    I = orc.equisolid_inverse_normal(A, N)
    np.testing.assert_allclose(np.linalg.norm(I, axis=1), 1, atol=1e-14)
    Ap = np.stack([A[:, 0] / np.sqrt(2), A[:, 1] / np.sqrt(2), np.sqrt(1 - np.sum(A * A, 1) / 2)], 1)
    np.testing.assert_allclose(np.sum(Ap * I, 1), np.sum(Ap * N, 1), atol=1e-14)


def test_eq4b_is_mirror_of_eq2c(orc):
    """Eq. 4b: the reflection vector is the Eq. 2c direction mirrored about the normal,
    R = 2 (I . N) N - I with N = z."""
    rng = np.random.default_rng(7)
    A = orc.unsquarify(rng.uniform(-1, 1, (5000, 2)))
    I = orc.equisolid_inverse(A)
    R = orc.reflection(A)
    N = np.array([0.0, 0.0, 1.0])
    np.testing.assert_allclose(R, 2 * (I @ N)[:, None] * N[None, :] - I, atol=1e-15)


def test_equal_area(orc):
    """Section 2: the equisolid projection preserves area -> uniform directions on the
    hemisphere map to a uniform density on the unit disc: |A|^2 ~ U[0, 1] and the
    azimuth is uniform."""
    rng = np.random.default_rng(8)
    I = unit_dirs(rng, 200000)
    A = orc.equisolid(I)
    r2 = np.sum(A * A, 1)
    assert abs(r2.mean() - 0.5) < 0.005
    hist, _ = np.histogram(r2, bins=20, range=(0, 1))
    expect = len(r2) / 20
    chi2 = np.sum((hist - expect) ** 2 / expect)
    assert chi2 < 50  # 19 dof; p ~ 1e-4
    # sub-disc areas: fraction inside radius rho equals rho^2
    for rho in (0.25, 0.5, 0.75):
        assert abs(np.mean(r2 <= rho * rho) - rho * rho) < 0.005


def test_texel_centres_and_clamp(orc):
    """Note after Eq. 3: the clamp range [1/n - 1, 1 - 1/n] is exactly the first and
    last texel centre of B_k = (2k + 1)/n - 1; the directions of the centres come back
    to the centres through Eq. 1b and Eq. 3."""
    for n in (1, 2, 3, 8, 16, 32):
        centres = (2 * np.arange(n) + 1) / n - 1
        assert centres[0] == pytest.approx(1 / n - 1, abs=1e-15)
        assert centres[-1] == pytest.approx(1 - 1 / n, abs=1e-15)
        dirs = orc.texel_directions(n)
        B = orc.squarify(orc.equisolid(dirs.reshape(-1, 3))).reshape(n, n, 2)
        np.testing.assert_allclose(B[..., 0], np.broadcast_to(centres[None, :], (n, n)), atol=1e-14)
        np.testing.assert_allclose(B[..., 1], np.broadcast_to(centres[:, None], (n, n)), atol=1e-14)


# ----------------------------------------------------------------------------
# Shading: texel centres, constants, brute force
# ----------------------------------------------------------------------------

def field_numpy(lobes, u, v, I):
    """The synthetic multi-lobe field, evaluated independently of the oracle."""
    out = np.zeros((len(u), 4))
    for P in lobes:
        spatial = 0.5 + 0.5 * np.cos(2 * np.pi * (P[4] * u + P[5] * v) + P[6])
        c = I @ P[7:10]
        lobe = np.where(c > 0, np.maximum(c, 0) ** P[10], 0.0)
        out += P[None, 0:4] * (spatial * lobe)[:, None]
    return out


def trig_centre_dir(s, t, n):
    """Direction of texel centre (s, t) from the paper's closed forms only:
    ring radius |A| = max(|B_x|, |B_y|) (Eq. 3 maps circles to squares), azimuth
    of B (radial), theta = 2 asin(|A| / sqrt 2) (Section 2)."""
    Bx = (2 * s + 1) / n - 1
    By = (2 * t + 1) / n - 1
    rA = np.maximum(np.abs(Bx), np.abs(By))
    phi = np.arctan2(By, Bx)
    theta = 2 * np.arcsin(rA / np.sqrt(2))
    return np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], -1)


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_texel_centre_reproduction(orc, filt):
    """A texture filled from an analytic field is reproduced exactly at bucket and texel centres."""
    W, H, n = 7, 5, 6
    lobes = synth.field_lobes(11)
    atlas = orc.fill_field(W, H, n, lobes)
    T = orc.Texture.from_f32(atlas, W, H, n, orc.F32)
    jj, ii, tt, ss = np.meshgrid(np.arange(H), np.arange(W), np.arange(n), np.arange(n), indexing="ij")
    ii, jj, ss, tt = (x.reshape(-1) for x in (ii, jj, ss, tt))
    uv = np.stack([(ii + 0.5) / W, (jj + 0.5) / H], 1)
    d = trig_centre_dir(ss, tt, n)
    out, flags = orc.shade([T], uv, d, np.zeros(len(ii), np.int32), filt, precise_inputs=True)
    assert flags == 0
    expect = field_numpy(lobes, uv[:, 0], uv[:, 1], d).astype(np.float32).astype(np.float64)
    if filt == 0:
        np.testing.assert_array_equal(out, expect)  # bitwise
    else:
        assert np.max(np.abs(out - expect)) <= 1e-12  # exact up to FP64 rounding of the weights


@pytest.mark.parametrize("fmt", [0, 1, 2, 3])
@pytest.mark.parametrize("filt", [0, 1, 2])
def test_constant_texture(orc, fmt, filt):
    """A constant texture returns that constant for every UV and direction."""
    W, H, n = 5, 3, 4
    c = np.array([0.25, 0.5, 0.75, 1.0], np.float32)
    atlas = np.broadcast_to(c, (H * n, W * n, 4)).copy()
    T = orc.Texture.from_f32(atlas, W, H, n, fmt)
    rng = np.random.default_rng(9)
    F = 4000
    uv = rng.uniform(-0.5, 1.5, (F, 2))
    d = unit_dirs(rng, F, lower=True)
    d[:3] = [[0, 0, 1], [0, 0, -1], [1, 0, 0]]
    out, flags = orc.shade([T], uv, d, np.zeros(F, np.int32), filt)
    assert flags == 0
    expect = T.values()[0, 0]
    np.testing.assert_allclose(out, np.broadcast_to(expect, out.shape), rtol=1e-15, atol=0)


def tent(x):
    return np.maximum(0.0, 1.0 - np.abs(x))


def brute_shade(vals, W, H, n, u, v, I, filt):
    """Brute force over every texel of the bucket matrix.

    B from the closed form sqrt(1 - I_z) I_xy / max(|I_x|, |I_y|) (unit I);
    spatial weights: clamped tent kernels sum_{p: clamp(p) = i} tent(u W - 1/2 - p);
    angular weights: tent kernels of width 2/n around the texel centres in B units;
    nearest: argmin of the distance to the centres, ties to the higher index."""
    m = max(abs(I[0]), abs(I[1]))
    B = np.zeros(2) if m == 0 else np.sqrt(max(0.0, 1 - I[2])) * np.array(I[:2]) / m
    Bc = np.clip(B, 1 / n - 1, 1 - 1 / n)
    centres = (2 * np.arange(n) + 1) / n - 1

    def spatial_w(x, size):
        if filt == 2:
            c = min(max(x * size - 0.5, -1.0), float(size))
            w = np.zeros(size)
            for p in range(-3, size + 3):
                w[min(max(p, 0), size - 1)] += tent(c - p)
            return w
        w = np.zeros(size)
        cen = (np.arange(size) + 0.5) / size
        dist = np.abs(min(max(x, 0.0), 1.0) - cen)
        best = np.flatnonzero(dist == dist.min()).max()
        w[best] = 1.0
        return w

    def angular_w(b):
        if filt >= 1:
            return tent((b - centres) * n / 2)
        w = np.zeros(n)
        dist = np.abs(b - centres)
        w[np.flatnonzero(dist == dist.min()).max()] = 1.0
        return w

    wu, wv = spatial_w(u, W), spatial_w(v, H)
    ws, wt = angular_w(Bc[0]), angular_w(Bc[1])
    # vals: atlas (H n) x (W n) x 4 -> [j, t, i, s, c]
    T = vals.reshape(H, n, W, n, 4)
    return np.einsum("j,t,i,s,jtisc->c", wv, wt, wu, ws, T)


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_brute_force_tiny(orc, filt):
    rng = np.random.default_rng(10 + filt)
    for W, H, n in [(1, 1, 1), (1, 2, 2), (2, 1, 3), (3, 2, 4), (2, 3, 2), (3, 3, 3), (4, 2, 4)]:
        vals = rng.uniform(0, 1, (H * n, W * n, 4))
        T = orc.Texture(W, H, n, orc.F64, vals)
        F = 300
        uv = rng.uniform(-0.25, 1.25, (F, 2))
        uv[:20] = rng.uniform(0, 1, (20, 2))
        # dyadic bucket boundaries and the ends of [0, 1]
        uv[20:26] = [[0, 0], [1, 1], [0.5, 0.5], [0.25, 0.75], [1, 0], [0.125, 0.875]]
        d = unit_dirs(rng, F, lower=True)
        d[:6] = [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, -1, 0], [np.sqrt(0.5), np.sqrt(0.5), 0], [0.6, 0, 0.8]]
        out, flags = orc.shade([T], uv, d, np.zeros(F, np.int32), filt, precise_inputs=True)
        assert flags == 0
        for f in range(F):
            ref = brute_shade(vals, W, H, n, uv[f, 0], uv[f, 1], d[f], filt)
            np.testing.assert_allclose(out[f], ref, atol=1e-14, err_msg=f"W{W} H{H} n{n} f{f}")


def test_background_and_errors(orc):
    W, H, n = 2, 2, 2
    T = orc.Texture.from_f32(np.ones((H * n, W * n, 4), np.float32), W, H, n, orc.F32)
    uv = np.array([[0.5, 0.5]] * 5, np.float32)
    d = np.array([[0, 0, 1]] * 5, np.float32)
    d[3, 0] = np.nan
    obj = np.array([-1, 0, 1, 0, -7], np.int32)
    out, flags = orc.shade([T, None], uv, d, obj, 2)
    np.testing.assert_array_equal(out[:, 0], [0, 1, 0, 0, 0])
    assert flags == orc.FLAG_BAD_OBJ | orc.FLAG_NONFINITE


# ----------------------------------------------------------------------------
# Gradients
# ----------------------------------------------------------------------------

def _kink_free(orc, W, H, n, uv, d, margin):
    """Mask of fragments at least `margin` away from every kink of the quadrilinear lookup."""
    I = d
    m = np.max(np.abs(I[:, :2]), 1)
    B = np.sqrt(np.maximum(0, 1 - I[:, 2]))[:, None] * I[:, :2] / m[:, None]
    lo, hi = 1 / n - 1, 1 - 1 / n
    cu = uv[:, 0] * W - 0.5
    cv = uv[:, 1] * H - 0.5
    cs = (np.clip(B[:, 0], lo, hi) + 1) * n / 2 - 0.5
    ct = (np.clip(B[:, 1], lo, hi) + 1) * n / 2 - 0.5
    ok = np.ones(len(uv), bool)
    for c, scale in ((cu, W), (cv, H), (cs, n / 2), (ct, n / 2)):
        ok &= np.abs(c - np.round(c)) > margin * scale * 4
    for b in (B[:, 0], B[:, 1]):
        ok &= (np.abs(b - lo) > margin * 4) & (np.abs(b - hi) > margin * 4)
    ok &= np.abs(np.abs(I[:, 0]) - np.abs(I[:, 1])) > margin * 8
    ok &= np.hypot(I[:, 0], I[:, 1]) > margin * 8
    return ok


@pytest.mark.parametrize("filt", [1, 2])
def test_gradient_uv_dir_vs_fd(orc, filt):
    """Analytic FP64 dL/duv and dL/ddir against central differences (eps 1e-7)."""
    rng = np.random.default_rng(20 + filt)
    W, H, n = 6, 5, 8
    vals = rng.uniform(0, 1, (H * n, W * n, 4))
    T = orc.Texture(W, H, n, orc.F64, vals)
    F = 400
    uv = rng.uniform(0.02, 0.98, (F, 2))
    d = unit_dirs(rng, F)
    d[:, 2] = np.maximum(d[:, 2], 0.05)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    g = rng.normal(size=(F, 4))
    obj = np.zeros(F, np.int32)
    _, guv, gdir, flags = orc.shade_backward([T], uv, d, obj, filt, g, want_tex=False, precise_inputs=True)
    assert flags == 0
    eps = 1e-7
    ok = _kink_free(orc, W, H, n, uv, d, 1e-5)
    assert ok.sum() > 250

    def L(uv_, d_):
        out, _ = orc.shade([T], uv_, d_, obj, filt, precise_inputs=True)
        return np.sum(out * g, 1)

    for k in range(2):
        e = np.zeros_like(uv)
        e[:, k] = eps
        fd = (L(uv + e, d) - L(uv - e, d)) / (2 * eps)
        np.testing.assert_allclose(guv[ok, k], fd[ok], rtol=1e-6, atol=1e-6 * (W + H))
    for k in range(3):
        e = np.zeros_like(d)
        e[:, k] = eps
        fd = (L(uv, d + e) - L(uv, d - e)) / (2 * eps)
        np.testing.assert_allclose(gdir[ok, k], fd[ok], rtol=1e-6, atol=1e-6 * n)


@pytest.mark.parametrize("filt", [1, 2])
def test_gradient_zero_through_the_clamp(orc, filt):
    """Inside the Note's clamp zone (|B| beyond the outer texel centre 1 - 1/n)
    the colour does not change with the clamped component of B, so dL/ddir
    equals central differences there too: the clamped axis contributes nothing,
    the other axis its usual derivative (reading R6).  At the low clamp the
    floor branch of the in-bucket coordinate would otherwise pass the texel
    difference through."""
    rng = np.random.default_rng(40 + filt)
    W, H, n = 5, 4, 8
    T = orc.Texture(W, H, n, orc.F64, rng.uniform(0, 1, (H * n, W * n, 4)))
    F = 200
    far = rng.uniform(0.9, 0.99, F) * rng.choice([-1.0, 1.0], F)  # beyond 1 - 1/n = 0.875
    free = rng.uniform(-0.8, 0.8, F)
    # keep the free component's in-bucket coordinate away from integers
    c = (free + 1) * n / 2 - 0.5
    free = np.where(np.abs(c - np.round(c)) < 0.05, free + 0.2 / n, free)
    axis = rng.integers(0, 2, F)
    B = np.where(axis[:, None] == 0, np.stack([far, free], 1), np.stack([free, far], 1))
    d = orc.equisolid_inverse(orc.unsquarify(B))
    assert np.all(d[:, 2] > 0.0)
    uv = rng.uniform(0.05, 0.95, (F, 2))
    cu, cv = uv[:, 0] * W - 0.5, uv[:, 1] * H - 0.5
    uv[:, 0] += np.where(np.abs(cu - np.round(cu)) < 0.05, 0.1 / W, 0.0)
    uv[:, 1] += np.where(np.abs(cv - np.round(cv)) < 0.05, 0.1 / H, 0.0)
    g = rng.normal(size=(F, 4))
    obj = np.zeros(F, np.int32)
    _, _, gdir, flags = orc.shade_backward([T], uv, d, obj, filt, g, want_tex=False, precise_inputs=True)
    assert flags == 0

    def L(d_):
        out, _ = orc.shade([T], uv, d_, obj, filt, precise_inputs=True)
        return np.sum(out * g, 1)

    eps = 1e-7
    for k in range(3):
        e = np.zeros_like(d)
        e[:, k] = eps
        fd = (L(d + e) - L(d - e)) / (2 * eps)
        np.testing.assert_allclose(gdir[:, k], fd, rtol=1e-6, atol=1e-6 * n)
    # not vacuous: the free axis still carries a gradient
    assert np.abs(gdir).max() > 1e-3


@pytest.mark.parametrize("filt", [1, 2])
def test_gradient_at_eq3_ties_takes_the_x_branch(orc, filt):
    """At |A_x| = |A_y| Eq. 3 has a kink; reading R6 takes the x branch
    (B = A |A| / |A_x|).  The oracle's dL/ddir at exact ties equals central
    differences taken just inside the x-dominant side, and differs from the
    y-dominant side's."""
    rng = np.random.default_rng(50 + filt)
    W, H, n = 4, 4, 8
    T = orc.Texture(W, H, n, orc.F64, rng.uniform(0, 1, (H * n, W * n, 4)))
    F = 60
    a = rng.uniform(0.15, 0.6, F)
    sx, sy = rng.choice([-1.0, 1.0], F), rng.choice([-1.0, 1.0], F)
    d = np.stack([sx * a, sy * a, np.sqrt(1 - 2 * a * a)], 1)
    assert np.all(np.abs(d[:, 0]) == np.abs(d[:, 1]))
    uv = rng.uniform(0.1, 0.9, (F, 2))
    g = rng.normal(size=(F, 4))
    obj = np.zeros(F, np.int32)
    # keep every in-bucket coordinate away from integers and the clamp
    B = orc.squarify(orc.equisolid(d))
    c = (B + 1) * n / 2 - 0.5
    keep = (np.abs(c - np.round(c)) > 0.02).all(1) & (np.abs(B) < 1 - 1.0 / n - 0.02).all(1)
    d, uv, g, obj = d[keep], uv[keep], g[keep], obj[keep]
    assert len(obj) > 20
    _, _, gdir, flags = orc.shade_backward([T], uv, d, obj, filt, g, want_tex=False, precise_inputs=True)
    assert flags == 0

    def L(d_):
        out, _ = orc.shade([T], uv, d_, obj, filt, precise_inputs=True)
        return np.sum(out * g, 1)

    delta, eps = 1e-6, 1e-9

    def fd_at(shift):
        base = d + shift
        out = np.empty_like(d)
        for k in range(3):
            e = np.zeros_like(d)
            e[:, k] = eps
            out[:, k] = (L(base + e) - L(base - e)) / (2 * eps)
        return out

    x_side = np.zeros_like(d)
    x_side[:, 0] = delta * np.sign(d[:, 0])  # |I_x| > |I_y|: |A_x| > |A_y|
    y_side = np.zeros_like(d)
    y_side[:, 1] = delta * np.sign(d[:, 1])
    fx, fy = fd_at(x_side), fd_at(y_side)
    scale = np.abs(fx).max()
    np.testing.assert_allclose(gdir, fx, rtol=0, atol=1e-4 * scale)
    assert np.abs(gdir - fy).max() > 1e-2 * scale


def test_gradient_nearest_is_zero(orc):
    rng = np.random.default_rng(30)
    W, H, n = 3, 3, 4
    T = orc.Texture(W, H, n, orc.F64, rng.uniform(0, 1, (H * n, W * n, 4)))
    F = 100
    uv = rng.uniform(0, 1, (F, 2))
    d = unit_dirs(rng, F)
    _, guv, gdir, _ = orc.shade_backward([T], uv, d, np.zeros(F, np.int32), 0, rng.normal(size=(F, 4)),
                                         want_tex=False, precise_inputs=True)
    assert np.all(guv == 0) and np.all(gdir == 0)


@pytest.mark.parametrize("filt", [0, 1, 2])
def test_gradient_texels_vs_fd(orc, filt):
    """L = sum g . colour is linear in the texels, so a central difference is exact up to rounding."""
    rng = np.random.default_rng(40 + filt)
    W, H, n = 4, 3, 4
    vals = rng.uniform(0, 1, (H * n, W * n, 4))
    F = 300
    uv = rng.uniform(-0.1, 1.1, (F, 2))
    d = unit_dirs(rng, F, lower=True)
    obj = np.zeros(F, np.int32)
    obj[:10] = -1
    g = rng.normal(size=(F, 4))
    T = orc.Texture(W, H, n, orc.F64, vals)
    gtex, _, _, _ = orc.shade_backward([T], uv, d, obj, filt, g, want_uv=False, want_dir=False,
                                       precise_inputs=True)
    eps = 1e-3
    flat = vals.reshape(-1)
    for e in rng.choice(flat.size, 60, replace=False):
        vp = flat.copy()
        vm = flat.copy()
        vp[e] += eps
        vm[e] -= eps
        op, _ = orc.shade([orc.Texture(W, H, n, orc.F64, vp.reshape(vals.shape))], uv, d, obj, filt,
                          precise_inputs=True)
        om, _ = orc.shade([orc.Texture(W, H, n, orc.F64, vm.reshape(vals.shape))], uv, d, obj, filt,
                          precise_inputs=True)
        fd = np.sum((op - om) * g) / (2 * eps)
        assert abs(gtex[0].reshape(-1)[e] - fd) < 1e-9 * max(1.0, abs(fd))


def test_gradient_texels_sum_rule(orc):
    """The weights of every fragment sum to 1, so the texel gradient, summed per
    channel, equals the sum of dL/dout over shaded fragments."""
    rng = np.random.default_rng(50)
    W, H, n = 5, 4, 3
    T = orc.Texture(W, H, n, orc.F64, rng.uniform(0, 1, (H * n, W * n, 4)))
    F = 500
    uv = rng.uniform(-0.2, 1.2, (F, 2))
    d = unit_dirs(rng, F, lower=True)
    obj = np.where(rng.uniform(size=F) < 0.2, -1, 0).astype(np.int32)
    g = rng.normal(size=(F, 4))
    gtex, _, _, _ = orc.shade_backward([T], uv, d, obj, 2, g, want_uv=False, want_dir=False, precise_inputs=True)
    np.testing.assert_allclose(gtex[0].reshape(-1, 4).sum(0), g[obj >= 0].sum(0), atol=1e-10)


# ----------------------------------------------------------------------------
# Storage formats
# ----------------------------------------------------------------------------

def _probe_floats(rng):
    x = np.concatenate([
        rng.uniform(-1, 1, 20000),
        rng.uniform(-70000, 70000, 5000),
        np.exp(rng.uniform(np.log(1e-9), np.log(1e-3), 5000)) * rng.choice([-1, 1], 5000),
        np.array([0.0, -0.0, 1.0, 65504.0, 65519.99, 65520.0, 1e-8, 2 ** -24, 2 ** -25, 3 * 2 ** -26]),
    ]).astype(np.float32)
    # exact ties between FP16 neighbours
    h = rng.uniform(-2, 2, 2000).astype(np.float16)
    nxt = np.nextafter(h, np.float16(np.inf))
    ties = ((h.astype(np.float64) + nxt.astype(np.float64)) / 2).astype(np.float32)
    return np.concatenate([x, ties])


def test_f16_encoder_matches_numpy(orc):
    rng = np.random.default_rng(60)
    x = _probe_floats(rng)
    ours = orc.encode(orc.F16, x)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).view(np.uint16)
    np.testing.assert_array_equal(ours, ref)
    np.testing.assert_array_equal(orc.decode(orc.F16, ref), ref.view(np.float16).astype(np.float64))


def test_bf16_encoder_matches_torch(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(61)
    x = np.concatenate([_probe_floats(rng), rng.normal(size=20000).astype(np.float32) * 1e30,
                        np.array([3.3895314e38, 3.39e38], np.float32)])
    # exact BF16 ties
    b = (rng.integers(0, 2 ** 16, 5000, dtype=np.uint32) << 16).view(np.float32)
    b = b[np.isfinite(b)]
    ties = (b.view(np.uint32) | np.uint32(0x8000)).view(np.float32)
    x = np.concatenate([x, ties])
    ours = orc.encode(orc.BF16, x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(ours, ref)
    np.testing.assert_array_equal(orc.decode(orc.BF16, ref),
                                  torch.from_numpy(ref.view(np.int16)).view(torch.bfloat16).float().numpy())


def test_e4m3_table_matches_torch(orc):
    torch = pytest.importorskip("torch")
    codes = np.arange(256, dtype=np.uint8)
    ours = orc.decode(orc.E4M3, codes)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).float().numpy().astype(np.float64)
    np.testing.assert_array_equal(np.isnan(ours), np.isnan(ref))
    ok = ~np.isnan(ref)
    np.testing.assert_array_equal(ours[ok], ref[ok])
    assert np.isnan(ours[0x7F]) and np.isnan(ours[0xFF]) and np.sum(np.isnan(ours)) == 2
    assert ours[0x7E] == 448.0 and ours[1] == 2.0 ** -9 and ours[0x08] == 2.0 ** -6


def test_e4m3_encoder_matches_torch(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(62)
    x = np.concatenate([rng.uniform(-448, 448, 20000), rng.uniform(-1, 1, 20000),
                        np.exp(rng.uniform(np.log(1e-4), np.log(448), 20000))]).astype(np.float32)
    # exact ties between E4M3 neighbours
    vals = orc.decode(orc.E4M3, np.arange(0, 0x7E, dtype=np.uint8))
    ties = ((vals[:-1] + vals[1:]) / 2).astype(np.float32)
    x = np.concatenate([x, ties, -ties, np.float32([0.0, 448.0, -448.0])])
    ours = orc.encode(orc.E4M3, x)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    np.testing.assert_array_equal(ours, ref)


def test_e4m3_saturates(orc):
    x = np.float32([449.0, 463.9, 464.0, 500.0, 1e6, np.inf, -1e6, -np.inf])
    np.testing.assert_array_equal(orc.encode(orc.E4M3, x), [0x7E] * 6 + [0xFE] * 2)


@pytest.mark.parametrize("fmt,rel", [(1, 2.0 ** -11), (2, 2.0 ** -8), (3, 2.0 ** -4)])
def test_quantisation_error_bounds(orc, fmt, rel):
    """Round-to-nearest bounds: half an ulp relative for normal values; E4M3 with a
    per-bucket scale s has |err| <= 2^-4 |v| in its normal range, 2^-10 s below it."""
    rng = np.random.default_rng(63)
    W, H, n = 8, 6, 4
    atlas = (rng.uniform(0, 1, (H * n, W * n, 4)) ** 3).astype(np.float32)
    atlas[:n, :n] = 0.0  # an all-zero bucket: scale 1
    T = orc.Texture.from_f32(atlas, W, H, n, fmt)
    err = np.abs(T.values() - atlas.astype(np.float64))
    v = np.abs(atlas.astype(np.float64))
    if fmt == 3:
        s = np.broadcast_to(np.repeat(np.repeat(T.scales.astype(np.float64), n, 0), n, 1)[..., None], v.shape)
        assert np.all(T.scales[0, 0] == 1.0)
        normal = v / s >= 2.0 ** -6
        assert np.all(err[normal] <= rel * v[normal] * (1 + 1e-6))
        assert np.all(err[~normal] <= 2.0 ** -10 * s[~normal] * (1 + 1e-6))
        # the largest magnitude of each bucket is represented by the top code (448 s)
        amax = atlas.reshape(H, n, W, n, 4).max(axis=(1, 3, 4))
        ok = amax > 0
        np.testing.assert_allclose(T.scales[ok] * 448.0, amax[ok], rtol=1e-6)
    else:
        normal = v >= (2.0 ** -14 if fmt == 1 else 2.0 ** -126)
        assert np.all(err[normal] <= rel * v[normal])
    # filtered error is a convex combination of the texel errors
    rng2 = np.random.default_rng(64)
    F = 2000
    uv = rng2.uniform(0, 1, (F, 2))
    d = unit_dirs(rng2, F)
    q, _ = orc.shade([T], uv, d, np.zeros(F, np.int32), 2)
    x, _ = orc.shade([orc.Texture(W, H, n, orc.F64, atlas.astype(np.float64))], uv, d, np.zeros(F, np.int32), 2)
    assert np.max(np.abs(q - x)) <= err.max() + 1e-15


def test_note_clamp_keeps_lookups_inside_the_texel_centres(orc):
    """The Note after Eq. 3 clamps B to [1/n - 1, 1 - 1/n], the first and last
    texel centres: the in-bucket coordinate of every direction lies in [0, n-1]
    (bilinear) or [1/2, n - 1/2] (nearest), and grazing directions, whose B
    reaches the edge of the square, land exactly on the outer centre."""
    n = 8
    T = orc.Texture(2, 2, n, orc.F64, np.zeros((2 * n, 2 * n, 4)))
    rng = np.random.default_rng(40)
    d = unit_dirs(rng, 2000, lower=True).astype(np.float32)
    phi = rng.uniform(0, 2 * np.pi, 200)
    d[:200] = np.stack([np.cos(phi), np.sin(phi), np.zeros(200)], 1)  # on the horizon: |B|_inf = 1
    uv = np.full((2000, 2), 0.5, np.float32)
    obj = np.zeros(2000, np.int32)
    for filt, lo, hi in ((1, 0.0, n - 1.0), (0, 0.5, n - 0.5)):
        idx, c, _ = orc.locate([T], uv, d, obj, filt)
        assert (c[:, 2:] >= lo).all() and (c[:, 2:] <= hi).all()
        edge = np.abs(c[:200, 2:] - np.where(c[:200, 2:] > n / 2, hi, lo)).min(axis=1)
        assert (edge == 0).all()


def test_bucket_lobe_fill_against_numpy(orc):
    """The per-bucket lobe fill of the large workloads (reading A11's form for
    them: rho max(0, I . d)^p, alpha the lobe itself) against an independent
    numpy evaluation at the texel-centre directions, atlas row j n + t, column
    i n + s (R4); the directions themselves are pinned by the texel-centre pins."""
    import synth

    W, H, n = 5, 3, 4
    params = synth.bucket_lobe_params(91, W, H)
    got = orc.fill_bucket_lobes(W, H, n, params)
    dirs = orc.texel_directions(n)  # [t, s, 3]
    want = np.zeros((H * n, W * n, 4))
    for j in range(H):
        for i in range(W):
            P = params[j, i].astype(np.float64)
            cosang = dirs @ P[3:6]
            lobe = np.where(cosang > 0, np.maximum(cosang, 0.0) ** P[6], 0.0)
            for c in range(3):
                want[j * n:(j + 1) * n, i * n:(i + 1) * n, c] = P[c] * lobe
            want[j * n:(j + 1) * n, i * n:(i + 1) * n, 3] = lobe
    np.testing.assert_allclose(got, want.astype(np.float32), rtol=2e-7, atol=1e-30)
