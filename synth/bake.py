"""Seeded analytic scenes for baking (sphere + ground plane + sky).

Only parameter draws: the geometry matches the sphere-plane G-buffer scene
(unit sphere at the origin, ground plane y = -1 with half extent 4)."""
from __future__ import annotations

import numpy as np


def bake_scene(seed: int, plane_height: float = -1.0, sphere_radius: float = 1.0) -> dict:
    """A seeded scene: albedos, reflectances, sun, sky and fog.  Colours stay in
    [0, 1] and the sun exponent is moderate, so baked texels lie in [0, 2]."""
    rng = np.random.default_rng(seed)
    sun = np.array([rng.uniform(-0.6, 0.6), 1.0, rng.uniform(-0.6, 0.6)])
    sun /= np.linalg.norm(sun)
    return {
        "sphere_centre": [0.0, 0.0, 0.0],
        "sphere_radius": sphere_radius,
        "plane_height": plane_height,
        "plane_half_extent": 4.0,
        "sphere_albedo": rng.uniform(0.2, 0.9, 3).tolist(),
        "sphere_reflectance": float(rng.uniform(0.2, 0.6)),
        "plane_albedo": rng.uniform(0.2, 0.9, 3).tolist(),
        "plane_reflectance": float(rng.uniform(0.2, 0.6)),
        "plane_frequency": float(rng.uniform(2.0, 6.0)),
        "sun_direction": sun.tolist(),
        "sun_rgb": rng.uniform(0.3, 0.8, 3).tolist(),
        "sun_exponent": float(rng.integers(4, 17)),
        "sky_zenith": rng.uniform(0.3, 0.8, 3).tolist(),
        "sky_horizon": rng.uniform(0.3, 0.8, 3).tolist(),
        "ambient": float(rng.uniform(0.1, 0.3)),
        "fog": float(rng.uniform(0.05, 0.15)),
        "ray_offset": 1e-4,
    }


def ao_directions(seed: int, K: int) -> np.ndarray:
    """K unit directions of the upper hemisphere (z >= 0), cosine-distributed and
    stratified (jittered cells of a near-square grid), FP32: the sample set of an
    ambient-occlusion estimate, drawn once and passed to the bake as an input."""
    rng = np.random.default_rng(seed)
    a = int(np.floor(np.sqrt(K)))
    while K % a:
        a -= 1
    b = K // a
    cells = np.stack(np.meshgrid(np.arange(a), np.arange(b), indexing="ij"), -1).reshape(-1, 2)
    u1 = (cells[:, 0] + rng.uniform(size=K)) / a
    u2 = (cells[:, 1] + rng.uniform(size=K)) / b
    r, phi = np.sqrt(u1), 2.0 * np.pi * u2
    d = np.stack([r * np.cos(phi), r * np.sin(phi), np.sqrt(np.maximum(1.0 - u1, 0.0))], 1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d.astype(np.float32)
