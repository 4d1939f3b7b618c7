"""Seeded parameters of the synthetic radiance fields (the paper gives none).

Two field families are drawn here; their evaluation belongs to whoever fills
the texture (the oracle on the CPU, the fill kernel on the GPU):

* ``field_lobes``: the multi-lobe analytic field of the tiny quad workload,
  f_c(u, v, I) = sum_k a_kc (1/2 + 1/2 cos(2 pi (alpha_k u + beta_k v) + gamma_k)) max(0, I . d_k)^p_k,
  returned as rows of 11 numbers (a_0..a_3, alpha, beta, gamma, d_x, d_y, d_z, p).
* ``bucket_lobe_params``: one cosine-power lobe per bucket for the large
  workloads, returned as h x w x 8 FP32 (rho_r, rho_g, rho_b, d_x, d_y, d_z, p, 0).

and one texel pattern, ``pattern_values``, for textures too large to hold as
a host-side atlas (the oracle evaluates it per texel instead of storing it).
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _hemisphere(rng: np.random.Generator, k: int) -> np.ndarray:
    """k directions uniform on the upper (z >= 0) unit hemisphere."""
    z = rng.uniform(0.0, 1.0, k)
    phi = rng.uniform(0.0, 2.0 * np.pi, k)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def field_lobes(seed: int, n_lobes: int = 4) -> np.ndarray:
    """n_lobes x 11 FP64 parameters; every channel gets its own amplitudes, so
    a channel swap changes the result, and f stays in [0, 1]."""
    rng = _rng(seed)
    a = rng.uniform(0.0, 0.25, (n_lobes, 4))
    alpha = rng.integers(1, 5, n_lobes).astype(np.float64)
    beta = rng.integers(1, 5, n_lobes).astype(np.float64)
    gamma = rng.uniform(0.0, 2.0 * np.pi, n_lobes)
    d = _hemisphere(rng, n_lobes)
    p = np.exp(rng.uniform(np.log(1.0), np.log(200.0), n_lobes))
    return np.concatenate([a, alpha[:, None], beta[:, None], gamma[:, None], d, p[:, None]], axis=1)


def _smooth_noise(rng: np.random.Generator, W: int, H: int, cells: int) -> np.ndarray:
    """Low-frequency value noise in [0, 1] at the W x H bucket centres: a
    (cells+1)^2 grid of U[0, 1] values, bilinearly upsampled."""
    grid = rng.uniform(0.0, 1.0, (cells + 1, cells + 1))
    x = (np.arange(W) + 0.5) / W * cells
    y = (np.arange(H) + 0.5) / H * cells
    x0 = np.minimum(np.floor(x).astype(np.int64), cells - 1)
    y0 = np.minimum(np.floor(y).astype(np.int64), cells - 1)
    fx = (x - x0)[None, :]
    fy = (y - y0)[:, None]
    g00 = grid[np.ix_(y0, x0)]
    g01 = grid[np.ix_(y0, x0 + 1)]
    g10 = grid[np.ix_(y0 + 1, x0)]
    g11 = grid[np.ix_(y0 + 1, x0 + 1)]
    return (g00 * (1 - fx) + g01 * fx) * (1 - fy) + (g10 * (1 - fx) + g11 * fx) * fy


def bucket_lobe_params(seed: int, W: int, H: int, cells: int = 8, jitter: float = 0.05) -> np.ndarray:
    """Per-bucket lobes: albedo rho ~ U[0, 1]^3 per bucket; lobe direction and
    exponent vary smoothly over (u, v) (value noise plus a small per-bucket
    jitter), the exponent log-uniform-ish in [1, 200].  Returns H x W x 8 FP32."""
    rng = _rng(seed)
    rho = rng.uniform(0.0, 1.0, (H, W, 3))

    def field():
        return np.clip(_smooth_noise(rng, W, H, cells) + rng.uniform(-jitter, jitter, (H, W)), 0.0, 1.0)

    z = field()
    phi = 2.0 * np.pi * field()
    e = field()
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=-1)
    p = np.exp(np.log(200.0) * e)
    out = np.zeros((H, W, 8), dtype=np.float32)
    out[..., 0:3] = rho
    out[..., 3:6] = d
    out[..., 6] = p
    return out


def eval_field_lobes(lobes: np.ndarray, uv: np.ndarray, dirs: np.ndarray, chunk: int = 1 << 20) -> np.ndarray:
    """The multi-lobe field at arbitrary (u, v, I) in FP64 (target renders of the
    fitting workload): F x 4."""
    lobes = np.asarray(lobes, dtype=np.float64).reshape(-1, 11)
    uv = np.asarray(uv)
    dirs = np.asarray(dirs)
    out = np.zeros((uv.shape[0], 4))
    for a in range(0, uv.shape[0], chunk):
        u = uv[a:a + chunk, 0].astype(np.float64)
        v = uv[a:a + chunk, 1].astype(np.float64)
        I = dirs[a:a + chunk].astype(np.float64)
        acc = np.zeros((u.shape[0], 4))
        for P in lobes:
            spatial = 0.5 + 0.5 * np.cos(2.0 * np.pi * (P[4] * u + P[5] * v) + P[6])
            c = I @ P[7:10]
            lobe = np.where(c > 0.0, np.maximum(c, 0.0) ** P[10], 0.0)
            acc += P[None, 0:4] * (spatial * lobe)[:, None]
        out[a:a + chunk] = acc
    return out


# A texel pattern for textures too large for a host-side atlas: channel c of
# atlas texel (X, Y) is the triangle wave |((a_c X + b_c Y + k_c) mod 2m) - m| / m.
# Its values j / m (m = 2048) are exact in FP32, FP16 and BF16 alike, and its
# slope (at most 7 / 2048 per texel) keeps the colour's sensitivity to FP32
# coordinate rounding far below the colour tolerance, while a texel read from a
# wrong address differs from the right one.
PATTERN_A = (1, 3, 5, 7)
PATTERN_B = (3, 1, 7, 5)
PATTERN_K = (0, 517, 1031, 1543)
PATTERN_M = 2048


def pattern_values(X, Y, c: int):
    """Channel c of the pattern at integer atlas coordinates X, Y (broadcastable
    numpy arrays or torch tensors of a 64-bit integer type; only operators are
    used, so the same code fills a host array or a device tensor)."""
    m = PATTERN_M
    q = (PATTERN_A[c] * X + PATTERN_B[c] * Y + PATTERN_K[c]) % (2 * m)
    return abs(q - m) / m
