"""FP64 CPU oracle for radiance-texture synthesis -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package.  The product path (the CUDA library
and its Python binding) never imports it, and this package imports nothing
from the product path.

The arithmetic lives in ``radtex_oracle.c`` (plain C11, FP64, OpenMP over
fragments); this module only compiles it with gcc and marshals numpy arrays
through ctypes.  Every function cites the passage of Fober, "Radiance Textures
for Rasterizing Ray-Traced Data" (arXiv 2301.01719) it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

F32, F16, BF16, E4M3, F64, BIT1, PATTERN = 0, 1, 2, 3, 4, 5, 6
NEAREST, ANGULAR_BILINEAR, QUADRILINEAR = 0, 1, 2
FLAG_BAD_OBJ, FLAG_NONFINITE = 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "radtex_oracle.c")
_LIB = os.path.join(_HERE, "libradtex_oracle.so")
_lock = threading.Lock()
_lib = None

_CODE_DTYPE = {F32: np.float32, F16: np.uint16, BF16: np.uint16, E4M3: np.uint8, F64: np.float64, BIT1: np.uint8}


# The mutation tests point the package at a deliberately broken build of the
# oracle through this variable, to check that the pins catch each mistake.
_OVERRIDE = os.environ.get("RADTEX_ORACLE_LIB")


def compile_oracle(src: str, out: str) -> str:
    """gcc -std=c11 -O2, FP contraction off, OpenMP: src -> shared library out."""
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
           "-Wall", "-Wextra", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (C11, FP contraction off, OpenMP)."""
    if _OVERRIDE:
        return _OVERRIDE
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    return compile_oracle(_SRC, _LIB)


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P, I32, I64, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
            sig = {
                "oracle_equisolid": (None, [I64, P, P]),
                "oracle_equisolid_normal": (None, [I64, P, P, P]),
                "oracle_squarify": (None, [I64, P, P]),
                "oracle_unsquarify": (None, [I64, P, P]),
                "oracle_equisolid_inverse": (None, [I64, P, P]),
                "oracle_equisolid_inverse_normal": (None, [I64, P, P, P]),
                "oracle_reflection": (None, [I64, P, P]),
                "oracle_texel_directions": (None, [I32, P]),
                "oracle_encode": (None, [I32, I64, P, P]),
                "oracle_decode": (None, [I32, I64, P, P]),
                "oracle_encode_e4m3_buckets": (None, [I32, I32, I32, P, P, P]),
                "oracle_locate": (U32, [P, P, I32, I64, P, P, P, I32, P, P]),
                "oracle_taps": (U32, [P, P, I32, I64, P, P, P, I32, P, P]),
                "oracle_shade": (U32, [P, P, P, I32, I64, P, P, P, I32, P]),
                "oracle_shade64": (U32, [P, P, P, I32, I64, P, P, P, I32, P]),
                "oracle_shade_backward": (U32, [P, P, P, I32, I64, P, P, P, I32, P, P, P, P]),
                "oracle_shade_backward64": (U32, [P, P, P, I32, I64, P, P, P, I32, P, P, P, P]),
                "oracle_eval_field": (None, [P, I32, I64, P, P, P]),
                "oracle_fill_field": (None, [I32, I32, I32, P, I32, P]),
                "oracle_fill_bucket_lobes": (None, [I32, I32, I32, P, P]),
                "oracle_bake": (None, [I32, I32, I32, I32, P, ctypes.c_double, P, P, P]),
                "oracle_bake_ray": (None, [I32, I32, P, ctypes.c_double, ctypes.c_double, I32, I32, P, P, P]),
                "oracle_trace": (None, [P, I64, P, P, P]),
                "oracle_bake_texels": (None, [I32, I32, I32, I32, P, ctypes.c_double, I64, P, P, P, P]),
                "oracle_palette_expand": (None, [I32, I32, I32, I32, I32, P, P, P, P, P]),
                "oracle_kmeans_assign": (None, [I64, I64, P, I64, P, P, P, P]),
                "oracle_kmeans_update": (None, [I64, I64, P, I64, P, P, P]),
                "oracle_locate_world": (U32, [P, P, I32, I64, P, P, P, P, I32, P, P]),
                "oracle_shade_world": (U32, [P, P, P, I32, I64, P, P, P, P, I32, P]),
                "oracle_shade_world64": (U32, [P, P, P, I32, I64, P, P, P, P, I32, P]),
                "oracle_shade_world_backward": (U32, [P, P, P, I32, I64, P, P, P, P, I32, P, P, P, P, P]),
                "oracle_shade_world_backward64": (U32, [P, P, P, I32, I64, P, P, P, P, I32, P, P, P, P, P]),
                "oracle_bake_shadow": (None, [I32, I32, I32, I32, P, ctypes.c_double, P, P]),
                "oracle_bake_shadow_texels": (None, [I32, I32, I32, I32, P, ctypes.c_double, I64, P, P, P]),
                "oracle_bake_deferred": (None, [I32, I32, I32, I32, P, I32, P, ctypes.c_double, P, P, P]),
                "oracle_bake_deferred_texels": (None, [I32, I32, I32, I32, P, I32, P, ctypes.c_double, I64, P, P,
                                                       P, P]),
                "oracle_ambient_occlusion": (None, [P, I32, I64, P, P, I32, P, P]),
                "oracle_onb": (None, [I64, P, P, P]),
                "oracle_num_threads": (I32, []),
                "oracle_set_num_threads": (None, [I32]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
# Section 2.1 mapping functions (rows of vectors).
# --------------------------------------------------------------------------

def _map(name: str, x, width_in: int, width_out: int, extra=None) -> np.ndarray:
    x = _c(x, np.float64).reshape(-1, width_in)
    out = np.empty((x.shape[0], width_out))
    if extra is None:
        getattr(lib(), name)(x.shape[0], _p(x), _p(out))
    else:
        e = _c(extra, np.float64).reshape(-1, 3)
        e = np.broadcast_to(e, (x.shape[0], 3)).copy()
        getattr(lib(), name)(x.shape[0], _p(x), _p(e), _p(out))
    return out


def equisolid(I) -> np.ndarray:
    """Eq. 1b: tangent-space incidence (k x 3) -> equisolid coordinate A (k x 2)."""
    return _map("oracle_equisolid", I, 3, 2)


def equisolid_normal(I, N) -> np.ndarray:
    """Eq. 1a: sqrt(2) normalize(I + N), k x 3."""
    return _map("oracle_equisolid_normal", I, 3, 3, N)


def squarify(A) -> np.ndarray:
    """Eq. 3: disc -> square, A (k x 2) -> B (k x 2)."""
    return _map("oracle_squarify", A, 2, 2)


def unsquarify(B) -> np.ndarray:
    """Eq. 4a: square -> disc, B (k x 2) -> A (k x 2)."""
    return _map("oracle_unsquarify", B, 2, 2)


def equisolid_inverse(A) -> np.ndarray:
    """Eq. 2c: A (k x 2) -> incidence I (k x 3), tangent space."""
    return _map("oracle_equisolid_inverse", A, 2, 3)


def equisolid_inverse_normal(A, N) -> np.ndarray:
    """Eq. 2a-2b: A (k x 2) and a normal N -> incidence I (k x 3)."""
    return _map("oracle_equisolid_inverse_normal", A, 2, 3, N)


def reflection(A) -> np.ndarray:
    """Eq. 4b: A (k x 2) -> equisolid reflection vector R (k x 3)."""
    return _map("oracle_reflection", A, 2, 3)


def texel_directions(n: int) -> np.ndarray:
    """Directions of the n x n texel centres of a bucket (Eq. 4a then Eq. 2c), shape (n, n, 3) indexed [t, s]."""
    out = np.empty((n, n, 3))
    lib().oracle_texel_directions(n, _p(out))
    return out


# --------------------------------------------------------------------------
# Storage formats.
# --------------------------------------------------------------------------

def encode(fmt: int, x) -> np.ndarray:
    """FP32 values -> codes of F32 / F16 / BF16 / E4M3 (no scale), round to nearest even."""
    x = _c(x, np.float32)
    out = np.empty(x.shape, dtype=_CODE_DTYPE[fmt])
    lib().oracle_encode(fmt, x.size, _p(x), _p(out))
    return out


def decode(fmt: int, codes) -> np.ndarray:
    codes = _c(codes, _CODE_DTYPE[fmt])
    out = np.empty(codes.shape, dtype=np.float64)
    lib().oracle_decode(fmt, codes.size, _p(codes), _p(out))
    return out


def encode_e4m3_buckets(atlas: np.ndarray, W: int, H: int, n: int):
    """FP32 atlas ((h n) x (w n) x 4) -> (E4M3 codes, per-bucket FP32 scales (h x w))."""
    atlas = _c(atlas, np.float32)
    assert atlas.shape == (H * n, W * n, 4)
    codes = np.empty(atlas.shape, dtype=np.uint8)
    scales = np.empty((H, W), dtype=np.float32)
    lib().oracle_encode_e4m3_buckets(W, H, n, _p(atlas), _p(codes), _p(scales))
    return codes, scales


class Texture:
    """A texture as the oracle sees it: stored codes in the atlas layout plus E4M3 scales."""

    def __init__(self, W: int, H: int, n: int, fmt: int, codes: np.ndarray, scales: np.ndarray | None = None,
                 wrap: int = 0):
        self.W, self.H, self.n, self.fmt = int(W), int(H), int(n), int(fmt)
        self.wrap = int(wrap)  # reading R12: bit 0 repeats u, bit 1 repeats v
        self.codes = _c(codes, _CODE_DTYPE[fmt])
        assert self.codes.shape == (H * n, W * n, 4), self.codes.shape
        self.scales = None if scales is None else _c(scales, np.float32)

    @classmethod
    def from_f32(cls, atlas: np.ndarray, W: int, H: int, n: int, fmt: int) -> "Texture":
        """Quantise an FP32 atlas with the oracle's own encoders."""
        if fmt == E4M3:
            codes, scales = encode_e4m3_buckets(atlas, W, H, n)
            return cls(W, H, n, fmt, codes, scales)
        if fmt == F64:
            return cls(W, H, n, fmt, np.asarray(atlas, dtype=np.float64))
        return cls(W, H, n, fmt, encode(fmt, atlas))

    def values(self) -> np.ndarray:
        """The stored texels decoded exactly to FP64, atlas layout."""
        v = decode(self.fmt, self.codes)
        if self.fmt == E4M3:
            v = v * np.repeat(np.repeat(self.scales.astype(np.float64), self.n, 0), self.n, 1)[..., None]
        return v


class PatternTexture:
    """An oracle-only procedural texture for sizes whose atlas would not fit in
    host memory (test infrastructure).  Channel c of atlas texel (X, Y) =
    (i n + s, j n + t) is the triangle wave |((a_c X + b_c Y + k_c) mod 2m) - m| / m,
    read by the same lookup as stored textures; no codes are held."""

    def __init__(self, W: int, H: int, n: int, a, b, k, m: int):
        self.W, self.H, self.n, self.fmt, self.wrap = int(W), int(H), int(n), PATTERN, 0
        p = [int(x) for x in (*a, *b, *k, m)]
        assert len(p) == 13 and min(p) >= 0 and p[12] >= 1
        self.codes = np.array(p, dtype=np.int64)
        self.scales = None


def _tables(textures):
    dims = np.zeros((max(len(textures), 1), 4), dtype=np.int32)
    codes = (ctypes.c_void_p * max(len(textures), 1))()
    scales = (ctypes.c_void_p * max(len(textures), 1))()
    for o, T in enumerate(textures):
        if T is None:
            continue
        dims[o] = (T.W, T.H, T.n, T.fmt | (getattr(T, "wrap", 0) << 8))
        codes[o] = T.codes.ctypes.data
        scales[o] = None if T.scales is None else T.scales.ctypes.data
    return dims, codes, scales


def _gbuf(uv, dirs, obj, dtype):
    uv = _c(uv, dtype).reshape(-1, 2)
    dirs = _c(dirs, dtype).reshape(-1, 3)
    obj = _c(obj, np.int32).reshape(-1)
    assert uv.shape[0] == dirs.shape[0] == obj.shape[0]
    return uv, dirs, obj


def shade(textures, uv, dirs, obj, filt: int, precise_inputs: bool = False):
    """Forward synthesis (Section 2): F x 4 FP64 colours and the OR of the error flags.

    textures: list indexed by object id (None for a missing object).
    uv: F x 2, dirs: F x 3 (FP32 unless precise_inputs), obj: F int32 (< 0 = background).
    """
    dtype = np.float64 if precise_inputs else np.float32
    uv, dirs, obj = _gbuf(uv, dirs, obj, dtype)
    dims, codes, scales = _tables(textures)
    out = np.empty((obj.shape[0], 4))
    fn = lib().oracle_shade64 if precise_inputs else lib().oracle_shade
    flags = fn(_p(dims), codes, scales, len(textures), obj.shape[0], _p(uv), _p(dirs), _p(obj), filt, _p(out))
    return out, int(flags)


def locate(textures, uv, dirs, obj, filt: int):
    """Floors (F x 4 int32: u, v, s, t) and continuous coordinates (F x 4 FP64) of every fragment."""
    uv, dirs, obj = _gbuf(uv, dirs, obj, np.float32)
    dims, codes, _ = _tables(textures)
    idx = np.empty((obj.shape[0], 4), dtype=np.int32)
    coord = np.empty((obj.shape[0], 4))
    flags = lib().oracle_locate(_p(dims), codes, len(textures), obj.shape[0], _p(uv), _p(dirs), _p(obj), filt,
                                _p(idx), _p(coord))
    return idx, coord, int(flags)


def taps(textures, uv, dirs, obj, filt: int):
    """The taps the colour sums (Section 2, the filters of reading R5): F x 16
    atlas texel indices Y (w n) + X (int64, -1 for no tap) and their FP64
    weights w_u w_v w_s w_t, in (u, v, s, t) tap order."""
    uv, dirs, obj = _gbuf(uv, dirs, obj, np.float32)
    dims, codes, _ = _tables(textures)
    index = np.empty((obj.shape[0], 16), dtype=np.int64)
    weight = np.empty((obj.shape[0], 16))
    flags = lib().oracle_taps(_p(dims), codes, len(textures), obj.shape[0], _p(uv), _p(dirs), _p(obj), filt,
                              _p(index), _p(weight))
    return index, weight, int(flags)


def shade_backward(textures, uv, dirs, obj, filt: int, dL_dout, want_tex=True, want_uv=True, want_dir=True,
                   precise_inputs: bool = False):
    """Analytic FP64 gradients: (dL/dtex list of FP64 atlases or None, dL/duv F x 2, dL/ddir F x 3, flags)."""
    dtype = np.float64 if precise_inputs else np.float32
    uv, dirs, obj = _gbuf(uv, dirs, obj, dtype)
    dims, codes, scales = _tables(textures)
    g = _c(dL_dout, np.float64).reshape(-1, 4)
    F = obj.shape[0]
    gtex = [None] * len(textures)
    gptr = (ctypes.c_void_p * max(len(textures), 1))()
    if want_tex:
        for o, T in enumerate(textures):
            if T is not None:
                gtex[o] = np.zeros((T.H * T.n, T.W * T.n, 4))
                gptr[o] = gtex[o].ctypes.data
    guv = np.empty((F, 2)) if want_uv else None
    gdir = np.empty((F, 3)) if want_dir else None
    fn = lib().oracle_shade_backward64 if precise_inputs else lib().oracle_shade_backward
    flags = fn(_p(dims), codes, scales, len(textures), F, _p(uv), _p(dirs), _p(obj), filt, _p(g),
               gptr if want_tex else None, _p(guv), _p(gdir))
    return (gtex if want_tex else None), guv, gdir, int(flags)


# --------------------------------------------------------------------------
# World-space variant (Eq. 1a with a per-fragment normal).
# --------------------------------------------------------------------------

def _normals(nrm, F, dtype):
    nrm = _c(nrm, dtype).reshape(-1, 3)
    assert nrm.shape[0] == F
    return nrm


def locate_world(textures, uv, dirs, nrm, obj, filt: int):
    """Floors and continuous coordinates with A from Eq. 1a (I, N in one frame)."""
    uv, dirs, obj = _gbuf(uv, dirs, obj, np.float32)
    nrm = _normals(nrm, obj.shape[0], np.float32)
    dims, codes, _ = _tables(textures)
    idx = np.empty((obj.shape[0], 4), dtype=np.int32)
    coord = np.empty((obj.shape[0], 4))
    flags = lib().oracle_locate_world(_p(dims), codes, len(textures), obj.shape[0], _p(uv), _p(dirs), _p(nrm),
                                      _p(obj), filt, _p(idx), _p(coord))
    return idx, coord, int(flags)


def shade_world(textures, uv, dirs, nrm, obj, filt: int, precise_inputs: bool = False):
    """World-space synthesis: like shade, with A the first two entries of Eq. 1a."""
    dtype = np.float64 if precise_inputs else np.float32
    uv, dirs, obj = _gbuf(uv, dirs, obj, dtype)
    nrm = _normals(nrm, obj.shape[0], dtype)
    dims, codes, scales = _tables(textures)
    out = np.empty((obj.shape[0], 4))
    fn = lib().oracle_shade_world64 if precise_inputs else lib().oracle_shade_world
    flags = fn(_p(dims), codes, scales, len(textures), obj.shape[0], _p(uv), _p(dirs), _p(nrm), _p(obj), filt,
               _p(out))
    return out, int(flags)


def shade_world_backward(textures, uv, dirs, nrm, obj, filt: int, dL_dout, want_tex=True,
                         precise_inputs: bool = False):
    """(dL/dtex list, dL/duv, dL/ddir, dL/dnrm, flags) of the world-space synthesis."""
    dtype = np.float64 if precise_inputs else np.float32
    uv, dirs, obj = _gbuf(uv, dirs, obj, dtype)
    nrm = _normals(nrm, obj.shape[0], dtype)
    dims, codes, scales = _tables(textures)
    g = _c(dL_dout, np.float64).reshape(-1, 4)
    F = obj.shape[0]
    gtex = [None] * len(textures)
    gptr = (ctypes.c_void_p * max(len(textures), 1))()
    if want_tex:
        for o, T in enumerate(textures):
            if T is not None:
                gtex[o] = np.zeros((T.H * T.n, T.W * T.n, 4))
                gptr[o] = gtex[o].ctypes.data
    guv, gdir, gnrm = np.empty((F, 2)), np.empty((F, 3)), np.empty((F, 3))
    fn = lib().oracle_shade_world_backward64 if precise_inputs else lib().oracle_shade_world_backward
    flags = fn(_p(dims), codes, scales, len(textures), F, _p(uv), _p(dirs), _p(nrm), _p(obj), filt, _p(g),
               gptr if want_tex else None, _p(guv), _p(gdir), _p(gnrm))
    return (gtex if want_tex else None), guv, gdir, gnrm, int(flags)


# --------------------------------------------------------------------------
# Fills.
# --------------------------------------------------------------------------

def fill_field(W: int, H: int, n: int, lobes: np.ndarray) -> np.ndarray:
    """FP32 atlas filled from the analytic multi-lobe field (rows of 11 parameters)."""
    lobes = _c(lobes, np.float64).reshape(-1, 11)
    atlas = np.empty((H * n, W * n, 4), dtype=np.float32)
    lib().oracle_fill_field(W, H, n, _p(lobes), lobes.shape[0], _p(atlas))
    return atlas


def eval_field(lobes: np.ndarray, uv, dirs) -> np.ndarray:
    lobes = _c(lobes, np.float64).reshape(-1, 11)
    uv = _c(uv, np.float64).reshape(-1, 2)
    dirs = _c(dirs, np.float64).reshape(-1, 3)
    out = np.empty((uv.shape[0], 4))
    lib().oracle_eval_field(_p(lobes), lobes.shape[0], uv.shape[0], _p(uv), _p(dirs), _p(out))
    return out


def fill_bucket_lobes(W: int, H: int, n: int, params: np.ndarray) -> np.ndarray:
    """FP32 atlas from one cosine-power lobe per bucket (params: h x w x 8 FP32)."""
    params = _c(params, np.float32).reshape(H * W, 8)
    atlas = np.empty((H * n, W * n, 4), dtype=np.float32)
    lib().oracle_fill_bucket_lobes(W, H, n, _p(params), _p(atlas))
    return atlas


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_num_threads(k: int) -> None:
    lib().oracle_set_num_threads(int(k))


# --------------------------------------------------------------------------
# Baking (Section 2.2, Eq. 4a, Eq. 4b): texel centre -> reflection vector ->
# ray traced through an analytic sphere + plane + sky scene (reading R10).
# --------------------------------------------------------------------------

SURFACE_SPHERE, SURFACE_PLANE = 0, 1
# (key, width) in the order of the oracle's flat parameter array
_SCENE_KEYS = (("sphere_centre", 3), ("sphere_radius", 1), ("plane_height", 1), ("plane_half_extent", 1),
               ("sphere_albedo", 3), ("sphere_reflectance", 1), ("plane_albedo", 3), ("plane_reflectance", 1),
               ("plane_frequency", 1), ("sun_direction", 3), ("sun_rgb", 3), ("sun_exponent", 1),
               ("sky_zenith", 3), ("sky_horizon", 3), ("ambient", 1), ("fog", 1), ("ray_offset", 1))


def scene_array(scene: dict) -> np.ndarray:
    """The scene dictionary as the oracle's flat parameter array (31 doubles)."""
    out = []
    for key, width in _SCENE_KEYS:
        v = np.atleast_1d(np.asarray(scene[key], np.float64))
        assert v.size == width, key
        out.extend(v.tolist())
    return np.array(out, np.float64)


def bake(W: int, H: int, n: int, surface: int, scene: dict, delta: float | None = None):
    """Baked texture as an FP64 atlas ((H n) x (W n) x 4), following Eq. 4a and
    Eq. 4b per texel centre.  With `delta`, also the per-texel range (lo, hi) of
    the value over rays perturbed by +-delta (origin along T, B; direction along
    T, B, N, renormalised)."""
    S = scene_array(scene)
    val = np.empty((H * n, W * n, 4))
    lo = hi = None
    if delta is not None:
        lo = np.empty_like(val)
        hi = np.empty_like(val)
    lib().oracle_bake(W, H, n, surface, _p(S), float(delta or 0.0), _p(val), _p(lo), _p(hi))
    return val if delta is None else (val, lo, hi)


def bake_texels(W: int, H: int, n: int, surface: int, scene: dict, ijst, delta: float | None = 2.0 ** -17):
    """Baked values of selected texels (rows i, j, s, t) and their perturbed-ray
    range: (val, lo, hi), each k x 4; with delta None only val."""
    S = scene_array(scene)
    q = _c(ijst, np.int32).reshape(-1, 4)
    val = np.empty((q.shape[0], 4))
    lo = hi = None
    if delta is not None:
        lo, hi = np.empty_like(val), np.empty_like(val)
    lib().oracle_bake_texels(W, H, n, surface, _p(S), float(delta or 0.0), q.shape[0], _p(q), _p(val), _p(lo),
                             _p(hi))
    return val if delta is None else (val, lo, hi)


def bake_ray(n: int, surface: int, scene: dict, u: float, v: float, s: int, t: int):
    """World-space origin P, direction d of the reflection ray of texel (s, t) at
    (u, v), and the tangent frame (rows T, B, N)."""
    S = scene_array(scene)
    P = np.empty(3)
    d = np.empty(3)
    F = np.empty((3, 3))
    lib().oracle_bake_ray(n, surface, _p(S), float(u), float(v), int(s), int(t), _p(P), _p(d), _p(F))
    return P, d, F


def trace(scene: dict, P, d) -> np.ndarray:
    """Radiance and fog transmittance (k x 4) along rays P + t d (rows of 3)."""
    S = scene_array(scene)
    P = _c(P, np.float64).reshape(-1, 3)
    d = _c(d, np.float64).reshape(-1, 3)
    out = np.empty((P.shape[0], 4))
    lib().oracle_trace(_p(S), P.shape[0], _p(P), _p(d), _p(out))
    return out


# --------------------------------------------------------------------------
# Bucket compression (Section 2; reading R11): palette + index map, k-means.
# --------------------------------------------------------------------------

def palette_expand(palette: "Texture", index, W: int, H: int) -> "Texture":
    """The dense texture a palette texture stands for: bucket (i, j) = palette
    bucket index[j, i].  palette: a K x 1 texture (its codes an n x K n atlas)."""
    n, K = palette.n, palette.W
    assert palette.H == 1
    index = _c(index, np.uint32).reshape(H, W)
    assert index.max(initial=0) < K
    dense = np.empty((H * n, W * n, 4), dtype=palette.codes.dtype)
    scales = np.empty((H, W), np.float32) if palette.scales is not None else None
    lib().oracle_palette_expand(W, H, n, K, palette.codes.dtype.itemsize, _p(palette.codes), _p(palette.scales),
                                _p(index), _p(dense), _p(scales))
    return Texture(W, H, n, palette.fmt, dense, scales)


def bucket_vectors(values: np.ndarray, W: int, H: int, n: int) -> np.ndarray:
    """Atlas-layout texel values ((H n) x (W n) x 4) -> one row per bucket
    (row b = j W + i), the n^2 x 4 values in (t, s, channel) order."""
    v = np.asarray(values, np.float64).reshape(H, n, W, n, 4)
    return np.ascontiguousarray(v.transpose(0, 2, 1, 3, 4).reshape(H * W, n * n * 4))


def kmeans_assign(X, C, all_distances: bool = False):
    """Nearest centroid of every row of X (B x D) among C (K x D), ties to the
    lowest index: (index, squared distance[, all squared distances B x K])."""
    X = _c(X, np.float64)
    C = _c(C, np.float64)
    B, D = X.shape
    K = C.shape[0]
    index = np.empty(B, np.uint32)
    dist = np.empty(B)
    dall = np.empty((B, K)) if all_distances else None
    lib().oracle_kmeans_assign(B, D, _p(X), K, _p(C), _p(index), _p(dist), _p(dall))
    return (index, dist, dall) if all_distances else (index, dist)


def kmeans_update(X, index, C_prev):
    """Means of the rows of X per assigned centroid; empty centroids keep C_prev."""
    X = _c(X, np.float64)
    C = np.array(C_prev, dtype=np.float64, copy=True, order="C")
    index = _c(index, np.uint32)
    counts = np.empty(C.shape[0], np.int64)
    lib().oracle_kmeans_update(X.shape[0], X.shape[1], _p(X), C.shape[0], _p(index), _p(C), _p(counts))
    return C, counts


# --------------------------------------------------------------------------
# Shadow textures (Section 5, "Shadowing"; reading R13).
# --------------------------------------------------------------------------

def bake_shadow(W: int, H: int, n: int, surface: int, scene: dict, delta: float = 2.0 ** -17):
    """Visibility bits ((H n) x (W n) uint8, atlas order) towards every texel
    direction (Eq. 4a, Eq. 2c), and the band of texels whose bit changes under
    perturbed rays."""
    S = scene_array(scene)
    vis = np.empty((H * n, W * n), np.uint8)
    band = np.empty_like(vis)
    lib().oracle_bake_shadow(W, H, n, surface, _p(S), float(delta), _p(vis), _p(band))
    return vis, band.astype(bool)


def bake_shadow_texels(W: int, H: int, n: int, surface: int, scene: dict, ijst, delta: float = 2.0 ** -17):
    S = scene_array(scene)
    q = _c(ijst, np.int32).reshape(-1, 4)
    vis = np.empty(q.shape[0], np.uint8)
    band = np.empty_like(vis)
    lib().oracle_bake_shadow_texels(W, H, n, surface, _p(S), float(delta), q.shape[0], _p(q), _p(vis), _p(band))
    return vis, band.astype(bool)


# --------------------------------------------------------------------------
# Deferred payloads (Section 1: deferred ambient occlusion and reflections;
# reading R15).
# --------------------------------------------------------------------------

def _dirs(dirs) -> np.ndarray:
    d = _c(dirs, np.float64).reshape(-1, 3)
    assert 1 <= d.shape[0]
    return d


def bake_deferred(W: int, H: int, n: int, surface: int, scene: dict, dirs, delta: float | None = 2.0 ** -17):
    """Deferred payload of every texel ((H n) x (W n) x 4, atlas order): the unlit albedo
    of the reflected ray's first hit and the ambient occlusion there over the K local
    directions dirs (K x 3); (0, 0, 0, 1) where the ray reaches the sky.  With delta, also
    the range [lo, hi] over perturbed rays and ambiguous AO directions."""
    S = scene_array(scene)
    d = _dirs(dirs)
    val = np.empty((H * n, W * n, 4))
    if delta is None:
        lib().oracle_bake_deferred(W, H, n, surface, _p(S), d.shape[0], _p(d), 0.0, _p(val), None, None)
        return val
    lo, hi = np.empty_like(val), np.empty_like(val)
    lib().oracle_bake_deferred(W, H, n, surface, _p(S), d.shape[0], _p(d), float(delta), _p(val), _p(lo), _p(hi))
    return val, lo, hi


def bake_deferred_texels(W: int, H: int, n: int, surface: int, scene: dict, dirs, ijst,
                         delta: float | None = 2.0 ** -17):
    """bake_deferred for a list of texels ijst (count x 4: i, j, s, t): val, lo, hi rows
    (val alone when delta is None)."""
    S = scene_array(scene)
    d = _dirs(dirs)
    q = _c(ijst, np.int32).reshape(-1, 4)
    val = np.empty((q.shape[0], 4))
    if delta is None:
        lib().oracle_bake_deferred_texels(W, H, n, surface, _p(S), d.shape[0], _p(d), 0.0, q.shape[0], _p(q),
                                          _p(val), None, None)
        return val
    lo, hi = np.empty_like(val), np.empty_like(val)
    lib().oracle_bake_deferred_texels(W, H, n, surface, _p(S), d.shape[0], _p(d), float(delta), q.shape[0], _p(q),
                                      _p(val), _p(lo), _p(hi))
    return val, lo, hi


def ambient_occlusion(scene: dict, X, N, dirs, surface: int = -1) -> np.ndarray:
    """Fraction of the K local directions (frame of the unit normal N) unblocked from X;
    `surface` (SURFACE_SPHERE / SURFACE_PLANE) is the one X lies on, which the rays skip
    (-1: both surfaces are tested)."""
    S = scene_array(scene)
    X = _c(X, np.float64).reshape(-1, 3)
    N = _c(N, np.float64).reshape(-1, 3)
    d = _dirs(dirs)
    out = np.empty(X.shape[0])
    lib().oracle_ambient_occlusion(_p(S), int(surface), X.shape[0], _p(X), _p(N), d.shape[0], _p(d), _p(out))
    return out


def onb(N):
    """The orthonormal basis (b1, b2) the deferred payload uses around unit normals N."""
    N = _c(N, np.float64).reshape(-1, 3)
    b1, b2 = np.empty_like(N), np.empty_like(N)
    lib().oracle_onb(N.shape[0], _p(N), _p(b1), _p(b2))
    return b1, b2


def bit_texture(bits: np.ndarray, W: int, H: int, n: int) -> "Texture":
    """A 1-bit texture from per-texel bits ((H n) x (W n)), value in every channel."""
    b = np.asarray(bits, np.uint8).reshape(H * n, W * n)
    return Texture(W, H, n, BIT1, np.repeat(b[..., None], 4, axis=2))
