"""Python binding of libradtex for PyTorch tensors.

Every function has the name of the C entry point it calls (include/radtex.h)
and only marshals arguments: tensors become device pointers, sizes come from
their shapes, and the stream defaults to PyTorch's current stream on the
tensors' device.  All the work happens in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import (RT_ACCUMULATE, RT_ACCUMULATE_TEXELS, RT_ANGULAR_BILINEAR, RT_BF16, RT_BIT1,  # noqa: F401
                   RT_BORROW, RT_DETERMINISTIC, RT_E4M3_BUCKET_SCALE, RT_ERR_BAD_OBJ_ID, RT_ERR_CUDA,
                   RT_ERR_INVALID_ARG, RT_ERR_NONFINITE, RT_ERR_OOM, RT_ERR_OUT_OF_BOUNDS, RT_ERR_TIMEOUT,
                   RT_ERR_UNSUPPORTED, RT_F16, RT_F32,
                   RT_FIXED_POINT_GRADS, RT_LAYOUT_ATLAS, RT_LAYOUT_PALETTE, RT_LAYOUT_PLANES, RT_LAYOUT_QUADS,
                   RT_MAX_AO_DIRECTIONS,
                   RT_MAX_OBJECTS, RT_NEAREST, RT_OK, RT_QUADRILINEAR, RT_SURFACE_PLANE, RT_SURFACE_SPHERE, RT_WRAP_U,
                   RT_WRAP_V, RadtexError)

FORMAT_BYTES = {RT_F32: 16, RT_F16: 8, RT_BF16: 8, RT_E4M3_BUCKET_SCALE: 4, RT_BIT1: 1 / 8}
CODE_DTYPE = {RT_F32: torch.float32, RT_F16: torch.int16, RT_BF16: torch.int16, RT_E4M3_BUCKET_SCALE: torch.uint8,
              RT_BIT1: torch.uint8}
FORMAT_NAMES = {"f32": RT_F32, "f16": RT_F16, "bf16": RT_BF16, "e4m3": RT_E4M3_BUCKET_SCALE, "bit1": RT_BIT1}
FILTER_NAMES = {"nearest": RT_NEAREST, "angular_bilinear": RT_ANGULAR_BILINEAR, "quadrilinear": RT_QUADRILINEAR}


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream, device) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream(device)
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    return ctypes.c_void_p(handle)


def _check(t: torch.Tensor, name: str, dtype, last_dim: int | None = None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if last_dim is not None and (t.dim() < 1 or t.shape[-1] != last_dim):
        raise ValueError(f"{name} must have last dimension {last_dim}, got {tuple(t.shape)}")


class Context:
    """An rt_ctx on one CUDA device; destroyed with the object (or .close())."""

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        _lib.call("rt_context_create", int(device), ctypes.byref(h))
        self.handle = h
        self.device = int(device)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.lib().rt_context_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rt_context_create(device: int = 0) -> Context:
    return Context(device)


def rt_context_destroy(ctx: Context) -> None:
    ctx.close()


def rt_create_texture(ctx: Context, w: int, h: int, n: int, storage: int = RT_F32, src_layout: int = RT_LAYOUT_ATLAS,
                      src: torch.Tensor | None = None, flags: int = 0) -> int:
    """src: FP32 CUDA tensor shaped by layout_shape(src_layout, w, h, n) (or None).  Returns the object id."""
    if src is not None:
        _check(src, "src", torch.float32)
        want = layout_numel(src_layout, w, h, n)
        if src.numel() != want:
            raise ValueError(f"src has {src.numel()} elements, expected {want}")
    out = ctypes.c_int32(-1)
    _lib.call("rt_create_texture", ctx.handle, int(w), int(h), int(n), int(storage), int(src_layout), _ptr(src),
              int(flags), ctypes.byref(out))
    return out.value


def rt_create_palette_texture(ctx: Context, w: int, h: int, n: int, K: int, storage: int, src_layout: int,
                              palette: torch.Tensor, index: torch.Tensor, flags: int = 0) -> int:
    """Palette texture (bucket compression): palette = FP32 CUDA tensor of K x n x n x 4
    values (a K x 1 texture in src_layout), index = CUDA int32/uint32 (h, w) map of
    palette buckets.  Returns the object id."""
    _check(palette, "palette", torch.float32)
    if palette.numel() != K * n * n * 4:
        raise ValueError(f"palette has {palette.numel()} elements, expected {K * n * n * 4}")
    if index.dtype not in (torch.int32, torch.uint32) or not index.is_cuda or not index.is_contiguous():
        raise ValueError("index must be a contiguous CUDA int32 / uint32 tensor")
    if index.numel() != w * h:
        raise ValueError(f"index has {index.numel()} entries, expected {w * h}")
    out = ctypes.c_int32(-1)
    _lib.call("rt_create_palette_texture", ctx.handle, int(w), int(h), int(n), int(K), int(storage),
              int(src_layout), _ptr(palette), _ptr(index), int(flags), ctypes.byref(out))
    return out.value


def rt_palette_size(ctx: Context, obj_id: int) -> int:
    K = ctypes.c_int32(0)
    _lib.call("rt_palette_size", ctx.handle, int(obj_id), ctypes.byref(K))
    return K.value


def rt_set_wait_limit(ctx: Context, polls: int = 0) -> None:
    """Polls before a bounded device wait gives up with RT_ERR_TIMEOUT (0: the default)."""
    _lib.call("rt_set_wait_limit", ctx.handle, int(polls))


def rt_kmeans_init(ctx: Context, obj_id: int, K: int, buckets: torch.Tensor, centroids: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
    """Centroids (n, n, K, 4) FP32 initialised from the buckets numbered `buckets` (CUDA int32, K)."""
    info = rt_texture_info(ctx, obj_id)
    n = info["n"]
    _check(buckets, "buckets", torch.int32)
    if buckets.numel() != K:
        raise ValueError("buckets must hold K bucket numbers")
    if centroids is None:
        centroids = torch.empty((n, n, K, 4), dtype=torch.float32, device=buckets.device)
    _check(centroids, "centroids", torch.float32, 4)
    _lib.call("rt_kmeans_init", ctx.handle, int(obj_id), int(K), _ptr(buckets), _ptr(centroids),
              _stream(stream, buckets.device))
    return centroids


def rt_kmeans_assign(ctx: Context, obj_id: int, K: int, centroids: torch.Tensor, index: torch.Tensor | None = None,
                     dist: torch.Tensor | None = None, want_dist: bool = False, stream=None):
    """Nearest centroid of every bucket: index (h, w) int32 [, squared distance (h, w) FP32]."""
    info = rt_texture_info(ctx, obj_id)
    _check(centroids, "centroids", torch.float32, 4)
    if centroids.numel() != K * info["n"] ** 2 * 4:
        raise ValueError("centroids must hold K x n x n x 4 values")
    dev = centroids.device
    if index is None:
        index = torch.empty((info["h"], info["w"]), dtype=torch.int32, device=dev)
    if want_dist and dist is None:
        dist = torch.empty((info["h"], info["w"]), dtype=torch.float32, device=dev)
    _lib.call("rt_kmeans_assign", ctx.handle, int(obj_id), int(K), _ptr(centroids), _ptr(index), _ptr(dist),
              _stream(stream, dev))
    return (index, dist) if want_dist else index


class TcScratch:
    """Device scratch of rt_kmeans_assign_tc, 1024-byte aligned."""

    def __init__(self, nbytes: int, device):
        self.buf = torch.empty(nbytes + 1024, dtype=torch.uint8, device=device)
        self.ptr = (self.buf.data_ptr() + 1023) & ~1023
        self.nbytes = nbytes


def rt_kmeans_tc_scratch_bytes(w: int, h: int, n: int, K: int) -> int:
    return int(_lib.lib().rt_kmeans_tc_scratch_bytes(int(w), int(h), int(n), int(K)))


def rt_kmeans_assign_tc(ctx: Context, obj_id: int, K: int, centroids: torch.Tensor, index: torch.Tensor | None = None,
                        dist: torch.Tensor | None = None, want_dist: bool = False, scratch: TcScratch | None = None,
                        stream=None):
    """rt_kmeans_assign on the tensor cores (FP16 operands, FP32 accumulation)."""
    info = rt_texture_info(ctx, obj_id)
    _check(centroids, "centroids", torch.float32, 4)
    if centroids.numel() != K * info["n"] ** 2 * 4:
        raise ValueError("centroids must hold K x n x n x 4 values")
    dev = centroids.device
    if index is None:
        index = torch.empty((info["h"], info["w"]), dtype=torch.int32, device=dev)
    if want_dist and dist is None:
        dist = torch.empty((info["h"], info["w"]), dtype=torch.float32, device=dev)
    if scratch is None:
        scratch = TcScratch(rt_kmeans_tc_scratch_bytes(info["w"], info["h"], info["n"], K), dev)
    _lib.call("rt_kmeans_assign_tc", ctx.handle, int(obj_id), int(K), _ptr(centroids), _ptr(index), _ptr(dist),
              ctypes.c_void_p(scratch.ptr), int(scratch.nbytes), _stream(stream, dev))
    return (index, dist) if want_dist else index


def rt_kmeans_update(ctx: Context, obj_id: int, K: int, index: torch.Tensor, centroids: torch.Tensor,
                     scratch: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Centroids <- means of their members (in place); empty centroids are kept."""
    info = rt_texture_info(ctx, obj_id)
    B = info["w"] * info["h"]
    _check(centroids, "centroids", torch.float32, 4)
    if index.numel() != B:
        raise ValueError("index must hold one entry per bucket")
    if scratch is None:
        scratch = torch.empty(B + 3 * K + 1, dtype=torch.int32, device=centroids.device)
    if scratch.numel() < B + 3 * K + 1:
        raise ValueError("scratch needs w h + 3 K + 1 entries")
    _lib.call("rt_kmeans_update", ctx.handle, int(obj_id), int(K), _ptr(index), _ptr(centroids), _ptr(scratch),
              _stream(stream, centroids.device))
    return centroids


def palette_encode(ctx: Context, obj_id: int, K: int, iterations: int, seed: int = 0, stream=None,
                   tensor_cores: bool = True):
    """k-means palette of a dense texture: K centroids seeded at K distinct random
    buckets, `iterations` Lloyd steps, assignments on the tensor cores (FP16
    operands) unless tensor_cores is False (FP32 on the CUDA cores).  Returns
    (centroids (n, n, K, 4), index (h, w), per-step sums of squared distances)."""
    import numpy as np

    info = rt_texture_info(ctx, obj_id)
    B = info["w"] * info["h"]
    dev = torch.device("cuda", ctx.device)
    pick = np.random.default_rng(seed).choice(B, size=K, replace=False).astype(np.int32)
    C = rt_kmeans_init(ctx, obj_id, K, torch.from_numpy(pick).to(dev), stream=stream)
    scratch = torch.empty(B + 3 * K + 1, dtype=torch.int32, device=dev)
    index = torch.empty((info["h"], info["w"]), dtype=torch.int32, device=dev)
    dist = torch.empty((info["h"], info["w"]), dtype=torch.float32, device=dev)
    sse = []
    tc = TcScratch(rt_kmeans_tc_scratch_bytes(info["w"], info["h"], info["n"], K), dev) if tensor_cores else None

    def assign():
        if tensor_cores:
            rt_kmeans_assign_tc(ctx, obj_id, K, C, index, dist, scratch=tc, stream=stream)
        else:
            rt_kmeans_assign(ctx, obj_id, K, C, index, dist, stream=stream)

    for _ in range(iterations):
        assign()
        sse.append(dist.double().sum())
        rt_kmeans_update(ctx, obj_id, K, index, C, scratch, stream=stream)
    assign()
    sse.append(dist.double().sum())
    return C, index, [float(x) for x in sse]


def rt_destroy_texture(ctx: Context, obj_id: int) -> None:
    _lib.call("rt_destroy_texture", ctx.handle, int(obj_id))


def rt_texture_info(ctx: Context, obj_id: int) -> dict:
    vals = [ctypes.c_int32() for _ in range(5)]
    nbytes = ctypes.c_int64()
    _lib.call("rt_texture_info", ctx.handle, int(obj_id), *[ctypes.byref(v) for v in vals], ctypes.byref(nbytes))
    w, h, n, storage, layout = (v.value for v in vals)
    return {"w": w, "h": h, "n": n, "storage": storage, "layout": layout, "bytes": nbytes.value}


def layout_shape(layout: int, w: int, h: int, n: int) -> tuple:
    """Tensor shape of a 4-channel texture buffer: atlas (h n, w n, 4); planes
    (n, n, h, w, 4); quads (n, n, ceil(h/2), ceil(w/2), 2, 2, 4), i.e. (t, s, j // 2,
    i // 2, j mod 2, i mod 2, channel), an odd side padded."""
    if layout == RT_LAYOUT_ATLAS:
        return (h * n, w * n, 4)
    if layout == RT_LAYOUT_QUADS:
        return (n, n, (h + 1) // 2, (w + 1) // 2, 2, 2, 4)
    return (n, n, h, w, 4)


def layout_numel(layout: int, w: int, h: int, n: int) -> int:
    return int(np.prod(layout_shape(layout, w, h, n)))


def storage_numel(ctx: Context, obj_id: int) -> int:
    """Values (4 per texel) of a buffer in the object's storage layout: its texel
    gradients (rt_shade_backward's dL_dtex) and its stored codes."""
    info = rt_texture_info(ctx, obj_id)
    K = rt_palette_size(ctx, obj_id)
    if K:
        return K * info["n"] ** 2 * 4
    return layout_numel(info["layout"], info["w"], info["h"], info["n"])


def rt_read_texture(ctx: Context, obj_id: int, dst_layout: int = RT_LAYOUT_ATLAS, stream=None):
    """Stored codes (and E4M3 scales) of an owned texture, as new CUDA tensors.

    Codes are shaped by layout_shape(dst_layout, ...) and are float32 (F32),
    int16 bit patterns (F16 / BF16) or uint8 (E4M3)."""
    info = rt_texture_info(ctx, obj_id)
    w, h, n, fmt = info["w"], info["h"], info["n"], info["storage"]
    K = rt_palette_size(ctx, obj_id)
    if K:  # a palette reads as its K x 1 texture
        w, h = K, 1
    dev = torch.device("cuda", ctx.device)
    shape = layout_shape(dst_layout, w, h, n)
    if fmt == RT_BIT1:  # one byte (0 or 1) per texel, no channels
        shape = shape[:-1]
    codes = torch.zeros(shape, dtype=CODE_DTYPE[fmt], device=dev)  # the padding of quads stays zero
    scales = torch.empty((h, w), dtype=torch.float32, device=dev) if fmt == RT_E4M3_BUCKET_SCALE else None
    _lib.call("rt_read_texture", ctx.handle, int(obj_id), int(dst_layout), _ptr(codes), _ptr(scales),
              _stream(stream, dev))
    return codes, scales


def rt_fill_bucket_lobes(ctx: Context, obj_id: int, params: torch.Tensor, stream=None) -> None:
    """params: CUDA float32 (h, w, 8) per-bucket lobe parameters."""
    _check(params, "params", torch.float32, 8)
    info = rt_texture_info(ctx, obj_id)
    if params.numel() != info["w"] * info["h"] * 8:
        raise ValueError(f"params must hold h x w x 8 = {info['h']} x {info['w']} x 8 floats")
    _lib.call("rt_fill_bucket_lobes", ctx.handle, int(obj_id), _ptr(params), _stream(stream, params.device))


def bake_scene_struct(scene: dict) -> _lib.BakeScene:
    """The scene dictionary (keys as rt_bake_scene's fields) as the C struct."""
    S = _lib.BakeScene()
    for name, ctype in _lib.BakeScene._fields_:
        value = scene[name]
        if hasattr(ctype, "_length_"):
            vals = [float(x) for x in value]
            if len(vals) != ctype._length_:
                raise ValueError(f"{name} needs {ctype._length_} values")
            setattr(S, name, ctype(*vals))
        else:
            setattr(S, name, float(value))
    return S


def rt_bake(ctx: Context, obj_id: int, surface: int, scene: dict, stream=None) -> None:
    """Bakes object obj_id from the analytic scene (Eq. 4a, Eq. 4b, one traced
    ray per texel); surface is RT_SURFACE_SPHERE or RT_SURFACE_PLANE."""
    S = bake_scene_struct(scene)
    dev = torch.device("cuda", ctx.device)
    _lib.call("rt_bake", ctx.handle, int(obj_id), int(surface), ctypes.byref(S), _stream(stream, dev))


def rt_bake_deferred(ctx: Context, obj_id: int, surface: int, scene: dict, ao_dirs: torch.Tensor,
                     stream=None) -> None:
    """Bakes the deferred payload (unlit albedo and ambient occlusion of the reflected
    ray's first hit) into object obj_id; ao_dirs: (K, 3) float32 local unit directions
    on the object's device."""
    S = bake_scene_struct(scene)
    _check(ao_dirs, "ao_dirs", torch.float32, 3)
    if ao_dirs.device != torch.device("cuda", ctx.device):
        raise ValueError("ao_dirs must live on the context's device")
    _lib.call("rt_bake_deferred", ctx.handle, int(obj_id), int(surface), ctypes.byref(S), _ptr(ao_dirs),
              int(ao_dirs.numel() // 3), _stream(stream, ao_dirs.device))


def _gbuffer(uv, dirs, obj):
    _check(uv, "uv", torch.float32, 2)
    _check(dirs, "dir", torch.float32, 3)
    _check(obj, "obj", torch.int32)
    F = obj.numel()
    if uv.numel() != 2 * F or dirs.numel() != 3 * F:
        raise ValueError("uv, dir and obj must describe the same number of fragments")
    return F


def rt_shade(ctx: Context, uv: torch.Tensor, dirs: torch.Tensor, obj: torch.Tensor, filter: int = RT_QUADRILINEAR,
             out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Forward synthesis: (F, 4) float32 colours."""
    F = _gbuffer(uv, dirs, obj)
    if out is None:
        out = torch.empty((F, 4), dtype=torch.float32, device=uv.device)
    _check(out, "out", torch.float32, 4)
    if out.numel() != 4 * F:
        raise ValueError("out must hold F x 4 floats")
    _lib.call("rt_shade", ctx.handle, _ptr(uv), _ptr(dirs), _ptr(obj), F, int(filter), _ptr(out),
              _stream(stream, uv.device))
    return out


def _frames(uv, dirs, obj):
    """(views, height, width) of G-buffer tensors shaped (V, H, W, k) / (V, H, W)."""
    if obj.dim() != 3:
        raise ValueError("batched G-buffers are shaped (views, height, width[, k])")
    V, H, W = obj.shape
    if tuple(uv.shape) != (V, H, W, 2) or tuple(dirs.shape) != (V, H, W, 3):
        raise ValueError("uv must be (V, H, W, 2) and dir (V, H, W, 3)")
    return V, H, W


def rt_shade_batched(ctx: Context, uv, dirs, obj, filter: int = RT_QUADRILINEAR, out=None, stream=None):
    """Synthesis of views x height x width fragments; uv (V, H, W, 2), dir (V, H, W, 3), obj (V, H, W)."""
    F = _gbuffer(uv, dirs, obj)
    V, H, W = _frames(uv, dirs, obj)
    if out is None:
        out = torch.empty((V, H, W, 4), dtype=torch.float32, device=uv.device)
    _check(out, "out", torch.float32, 4)
    if out.numel() != 4 * F:
        raise ValueError("out must hold V x H x W x 4 floats")
    _lib.call("rt_shade_batched", ctx.handle, _ptr(uv), _ptr(dirs), _ptr(obj), V, H, W, int(filter), _ptr(out),
              _stream(stream, uv.device))
    return out


def rt_shade_batched_backward(ctx: Context, uv, dirs, obj, filter: int, dL_dout, dL_dtex=None, dL_duv=None,
                              dL_ddir=None, flags: int = 0, stream=None) -> None:
    F = _gbuffer(uv, dirs, obj)
    V, H, W = _frames(uv, dirs, obj)
    arr, n_dtex = _grad_args(ctx, F, dL_dout, dL_dtex, dL_duv, dL_ddir, flags)
    _lib.call("rt_shade_batched_backward", ctx.handle, _ptr(uv), _ptr(dirs), _ptr(obj), V, H, W, int(filter),
              _ptr(dL_dout), arr, n_dtex, _ptr(dL_duv), _ptr(dL_ddir), int(flags), _stream(stream, uv.device))


def rt_zero_texture_grads(ctx: Context, dL_dtex: dict, stream=None) -> None:
    """Zeroes each object's texel-gradient buffer ({object id: FP32 tensor}) on the stream."""
    if not dL_dtex:
        return
    n_dtex = max(dL_dtex) + 1
    arr = (ctypes.c_void_p * n_dtex)()
    dev = None
    for o, t in dL_dtex.items():
        _check(t, f"dL_dtex[{o}]", torch.float32)
        want = storage_numel(ctx, o)
        if t.numel() != want:
            raise ValueError(f"dL_dtex[{o}] must hold {want} floats (the object's storage layout)")
        arr[o] = t.data_ptr()
        dev = t.device
    _lib.call("rt_zero_texture_grads", ctx.handle, arr, n_dtex, _stream(stream, dev))


def rt_shade_batched_l2_step(ctx: Context, uv, dirs, obj, filter: int, target, scale: float = 1.0, out=None,
                             sums=None, dL_dtex=None, dL_duv=None, dL_ddir=None, flags: int = 0, stream=None):
    """Fused forward + L2 loss + backward over (V, H, W) frames: writes `out` (if given),
    adds sum |out - target|^2 and the shaded count to `sums` (float64 (2,), if given) and
    the gradients of dL/dout = scale (out - target).  Returns out."""
    F = _gbuffer(uv, dirs, obj)
    V, H, W = _frames(uv, dirs, obj)
    _check(target, "target", torch.float32, 4)
    if target.numel() != 4 * F:
        raise ValueError("target must hold V x H x W x 4 floats")
    if out is not None:
        _check(out, "out", torch.float32, 4)
        if out.numel() != 4 * F:
            raise ValueError("out must hold V x H x W x 4 floats")
    if sums is not None and (sums.dtype != torch.float64 or sums.numel() < 2 or not sums.is_cuda):
        raise TypeError("sums must be a CUDA float64 tensor of 2 elements")
    arr, n_dtex = _grad_args(ctx, F, target, dL_dtex, dL_duv, dL_ddir, flags)
    _lib.call("rt_shade_batched_l2_step", ctx.handle, _ptr(uv), _ptr(dirs), _ptr(obj), V, H, W, int(filter),
              _ptr(target), float(scale), _ptr(out), _ptr(sums), arr, n_dtex, _ptr(dL_duv), _ptr(dL_ddir),
              int(flags), _stream(stream, uv.device))
    return out


def rt_prepare_deterministic(ctx: Context) -> None:
    _lib.call("rt_prepare_deterministic", ctx.handle)


def rt_set_tile(ctx: Context, filter: int, tw: int, th: int, bx: int, by: int) -> None:
    _lib.call("rt_set_tile", ctx.handle, int(filter), int(tw), int(th), int(bx), int(by))


def rt_set_backward_tile(ctx: Context, filter: int, tw: int, th: int, bx: int, by: int) -> None:
    _lib.call("rt_set_backward_tile", ctx.handle, int(filter), int(tw), int(th), int(bx), int(by))


def rt_get_tile(ctx: Context, filter: int) -> tuple:
    t = (ctypes.c_int32 * 4)()
    _lib.call("rt_get_tile", ctx.handle, int(filter), t)
    return tuple(int(x) for x in t)


def rt_get_backward_tile(ctx: Context, filter: int) -> tuple:
    t = (ctypes.c_int32 * 4)()
    _lib.call("rt_get_backward_tile", ctx.handle, int(filter), t)
    return tuple(int(x) for x in t)


def rt_autotune(ctx: Context, uv, dirs, obj, filter: int = RT_QUADRILINEAR, out=None, reps: int = 3, stream=None):
    """Picks the fastest screen tile for batched synthesis; returns ((tw, th, bx, by), mean ms)."""
    F = _gbuffer(uv, dirs, obj)
    V, H, W = _frames(uv, dirs, obj)
    if out is None:
        out = torch.empty((V, H, W, 4), dtype=torch.float32, device=uv.device)
    if out.numel() != 4 * F:
        raise ValueError("out must hold V x H x W x 4 floats")
    t = (ctypes.c_int32 * 4)()
    ms = ctypes.c_float()
    _lib.call("rt_autotune", ctx.handle, _ptr(uv), _ptr(dirs), _ptr(obj), V, H, W, int(filter), _ptr(out), int(reps),
              _stream(stream, uv.device), t, ctypes.byref(ms))
    return tuple(int(x) for x in t), float(ms.value)


def rt_autotune_backward(ctx: Context, uv, dirs, obj, filter: int, dL_dout, dL_dtex=None, dL_duv=None, dL_ddir=None,
                         flags: int = 0, reps: int = 3, stream=None):
    """Picks the fastest screen tile for the batched backward; returns ((tw, th, bx, by), mean ms).
    The gradient buffers are left holding the timed launches' results: clear them before use."""
    F = _gbuffer(uv, dirs, obj)
    V, H, W = _frames(uv, dirs, obj)
    arr, n_dtex = _grad_args(ctx, F, dL_dout, dL_dtex, dL_duv, dL_ddir, flags)
    t = (ctypes.c_int32 * 4)()
    ms = ctypes.c_float()
    _lib.call("rt_autotune_backward", ctx.handle, _ptr(uv), _ptr(dirs), _ptr(obj), V, H, W, int(filter),
              _ptr(dL_dout), arr, n_dtex, _ptr(dL_duv), _ptr(dL_ddir), int(flags), int(reps),
              _stream(stream, uv.device), t, ctypes.byref(ms))
    return tuple(int(x) for x in t), float(ms.value)


def rt_locate(ctx: Context, uv, dirs, obj, filter: int = RT_QUADRILINEAR, stream=None):
    """(idx (F, 4) int32 floors, coord (F, 4) float32 continuous coordinates)."""
    F = _gbuffer(uv, dirs, obj)
    idx = torch.empty((F, 4), dtype=torch.int32, device=uv.device)
    coord = torch.empty((F, 4), dtype=torch.float32, device=uv.device)
    _lib.call("rt_locate", ctx.handle, _ptr(uv), _ptr(dirs), _ptr(obj), F, int(filter), _ptr(idx), _ptr(coord),
              _stream(stream, uv.device))
    return idx, coord


def _grad_args(ctx, F, dL_dout, dL_dtex, dL_duv, dL_ddir, flags=0):
    _check(dL_dout, "dL_dout", torch.float32, 4)
    if dL_dout.numel() != 4 * F:
        raise ValueError("dL_dout must hold F x 4 floats")
    if dL_duv is not None:
        _check(dL_duv, "dL_duv", torch.float32, 2)
        if dL_duv.numel() != 2 * F:
            raise ValueError("dL_duv must hold F x 2 floats")
    if dL_ddir is not None:
        _check(dL_ddir, "dL_ddir", torch.float32, 3)
        if dL_ddir.numel() != 3 * F:
            raise ValueError("dL_ddir must hold F x 3 floats")
    n_dtex = 0
    arr = None
    if dL_dtex:
        n_dtex = max(dL_dtex) + 1
        arr = (ctypes.c_void_p * n_dtex)()
        dtype = torch.int64 if flags & RT_FIXED_POINT_GRADS else torch.float32
        for o, t in dL_dtex.items():
            _check(t, f"dL_dtex[{o}]", dtype)
            want = storage_numel(ctx, o)
            if t.numel() != want:
                raise ValueError(f"dL_dtex[{o}] must hold {want} values (the object's storage layout)")
            arr[o] = t.data_ptr()
    return arr, n_dtex


def rt_fixed_to_float(acc: torch.Tensor, dst: torch.Tensor | None = None, flags: int = 0, stream=None,
                      scale: float = 1.0) -> torch.Tensor:
    """FP32 gradients (times `scale`) from the int64 fixed-point sums of RT_FIXED_POINT_GRADS (same shape)."""
    _check(acc, "acc", torch.int64)
    if dst is None:
        dst = torch.empty(acc.shape, dtype=torch.float32, device=acc.device)
    _check(dst, "dst", torch.float32)
    if dst.numel() != acc.numel():
        raise ValueError("dst must hold as many values as acc")
    _lib.call("rt_fixed_to_float", _ptr(acc), _ptr(dst), acc.numel(), float(scale), int(flags),
              _stream(stream, acc.device))
    return dst


def rt_shade_backward(ctx: Context, uv, dirs, obj, filter: int, dL_dout: torch.Tensor, dL_dtex=None,
                      dL_duv: torch.Tensor | None = None, dL_ddir: torch.Tensor | None = None, flags: int = 0,
                      stream=None) -> None:
    """dL_dtex: dict {object id: FP32 CUDA tensor in the object's storage layout} or None."""
    F = _gbuffer(uv, dirs, obj)
    arr, n_dtex = _grad_args(ctx, F, dL_dout, dL_dtex, dL_duv, dL_ddir, flags)
    _lib.call("rt_shade_backward", ctx.handle, _ptr(uv), _ptr(dirs), _ptr(obj), F, int(filter), _ptr(dL_dout),
              arr, n_dtex, _ptr(dL_duv), _ptr(dL_ddir), int(flags), _stream(stream, uv.device))


def rt_bake_shadow(ctx: Context, obj_id: int, surface: int, scene: dict, stream=None) -> None:
    """Visibility bits of an RT_BIT1 texture towards every texel direction (Section 5)."""
    S = bake_scene_struct(scene)
    dev = torch.device("cuda", ctx.device)
    _lib.call("rt_bake_shadow", ctx.handle, int(obj_id), int(surface), ctypes.byref(S), _stream(stream, dev))


def rt_shade_multi(ctx: Context, uv, dirs, obj, filter: int = RT_QUADRILINEAR, out: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
    """Mean of S lookups per fragment: dirs (F, S, 3).  Returns (F, 4)."""
    _check(uv, "uv", torch.float32, 2)
    _check(dirs, "dirs", torch.float32, 3)
    _check(obj, "obj", torch.int32)
    F = obj.numel()
    if uv.numel() != 2 * F or dirs.numel() % (3 * max(F, 1)) != 0:
        raise ValueError("uv must hold F x 2 and dirs F x S x 3 floats")
    S = dirs.numel() // (3 * F) if F else 1
    if out is None:
        out = torch.empty((F, 4), dtype=torch.float32, device=uv.device)
    _check(out, "out", torch.float32, 4)
    _lib.call("rt_shade_multi", ctx.handle, _ptr(uv), _ptr(dirs), int(S), _ptr(obj), F, int(filter), _ptr(out),
              _stream(stream, uv.device))
    return out


def _normals(nrm, F):
    _check(nrm, "nrm", torch.float32, 3)
    if nrm.numel() != 3 * F:
        raise ValueError("nrm must hold F x 3 floats")


def rt_shade_world(ctx: Context, uv, dirs, nrm, obj, filter: int = RT_QUADRILINEAR, out: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
    """World-space synthesis (Eq. 1a, I and N in one frame): (F, 4) float32 colours."""
    F = _gbuffer(uv, dirs, obj)
    _normals(nrm, F)
    if out is None:
        out = torch.empty((F, 4), dtype=torch.float32, device=uv.device)
    _check(out, "out", torch.float32, 4)
    _lib.call("rt_shade_world", ctx.handle, _ptr(uv), _ptr(dirs), _ptr(nrm), _ptr(obj), F, int(filter), _ptr(out),
              _stream(stream, uv.device))
    return out


def rt_locate_world(ctx: Context, uv, dirs, nrm, obj, filter: int = RT_QUADRILINEAR, stream=None):
    F = _gbuffer(uv, dirs, obj)
    _normals(nrm, F)
    idx = torch.empty((F, 4), dtype=torch.int32, device=uv.device)
    coord = torch.empty((F, 4), dtype=torch.float32, device=uv.device)
    _lib.call("rt_locate_world", ctx.handle, _ptr(uv), _ptr(dirs), _ptr(nrm), _ptr(obj), F, int(filter), _ptr(idx),
              _ptr(coord), _stream(stream, uv.device))
    return idx, coord


def rt_shade_world_backward(ctx: Context, uv, dirs, nrm, obj, filter: int, dL_dout: torch.Tensor, dL_dtex=None,
                            dL_duv: torch.Tensor | None = None, dL_ddir: torch.Tensor | None = None,
                            dL_dnrm: torch.Tensor | None = None, flags: int = 0, stream=None) -> None:
    F = _gbuffer(uv, dirs, obj)
    _normals(nrm, F)
    arr, n_dtex = _grad_args(ctx, F, dL_dout, dL_dtex, dL_duv, dL_ddir, flags)
    if dL_dnrm is not None:
        _normals(dL_dnrm, F)
    _lib.call("rt_shade_world_backward", ctx.handle, _ptr(uv), _ptr(dirs), _ptr(nrm), _ptr(obj), F, int(filter),
              _ptr(dL_dout), arr, n_dtex, _ptr(dL_duv), _ptr(dL_ddir), _ptr(dL_dnrm), int(flags),
              _stream(stream, uv.device))


def rt_shade_world_batched(ctx: Context, uv, dirs, nrm, obj, filter: int = RT_QUADRILINEAR, out=None, stream=None):
    """World-space synthesis of views x height x width fragments in screen tiles; uv (V, H, W, 2), dir and
    nrm (V, H, W, 3), obj (V, H, W); returns (V, H, W, 4) colours."""
    F = _gbuffer(uv, dirs, obj)
    V, H, W = _frames(uv, dirs, obj)
    _normals(nrm, F)
    if out is None:
        out = torch.empty((V, H, W, 4), dtype=torch.float32, device=uv.device)
    _check(out, "out", torch.float32, 4)
    _lib.call("rt_shade_world_batched", ctx.handle, _ptr(uv), _ptr(dirs), _ptr(nrm), _ptr(obj), V, H, W,
              int(filter), _ptr(out), _stream(stream, uv.device))
    return out


def rt_shade_world_batched_backward(ctx: Context, uv, dirs, nrm, obj, filter: int, dL_dout: torch.Tensor,
                                    dL_dtex=None, dL_duv=None, dL_ddir=None, dL_dnrm=None, flags: int = 0,
                                    stream=None) -> None:
    F = _gbuffer(uv, dirs, obj)
    V, H, W = _frames(uv, dirs, obj)
    _normals(nrm, F)
    arr, n_dtex = _grad_args(ctx, F, dL_dout, dL_dtex, dL_duv, dL_ddir, flags)
    if dL_dnrm is not None:
        _normals(dL_dnrm, F)
    _lib.call("rt_shade_world_batched_backward", ctx.handle, _ptr(uv), _ptr(dirs), _ptr(nrm), _ptr(obj), V, H, W,
              int(filter), _ptr(dL_dout), arr, n_dtex, _ptr(dL_duv), _ptr(dL_ddir), _ptr(dL_dnrm), int(flags),
              _stream(stream, uv.device))


def rt_footprint(ctx: Context, uv, dirs, obj, filter: int = RT_QUADRILINEAR, n_counts: int = RT_MAX_OBJECTS,
                 stream=None) -> list[int]:
    """Distinct texels read, per object id (synchronises)."""
    F = _gbuffer(uv, dirs, obj)
    counts = (ctypes.c_uint64 * n_counts)()
    _lib.call("rt_footprint", ctx.handle, _ptr(uv), _ptr(dirs), _ptr(obj), F, int(filter), counts, n_counts,
              _stream(stream, uv.device))
    return [int(c) for c in counts]


def rt_convert_layout(src: torch.Tensor, src_layout: int, dst_layout: int, w: int, h: int, n: int,
                      dst: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    _check(src, "src", torch.float32)
    if src.numel() != layout_numel(src_layout, w, h, n):
        raise ValueError("src must be shaped by layout_shape(src_layout, w, h, n)")
    if dst is None:  # zeros: the padding of a quads buffer is not written
        dst = torch.zeros(layout_shape(dst_layout, w, h, n), dtype=torch.float32, device=src.device)
    _check(dst, "dst", torch.float32)
    if dst.numel() != layout_numel(dst_layout, w, h, n):
        raise ValueError("dst must be shaped by layout_shape(dst_layout, w, h, n)")
    _lib.call("rt_convert_layout", _ptr(src), int(src_layout), _ptr(dst), int(dst_layout), int(w), int(h), int(n),
              _stream(stream, src.device))
    return dst


def rt_l2_loss_grad(out: torch.Tensor, target: torch.Tensor, obj: torch.Tensor, scale: float,
                    dL_dout: torch.Tensor | None = None, sums: torch.Tensor | None = None, stream=None) -> None:
    """dL/dout = scale (out - target) on shaded fragments; sums (float64[2]) += (sum of squares, count)."""
    F = obj.numel()
    _check(out, "out", torch.float32, 4)
    _check(target, "target", torch.float32, 4)
    _check(obj, "obj", torch.int32)
    if out.numel() != 4 * F or target.numel() != 4 * F:
        raise ValueError("out and target must hold F x 4 floats")
    if dL_dout is not None:
        _check(dL_dout, "dL_dout", torch.float32, 4)
        if dL_dout.numel() != 4 * F:
            raise ValueError("dL_dout must hold F x 4 floats")
    if sums is not None:
        _check(sums, "sums", torch.float64)
        if sums.numel() < 2:
            raise ValueError("sums holds 2 doubles")
    _lib.call("rt_l2_loss_grad", _ptr(out), _ptr(target), _ptr(obj), F, float(scale), _ptr(dL_dout), _ptr(sums),
              _stream(stream, out.device))


def rt_adam_step(param: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, lr: float, beta1: float,
                 beta2: float, eps: float, step: int, stream=None) -> None:
    for name, t in (("param", param), ("grad", grad), ("m", m), ("v", v)):
        _check(t, name, torch.float32)
        if t.numel() != param.numel():
            raise ValueError("param, grad, m and v must have the same size")
    _lib.call("rt_adam_step", _ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(), float(lr), float(beta1),
              float(beta2), float(eps), int(step), _stream(stream, param.device))


def rt_get_error(ctx: Context, stream=None) -> int:
    """Synchronises the stream and returns (and clears) the sticky device status."""
    st = ctypes.c_int32(0)
    dev = torch.device("cuda", ctx.device)
    _lib.call("rt_get_error", ctx.handle, _stream(stream, dev), ctypes.byref(st))
    return st.value


def rt_checked_limit_extent(ctx: Context, obj_id: int, texels: int) -> int:
    """Checked build: lowers the extent the bounds checks allow for one object
    (returns the status; RT_ERR_UNSUPPORTED from the normal build)."""
    return _lib.lib().rt_checked_limit_extent(ctx.handle, int(obj_id), int(texels))


def rt_status_string(status: int) -> str:
    return _lib.lib().rt_status_string(int(status)).decode()
