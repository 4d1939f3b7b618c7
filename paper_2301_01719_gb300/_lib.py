"""ctypes binding of libradtex (include/radtex.h): the C entry points, same names.

Argument marshalling only.  The library must have been built (``build.build()``
or ``__graft_entry__.build()``); if it is missing, loading raises instead of
falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# RADTEX_CHECKED=1 in the environment loads the bounds-checked build instead
# (libradtex_checked.so: the same entry points, every computed texel address
# checked on the device).
CHECKED = os.environ.get("RADTEX_CHECKED", "0") not in ("", "0")
LIB_PATH = os.path.join(HERE, "libradtex_checked.so" if CHECKED else "libradtex.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "radtex.h")

# rt_status
RT_OK, RT_ERR_INVALID_ARG, RT_ERR_OOM, RT_ERR_CUDA, RT_ERR_BAD_OBJ_ID, RT_ERR_NONFINITE, RT_ERR_TIMEOUT, \
    RT_ERR_UNSUPPORTED, RT_ERR_OUT_OF_BOUNDS = range(9)
# rt_format
RT_F32, RT_F16, RT_BF16, RT_E4M3_BUCKET_SCALE, RT_BIT1 = range(5)
# rt_filter
RT_NEAREST, RT_ANGULAR_BILINEAR, RT_QUADRILINEAR = range(3)
# rt_layout
RT_LAYOUT_ATLAS, RT_LAYOUT_PLANES, RT_LAYOUT_PALETTE, RT_LAYOUT_QUADS = range(4)  # PALETTE: reported by rt_texture_info
RT_BORROW = 1
RT_WRAP_U = 2
RT_WRAP_V = 4
RT_ACCUMULATE = 1
RT_DETERMINISTIC = 2
RT_FIXED_POINT_GRADS = 4
RT_ACCUMULATE_TEXELS = 8
RT_MAX_OBJECTS = 1024
RT_MAX_AO_DIRECTIONS = 1024
RT_SURFACE_SPHERE, RT_SURFACE_PLANE = range(2)


class BakeScene(ctypes.Structure):
    """rt_bake_scene: the analytic scene that rt_bake ray traces (all floats)."""
    _fields_ = [("sphere_centre", ctypes.c_float * 3), ("sphere_radius", ctypes.c_float),
                ("plane_height", ctypes.c_float), ("plane_half_extent", ctypes.c_float),
                ("sphere_albedo", ctypes.c_float * 3), ("sphere_reflectance", ctypes.c_float),
                ("plane_albedo", ctypes.c_float * 3), ("plane_reflectance", ctypes.c_float),
                ("plane_frequency", ctypes.c_float), ("sun_direction", ctypes.c_float * 3),
                ("sun_rgb", ctypes.c_float * 3), ("sun_exponent", ctypes.c_float),
                ("sky_zenith", ctypes.c_float * 3), ("sky_horizon", ctypes.c_float * 3),
                ("ambient", ctypes.c_float), ("fog", ctypes.c_float), ("ray_offset", ctypes.c_float)]

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64

SIGNATURES = {
    "rt_context_create": (_I32, [ctypes.c_int, ctypes.POINTER(_P)]),
    "rt_context_destroy": (None, [_P]),
    "rt_create_texture": (_I32, [_P, _I32, _I32, _I32, _I32, _I32, _P, _I32, ctypes.POINTER(_I32)]),
    "rt_destroy_texture": (_I32, [_P, _I32]),
    "rt_texture_info": (_I32, [_P, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                               ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I64)]),
    "rt_read_texture": (_I32, [_P, _I32, _I32, _P, _P, _P]),
    "rt_fill_bucket_lobes": (_I32, [_P, _I32, _P, _P]),
    "rt_bake": (_I32, [_P, _I32, _I32, _P, _P]),
    "rt_bake_deferred": (_I32, [_P, _I32, _I32, _P, _P, _I32, _P]),
    "rt_shade_world": (_I32, [_P, _P, _P, _P, _P, _I64, _I32, _P, _P]),
    "rt_bake_shadow": (_I32, [_P, _I32, _I32, _P, _P]),
    "rt_shade_multi": (_I32, [_P, _P, _P, _I32, _P, _I64, _I32, _P, _P]),
    "rt_locate_world": (_I32, [_P, _P, _P, _P, _P, _I64, _I32, _P, _P, _P]),
    "rt_shade_world_backward": (_I32, [_P, _P, _P, _P, _P, _I64, _I32, _P, _P, _I32, _P, _P, _P, _I32, _P]),
    "rt_shade_world_batched": (_I32, [_P, _P, _P, _P, _P, _I32, _I32, _I32, _I32, _P, _P]),
    "rt_shade_world_batched_backward": (_I32, [_P, _P, _P, _P, _P, _I32, _I32, _I32, _I32, _P, ctypes.POINTER(_P),
                                               _I32, _P, _P, _P, _I32, _P]),
    "rt_create_palette_texture": (_I32, [_P, _I32, _I32, _I32, _I32, _I32, _I32, _P, _P, _I32, _P]),
    "rt_palette_size": (_I32, [_P, _I32, _P]),
    "rt_kmeans_init": (_I32, [_P, _I32, _I32, _P, _P, _P]),
    "rt_kmeans_tc_scratch_bytes": (_I64, [_I32, _I32, _I32, _I32]),
    "rt_kmeans_assign_tc": (_I32, [_P, _I32, _I32, _P, _P, _P, _P, _I64, _P]),
    "rt_kmeans_assign": (_I32, [_P, _I32, _I32, _P, _P, _P, _P]),
    "rt_kmeans_update": (_I32, [_P, _I32, _I32, _P, _P, _P, _P]),
    "rt_shade": (_I32, [_P, _P, _P, _P, _I64, _I32, _P, _P]),
    "rt_locate": (_I32, [_P, _P, _P, _P, _I64, _I32, _P, _P, _P]),
    "rt_shade_backward": (_I32, [_P, _P, _P, _P, _I64, _I32, _P, ctypes.POINTER(_P), _I32, _P, _P, _I32, _P]),
    "rt_shade_batched": (_I32, [_P, _P, _P, _P, _I32, _I32, _I32, _I32, _P, _P]),
    "rt_shade_batched_backward": (_I32, [_P, _P, _P, _P, _I32, _I32, _I32, _I32, _P, ctypes.POINTER(_P), _I32, _P,
                                         _P, _I32, _P]),
    "rt_shade_batched_l2_step": (_I32, [_P, _P, _P, _P, _I32, _I32, _I32, _I32, _P, ctypes.c_float, _P, _P,
                                        ctypes.POINTER(_P), _I32, _P, _P, _I32, _P]),
    "rt_prepare_deterministic": (_I32, [_P]),
    "rt_set_tile": (_I32, [_P, _I32, _I32, _I32, _I32, _I32]),
    "rt_set_backward_tile": (_I32, [_P, _I32, _I32, _I32, _I32, _I32]),
    "rt_get_tile": (_I32, [_P, _I32, ctypes.POINTER(_I32)]),
    "rt_get_backward_tile": (_I32, [_P, _I32, ctypes.POINTER(_I32)]),
    "rt_autotune": (_I32, [_P, _P, _P, _P, _I32, _I32, _I32, _I32, _P, _I32, _P, ctypes.POINTER(_I32),
                           ctypes.POINTER(ctypes.c_float)]),
    "rt_autotune_backward": (_I32, [_P, _P, _P, _P, _I32, _I32, _I32, _I32, _P, ctypes.POINTER(_P), _I32, _P, _P,
                                    _I32, _I32, _P, ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_float)]),
    "rt_footprint": (_I32, [_P, _P, _P, _P, _I64, _I32, ctypes.POINTER(ctypes.c_uint64), _I32, _P]),
    "rt_footprint_noalloc": (_I32, [_P, _P, _P, _P, _I64, _I32, _P, _I32, _P]),
    "rt_zero_texture_grads": (_I32, [_P, _P, _I32, _P]),
    "rt_set_wait_limit": (_I32, [_P, ctypes.c_uint32]),
    "rt_fixed_to_float": (_I32, [_P, _P, _I64, ctypes.c_double, _I32, _P]),
    "rt_l2_loss_grad": (_I32, [_P, _P, _P, _I64, ctypes.c_float, _P, _P, _P]),
    "rt_adam_step": (_I32, [_P, _P, _P, _P, _I64, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                            _I32, _P]),
    "rt_convert_layout": (_I32, [_P, _I32, _P, _I32, _I32, _I32, _I32, _P]),
    "rt_get_error": (_I32, [_P, _P, ctypes.POINTER(_I32)]),
    "rt_status_string": (ctypes.c_char_p, [_I32]),
    "rt_checked_limit_extent": (_I32, [_P, _I32, _I64]),
}

_lock = threading.Lock()
_lib = None


class RadtexError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        msg = lib().rt_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{fn} failed: {msg} (status {status})")


def header_symbols() -> list[str]:
    """Every function the public header declares."""
    with open(HEADER) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:rt_status|void|int64_t|const char\*)\s+(rt_\w+)\s*\(", text, flags=re.M)))


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is not built; run paper_2301_01719_gb300.build.build() "
                                   "(or __graft_entry__.build()) first")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def check(fn: str, status: int) -> None:
    if status != RT_OK:
        raise RadtexError(fn, status)


def call(name: str, *args) -> None:
    check(name, getattr(lib(), name)(*args))
