"""ctypes binding of libgs_b300.so (the C ABI in include/gs.h).

Argument marshalling only: every step of the rendering path runs in the
library's CUDA kernels. The library must have been built (``build()`` in
``paper_2603_18707_b300.build``); there is no fallback — a missing library
raises immediately.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgs_b300.so")

GS_OK, GS_ERR_ARG, GS_ERR_CUDA, GS_ERR_CAPACITY, GS_ERR_TIMEOUT, GS_ERR_UNSUPPORTED = 0, 1, 2, 4, 8, 16
GS_K_EXP, GS_K_POLY1, GS_K_POLY2, GS_K_POLY3 = 0, 1, 2, 3
GS_CULL_UNIVERSAL, GS_CULL_OPACITY, GS_CULL_LEGACY3 = 0, 1, 2
GS_RECT_AABB, GS_RECT_CIRCLE, GS_RECT_ELLIPSE = 0, 1, 2
GS_MAX_CAMERAS = 64
GS_SELFTEST_SCRATCH_BYTES = 4096

KIND = {"exp": GS_K_EXP, "poly1": GS_K_POLY1, "poly2": GS_K_POLY2, "poly3": GS_K_POLY3}
CULL = {"universal": GS_CULL_UNIVERSAL, "opacity": GS_CULL_OPACITY, "legacy3": GS_CULL_LEGACY3}


class GsCamera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 16), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32),
                ("height", C.c_int32), ("znear", C.c_float), ("reserved", C.c_int32)]


class GsConfig(C.Structure):
    _fields_ = [("kind", C.c_int32), ("c", C.c_float * 4), ("cull", C.c_int32),
                ("eps", C.c_float), ("alpha_max", C.c_float), ("t_min", C.c_float),
                ("aa_normalize", C.c_int32), ("aa_dilation", C.c_float), ("tile_w", C.c_int32),
                ("tile_h", C.c_int32), ("rect_mode", C.c_int32), ("batch", C.c_int32),
                ("px_per_thread", C.c_int32), ("fp16x2", C.c_int32), ("tensor_alpha", C.c_int32),
                ("reserved", C.c_int32 * 3)]


class GsError(RuntimeError):
    def __init__(self, where: str, status: int):
        super().__init__(f"{where}: status {status} ({status_string(status)})")
        self.status = status


_lib = None
_vp, _i32, _i64, _sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
_SIGS = {
    "gs_config_default": (_i32, [_i32, _i32, C.POINTER(GsConfig)]),
    "gs_splat2d_bytes": (_sz, [_i32, _i32]),
    "gs_preprocess": (_i32, [_vp, C.POINTER(GsCamera), _i32, _i32, _vp, _vp, _vp, _vp, _vp, _i32,
                             C.POINTER(GsConfig), _vp]),
    "gs_total_tiles": (_i64, [C.POINTER(GsCamera), _i32, C.POINTER(GsConfig)]),
    "gs_bin_sort_workspace_bytes": (_sz, [C.POINTER(GsCamera), _i32, _i32, C.POINTER(GsConfig), _i64]),
    "gs_bin_sort": (_i32, [_vp, C.POINTER(GsCamera), _i32, _i32, C.POINTER(GsConfig), _vp, _i64,
                           _vp, _sz, _vp, _vp, _vp, _vp]),
    "gs_bin_sort_noalloc": (_i32, [_vp, C.POINTER(GsCamera), _i32, _i32, C.POINTER(GsConfig), _vp,
                                   _i64, _vp, _vp, _vp, _vp, _vp]),
    "gs_render_work_bytes": (_sz, []),
    "gs_render": (_i32, [_vp, C.POINTER(GsCamera), _i32, _i32, C.POINTER(GsConfig), _vp, _vp, _vp,
                         C.POINTER(C.c_float), _vp, _vp, _vp, _vp, _vp]),
    "gs_grad2d_bytes": (_sz, [_i32, _i32]),
    "gs_render_backward": (_i32, [_vp, C.POINTER(GsCamera), _i32, _i32, C.POINTER(GsConfig),
                                  _vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp,
                                  C.POINTER(C.c_float), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                  _vp]),
    "gs_workspace_status": (_i32, [_vp, _vp, C.POINTER(_i32)]),
    "gs_workspace_status_async": (_i32, [_vp, _vp, _vp]),
    "gs_render_status_async": (_i32, [_vp, _vp]),
    "gs_spatial_order_workspace_bytes": (_sz, [_i32]),
    "gs_spatial_order": (_i32, [_vp, _i32, _vp, _vp, _vp]),
    "gs_gather_rows": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp]),
    "gs_fma_peak": (_i32, [_vp, _i32, _i32, _i32, _vp, C.POINTER(C.c_double)]),
    "gs_selftest_lookback_timeout": (_i32, [_vp, _i32, _vp, _i32]),
    "gs_launch_count": (C.c_uint64, []),
    "gs_status_string": (C.c_char_p, [_i32]),
}


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2603_18707_b300.build` (nvcc, sm_103a)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_string(status: int) -> str:
    try:
        return lib().gs_status_string(int(status)).decode()
    except Exception:  # noqa: BLE001 - message only
        return "?"


def check(where: str, status: int):
    if status != GS_OK:
        raise GsError(where, status)
