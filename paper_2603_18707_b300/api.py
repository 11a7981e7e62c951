"""Python binding of the C ABI with the same entry-point names.

Marshalling only: torch tensors are passed as device pointers, the current
torch CUDA stream is passed as the stream, cameras and configs as ctypes
structs. Nothing here computes any part of the rendering path.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import GsCamera, GsConfig, check, lib


def make_camera(d: dict) -> GsCamera:
    """ctypes camera from a dict with viewmat (4x4 world->camera, row-major),
    fx, fy, cx, cy, width, height and optional znear."""
    c = GsCamera()
    vm = np.asarray(d["viewmat"], dtype=np.float64).reshape(16)
    for i in range(16):
        c.viewmat[i] = float(vm[i])
    c.fx, c.fy, c.cx, c.cy = float(d["fx"]), float(d["fy"]), float(d["cx"]), float(d["cy"])
    c.width, c.height = int(d["width"]), int(d["height"])
    c.znear = float(d.get("znear", 0.2))
    return c


def camera_array(cams) -> C.Array:
    cams = list(cams)
    if not 1 <= len(cams) <= _lib.GS_MAX_CAMERAS:
        raise ValueError(f"1..{_lib.GS_MAX_CAMERAS} cameras per call")
    arr = (GsCamera * len(cams))()
    for i, d in enumerate(cams):
        arr[i] = d if isinstance(d, GsCamera) else make_camera(d)
    return arr


# f2 = max(c0 + c1 x + c2 x^2, 0) fitted by the Sec. 3.1 L1 procedure over the
# quadric range a tile renderer evaluates, [0, x_max(tile)] with
# x_max = (sqrt(2) tile / sqrt(0.3) + sqrt(-2 ln(1/255)))^2 (App. A), per tile
# size in pixels. The second root sits at x_max, so GS_K_POLY2 (cut at the
# first root) renders it exactly: make_config("poly2", coeffs=F2_RANGE[16]).
F2_RANGE = {8: (0.7706480720543922, -0.1763059655625171, 0.0003041422547261449),
            16: (0.7700231846428013, -0.17549960677781712, 8.787264296324024e-05)}


def make_config(kind="poly1", cull="opacity", **over) -> GsConfig:
    """Library defaults for a kernel kind and cull mode (gs_config_default),
    then field overrides, e.g. tile=(8, 8), coeffs=(...), aa=False."""
    cfg = GsConfig()
    k = _lib.KIND[kind] if isinstance(kind, str) else int(kind)
    cu = _lib.CULL[cull] if isinstance(cull, str) else int(cull)
    check("gs_config_default", lib().gs_config_default(k, cu, C.byref(cfg)))
    for key, val in over.items():
        if key == "tile":
            cfg.tile_w, cfg.tile_h = int(val[0]), int(val[1])
        elif key == "coeffs":
            vals = list(val) + [0.0] * (4 - len(val))
            for i in range(4):
                cfg.c[i] = float(vals[i])
        elif key == "aa":
            cfg.aa_normalize = int(bool(val))
        elif key == "rect":
            cfg.rect_mode = {"aabb": _lib.GS_RECT_AABB, "circle": _lib.GS_RECT_CIRCLE,
                             "ellipse": _lib.GS_RECT_ELLIPSE}[val]
        else:
            setattr(cfg, key, val)
    return cfg


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _p(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return t.data_ptr()


def _f32(t):
    if t is not None and t.dtype != torch.float32:
        raise ValueError("float32 tensor expected")
    return _p(t)


def gs_splat2d_bytes(ncam: int, P: int) -> int:
    return int(lib().gs_splat2d_bytes(ncam, P))


def gs_total_tiles(cams, cfg: GsConfig) -> int:
    arr = camera_array(cams)
    return int(lib().gs_total_tiles(arr, len(arr), C.byref(cfg)))


def gs_bin_sort_workspace_bytes(cams, P: int, cfg: GsConfig, capacity: int) -> int:
    arr = camera_array(cams)
    return int(lib().gs_bin_sort_workspace_bytes(arr, len(arr), int(P), C.byref(cfg), int(capacity)))


def gs_grad2d_bytes(ncam: int, P: int) -> int:
    return int(lib().gs_grad2d_bytes(ncam, P))


def gs_preprocess(cams, P, means, scales, quats, opacities, sh, sh_degree, cfg, splat2d, stream=None):
    arr = camera_array(cams)
    check("gs_preprocess", lib().gs_preprocess(
        _stream(stream), arr, len(arr), int(P), _f32(means), _f32(scales), _f32(quats),
        _f32(opacities), _f32(sh), int(sh_degree), C.byref(cfg), _p(splat2d)))


def gs_bin_sort(cams, P, cfg, splat2d, capacity, workspace, vals, ranges, keys64=None, count=None,
                stream=None):
    arr = camera_array(cams)
    check("gs_bin_sort", lib().gs_bin_sort(
        _stream(stream), arr, len(arr), int(P), C.byref(cfg), _p(splat2d), int(capacity),
        _p(workspace), workspace.numel() * workspace.element_size(), _p(vals), _p(ranges),
        _p(keys64), _p(count)))


def gs_bin_sort_noalloc(cams, P, cfg, splat2d, capacity, vals, ranges, keys64=None, count=None,
                        error=None, stream=None):
    """gs_bin_sort for callers that cannot allocate device memory: the
    scratch is the library's static device array (GS_NOALLOC_WORKSPACE_BYTES),
    shared by every call on a device. error: optional uint32 buffer that
    receives this call's device error word."""
    arr = camera_array(cams)
    check("gs_bin_sort_noalloc", lib().gs_bin_sort_noalloc(
        _stream(stream), arr, len(arr), int(P), C.byref(cfg), _p(splat2d), int(capacity),
        _p(vals), _p(ranges), _p(keys64), _p(count), _p(error)))


def gs_render_work_bytes() -> int:
    return int(lib().gs_render_work_bytes())


def gs_render(cams, P, cfg, splat2d, vals, ranges, bg, out_rgb, final_T=None, last=None,
              n_eval=None, work=None, stream=None):
    """work: None (one CTA per tile) or a device buffer of
    gs_render_work_bytes() bytes (one persistent launch)."""
    arr = camera_array(cams)
    bgc = (C.c_float * 3)(*[float(v) for v in bg])
    check("gs_render", lib().gs_render(
        _stream(stream), arr, len(arr), int(P), C.byref(cfg), _p(splat2d), _p(vals), _p(ranges),
        bgc, _f32(out_rgb), _f32(final_T), _p(last), _p(n_eval), _p(work)))


def gs_render_backward(cams, P, cfg, means, scales, quats, opacities, sh, sh_degree, splat2d, vals,
                       ranges, bg, final_T, last, grad_out, grad2d, grad_means, grad_scales,
                       grad_quats, grad_opacities, grad_sh, stream=None):
    arr = camera_array(cams)
    bgc = (C.c_float * 3)(*[float(v) for v in bg])
    check("gs_render_backward", lib().gs_render_backward(
        _stream(stream), arr, len(arr), int(P), C.byref(cfg), _f32(means), _f32(scales),
        _f32(quats), _f32(opacities), _f32(sh), int(sh_degree), _p(splat2d), _p(vals),
        _p(ranges), bgc, _f32(final_T), _p(last), _f32(grad_out), _p(grad2d), _f32(grad_means),
        _f32(grad_scales), _f32(grad_quats), _f32(grad_opacities), _f32(grad_sh)))


def gs_workspace_status(workspace, stream=None) -> int:
    code = C.c_int32(0)
    check("gs_workspace_status", lib().gs_workspace_status(_stream(stream), _p(workspace),
                                                           C.byref(code)))
    return int(code.value)


def gs_workspace_status_async(workspace, dst, stream=None) -> None:
    """Enqueues a copy of the workspace's error word into dst (a 4-byte
    device or pinned host tensor) and clears the word, without waiting."""
    check("gs_workspace_status_async", lib().gs_workspace_status_async(_stream(stream), _p(workspace),
                                                                       _p(dst)))


def gs_render_status_async(dst, stream=None) -> None:
    """Enqueues a copy of the blend's device error word (GS_ERR_TIMEOUT when
    a wait of the tcgen05 variant gave up) into dst (a 4-byte device or
    pinned host tensor) and clears it."""
    check("gs_render_status_async", lib().gs_render_status_async(_stream(stream), _p(dst)))


def gs_spatial_order(means, stream=None):
    """Z-order permutation of the splats (int32 tensor [P]; see gs.h):
    store a scene in this order once when it is loaded."""
    P = int(means.shape[0])
    perm = torch.empty(max(P, 1), dtype=torch.int32, device=means.device)
    if P:
        ws = torch.empty(lib().gs_spatial_order_workspace_bytes(P), dtype=torch.uint8, device=means.device)
        check("gs_spatial_order", lib().gs_spatial_order(_stream(stream), P, _f32(means), _p(ws), _p(perm)))
    return perm[:P]


def gs_gather_rows(src, perm, dst=None, stream=None):
    """dst[k] = src[perm[k]] row-wise (any 4-byte dtype layout; rows are the
    first dimension)."""
    n = int(perm.shape[0])
    if dst is None:
        dst = torch.empty((n,) + tuple(src.shape[1:]), dtype=src.dtype, device=src.device)
    row = src[0].numel() * src.element_size() if src.shape[0] else 4
    if dst.shape[1:] != src.shape[1:] or dst.dtype != src.dtype or dst.shape[0] != n:
        raise ValueError("dst must have perm's length and src's row shape and dtype")
    check("gs_gather_rows", lib().gs_gather_rows(_stream(stream), n, int(row), _p(src), _p(perm), _p(dst)))
    return dst


def gs_selftest_lookback_timeout(which: int, scratch, spin_limit: int, stream=None) -> None:
    """Runs a look-back against a predecessor that never publishes (which 0:
    scalar, 1: per digit); the error word scratch[0] then holds
    GS_ERR_TIMEOUT. scratch: int32/uint32 device tensor of
    GS_SELFTEST_SCRATCH_BYTES bytes."""
    check("gs_selftest_lookback_timeout",
          lib().gs_selftest_lookback_timeout(_stream(stream), int(which), _p(scratch), int(spin_limit)))


def gs_fma_peak(half2: bool, blocks: int, iters: int, sink, stream=None) -> float:
    """Launches the FFMA (half2=False) or HFMA2 peak microbenchmark on the
    stream; returns the FLOP it performs (time it with events)."""
    flop = C.c_double(0.0)
    check("gs_fma_peak", lib().gs_fma_peak(_stream(stream), int(bool(half2)), int(blocks), int(iters),
                                           _p(sink), C.byref(flop)))
    return float(flop.value)


def gs_launch_count() -> int:
    return int(lib().gs_launch_count())
