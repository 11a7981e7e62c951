"""FP64 CPU oracle for Gaussian splatting with polynomial kernels (arXiv 2603.18707).

TEST INFRASTRUCTURE ONLY. The test suite, the smoke check and the benchmark's
CPU-baseline leg use it; the rendering package never imports it, and this
package imports nothing from the rendering package.

The arithmetic lives in ``gs_oracle.c`` (plain C, double precision, built with
gcc by :func:`build`). This module marshals numpy arrays in and out and applies
the parameter activations of 3DGS (scale = exp(log-scale), opacity =
sigmoid(logit)) in float64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_HDR = os.path.join(_HERE, "gs_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

EXP, POLY1, POLY2CUT, POLY3 = 0, 1, 2, 3
CULL_UNIVERSAL, CULL_OPACITY, CULL_LEGACY3 = 0, 1, 2
RECT_AABB, RECT_CIRCLE = 0, 1
KIND_NAMES = {"exp": EXP, "poly1": POLY1, "poly2": POLY2CUT, "poly3": POLY3}
CULL_NAMES = {"universal": CULL_UNIVERSAL, "opacity": CULL_OPACITY, "legacy3": CULL_LEGACY3}


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (-O2, OpenMP, IEEE semantics)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-std=c11", "-D_DEFAULT_SOURCE",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Camera(C.Structure):
    _fields_ = [("viewmat", C.c_double * 16), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("width", C.c_int),
                ("height", C.c_int), ("znear", C.c_double)]


class Config(C.Structure):
    _fields_ = [("kind", C.c_int), ("c", C.c_double * 4), ("cull", C.c_int),
                ("eps", C.c_double), ("alpha_max", C.c_double), ("t_min", C.c_double),
                ("aa", C.c_int), ("dilation", C.c_double), ("tile_w", C.c_int),
                ("tile_h", C.c_int), ("rect_mode", C.c_int)]


class Splat2D(C.Structure):
    _fields_ = [("visible", C.c_int), ("pad_", C.c_int), ("mean2d", C.c_double * 2),
                ("cov2d", C.c_double * 3), ("conic", C.c_double * 3), ("rho", C.c_double),
                ("opacity", C.c_double), ("depth", C.c_double), ("color", C.c_double * 3),
                ("color_raw", C.c_double * 3), ("xcut", C.c_double), ("rect", C.c_int * 4),
                ("tiles", C.c_longlong)]


_lib = None
_DP = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I64P = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_U64P = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_I32P = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_order.argtypes = [C.c_int]
        L.orc_order.restype = C.c_int
        L.orc_poly.argtypes = [_DP, C.c_int, C.c_double]
        L.orc_poly.restype = C.c_double
        L.orc_first_root.argtypes = [_DP, C.c_int, C.c_double]
        L.orc_first_root.restype = C.c_double
        L.orc_universal_root.argtypes = [C.POINTER(Config)]
        L.orc_universal_root.restype = C.c_double
        L.orc_kernel.argtypes = [C.POINTER(Config), C.c_double, C.c_double]
        L.orc_kernel.restype = C.c_double
        L.orc_kernel_deriv.argtypes = [C.POINTER(Config), C.c_double, C.c_double]
        L.orc_kernel_deriv.restype = C.c_double
        L.orc_xcut.argtypes = [C.POINTER(Config), C.c_double, C.c_double]
        L.orc_xcut.restype = C.c_double
        L.orc_sh_basis.argtypes = [C.c_int, _DP, _DP]
        L.orc_sh_basis.restype = C.c_int
        L.orc_project.argtypes = [C.c_int, _DP, _DP, _DP, _DP, _DP, C.c_int,
                                  C.POINTER(Camera), C.POINTER(Config), C.c_void_p]
        L.orc_project.restype = None
        L.orc_render_untiled.argtypes = [C.c_int, C.c_void_p, C.POINTER(Camera), C.POINTER(Config),
                                         _DP, _DP, _DP, _I64P]
        L.orc_render_untiled.restype = None
        L.orc_render_tiled.argtypes = [C.c_int, C.c_void_p, C.POINTER(Camera), C.POINTER(Config),
                                       _DP, C.c_int, _I32P, _DP, _DP, _I64P, _I64P, _I64P, _DP]
        L.orc_render_tiled.restype = None
        L.orc_render_backward.argtypes = [C.c_int, _DP, _DP, _DP, _DP, _DP, C.c_int,
                                          C.POINTER(Camera), C.POINTER(Config), _DP, _DP,
                                          _DP, _DP, _DP, _DP, _DP, _DP, _DP, _DP, _DP]
        L.orc_render_backward.restype = None
        L.orc_decisions.argtypes = [C.c_int, C.c_void_p, C.POINTER(Camera), C.POINTER(Config), _U64P]
        L.orc_decisions.restype = None
        _lib = L
    return _lib


# --------------------------------------------------------------------------
# Descriptors
# --------------------------------------------------------------------------

def make_camera(viewmat, fx, fy, cx, cy, width, height, znear=0.2) -> Camera:
    cam = Camera()
    vm = np.asarray(viewmat, dtype=np.float64).reshape(16)
    for i in range(16):
        cam.viewmat[i] = float(vm[i])
    cam.fx, cam.fy, cam.cx, cam.cy = float(fx), float(fy), float(cx), float(cy)
    cam.width, cam.height, cam.znear = int(width), int(height), float(znear)
    return cam


def camera_from_dict(d: dict) -> Camera:
    return make_camera(d["viewmat"], d["fx"], d["fy"], d["cx"], d["cy"], d["width"], d["height"],
                       d.get("znear", 0.2))


def make_config(kind="poly1", coeffs=(0.0, 0.0, 0.0, 0.0), cull="opacity", eps=1.0 / 255.0,
                alpha_max=0.99, t_min=1e-4, aa=True, dilation=0.3, tile=(16, 16),
                rect_mode=RECT_AABB) -> Config:
    cfg = Config()
    cfg.kind = KIND_NAMES[kind] if isinstance(kind, str) else int(kind)
    cs = list(coeffs) + [0.0] * (4 - len(coeffs))
    for i in range(4):
        cfg.c[i] = float(cs[i])
    cfg.cull = CULL_NAMES[cull] if isinstance(cull, str) else int(cull)
    cfg.eps, cfg.alpha_max, cfg.t_min = float(eps), float(alpha_max), float(t_min)
    cfg.aa, cfg.dilation = int(bool(aa)), float(dilation)
    cfg.tile_w, cfg.tile_h = int(tile[0]), int(tile[1])
    cfg.rect_mode = int(rect_mode)
    return cfg


# --------------------------------------------------------------------------
# Kernel math
# --------------------------------------------------------------------------

def _c4(c):
    a = np.zeros(4)
    a[:len(c)] = c
    return a


def poly(c, x: float) -> float:
    c = _c4(c)
    return lib().orc_poly(c, len([v for v in c]) - 1, float(x))


def first_root(c, order: int, rhs: float = 0.0) -> float:
    return lib().orc_first_root(_c4(c), int(order), float(rhs))


def universal_root(cfg: Config) -> float:
    return lib().orc_universal_root(C.byref(cfg))


def kernel(cfg: Config, x: float) -> float:
    return lib().orc_kernel(C.byref(cfg), universal_root(cfg), float(x))


def kernel_deriv(cfg: Config, x: float) -> float:
    return lib().orc_kernel_deriv(C.byref(cfg), universal_root(cfg), float(x))


def xcut(cfg: Config, opacity: float) -> float:
    return lib().orc_xcut(C.byref(cfg), universal_root(cfg), float(opacity))


def sh_basis(degree: int, direction) -> np.ndarray:
    d = np.ascontiguousarray(direction, dtype=np.float64)
    Y = np.zeros(16)
    n = lib().orc_sh_basis(int(degree), d, Y)
    return Y[:n].copy()


# --------------------------------------------------------------------------
# Scenes
# --------------------------------------------------------------------------

def activate(scene: dict) -> dict:
    """3DGS parameter activations in float64: exp of log-scales, sigmoid of
    opacity logits. Quaternions are passed raw (the projection normalises)."""
    out = {
        "means": np.ascontiguousarray(scene["means"], dtype=np.float64).reshape(-1, 3),
        "scales": np.exp(np.asarray(scene["log_scales"], dtype=np.float64)).reshape(-1, 3),
        "quats": np.ascontiguousarray(scene["quats"], dtype=np.float64).reshape(-1, 4),
        "opacities": 1.0 / (1.0 + np.exp(-np.asarray(scene["opacity_logits"], dtype=np.float64))),
        "sh": np.ascontiguousarray(scene["sh"], dtype=np.float64),
        "sh_degree": int(scene["sh_degree"]),
    }
    out["sh"] = out["sh"].reshape(out["means"].shape[0], -1, 3)
    return out


def _arrs(sc):
    return (np.ascontiguousarray(sc["means"], dtype=np.float64).reshape(-1),
            np.ascontiguousarray(sc["scales"], dtype=np.float64).reshape(-1),
            np.ascontiguousarray(sc["quats"], dtype=np.float64).reshape(-1),
            np.ascontiguousarray(sc["opacities"], dtype=np.float64).reshape(-1),
            np.ascontiguousarray(sc["sh"], dtype=np.float64).reshape(-1))


def project(sc: dict, cam: Camera, cfg: Config):
    """Per-splat projection records (ctypes array of Splat2D) for activated
    scene arrays ``sc`` (keys means, scales, quats, opacities, sh, sh_degree)."""
    m, s, q, o, sh = _arrs(sc)
    P = m.size // 3
    out = (Splat2D * max(P, 1))()
    lib().orc_project(P, m, s, q, o, sh, int(sc["sh_degree"]), C.byref(cam), C.byref(cfg),
                      C.addressof(out))
    return out


def splats_to_numpy(s2d, P: int) -> dict:
    """Struct-of-arrays view of projection records."""
    dt = np.dtype({"names": [f[0] for f in Splat2D._fields_],
                   "formats": [_np_fmt(f[1]) for f in Splat2D._fields_],
                   "offsets": [getattr(Splat2D, f[0]).offset for f in Splat2D._fields_],
                   "itemsize": C.sizeof(Splat2D)})
    buf = np.frombuffer((C.c_char * (C.sizeof(Splat2D) * max(P, 1))).from_address(C.addressof(s2d)),
                        dtype=dt, count=max(P, 1))[:P]
    return {k: np.array(buf[k]) for k in dt.names if k != "pad_"}


def _np_fmt(ct):
    if hasattr(ct, "_length_"):
        return (_np_fmt(ct._type_), (ct._length_,))
    return {C.c_double: np.float64, C.c_int: np.int32, C.c_longlong: np.int64}[ct]


def render_untiled(sc: dict, cam: Camera, cfg: Config, bg=(0.0, 0.0, 0.0), s2d=None):
    """Unculled per-pixel render over all visible splats (the definition)."""
    if s2d is None:
        s2d = project(sc, cam, cfg)
    P = np.asarray(sc["means"]).size // 3
    H, W = cam.height, cam.width
    img = np.zeros((H, W, 3))
    T = np.zeros((H, W))
    nc = np.zeros((H, W), dtype=np.int64)
    lib().orc_render_untiled(P, C.addressof(s2d), C.byref(cam), C.byref(cfg),
                             np.asarray(bg, dtype=np.float64), img.reshape(-1), T.reshape(-1),
                             nc.reshape(-1))
    return img, T, nc


def render_tiled(sc: dict, cam: Camera, cfg: Config, bg=(0.0, 0.0, 0.0), tiles=None, s2d=None,
                 with_margin: bool = False):
    """Tile-binned render; ``tiles``: iterable of tile ids (default all).
    Returns image, final T, last contributor, evaluations per pixel, list
    length per tile (and, with ``with_margin``, the per-pixel decision
    margin: distance of the closest skip / stop decision from its threshold,
    relative to the threshold plus the change a 0.3 px shift of the splats
    causes; diagnostic, see gs_oracle.c)."""
    if s2d is None:
        s2d = project(sc, cam, cfg)
    P = np.asarray(sc["means"]).size // 3
    H, W = cam.height, cam.width
    tx = (W + cfg.tile_w - 1) // cfg.tile_w
    ty = (H + cfg.tile_h - 1) // cfg.tile_h
    img = np.zeros((H, W, 3))
    T = np.ones((H, W))
    last = np.zeros((H, W), dtype=np.int64)
    nev = np.zeros((H, W), dtype=np.int64)
    llen = np.zeros(tx * ty, dtype=np.int64)
    margin = np.full((H, W), np.inf)
    if tiles is None:
        sel = np.zeros(1, dtype=np.int32)
        nsel = -1
    else:
        sel = np.ascontiguousarray(np.asarray(list(tiles), dtype=np.int32))
        nsel = sel.size
        if nsel == 0:
            sel = np.zeros(1, dtype=np.int32)
    lib().orc_render_tiled(P, C.addressof(s2d), C.byref(cam), C.byref(cfg),
                           np.asarray(bg, dtype=np.float64), nsel, sel, img.reshape(-1),
                           T.reshape(-1), last.reshape(-1), nev.reshape(-1), llen, margin.reshape(-1))
    if with_margin:
        return img, T, last, nev, llen, margin
    return img, T, last, nev, llen


def decisions(sc: dict, cam: Camera, cfg: Config, s2d=None) -> np.ndarray:
    if s2d is None:
        s2d = project(sc, cam, cfg)
    P = np.asarray(sc["means"]).size // 3
    sig = np.zeros(cam.height * cam.width, dtype=np.uint64)
    lib().orc_decisions(P, C.addressof(s2d), C.byref(cam), C.byref(cfg), sig)
    return sig.reshape(cam.height, cam.width)


def render_backward(sc: dict, cam: Camera, cfg: Config, dL_dimg, bg=(0.0, 0.0, 0.0)) -> dict:
    """Analytic reverse pass of the untiled render: gradients with respect to
    means, scales, quaternions (as given), opacities, SH and the 2D
    quantities (mean2d, conic (A, B, C), o', colour)."""
    m, s, q, o, sh = _arrs(sc)
    P = m.size // 3
    K = (int(sc["sh_degree"]) + 1) ** 2
    g = {k: np.zeros(n) for k, n in [("means", 3 * P), ("scales", 3 * P), ("quats", 4 * P),
                                      ("opacities", P), ("sh", K * 3 * P), ("mean2d", 2 * P),
                                      ("conic", 3 * P), ("opacity2d", P), ("color", 3 * P)]}
    lib().orc_render_backward(P, m, s, q, o, sh, int(sc["sh_degree"]), C.byref(cam), C.byref(cfg),
                              np.asarray(bg, dtype=np.float64),
                              np.ascontiguousarray(dL_dimg, dtype=np.float64).reshape(-1),
                              g["means"], g["scales"], g["quats"], g["opacities"], g["sh"],
                              g["mean2d"], g["conic"], g["opacity2d"], g["color"])
    shapes = {"means": (P, 3), "scales": (P, 3), "quats": (P, 4), "opacities": (P,),
              "sh": (P, K, 3), "mean2d": (P, 2), "conic": (P, 3), "opacity2d": (P,),
              "color": (P, 3)}
    return {k: v.reshape(shapes[k]) for k, v in g.items()}
