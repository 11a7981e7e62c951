"""The C-ABI library loads on a CPU-only host, exports every entry point
include/*.h declares, and rejects bad arguments on the host (no kernel is
launched in any of these calls)."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2603_18707_b300 import build
    build.build()
    from paper_2603_18707_b300 import _lib
    return _lib


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert "gs_preprocess" in names and "gs_render_backward" in names
    lib = C.CDLL(L.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header(L):
    assert set(_declared()) <= set(L._SIGS)


def test_struct_sizes_match_header(L):
    assert C.sizeof(L.GsCamera) == 16 * 4 + 4 * 4 + 2 * 4 + 4 + 4
    assert C.sizeof(L.GsConfig) == 4 + 16 + 4 * 4 + 4 + 4 + 4 * 3 + 4 * 3 + 16


def test_config_defaults(L):
    from paper_2603_18707_b300 import api
    c = api.make_config("poly1", "opacity")
    assert c.c[0] == pytest.approx(0.773) and c.c[1] == pytest.approx(-0.773 / 4.386)
    assert c.eps == pytest.approx(1 / 255) and c.alpha_max == pytest.approx(0.99)
    assert c.t_min == pytest.approx(1e-4) and c.aa_dilation == pytest.approx(0.3)
    assert (c.tile_w, c.tile_h) == (16, 16) and c.aa_normalize == 1
    e = api.make_config("exp", "universal")
    assert list(e.c) == [0.0, 0.0, 0.0, 0.0]


def test_default_coefficients_match_golden(L):
    """The library's frozen f'2 / f3 coefficients are the oracle fit's."""
    import json
    from paper_2603_18707_b300 import api
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "coeffs.json")))
    for kind in ("poly1", "poly2", "poly3"):
        c = api.make_config(kind, "opacity")
        assert list(c.c) == pytest.approx(gold[kind], rel=1e-6, abs=1e-9)
    for tile, c in api.F2_RANGE.items():
        assert list(c) == pytest.approx(gold["poly2_range"][str(tile)][:3], rel=1e-12)


def test_sizes_and_tiles(L):
    from paper_2603_18707_b300 import api, synth
    cams = [synth.camera_small(128, 128), synth.camera_small(100, 75)]
    cfg = api.make_config("poly1", "opacity")
    assert api.gs_total_tiles(cams, cfg) == 64 + 7 * 5
    cfg8 = api.make_config("poly1", "opacity", tile=(8, 8))
    assert api.gs_total_tiles(cams, cfg8) == 256 + 13 * 10
    assert api.gs_splat2d_bytes(2, 1000) >= 2 * 1000 * 64
    assert api.gs_bin_sort_workspace_bytes(cams, 500, cfg, 5000) > 8 * 5000 + 16 * 1000
    assert api.gs_bin_sort_workspace_bytes(cams, -1, cfg, 5000) == 0
    assert api.gs_bin_sort_workspace_bytes(cams, 500, cfg, -1) == 0


def test_host_argument_checks(L):
    """Every entry point rejects invalid arguments before touching the GPU."""
    from paper_2603_18707_b300 import api
    from paper_2603_18707_b300._lib import GS_ERR_ARG, GS_ERR_UNSUPPORTED, lib
    lb = lib()
    cams = api.camera_array([{"viewmat": [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 3], [0, 0, 0, 1]],
                              "fx": 100, "fy": 100, "cx": 64, "cy": 64, "width": 128,
                              "height": 128}])
    cfg = api.make_config("poly1", "opacity")
    ptr = C.c_void_p(256)
    # null pointers / negative sizes / too many cameras
    assert lb.gs_preprocess(None, cams, 1, 10, None, None, None, None, None, 0, C.byref(cfg), None) == GS_ERR_ARG
    assert lb.gs_preprocess(None, cams, 0, 10, ptr, ptr, ptr, ptr, ptr, 0, C.byref(cfg), ptr) == GS_ERR_ARG
    assert lb.gs_preprocess(None, cams, 65, 10, ptr, ptr, ptr, ptr, ptr, 0, C.byref(cfg), ptr) == GS_ERR_ARG
    assert lb.gs_preprocess(None, cams, 1, 10, ptr, ptr, ptr, ptr, ptr, 4, C.byref(cfg), ptr) == GS_ERR_ARG
    # misaligned record buffer
    assert lb.gs_preprocess(None, cams, 1, 10, ptr, ptr, ptr, ptr, ptr, 0, C.byref(cfg),
                            C.c_void_p(260)) == GS_ERR_ARG
    # bad config fields
    for field, val in (("kind", 7), ("cull", 5), ("eps", 0.0), ("alpha_max", 1.5), ("tile_w", 12),
                       ("tile_h", 64), ("t_min", -1.0)):
        bad = api.make_config("poly1", "opacity")
        setattr(bad, field, val)
        assert lb.gs_preprocess(None, cams, 1, 10, ptr, ptr, ptr, ptr, ptr, 0, C.byref(bad), ptr) == GS_ERR_ARG
    # polynomial that never reaches zero
    bad = api.make_config("poly1", "opacity", coeffs=(0.5, 0.1))
    assert lb.gs_preprocess(None, cams, 1, 10, ptr, ptr, ptr, ptr, ptr, 0, C.byref(bad), ptr) == GS_ERR_ARG
    # camera with non-positive focal length / near plane
    badcam = api.camera_array([{"viewmat": [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 3], [0, 0, 0, 1]],
                                "fx": 0.0, "fy": 100, "cx": 64, "cy": 64, "width": 128,
                                "height": 128}])
    assert lb.gs_preprocess(None, badcam, 1, 10, ptr, ptr, ptr, ptr, ptr, 0, C.byref(cfg), ptr) == GS_ERR_ARG
    # workspace too small / unaligned; capacity beyond 2^30
    assert lb.gs_bin_sort(None, cams, 1, 10, C.byref(cfg), ptr, 100, ptr, 16, ptr, ptr, None, None) == GS_ERR_ARG
    assert lb.gs_bin_sort(None, cams, 1, 10, C.byref(cfg), ptr, 1 << 31, ptr, 1 << 40, ptr, ptr, None, None) == GS_ERR_ARG
    assert lb.gs_bin_sort(None, cams, 1, 10, C.byref(cfg), ptr, 100, C.c_void_p(300), 1 << 30, ptr, ptr, None, None) == GS_ERR_ARG
    bg = (C.c_float * 3)(0, 0, 0)
    assert lb.gs_render(None, cams, 1, 10, C.byref(cfg), None, None, None, bg, None, None, None, None,
                        None) == GS_ERR_ARG
    bad = api.make_config("poly1", "opacity")
    bad.batch = 512
    assert lb.gs_render(None, cams, 1, 10, C.byref(bad), ptr, ptr, ptr, bg, ptr, None, None, None,
                        None) == GS_ERR_ARG
    bad = api.make_config("poly1", "opacity", tensor_alpha=3)
    assert lb.gs_render(None, cams, 1, 10, C.byref(bad), ptr, ptr, ptr, bg, ptr, None, None, None,
                        None) == GS_ERR_ARG
    bad = api.make_config("poly1", "opacity", tensor_alpha=1, tile=(8, 8))
    assert lb.gs_render(None, cams, 1, 10, C.byref(bad), ptr, ptr, ptr, bg, ptr, None, None, None,
                        None) == GS_ERR_UNSUPPORTED
    bad = api.make_config("poly1", "opacity", px_per_thread=3)
    assert lb.gs_render(None, cams, 1, 10, C.byref(bad), ptr, ptr, ptr, bg, ptr, None, None, None,
                        None) == GS_ERR_ARG
    code = C.c_int32()
    assert lb.gs_workspace_status(None, None, C.byref(code)) == GS_ERR_ARG
    assert lb.gs_selftest_lookback_timeout(None, 0, None, 100) == GS_ERR_ARG
    assert lb.gs_selftest_lookback_timeout(None, 3, ptr, 100) == GS_ERR_ARG
    assert lb.gs_render_status_async(None, None) == GS_ERR_ARG
    assert lb.gs_selftest_lookback_timeout(None, 1, ptr, 0) == GS_ERR_ARG
    assert lb.gs_selftest_lookback_timeout(None, 1, ptr, (1 << 20) + 1) == GS_ERR_ARG
    flop = C.c_double()
    assert lb.gs_fma_peak(None, 0, 0, 10, ptr, C.byref(flop)) == GS_ERR_ARG
    assert lb.gs_fma_peak(None, 2, 1, 10, ptr, C.byref(flop)) == GS_ERR_ARG
    assert lb.gs_fma_peak(None, 0, 1, 0, ptr, C.byref(flop)) == GS_ERR_ARG
    assert lb.gs_fma_peak(None, 1, 1, 10, None, C.byref(flop)) == GS_ERR_ARG
    # scene preparation: sizes, null / misaligned pointers; P = 0 and n = 0 do nothing
    assert lb.gs_spatial_order_workspace_bytes(-1) == 0
    assert lb.gs_spatial_order_workspace_bytes(1000) > 1000 * 12
    assert lb.gs_spatial_order(None, -1, ptr, ptr, ptr) == GS_ERR_ARG
    assert lb.gs_spatial_order(None, 1 << 30, ptr, ptr, ptr) == GS_ERR_ARG
    assert lb.gs_spatial_order(None, 10, None, ptr, ptr) == GS_ERR_ARG
    assert lb.gs_spatial_order(None, 10, ptr, C.c_void_p(260), ptr) == GS_ERR_ARG
    assert lb.gs_spatial_order(None, 0, None, None, None) == 0
    assert lb.gs_gather_rows(None, 10, 6, ptr, ptr, ptr) == GS_ERR_ARG
    assert lb.gs_gather_rows(None, 10, 0, ptr, ptr, ptr) == GS_ERR_ARG
    assert lb.gs_gather_rows(None, -1, 4, ptr, ptr, ptr) == GS_ERR_ARG
    assert lb.gs_gather_rows(None, 10, 4, ptr, None, ptr) == GS_ERR_ARG
    assert lb.gs_gather_rows(None, 10, 4, C.c_void_p(258), ptr, ptr) == GS_ERR_ARG
    assert lb.gs_gather_rows(None, 0, 4, None, None, None) == 0
    assert lb.gs_status_string(4) == b"overlap capacity exceeded"


def test_missing_library_fails_loudly(L, monkeypatch):
    """No CPU fallback: without the built library every entry point raises."""
    from paper_2603_18707_b300 import _lib, api
    monkeypatch.setattr(_lib, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libgs_b300.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        _lib.lib()
    with pytest.raises(RuntimeError, match="missing"):
        api.make_config("poly1", "opacity")
