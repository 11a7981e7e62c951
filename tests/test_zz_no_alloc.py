"""gs_bin_sort_noalloc: binning for callers that cannot allocate device
memory (a plugin whose host application owns every allocation, a frame loop
that may not allocate once it is running). Through the C ABI it must give
exactly what gs_bin_sort gives with a caller-allocated workspace, call after
call, although every call shares one static scratch array. This file is
collected last on purpose."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2603_18707_b300 import build
    build.build()
    from paper_2603_18707_b300 import api, render, synth
    return api, render, synth


def _noalloc(api, R, capacity):
    """Output buffers pre-filled with garbage, then one no-alloc call. The
    buffers are allocated by torch before the call; around the call itself
    the device's free memory must not change (the call allocates nothing)."""
    vals = torch.full((capacity,), -1, dtype=torch.int32, device="cuda")
    ranges = torch.full((2 * R.total_tiles,), -7, dtype=torch.int32, device="cuda")
    keys = torch.full((capacity,), -3, dtype=torch.int64, device="cuda")
    count = torch.full((3,), -5, dtype=torch.int32, device="cuda")
    err = torch.full((1,), -9, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    api.gs_bin_sort_noalloc(R.cams, R.P, R.cfg, R.splat2d, capacity, vals, ranges, keys, count, err)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    return vals, ranges, keys, count, int(err.item()), free0 - free1


def test_noalloc_matches_workspace_path_twice(gs):
    api, render, synth = gs
    cams = [synth.camera_small(128, 128), synth.camera_small(100, 75)]
    cfg = api.make_config("poly1", "opacity")
    # set-up call (P = 0): the first call on a device may load the library's
    # static array; every call after it must leave free memory unchanged
    ranges0 = torch.zeros(2 * api.gs_total_tiles(cams, cfg), dtype=torch.int32, device="cuda")
    api.gs_bin_sort_noalloc(cams, 0, cfg, None, 0, None, ranges0)
    torch.cuda.synchronize()
    for seed in (0, 1):  # two calls in a row, different scenes, one shared scratch
        raw = synth.scene_uniform(4096, seed)
        R = render.Rasterizer(cams, cfg, 4096, keep_keys=True)
        R.forward(render.activate(raw))  # records + the workspace path's binning
        torch.cuda.synchronize()
        n_over = R.n_records()[1]
        capacity = n_over + 1000
        assert api.gs_bin_sort_workspace_bytes(R.cams, R.P, cfg, capacity) <= 32 << 20
        vals, ranges, keys, count, err, grew = _noalloc(api, R, capacity)
        assert err == 0
        assert grew == 0, f"free device memory fell by {grew} bytes during the call"
        assert torch.equal(count, R.count)
        assert torch.equal(vals[:n_over], R.vals[:n_over])
        assert torch.equal(keys[:n_over], R.keys64[:n_over])
        assert torch.equal(ranges, R.ranges)
        out = torch.empty_like(R.out)
        api.gs_render(R.cams, R.P, cfg, R.splat2d, vals, ranges, (0.0, 0.0, 0.0), out)
        torch.cuda.synchronize()
        assert torch.equal(out, R.out)


def test_noalloc_reports_capacity_overflow_in_its_error_word(gs):
    """The error word lives in the static array, so the call hands it out
    through d_error: an overflowing capacity reads GS_ERR_CAPACITY, and the
    next call that fits reads 0 again (each call starts from a clear word)."""
    api, render, synth = gs
    from paper_2603_18707_b300._lib import GS_ERR_CAPACITY
    cams = [synth.camera_small(128, 128)]
    cfg = api.make_config("poly1", "opacity")
    R = render.Rasterizer(cams, cfg, 4096, keep_keys=True)
    R.forward(render.activate(synth.scene_uniform(4096, 2)))
    torch.cuda.synchronize()
    n_over = R.n_records()[1]
    _, _, _, count, err, _ = _noalloc(api, R, n_over // 2)
    assert err == GS_ERR_CAPACITY
    assert int(count[2]) == n_over  # overlaps counted: the capacity a retry needs
    vals, ranges, _, count, err, _ = _noalloc(api, R, n_over)
    assert err == 0
    assert torch.equal(vals[:n_over], R.vals[:n_over]) and torch.equal(ranges, R.ranges)


def test_noalloc_rejects_sizes_beyond_the_static_scratch(gs):
    api, render, synth = gs
    from paper_2603_18707_b300._lib import GS_ERR_ARG, GsError
    cams = [synth.camera_small(128, 128)]
    cfg = api.make_config("poly1", "opacity")
    R = render.Rasterizer(cams, cfg, 4096)
    too_many = 4 << 20  # overlaps: at 13 bytes each they alone exceed 32 MiB
    with pytest.raises(GsError) as e:
        api.gs_bin_sort_noalloc(cams, 4096, cfg, R.splat2d, too_many, R.vals, R.ranges)
    assert e.value.status == GS_ERR_ARG
