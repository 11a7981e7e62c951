"""Failure detection on the GPU without a fault: the decoupled look-backs of
gs_bin_sort are run against a predecessor that never publishes (a flag that
nothing sets), and the tcgen05 blend's mbarrier wait against a barrier that
no arrival completes. The bounded wait must give up, report GS_ERR_TIMEOUT
through the error word and return, and the context must stay usable."""
import time

import pytest
import torch

from paper_2603_18707_b300 import _lib, api

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", [0, 1, 2])
def test_lookback_wait_gives_up_and_reports_timeout(which):
    from paper_2603_18707_b300 import build
    build.build()
    scratch = torch.full((_lib.GS_SELFTEST_SCRATCH_BYTES // 4,), -1, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    api.gs_selftest_lookback_timeout(which, scratch, 2000)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 10.0
    assert int(scratch[0].item()) == _lib.GS_ERR_TIMEOUT


def test_context_usable_after_timeout(orc):
    from paper_2603_18707_b300 import render, synth
    scratch = torch.zeros(_lib.GS_SELFTEST_SCRATCH_BYTES // 4, dtype=torch.int32, device="cuda")
    api.gs_selftest_lookback_timeout(1, scratch, 100)
    api.gs_selftest_lookback_timeout(2, scratch, 100)
    raw = synth.scene_uniform(512, 3)
    cam = synth.camera_small(64, 64)
    R = render.Rasterizer([cam], api.make_config("poly1", "opacity"), 512)
    R.forward(render.activate(raw))  # raises if the bin/sort error word is set
    torch.cuda.synchronize()
    img = R.images()[0].cpu().double().numpy()
    ref, _, _ = orc.render_untiled(orc.activate(raw), orc.camera_from_dict(cam),
                                   orc.make_config("poly1", (0.773, -0.773 / 4.386), "opacity"))
    assert abs(img - ref).max() < 1e-3
