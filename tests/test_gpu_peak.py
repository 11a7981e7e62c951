"""The arithmetic peak microbenchmark behind the blend's roofline denominator:
it runs through the C ABI, reports the FLOP it performs, and the rate it
measures is a plausible FP32 / packed-FP16 FMA rate for this GPU."""
import pytest
import torch

from paper_2603_18707_b300 import api

pytestmark = pytest.mark.gpu


def _rate(half2: bool, blocks: int, iters: int):
    sink = torch.empty(blocks * 256, device="cuda", dtype=torch.float32)
    api.gs_fma_peak(half2, blocks, 10, sink)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    flop = api.gs_fma_peak(half2, blocks, iters, sink)
    e1.record()
    torch.cuda.synchronize()
    assert torch.isfinite(sink).all()
    return flop, flop / (e0.elapsed_time(e1) / 1e3) / 1e12


def test_fma_peak_flop_count_and_rate():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks = sms * 8
    flop, ffma = _rate(False, blocks, 200)
    assert flop == blocks * 256 * 200 * 16 * 8 * 2
    # 128 FP32 lanes per SM at no more than 2.2 GHz bound it from above
    cap = sms * 128 * 2 * 2.2e9 / 1e12
    assert 0.3 * cap < ffma < 1.05 * cap, (ffma, cap)
    flop2, hfma2 = _rate(True, blocks, 200)
    assert flop2 == 2 * flop
    assert 0.3 * ffma < hfma2 < 2.1 * 1.05 * cap, (hfma2, ffma)
