"""The measured FP32 FMA ceiling (tomo_fp32_peak) that the benchmark divides
the operators' achieved FLOP rate by: plausible for one GB300 (152 SMs x 128
FP32 lanes x 2 FLOP at the measured SM clock bounds the scalar form from
above), the shared-memory bandwidth likewise, and refused on a stream that
is capturing a CUDA graph."""
import pytest
import torch

from gpu_common import need_gpu
from paper_2410_06106_gb300 import api

pytestmark = pytest.mark.gpu


def test_fp32_peak_is_plausible():
    need_gpu()
    r = api.fp32_peak(20)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert 300.0 <= r["sm_mhz"] <= 3000.0, r
    nominal = sms * 128 * 2 * r["sm_mhz"] * 1e6 / 1e12
    # dependent chains at full occupancy reach most of the pipe; nothing can exceed it
    # by more than the clock's variation between the two launches
    assert 0.5 * nominal <= r["scalar_tflops"] <= 1.1 * nominal, (r, nominal)
    assert r["packed_tflops"] > 0.5 * nominal, (r, nominal)


def test_fp32_peak_refuses_a_capturing_stream():
    need_gpu()
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        graph.capture_begin(capture_error_mode="relaxed")
        try:
            with pytest.raises(api.TomoError) as e:
                api.fp32_peak(5)
        finally:
            graph.capture_end()
    assert e.value.code == -1
    del graph


def test_smem_peak_is_plausible():
    """128 bytes per clock per SM is the shared-memory pipe's width; the
    measured bandwidth lies between half of that and that at the measured clock"""
    need_gpu()
    gbs = api.smem_peak(20)
    r = api.fp32_peak(5)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 128 * r["sm_mhz"] * 1e6 / 1e9
    assert 0.5 * nominal <= gbs <= 1.1 * nominal, (gbs, nominal)
