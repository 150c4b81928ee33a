"""The issue-rate microbenchmarks behind the arithmetic rooflines
(misa_measure_peaks): every figure measured, and ordered as the hardware
orders them."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    import torch
    assert torch.cuda.is_available()
    from paper_2107_07866_gb300 import build
    build.build()
    from paper_2107_07866_gb300 import misa
    p = misa.measure_peaks()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert p["num_sms"] == nsm
    assert 300.0 < p["sm_clock_mhz"] < 3000.0
    # at most 128 FP32 lanes x 2 flops per SM per clock for scalar FMA, and
    # the packed form cannot be slower than a third of it
    ceiling = nsm * 128 * 2 * p["sm_clock_mhz"] * 1e6 / 1e12
    assert 0.5 * ceiling < p["fp32_ffma_tflops"] < 1.1 * ceiling, (p, ceiling)
    assert p["fp32_ffma2_tflops"] > 0.3 * p["fp32_ffma_tflops"]
    assert 0.0 < p["fp64_dfma_tflops"] < p["fp32_ffma_tflops"]
    assert 0.0 < p["mufu_rsqrt_tops"] < p["fp32_ffma_tflops"] / 2
    assert p["lds128_tbps"] > 0.0
