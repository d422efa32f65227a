"""The measured arithmetic peaks that roofline fractions divide by (GPU, through the C ABI).

jtrlan_measure_peaks times FP64 FMA, FP64 mma.sync (m8n8k4) and FP32 FMA throughput loops.  The
figures must be positive and ordered as the hardware is built: FP32 far above FP64, and none above
what 152 SMs could issue at the 2.07 GHz maximum clock (FP32: 128 lanes x 2 flop per SM and clock).
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2001_07428_gb300 import binding as B
    p = B.jtrlan_measure_peaks(torch.cuda.current_stream().cuda_stream)
    fp32_bound = 152 * 128 * 2 * 2.07e9 / 1e12
    assert 0 < p["fp64_fma_tflops"] < p["fp32_fma_tflops"] / 8
    assert 0 < p["fp64_mma_tflops"]
    assert p["fp32_fma_tflops"] <= 1.02 * fp32_bound
