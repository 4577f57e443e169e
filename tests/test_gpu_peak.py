"""The measured FMA throughput (``-m gpu``), the denominator of the roofline
of the ALU-bound short range: plausible for a 152-SM GB300 (nominal float32
rate about 80 TFLOP/s at 2 GHz, float64 far below float32)."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_peak_is_plausible():
    import paper_2406_07366_gb300 as B
    f32 = B.bs_fma_peak(B.BS_MIXED)
    f64 = B.bs_fma_peak(B.BS_FP64)
    assert 5e12 < f32 < 2e14, f32
    assert 1e10 < f64 < f32, (f64, f32)
