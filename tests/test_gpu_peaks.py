"""The FMA-throughput diagnostic that supplies the ALU roofline denominators:
positive, finite, stable between calls, and in the range the SM count and
clock allow (FP64 far below FP32 on this part)."""
import math

import pytest

import paper_2604_25876_gb300 as sk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_measured_fma_peaks_are_plausible():
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    f32 = sk.measure_fma_peak(sk.PEAK_FP32)
    f64 = sk.measure_fma_peak(sk.PEAK_FP64)
    assert math.isfinite(f32) and math.isfinite(f64)
    # between a tenth of 128 FMA lanes per SM at 1 GHz and 256 lanes per SM at 3 GHz
    assert 0.1 * sms * 128 * 2 * 1.0e9 / 1e12 < f32 < sms * 256 * 2 * 3.0e9 / 1e12
    assert 0.0 < f64 < f32
    again = sk.measure_fma_peak(sk.PEAK_FP32)
    assert again == pytest.approx(f32, rel=0.25)
