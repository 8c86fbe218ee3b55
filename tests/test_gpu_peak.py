"""The FMA throughput self-test (dd_alu_peak_test) that supplies the FP64 and FP32 roofline
denominators: it runs, and its figures are those of a GB300-class part (2 FP64 FMA lanes per
SM per clock: about 1.2 TFLOP/s over 152 SMs at 2 GHz; FP32 64 times that)."""
import pytest

import paper_2311_08757_gb300 as dd

pytestmark = pytest.mark.gpu


def test_fma_peaks_are_measured():
    f64 = dd.dd_alu_peak_test(0, 3)
    f32 = dd.dd_alu_peak_test(1, 3)
    print(f"FP64 FMA {f64:.3f} TFLOP/s, FP32 FMA {f32:.1f} TFLOP/s")
    assert 0.3 < f64 < 5.0
    assert 10.0 < f32 < 200.0
    assert f32 > 10 * f64
