"""lb_fma_peak, the denominator of the ALU roofline in bench.py: plausible rates.

GB300 nominal: float32 152 SMs x 128 lanes x 2 flops x 2.07 GHz = 80.5
TFLOP/s; float64 far lower (about 1.2 TFLOP/s).  The bounds only catch a
broken measurement (wrong flop count, a dead-code launch, a unit error).
"""
import pytest

from tests.helpers import library

pytestmark = pytest.mark.gpu


def test_fma_rates_are_plausible():
    lb = library()
    f64 = max(lb.fma_peak(0) for _ in range(3))
    f32 = max(lb.fma_peak(1) for _ in range(3))
    print(f"FMA rate: float64 {f64:.3f} TFLOP/s, float32 {f32:.2f} TFLOP/s")
    assert 0.05 < f64 < 10.0
    assert 10.0 < f32 < 200.0
    assert f32 > 5 * f64
