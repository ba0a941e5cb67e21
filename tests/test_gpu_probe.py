"""The FMA-peak probe behind the FP64 step's ALU roofline: plausible rates,
FP32 well above FP64, and stable across calls."""
import pytest

from gpu_helpers import lib

pytestmark = pytest.mark.gpu


def test_fma_peak_is_plausible_and_repeatable():
    L = lib()
    f64 = L.lb_fma_peak("fp64")
    f32 = L.lb_fma_peak("fp32")
    # a GB300-class part: FP64 vector rate of order 1 TFLOP/s, FP32 tens of TFLOP/s
    assert 1e11 < f64 < 1e14
    assert 1e12 < f32 < 1e15
    assert f32 > 4 * f64
    again = L.lb_fma_peak("fp64")
    assert again == pytest.approx(f64, rel=0.15)
