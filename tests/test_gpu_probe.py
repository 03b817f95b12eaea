"""The FP32 FMA throughput probe (the roofline denominator of the FP32-bound force
kernels): its rate lies between a plausible floor and the unit-count formula
152 SMs x 128 lanes x 2 flop x 2070 MHz (a probe far above the formula would not
be doing the work it counts)."""
import pytest

from paper_1702_00440_gb300 import gravidy

pytestmark = pytest.mark.gpu


def test_fma_probe_rate_is_plausible():
    gravidy.load()
    tflops, ms = gravidy.gd_probe_fma(0, 1 << 16)
    formula = 152 * 128 * 2 * 2070e6 / 1e12
    print("FMA probe: %.1f TFLOP/s in %.3f ms (formula at the maximum clock %.2f)" % (tflops, ms, formula))
    assert ms > 0
    assert 0.5 * formula < tflops <= 1.02 * formula
