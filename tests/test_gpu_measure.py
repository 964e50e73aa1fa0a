"""Measurement utilities of the library."""
import pytest

import paper_1705_03141_gb300 as pkg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("packed", [False, True])
def test_fp32_peak_is_plausible(cuda, packed):
    # 152 SMs x 128 FP32 lanes x 2 FLOP x ~2 GHz ~ 80 TFLOP/s; allow clocks from 0.5 to 2.5 GHz
    # and any SM count of this device class
    v = pkg.measure_fp32_peak(packed)
    assert 10.0 < v < 200.0
