"""The integer-rate microbenchmark behind the rasterizer's roofline: a
positive rate of the order of the multiprocessors' integer lanes at their
clock (152 SMs x 128 lanes x ~2 GHz is about 4e13 operations/s)."""
import pytest

from paper_2602_07782_gb300 import tabi


@pytest.mark.gpu
def test_measure_int_rate():
    r = tabi.measure_int_rate(0)
    assert 1e12 < r < 1e15
    assert tabi.load().tabi_measure_int_rate(0, None) == tabi.TABI_ERR_INVALID_ARG
