"""The integer FP64 <-> FP32 conversions of the mixed-precision kernels give
the hardware conversions' bits (round to nearest even one way, exact the
other), on edge cases, rounding ties, subnormal results and raw words."""
import pytest

from paper_0809_3098_gb300 import lc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_integer_conversions_match_hardware(seed):
    assert lc.lc_selftest_conversions(1 << 26, seed) == (0, 0)


def test_selftest_detects_nothing_on_zero_values_and_rejects_bad_n():
    assert lc.lc_selftest_conversions(0) == (0, 0)
    with pytest.raises(lc.LCError):
        lc.lc_selftest_conversions(-1)
