"""The refinement kernels convert between FP32 and FP64 on the integer and
FP32 pipes (split of an FP64 value into its nearest FP32 value and the FP32
rounding of the remainder; exact FP32 to FP64 widening).  Their results must
be bit-identical to the hardware conversions (IEEE 754 round to nearest,
ties to even), checked on the device over seeded bit patterns that cover
every exponent, the rounding ties and the carries out of the significand."""

import pytest

from paper_2404_14864_gb300 import kfbi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [0, 1, 12345])
def test_conversions_match_hardware(seed):
    assert kfbi.kfbi_check_conversions(seed, 1 << 22) == 0


def test_conversions_reject_bad_arguments():
    with pytest.raises(kfbi.KfbiError):
        kfbi.kfbi_check_conversions(0, 0)
