"""Device self-checks.

Conversions: the refinement kernels convert between FP32 and FP64 on the
integer and FP32 pipes (split of an FP64 value into its nearest FP32 value
and the FP32 rounding of the remainder; exact FP32 to FP64 widening).  Their
results must be bit-identical to the hardware conversions (IEEE 754 round to
nearest, ties to even), checked on the device over seeded bit patterns that
cover every exponent, the rounding ties and the carries out of the
significand.

Bounded waits: the tensor-core passes wait on their pipeline with a cycle
limit and report KFBI_ERR_TIMEOUT instead of hanging.  The self-check runs
the same wait routine on an mbarrier that nothing completes, with a 10 ms
limit: the call must return KFBI_ERR_TIMEOUT and the device must stay usable
(a kernel launched afterwards runs and gives correct results)."""

import pytest

from paper_2404_14864_gb300 import kfbi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [0, 1, 12345])
def test_conversions_match_hardware(seed):
    assert kfbi.kfbi_check_conversions(seed, 1 << 22) == 0


def test_conversions_reject_bad_arguments():
    with pytest.raises(kfbi.KfbiError):
        kfbi.kfbi_check_conversions(0, 0)


def test_bounded_wait_gives_up_and_device_stays_usable():
    assert kfbi.kfbi_check_wait_timeout(0.01) == kfbi.KFBI_ERR_TIMEOUT
    assert kfbi.kfbi_check_wait_timeout(0.001) == kfbi.KFBI_ERR_TIMEOUT
    assert kfbi.kfbi_check_conversions(7, 1 << 16) == 0


@pytest.mark.parametrize("seconds", [0.0, -1.0, 2.0])
def test_bounded_wait_rejects_bad_limits(seconds):
    assert kfbi.kfbi_check_wait_timeout(seconds) == kfbi.KFBI_ERR_ARG
