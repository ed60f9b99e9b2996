"""slpic_philox_static, the allocation-free variant of slpic_philox, called
through the C ABI and compared with the allocating entry point.

The file name sorts last so that these tests also run after every other test
in the same process; each test sets up everything it uses, so the file also
passes alone in a fresh process.
"""
import numpy as np
import pytest


def _slpic():
    from paper_2103_12194_gb300 import build, slpic
    build.build()
    return slpic


def _counters(rng, n):
    return rng.integers(0, 1 << 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)


def test_oversize_call_is_rejected_before_any_device_work():
    slpic = _slpic()
    ctr = np.zeros((slpic.PHILOX_STATIC_MAX + 1, 4), dtype=np.uint32)
    with pytest.raises(slpic.SlpicError) as e:
        slpic.philox_static(ctr, 1)
    assert e.value.code == slpic.ERR_INVALID_ARG
    assert "SLPIC_PHILOX_STATIC_MAX" in str(e.value)


@pytest.mark.gpu
def test_two_calls_in_a_row_match_the_allocating_entry_point():
    slpic = _slpic()
    rng = np.random.default_rng(20210323)
    # first call fills the whole scratch, the second a ragged part of it with
    # other counters and another key: a stale word would show
    for n, seed in ((slpic.PHILOX_STATIC_MAX, 0x0123456789ABCDEF), (1000 + 37, 42)):
        ctr = _counters(rng, n)
        want = slpic.philox(ctr, seed)
        got = slpic.philox_static(ctr, seed)
        np.testing.assert_array_equal(got, want)


@pytest.mark.gpu
def test_small_and_empty_calls_and_rejection_leave_it_usable():
    slpic = _slpic()
    rng = np.random.default_rng(7)
    assert slpic.philox_static(np.zeros((0, 4), np.uint32), 5).shape == (0, 4)
    with pytest.raises(slpic.SlpicError):
        slpic.philox_static(_counters(rng, slpic.PHILOX_STATIC_MAX + 1), 5)
    ctr = _counters(rng, 3)
    np.testing.assert_array_equal(slpic.philox_static(ctr, 5), slpic.philox(ctr, 5))
