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


@pytest.mark.gpu
def test_calls_leave_free_device_memory_unchanged():
    """The entry point allocates nothing: free device memory is the same
    before and after a call, for the first call after a context was created
    on the device (slpic_create did the set-up) and for later calls."""
    torch = pytest.importorskip("torch")
    slpic = _slpic()
    torch.cuda.mem_get_info(0)  # the process's own context exists
    sim = slpic.Simulation(1, device=0)
    rng = np.random.default_rng(11)
    ctr = _counters(rng, 4096)
    for _ in range(2):
        free0, _ = torch.cuda.mem_get_info(0)
        got = slpic.philox_static(ctr, 77)
        free1, _ = torch.cuda.mem_get_info(0)
        assert free1 == free0
    np.testing.assert_array_equal(got, slpic.philox(ctr, 77))
    sim.close()


@pytest.mark.gpu
def test_call_returns_while_a_simulation_runs_on_another_stream():
    """The call's copies and kernel use a private non-blocking stream: it
    returns with the right words while steps queued on a simulation's
    non-blocking stream are still running."""
    torch = pytest.importorskip("torch")
    slpic = _slpic()
    from paper_2103_12194_gb300 import inputs
    stream = torch.cuda.Stream(device=0)
    sim = slpic.Simulation(1, device=0, stream=stream)
    spec = inputs.gap_spec(n_cells=4096, V=300.0, pd_torr_cm=1.0, field_mode=1)
    sim.configure(0, spec, capacity=(1 << 23, 1 << 22))
    sim.seed(0, slpic.ELECTRON, 4_000_000, 2)
    sim.step(40)
    sim.synchronize()
    rng = np.random.default_rng(12)
    ctr = _counters(rng, 2048)
    want = slpic.philox(ctr, 9)
    slpic.philox_static(ctr, 9)
    sim.step(800)  # queued on the simulation's stream
    got = slpic.philox_static(ctr, 9)
    busy = not stream.query()
    sim.synchronize()
    np.testing.assert_array_equal(got, want)
    assert busy, "the simulation's steps had finished before the call returned"
    sim.close()
