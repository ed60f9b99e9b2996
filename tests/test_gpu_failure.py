"""Failure detection and checkpoint/resume on the GPU, without faulting it.

- Bounded waits: a thread block of the single-CTA path leaves out its
  arrival at a grid barrier (a test hook); every block's wait there runs
  out after a short spin limit, the call returns SLPIC_ERR_TIMEOUT, and after
  slpic_clear_error and a fresh load the context steps as a new one does.
- Checkpoint/resume: N steps, slpic_save, a fresh context configured alike,
  slpic_load, N more steps equals 2N steps of the first context, bit for bit
  (markers, deposit, field, history, totals), in FP32 and FP64, for a batch
  with an imposed field and a Poisson instance, gas and emission on.
"""
import numpy as np
import pytest

from .test_gpu_shape import assert_same_state
from .test_gpu_small import SHAPES, items_for, load, same_totals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slpic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_12194_gb300 import build
    build.build()
    from paper_2103_12194_gb300 import slpic as mod
    return mod


def test_missing_barrier_arrival_times_out_and_the_context_recovers(slpic):
    items = items_for(SHAPES[:3])
    sim = load(slpic, items)
    sim.set_spin_limit(20000)
    assert sim.step_small(5) == 5
    sim.test_skip_barrier(1, 3)  # instance 1 leaves out barrier 3 of the next launch
    with pytest.raises(slpic.SlpicError) as e:
        sim.step_small(10)
    assert e.value.code == slpic.ERR_TIMEOUT
    # the error stays latched until it is cleared
    with pytest.raises(slpic.SlpicError) as e:
        sim.synchronize()
    assert e.value.code == slpic.ERR_TIMEOUT
    sim.clear_error()
    sim.set_spin_limit(0)
    # a fresh load makes the context usable again: it now steps as a new one
    fresh = load(slpic, items, seed0=95)
    for i, (spec, ne, ni) in enumerate(items):
        for s in (0, 1):
            sim.load(i, s, fresh.particles(i, s))
            sim.reset_counters(i)
    fresh_b = load(slpic, items, seed0=95)
    for i in range(len(items)):
        fresh_b.reset_counters(i)
    assert sim.step_small(30) == 30
    assert fresh_b.step_small(30) == 30
    for i in range(len(items)):
        for s in (0, 1):
            a, b = sim.particles(i, s), fresh_b.particles(i, s)
            for k in a:
                assert np.array_equal(a[k], b[k]), (i, s, k)
            assert np.array_equal(sim.charge(i, s), fresh_b.charge(i, s))
    sim.close()
    fresh.close()
    fresh_b.close()


@pytest.mark.parametrize("precision", [32, 64])
def test_checkpoint_resume_is_bit_exact(slpic, precision):
    items = items_for(SHAPES[:2]) + items_for(SHAPES[2:3], field_mode=1)
    for i, (spec, _, _) in enumerate(items):
        spec["instance"] = i
    n = len(items)
    a = load(slpic, items, precision)
    a.step(40)
    snap = a.save()
    a.step(40)
    b = load(slpic, items, precision, seed0=333)  # other markers, replaced by the load
    b.restore(snap)
    b.step(40)
    assert_same_state(a, b, n)
    same_totals(a, b, n)
    # through the single-CTA path as well
    c = load(slpic, items, precision, seed0=444)
    c.restore(snap)
    done = c.step_small(40)
    c.step(40 - done)
    assert_same_state(a, c, n)
    same_totals(a, c, n)
    # a snapshot into a context of another shape is refused
    d = load(slpic, items[:2], precision)
    with pytest.raises(slpic.SlpicError) as e:
        d.restore(snap)
    assert e.value.code == slpic.ERR_INVALID_ARG
    with pytest.raises(slpic.SlpicError):
        b.restore(snap[:100])
    for s in (a, b, c, d):
        s.close()
