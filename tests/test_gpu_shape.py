"""Launch shapes and the autotuner: the step's results are the same, bit for
bit, for every shape of the particle and collision kernels. The autotuner
therefore only changes speed. Its timing steps are real steps of the
simulation, equal to those slpic_step would have taken."""
import numpy as np
import pytest

from .test_gpu_batched import batch_items, load_batch, states_for

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


def assert_same_state(a, b, n_inst):
    for i in range(n_inst):
        for s in (0, 1):
            pa, pb = a.particles(i, s), b.particles(i, s)
            for k in pa:
                assert np.array_equal(pa[k], pb[k]), (i, s, k)
            assert np.array_equal(a.charge(i, s), b.charge(i, s)), (i, s)
        assert np.array_equal(a.history(i), b.history(i)), i
        assert np.array_equal(a.field(i)[1], b.field(i)[1]), i


def test_results_do_not_depend_on_launch_shape(slpic):
    items = batch_items()[:4]  # the grids fit next to 20 warps' stages
    states = states_for(items, seed0=60)
    ref = load_batch(slpic, items, states)
    w0, c0 = ref.launch_shape()
    assert w0 == 20 and c0 == 8
    ref.step(40)
    for shape in ((8, 4), (4, 16), (12, 1), (20, 2)):
        sim = load_batch(slpic, items, states)
        sim.set_launch_shape(*shape)
        assert sim.launch_shape() == shape
        sim.step(40)
        assert_same_state(ref, sim, len(items))
        sim.close()
    with pytest.raises(slpic.SlpicError):
        ref.set_launch_shape(6, 8)
    ref.close()


def test_autotune_keeps_the_results(slpic):
    items = batch_items()
    states = states_for(items, seed0=70)
    tuned = load_batch(slpic, items, states)
    w, cc = tuned.autotune(steps_each=8)
    assert w % 4 == 0 and 4 <= w <= 20 and cc in (2, 4, 8, 16)
    assert tuned.launch_shape() == (w, cc)
    steps = len(tuned.history(0))
    assert steps >= 8 * 6
    plain = load_batch(slpic, items, states)
    plain.step(steps)
    assert_same_state(tuned, plain, len(items))
    tuned.close()
    plain.close()


def test_more_warps_than_fit_beside_the_shared_grid_deposit_to_global_memory(slpic):
    """With the 16384-cell gap in the batch, a particle-kernel CTA fits at
    most 12 warps beside the shared charge grid; 16 and 20 warps deposit to
    global memory instead.  The integers, and so every result, are the
    same."""
    items = batch_items()
    assert max(spec["n_cells"] for spec, _, _ in items) == 16384
    states = states_for(items, seed0=80)
    ref = load_batch(slpic, items, states)
    assert ref.launch_shape() == (12, 8)
    ref.step(40)
    for shape in ((16, 8), (20, 4)):
        sim = load_batch(slpic, items, states)
        sim.set_launch_shape(*shape)
        assert sim.launch_shape() == shape
        sim.step(40)
        assert_same_state(ref, sim, len(items))
        sim.close()
    ref.close()


def test_contexts_of_different_grids_live_side_by_side(slpic):
    """A context with a large charge grid keeps stepping after a context
    with a small one was configured in the same process (the kernels'
    shared-memory limits are per process)."""
    items = batch_items()
    states = states_for(items, seed0=90)
    big = load_batch(slpic, items, states)
    big.step(3)
    small = load_batch(slpic, items[:1], states[:1])
    small.step(3)
    big.step(3)
    big.synchronize()
    small.close()
    big.close()
