"""Batched instances: independent gaps of different sizes (cells, pressure,
voltage, marker counts, field mode) advanced by the same kernel launches.

Each instance must match the oracle run alone with that instance's index
(the index is part of the random-number counter). An instance's results must
not depend on what the other instances of the batch hold.
"""
import numpy as np
import pytest

from paper_2103_12194_gb300 import inputs

from .test_gpu_parity import REL, assert_same_markers, mixed_state

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


# (cells, pd [Torr cm], V, electrons, ions, field mode): uneven like a sweep
SHAPES = (
    (64, 5.0, 400.0, 3_000, 500, 0),
    (300, 30.0, 300.0, 60_000, 20_000, 1),
    (1024, 10.0, 250.0, 150_000, 0, 0),
    (4096, 30.0, 350.0, 20_000, 40_000, 1),
    (16384, 3.0, 300.0, 90_000, 10_000, 1),
)


def batch_items(vacuum=False):
    items = []
    for i, (cells, pd, V, ne, ni, fm) in enumerate(SHAPES):
        spec = inputs.gap_spec(n_cells=cells, V=V, pd_torr_cm=pd, gamma_se=0.5,
                               field_mode=fm, seed=1000 + i, instance=i)
        if vacuum:
            spec["p_Pa"] = 0.0
        items.append((spec, ne, ni))
    return items


def states_for(items, seed0=20):
    out = []
    for i, (spec, ne, ni) in enumerate(items):
        e, ion = mixed_state(spec, ne, max(ni, 1), seed=seed0 + 2 * i)
        if ni == 0:
            ion = {k: v[:0] for k, v in ion.items()}
        out.append((e, ion))
    return out


def load_batch(slpic, items, states):
    # every instance is configured before the first load allocates the batch
    sim = slpic.Simulation(len(items))
    for i, (spec, _, _) in enumerate(items):
        sim.configure(i, spec)
    for i in range(len(items)):
        e, ion = states[i]
        sim.load(i, 0, e)
        sim.load(i, 1, ion)
    return sim


def oracle_for(oracle_mod, spec, state):
    ref = oracle_mod.Oracle(spec, precision=32)
    ref.load(0, state[0])
    ref.load(1, state[1])
    return ref


def test_batched_one_step_matches_oracle_per_instance(slpic, oracle_mod):
    items = batch_items()
    states = states_for(items)
    sim = load_batch(slpic, items, states)
    sim.step(1)
    total_coll = 0
    for i, (spec, _, _) in enumerate(items):
        ref = oracle_for(oracle_mod, spec, states[i])
        ref.step(1)
        hg, hr = sim.history(i)[-1], ref.history()[-1]
        for k in ("n_live", "n_coll", "n_candidates", "n_abs", "n_see", "n_clamp",
                  "marker_steps"):
            assert np.array_equal(hg[k], hr[k]), (i, k, hg[k], hr[k])
        total_coll += int(np.sum(hr["n_coll"]))
        for s in (0, 1):
            assert_same_markers(sim.particles(i, s), ref.particles(s), spec["vlim_e"],
                                exact_values=False)
            qg, qr = sim.charge(i, s), ref.charge(s)
            assert qg.shape == (spec["n_cells"] + 1,)
            assert np.allclose(qg, qr, rtol=REL, atol=REL * 2**32), (i, s)
        if spec["field_mode"] == 1:
            phi_g, _ = sim.field(i)
            phi_r, _ = ref.field()
            assert np.allclose(phi_g, phi_r, rtol=1e-6, atol=1e-6 * spec["V"]), i
    assert total_coll > 1000
    sim.close()


def test_batched_vacuum_steps_bit_exact(slpic, oracle_mod):
    """No gas: every instance agrees bit for bit with the FP32 mirror over
    many steps (single launches and a replayed graph of 32 steps), with
    absorption, emission births and compaction in every instance."""
    items = batch_items(vacuum=True)
    for spec, _, _ in items:
        spec["field_mode"] = 0
    states = states_for(items, seed0=40)
    sim = load_batch(slpic, items, states)
    refs = [oracle_for(oracle_mod, spec, states[i]) for i, (spec, _, _) in enumerate(items)]
    for chunk in (1, 4, 32, 2):
        sim.step(chunk)
        for ref in refs:
            ref.step(chunk)
        for i, (spec, _, _) in enumerate(items):
            for s in (0, 1):
                assert_same_markers(sim.particles(i, s), refs[i].particles(s),
                                    spec["vlim_e"], True)
                assert np.array_equal(sim.charge(i, s), refs[i].charge(s)), (i, s)
    see = sum(int(ref.history()["n_see"].sum()) for ref in refs)
    assert see > 20
    sim.close()


def test_instances_do_not_interact(slpic):
    """Replacing the markers of one instance changes nothing in the others,
    bit for bit, over 40 steps with collisions, births and the field solve."""
    items = batch_items()
    states = states_for(items)
    a = load_batch(slpic, items, states)
    other = list(states)
    e, ion = mixed_state(items[1][0], 5_000, 70_000, seed=99)
    other[1] = (e, ion)
    b = load_batch(slpic, items, other)
    a.step(40)
    b.step(40)
    for i in (0, 2, 3, 4):
        for s in (0, 1):
            pa, pb = a.particles(i, s), b.particles(i, s)
            for k in pa:
                assert np.array_equal(pa[k], pb[k]), (i, s, k)
            assert np.array_equal(a.charge(i, s), b.charge(i, s)), (i, s)
        assert np.array_equal(a.history(i), b.history(i)), i
    assert not np.array_equal(a.history(1)["n_live"], b.history(1)["n_live"])
    a.close()
    b.close()
