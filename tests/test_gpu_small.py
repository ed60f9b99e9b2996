"""The single-CTA path for small populations (slpic_step_small) against the
batched kernels of slpic_step.

The breakdown runs of Sec. V start from 100 electrons and stay at hundreds to
thousands of markers, where one CTA per instance runs whole steps in one
launch. Bars:
- every marker, the deposit, the field, the history and the totals equal the
  batched path's after the same steps, bit for bit: SLPIC and PIC, imposed
  field and Poisson, constant and Eq. sey emission, one and three excitation
  levels, FP32 and FP64, one instance and an uneven batch;
- the path stops before the first step at which a store holds more than its
  limit of tiles, at the same step for every instance of a batch, and the
  batched path carries on from there with the same results;
- the paper's ion-population test gives the same window means with and
  without it;
- against the oracle's FP32 mirror directly: many vacuum steps bit for bit,
  and one dense step with every collision process (counts, ids and cells
  bit-exact, velocities after scattering to 1e-5).
"""
import math

import numpy as np
import pytest

from paper_2103_12194_gb300 import inputs

from .test_gpu_parity import mixed_state
from .test_gpu_shape import assert_same_state

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


# (cells, pd [Torr cm], V, electrons, ions): small and uneven, like a sweep
SHAPES = ((128, 1.0, 300.0, 1500, 300), (219, 1.0, 170.0, 600, 0),
          (874, 4.0, 400.0, 2500, 900), (66, 0.3, 500.0, 100, 40))


def items_for(shapes, pic=False, field_mode=0, levels=1, model=0):
    items = []
    for i, (cells, pd, V, ne, ni) in enumerate(shapes):
        kw = {}
        if pic:  # dt = dx / v_max, no speed limit (Sec. IV)
            kw = dict(vlim_e=math.inf,
                      dt=0.01 / cells / math.sqrt(2 * inputs.QE * V / inputs.ME))
        spec = inputs.gap_spec(n_cells=cells, V=V, pd_torr_cm=pd, gamma_se=0.3,
                               field_mode=field_mode, seed=300 + i, instance=i,
                               table=inputs.make_table(levels=levels), **kw)
        spec["emission_model"] = model
        items.append((spec, ne, ni))
    return items


def load(slpic, items, precision=32, seed0=90):
    sim = slpic.Simulation(len(items), precision=precision)
    for i, (spec, _, _) in enumerate(items):
        sim.configure(i, spec, capacity=(1 << 18, 1 << 18))
    for i, (spec, ne, ni) in enumerate(items):
        e, ion = mixed_state(spec, ne, max(ni, 1), seed=seed0 + 2 * i)
        e["vx"] *= np.float32(0.2)  # a few eV to tens of eV: modest growth
        sim.load(i, 0, e)
        sim.load(i, 1, ion if ni else {k: v[:0] for k, v in ion.items()})
    return sim


def same_totals(a, b, n):
    for i in range(n):
        assert a.tallies(i).tobytes() == b.tallies(i).tobytes(), i
        for s in (0, 1):
            assert a.count(i, s) == b.count(i, s)


CASES = {
    "slpic_frozen": dict(),
    "pic_frozen": dict(pic=True),
    "slpic_poisson": dict(field_mode=1),
    "slpic_sey_three_levels": dict(levels=3, model=1),
    "pic_poisson_sey": dict(pic=True, field_mode=1, model=1),
}


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("case", sorted(CASES))
def test_small_path_equals_batched_steps(slpic, case, precision):
    items = items_for(SHAPES, **CASES[case])
    n = len(items)
    a = load(slpic, items, precision)
    b = load(slpic, items, precision)
    done = a.step_small(300)
    assert done >= 50, done
    b.step(done)
    assert_same_state(a, b, n)
    same_totals(a, b, n)
    # the batched path carries on from the small path's state
    a.step(9)
    b.step(9)
    assert_same_state(a, b, n)
    # and the small path from the batched path's
    d2 = a.step_small(40)
    b.step(d2)
    assert_same_state(a, b, n)
    same_totals(a, b, n)
    a.close()
    b.close()


def test_single_instance_from_100_electrons_at_rest(slpic):
    """The paper's own start (Sec. IV): 100 electrons at rest at the cathode,
    one instance, SLPIC with v_lim = v0 and dt = dx / v0."""
    V, cells = 170.0, 219
    v0 = inputs.ion_speed(V)
    spec = inputs.gap_spec(n_cells=cells, V=V, pd_torr_cm=1.0, gamma_se=0.07, field_mode=0,
                           vlim_e=v0, dt=0.01 / cells / v0)
    spec["emission_model"] = 1
    sims = []
    for _ in range(2):
        s = slpic.Simulation(1)
        s.configure(0, spec, capacity=(1 << 18, 1 << 18))
        s.seed(0, slpic.ELECTRON, 100, slpic.SEED_REST)
        sims.append(s)
    a, b = sims
    done = a.step_small(4000)
    b.step(done)
    assert done > 1000
    assert_same_state(a, b, 1)
    same_totals(a, b, 1)
    assert a.tallies(0)["n_coll"].sum() > 100
    a.close()
    b.close()


def test_small_path_stops_when_a_store_outgrows_it(slpic):
    spec = inputs.gap_spec(n_cells=512, V=300.0, pd_torr_cm=30.0, gamma_se=0.5, field_mode=0,
                           seed=5)
    small = inputs.gap_spec(n_cells=128, V=200.0, pd_torr_cm=1.0, gamma_se=0.1, field_mode=0,
                            seed=6, instance=1)
    sims = []
    for _ in range(2):
        s = slpic.Simulation(2)
        s.configure(0, spec, capacity=(1 << 20, 1 << 20))
        s.configure(1, small, capacity=(1 << 20, 1 << 20))
        e, _ = mixed_state(spec, 3000, 1, seed=7)
        e["vx"] = np.abs(e["vx"]) * 0 + np.float32(6e6)  # ~100 eV: an avalanche
        s.load(0, 0, e)
        e1, _ = mixed_state(small, 500, 1, seed=8)
        s.load(1, 0, e1)
        sims.append(s)
    a, b = sims
    done = a.step_small(1000)
    assert 0 < done < 1000
    # it stopped because the avalanche's stores passed 32 tiles of 128
    assert max(a.count(0, 0), a.count(0, 1)) > 32 * 128
    assert a.step_small(10) == 0  # and does not apply from there
    b.step(done)
    assert_same_state(a, b, 2)
    a.step(5)
    b.step(5)
    assert_same_state(a, b, 2)
    a.close()
    b.close()


def test_small_path_does_not_apply_to_small_stores(slpic):
    spec = inputs.gap_spec(n_cells=128, V=200.0, pd_torr_cm=1.0, field_mode=0)
    s = slpic.Simulation(1)
    s.configure(0, spec, capacity=(4096, 4096))  # one step's births could overflow
    s.seed(0, slpic.ELECTRON, 100, slpic.SEED_REST)
    assert s.step_small(10) == 0
    s.close()
    s = slpic.Simulation(1)
    s.configure(0, spec)
    s.seed(0, slpic.ELECTRON, 100, slpic.SEED_REST)
    s.set_small_limit(0)
    assert s.step_small(10) == 0
    s.set_small_limit(4)
    assert s.step_small(10) == 10
    with pytest.raises(slpic.SlpicError):
        s.set_small_limit(33)
    s.close()


def test_ion_trend_is_the_same_with_and_without_the_small_path(slpic):
    volts = (130.0, 160.0, 200.0)
    out = []
    for limit in (32, 0):
        sim = slpic.Simulation(len(volts))
        for j, V in enumerate(volts):
            sim.configure(j, inputs.gap_spec(n_cells=128, V=V, pd_torr_cm=1.0, gamma_se=0.07,
                                             field_mode=0, seed=41 + j, instance=j),
                          capacity=(1 << 20, 1 << 20))
        for j in range(len(volts)):
            sim.seed(j, 0, 500, slpic.SEED_REST)
        sim.set_small_limit(limit)
        means, above = sim.ion_trend(steps_per_window=512, n_windows=8)
        out.append((means, above, [sim.tallies(j) for j in range(len(volts))]))
        sim.close()
    (m1, a1, t1), (m0, a0, t0) = out
    assert np.array_equal(a1, a0)
    ok = (m1 >= 0).all(1) & (m0 >= 0).all(1)  # no store stopped at a third of its capacity
    assert ok.any()
    assert np.array_equal(m1[ok], m0[ok])
    for j in np.flatnonzero(ok):
        assert t1[j].tobytes() == t0[j].tobytes()


def test_small_path_matches_fp32_mirror_in_vacuum(slpic, oracle_mod):
    """No gas, imposed field, emission on: every operation of the step is
    + - * / sqrt, so the single-CTA path and the FP32 mirror agree bit for bit
    over many steps (speed-limited electrons, ions reaching the cathode,
    emitted electrons, compaction)."""
    from .test_gpu_parity import assert_same_markers
    spec = inputs.gap_spec(n_cells=219, V=170.0, pd_torr_cm=1.0, gamma_se=0.4, field_mode=0,
                           vlim_e=inputs.ion_speed(170.0), dt=0.01 / 219 / inputs.ion_speed(170.0))
    spec["p_Pa"] = 0.0
    e, i = mixed_state(spec, 2500, 1500, seed=71)
    sim = slpic.Simulation(1)
    sim.configure(0, spec, capacity=(1 << 18, 1 << 18))
    sim.load(0, 0, e)
    sim.load(0, 1, i)
    ref = oracle_mod.Oracle(spec, precision=32)
    ref.load(0, e)
    ref.load(1, i)
    total = 0
    for chunk in (1, 7, 40, 200):
        done = sim.step_small(chunk)
        assert done == chunk
        ref.step(chunk)
        total += chunk
        for s in (0, 1):
            assert_same_markers(sim.particles(0, s), ref.particles(s), spec["vlim_e"], True)
            assert np.array_equal(sim.charge(0, s), ref.charge(s))
    hg, hr = sim.history(0), ref.history()
    assert len(hg) == len(hr) == total
    for k in ("n_live", "n_abs", "n_see", "marker_steps"):
        assert np.array_equal(hg[k], hr[k]), k
    assert hr["n_see"].sum() > 50
    sim.close()


def test_small_path_matches_fp32_mirror_in_one_dense_step(slpic, oracle_mod):
    """One step with every collision process through the single-CTA path:
    counts, ids and cells bit-exact against the FP32 mirror; velocities (which
    pass through the elementary functions of the scattering) to 1e-5."""
    from .test_gpu_parity import assert_same_markers
    spec = inputs.gap_spec(n_cells=256, V=300.0, pd_torr_cm=30.0, gamma_se=0.5, field_mode=0,
                           table=inputs.make_table(levels=3))
    e, i = mixed_state(spec, 3500, 1200, seed=73)
    sim = slpic.Simulation(1)
    sim.configure(0, spec, capacity=(1 << 18, 1 << 18))
    sim.load(0, 0, e)
    sim.load(0, 1, i)
    assert sim.step_small(1) == 1
    ref = oracle_mod.Oracle(spec, precision=32)
    ref.load(0, e)
    ref.load(1, i)
    ref.step(1)
    hg, hr = sim.history(0)[-1], ref.history()[-1]
    for k in ("n_live", "n_coll", "n_candidates", "n_abs", "n_see", "n_clamp", "marker_steps"):
        assert np.array_equal(hg[k], hr[k]), (k, hg[k], hr[k])
    assert min(hr["n_coll"]) > 10 and hr["n_see"] > 3
    for s in (0, 1):
        assert_same_markers(sim.particles(0, s), ref.particles(s), spec["vlim_e"], False)
    sim.close()
