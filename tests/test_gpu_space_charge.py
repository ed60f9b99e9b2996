"""Space-charge regime (Sec. VI: in a glow discharge the discharge's own
charge alters the applied field): with the Poisson solve on, the field the
markers see departs far from the vacuum field, and the GPU follows the FP64
oracle through that feedback.

A quasi-neutral plasma fills a 1 cm gap at 1 Torr and 120 V: 2e4 electron
and 2e4 ion markers of flux weight 1.5e8 per m^2, a density of 3e14 m^-3.
The applied field sweeps electrons toward the anode and leaves the ions'
space charge, which raises the potential inside the gap by about 100 V (a
uniform ion density n alone would give a hump of e n d^2 / (8 eps0) = 68 V);
the hump then traps electrons, and the run settles into a glow-like plasma.

The same initial plasma runs under 16 Philox seeds on the GPU (one batched
context) and 16 in the FP64 oracle (a process pool).  The FP32 path and the
oracle take the same decisions at first and then drift apart through
threshold flips, so the comparison is of the ensembles.  Bars, after 300
steps:
- the oracle's potential departs from the vacuum line V x / d by more than
  half of V (the feedback dominates the field);
- the height of the potential's hump above the vacuum line, and the live
  electron and ion counts, have means that agree within two standard errors
  of the difference (each side's error from the scatter of its seeds).
"""
import math

import numpy as np
import pytest

from paper_2103_12194_gb300 import inputs

from . import oracle_ensemble as ens

pytestmark = pytest.mark.gpu

N_RUNS = 16


@pytest.fixture(scope="module")
def slpic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_12194_gb300 import build
    build.build()
    from paper_2103_12194_gb300 import slpic as mod
    return mod


def test_space_charge_feedback_matches_oracle(slpic):
    n, W, steps = 20_000, 1.5e8, 300

    def kw(seed, instance=0):
        return dict(n_cells=128, V=120.0, pd_torr_cm=1.0, gamma_se=0.07, field_mode=1,
                    charge_shift=11, seed=seed, instance=instance)

    sim = slpic.Simulation(N_RUNS)
    specs = [inputs.gap_spec(**kw(100 + k, k)) for k in range(N_RUNS)]
    for k, spec in enumerate(specs):
        sim.configure(k, spec, capacity=(1 << 20, 1 << 20))
    for k, spec in enumerate(specs):
        e = inputs.gap_state(n, spec, rng_seed=81, e_lo=1.0, e_hi=5.0, wj=W)
        i = inputs.gap_state(n, spec, rng_seed=82, e_lo=0.02, e_hi=0.05, species=1, wj=W,
                             first_id=0)
        sim.load(k, 0, e)
        sim.load(k, 1, i)
    sim.step(steps)
    gpu = [(sim.field(k)[0], [sim.count(k, 0), sim.count(k, 1)]) for k in range(N_RUNS)]
    sim.close()
    ref = ens.pool_map(ens.space_charge, [(kw(500 + k), n, W, steps) for k in range(N_RUNS)])
    V = specs[0]["V"]
    lin = V * np.arange(specs[0]["n_cells"] + 1) / specs[0]["n_cells"]
    hump_g = np.array([(phi - lin).max() for phi, _ in gpu])
    hump_r = np.array([(phi - lin).max() for phi, _ in ref])
    assert hump_r.mean() > 0.5 * V
    pairs = [("hump", hump_g, hump_r)]
    for s, name in ((0, "electrons"), (1, "ions")):
        pairs.append((name, np.array([c[s] for _, c in gpu], float),
                      np.array([c[s] for _, c in ref], float)))
    for name, g, r in pairs:
        se = math.hypot(g.std(ddof=1), r.std(ddof=1)) / math.sqrt(N_RUNS)
        assert abs(g.mean() - r.mean()) <= 2.0 * se, (name, g.mean(), r.mean(), se)
