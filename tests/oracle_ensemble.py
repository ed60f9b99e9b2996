"""Ensemble runs of the FP64 oracle for the parity tests of long-run
quantities (Townsend alpha, multiplication per ion transit, the breakdown
gain, the ion-population trend of Sec. V).

Each function runs one independent oracle instance from plain arguments, so
that a process pool can run many at once.  The pool is started with the
"spawn" method: a process forked after the parent has created a CUDA context
may hang, and spawned processes start clean.
"""
import multiprocessing
import os

import numpy as np

GAMMA = 0.07


def _spec(kw):
    from paper_2103_12194_gb300 import inputs
    kw = dict(kw)
    table_levels = kw.pop("table_levels", 1)
    emission_model = kw.pop("emission_model", 0)
    if table_levels != 1:
        kw["table"] = inputs.make_table(levels=table_levels)
    spec = inputs.gap_spec(**kw)
    spec["emission_model"] = emission_model
    return spec


def anode_electrons_per_seed(kw, n_seed, chunk=256, max_steps=400_000):
    """Avalanches without emission from n_seed electrons at rest at the
    cathode: the flux weight of electrons reaching the anode per seed
    electron, e^(alpha d) (Sec. II.A)."""
    import oracle
    o = oracle.Oracle(_spec(kw), precision=64)
    o.seed(0, n_seed, 1)
    steps = 0
    while o.count(0) and steps < max_steps:
        o.step(chunk)
        steps += chunk
    assert o.count(0) == 0
    return float(o.history()["w_abs"][:, 0, 1].sum()) / n_seed


def gain(kw, n_seed, chunk=256, max_steps=400_000):
    """First-generation gain G = gamma (flux weight of first-generation ions
    at the cathode) / (seeded weight), emission off, seeds at rest at the
    cathode (Sec. II.A Townsend criterion)."""
    import oracle
    kw = dict(kw)
    kw["gamma_se"] = 0.0
    o = oracle.Oracle(_spec(kw), precision=64)
    o.seed(0, n_seed, 1)
    steps = 0
    while (o.count(0) or o.count(1)) and steps < max_steps:
        o.step(chunk)
        steps += chunk
    assert o.count(0) == 0 and o.count(1) == 0
    return GAMMA * float(o.history()["w_cath_ion_gen0"].sum()) / n_seed


def multiplication(kw, n_seed, steps_per_window, n_windows):
    """Flux weight emitted at the cathode per window of one ion crossing
    time, per seed electron (seeds at rest at the cathode, emission on)."""
    import oracle
    o = oracle.Oracle(_spec(kw), precision=64)
    o.seed(0, n_seed, 1)
    see, _ = o.multiplication(steps_per_window, n_windows)
    return see / n_seed


def ion_trend(kw, n_seed, steps_per_window, n_windows, stop_markers):
    """Mean live ions per window (Sec. V), seeds at rest at the cathode; a run
    whose live markers pass stop_markers stops there (above breakdown) and its
    remaining windows read -1, as the library's trend does."""
    import oracle
    o = oracle.Oracle(_spec(kw), precision=64)
    o.seed(0, n_seed, 1)
    means = np.full(n_windows, -1.0)
    for w in range(n_windows):
        total = 0
        for _ in range(steps_per_window):
            o.step(1)
            total += o.count(1)
            if o.count(0) + o.count(1) > stop_markers:
                return means, True
        means[w] = total / steps_per_window
    grows = means[-1] > 0 and all(means[-1] > m for m in means[:-1])
    return means, bool(grows)


def space_charge(kw, n, W, steps):
    """The space-charge run of the Poisson-feedback test: a quasi-neutral
    plasma of n electron and n ion markers of flux weight W, stepped
    `steps` steps with the Poisson solve on.  Returns (phi, live counts)."""
    import oracle
    from paper_2103_12194_gb300 import inputs
    spec = _spec(kw)
    e = inputs.gap_state(n, spec, rng_seed=81, e_lo=1.0, e_hi=5.0, wj=W)
    i = inputs.gap_state(n, spec, rng_seed=82, e_lo=0.02, e_hi=0.05, species=1, wj=W,
                         first_id=0)
    o = oracle.Oracle(spec, precision=64)
    o.load(0, e)
    o.load(1, i)
    o.step(steps)
    return o.field()[0], [o.count(0), o.count(1)]


def pool_map(fn, args):
    """fn(*a) for every a in args, on a spawn-started process pool."""
    n = min(len(args), os.cpu_count() or 1, 16)
    if n <= 1:
        return [fn(*a) for a in args]
    with multiprocessing.get_context("spawn").Pool(n) as pool:
        return pool.starmap(fn, args)
