"""The FP64 marker path (slpic_set_precision(ctx, 64)) against the FP64 oracle.

The FP64 path runs the same kernels in double. Without a speed limit every
decision of a step is made with + - * / sqrt, table lookups and Philox
uniforms, which are exact in both, so counts, ids, cells and the deposit are
bit-exact against the oracle.

The speed-limited kick is solved by Halley steps on the GPU and from its
closed form (asinh) by the oracle; the two agree to rounding.  Values that
pass through it, or through an elementary function (scattering angles,
seeding directions, Box-Muller), may differ in the last bits; they are
compared to 1e-12 relative, and a deposit rounded from them to the nearest
fixed-point unit may differ by one unit now and then.
"""
import math

import numpy as np
import pytest

from paper_2103_12194_gb300 import inputs

from .test_gpu_parity import dense_spec, mixed_state

pytestmark = pytest.mark.gpu

REL64 = 1e-12


@pytest.fixture(scope="module")
def slpic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_12194_gb300 import build
    build.build()
    from paper_2103_12194_gb300 import slpic as mod
    return mod


def make_sim64(slpic, spec, cap=(1 << 20, 1 << 20)):
    sim = slpic.Simulation(1, precision=64)
    sim.configure(0, spec, capacity=cap)
    return sim


def same_markers64(g, r, exact):
    """Same markers in the same order.  exact: every field bit for bit.
    Otherwise the position x = cell + offset to 1e-12 of a cell (a marker
    that moves exactly one cell per step, as one speed-limited on the field
    axis does, sits on a cell boundary, where a last-bit difference puts it at
    offset 0 of cell k or offset 1 - 2^-53 of cell k - 1: the same position)
    and velocities to 1e-12 relative."""
    assert np.array_equal(g["id"], r["id"].astype(np.uint32))
    assert g["off"].dtype == np.float64
    if exact:
        assert np.array_equal(g["cell"], r["cell"])
        for k in ("off", "vx", "vy", "vz", "wj"):
            assert np.array_equal(g[k], r[k]), k
    else:
        assert np.array_equal(g["wj"], r["wj"])
        xg, xr = g["cell"] + g["off"], r["cell"] + r["off"]
        worst = int(np.argmax(np.abs(xg - xr))) if xg.size else 0
        assert np.allclose(xg, xr, rtol=0, atol=REL64), (worst, xg[worst], xr[worst])
        assert np.abs(g["cell"] - r["cell"]).max(initial=0) <= 1
        vg = np.stack([g["vx"], g["vy"], g["vz"]])
        vr = np.stack([r["vx"], r["vy"], r["vz"]])
        err = np.linalg.norm(vg - vr, axis=0) / np.maximum(np.linalg.norm(vr, axis=0), 1.0)
        assert err.max() <= REL64, err.max()


def test_fp32_calls_are_refused_on_an_fp64_context(slpic):
    spec, _ = inputs.small_gap_config()
    sim = make_sim64(slpic, spec)
    st = inputs.gap_state(10, spec)
    soa = slpic.SoA(*[np.ascontiguousarray(st[k]).ctypes.data for k in slpic.FIELDS])
    import ctypes
    rc = sim._L.slpic_load_particles(sim._h, 0, 0, ctypes.byref(soa), 10, 10)
    assert rc == slpic.ERR_STATE
    sim.load(0, 0, st)  # the FP64 call takes the same values
    assert sim.count(0, 0) == 10
    sim.close()


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_fp64_seed_matches_oracle(slpic, oracle_mod, mode):
    spec = inputs.gap_spec(n_cells=4096, V=300.0, seed=777)
    sim = make_sim64(slpic, spec)
    n = 50_001
    sp = 1 if mode == 3 else 0
    sim.seed(0, sp, n, mode, e0=1.0, e_lo=0.1, e_hi=200.0, wj=0.75)
    ref = oracle_mod.Oracle(spec, precision=64)
    ref.seed(sp, n, mode, e0=1.0, e_lo=0.1, e_hi=200.0, wj=0.75)
    g, r = sim.particles(0, sp), ref.particles(sp)
    assert np.array_equal(g["id"], r["id"])
    assert np.array_equal(g["cell"], r["cell"])
    assert np.array_equal(g["off"], r["off"])
    assert np.array_equal(g["wj"], r["wj"])
    scale = np.abs(r["vx"]).max() + 1e-300
    for k in ("vx", "vy", "vz"):
        assert np.allclose(g[k], r[k], rtol=REL64, atol=REL64 * scale), k
    sim.close()


def test_fp64_deposit_bit_exact(slpic, oracle_mod):
    spec = dense_spec(n_cells=4096)
    spec["dt"] = 0.0
    e, i = mixed_state(spec, 200_001, 50_000, seed=31)
    sim = make_sim64(slpic, spec)
    sim.load(0, 0, e)
    sim.load(0, 1, i)
    sim.step(1)
    ref = oracle_mod.Oracle(spec, precision=64)
    ref.load(0, e)
    ref.load(1, i)
    ref.deposit()
    for s in (0, 1):
        assert np.array_equal(sim.charge(0, s), ref.charge(s))
    sim.close()


@pytest.mark.parametrize("vlim_e", [None, math.inf])
def test_fp64_vacuum_steps_match_oracle(slpic, oracle_mod, vlim_e):
    """Many steps without gas: bit-exact without a speed limit; with one,
    ids and counts exact, positions and velocities to 1e-12 (the kick's two
    solutions agree to rounding), the deposit to 1e-6 of each node's charge
    and the total to 64 fixed-point units."""
    exact = vlim_e == math.inf
    spec = inputs.gap_spec(n_cells=300, V=250.0, gamma_se=0.4, field_mode=0, vlim_e=vlim_e)
    spec["p_Pa"] = 0.0
    if vlim_e == math.inf:
        spec["dt"] = 2e-12
    e, i = mixed_state(spec, 40_000, 30_000, seed=33)
    sim = make_sim64(slpic, spec)
    sim.load(0, 0, e)
    sim.load(0, 1, i)
    ref = oracle_mod.Oracle(spec, precision=64)
    ref.load(0, e)
    ref.load(1, i)
    for chunk in (1, 5, 40):
        sim.step(chunk)
        ref.step(chunk)
        for s in (0, 1):
            same_markers64(sim.particles(0, s), ref.particles(s), exact=exact)
            qg, qr = sim.charge(0, s), ref.charge(s)
            if exact:
                assert np.array_equal(qg, qr)
            else:
                # a marker on a cell boundary (above) moves about 2^-24 of its
                # charge between two nodes (the electrons emitted at rest do
                # so every step); a last-bit difference of beta moves one
                # fixed-point unit
                assert np.all(np.abs(qg - qr) <= 1e-6 * np.abs(qr) + 64)
                assert abs(int(qg.sum()) - int(qr.sum())) <= 64
    hg, hr = sim.history(0), ref.history()
    for k in ("n_live", "n_abs", "n_see"):
        assert np.array_equal(hg[k], hr[k]), k
    assert hr["n_see"].sum() > 20
    sim.close()


def test_fp64_one_step_matches_oracle(slpic, oracle_mod):
    spec = dense_spec(n_cells=512, pd=30.0)
    e, i = mixed_state(spec, 150_000, 50_000, seed=35)
    sim = make_sim64(slpic, spec)
    sim.load(0, 0, e)
    sim.load(0, 1, i)
    sim.step(1)
    ref = oracle_mod.Oracle(spec, precision=64)
    ref.load(0, e)
    ref.load(1, i)
    ref.step(1)
    hg, hr = sim.history(0)[-1], ref.history()[-1]
    for k in ("n_live", "n_coll", "n_candidates", "n_abs", "n_see", "n_clamp", "n_majorant",
              "marker_steps"):
        assert np.array_equal(hg[k], hr[k]), (k, hg[k], hr[k])
    assert min(hr["n_coll"]) > 100 and hr["n_see"] > 100
    for s in (0, 1):
        same_markers64(sim.particles(0, s), ref.particles(s), exact=False)
        qg, qr = sim.charge(0, s), ref.charge(s)
        assert np.allclose(qg, qr, rtol=1e-11, atol=1e-11 * 2**32)
    sim.close()


def test_fp64_breakdown_search_runs(slpic):
    """The batched breakdown search on an FP64 context (the plain form the
    FP32 sweep is compared with) brackets the same crossing as FP32 within
    the statistics of the seeds."""
    res = {}
    for prec in (32, 64):
        sim = slpic.Simulation(4, precision=prec)
        for j in range(4):
            sim.configure(j, inputs.gap_spec(n_cells=128, V=300.0, pd_torr_cm=1.0, gamma_se=0.07,
                                             field_mode=0, seed=3 + j, instance=j),
                          capacity=(256 * 2000, 512 * 2000))
        res[prec] = sim.paschen_bisect([100.0], [400.0], n_v=4, rounds=2, n_seed=2000)
        sim.close()
    lo32, hi32, _ = res[32]
    lo64, hi64, _ = res[64]
    width = 300.0 / 25.0
    assert abs(lo32[0] - lo64[0]) <= 2 * width
