"""Seeded synthetic inputs for the SLPIC-MCC step, shared by the CUDA path's
tests and benchmark and by the CPU oracle.

This module holds no arithmetic of the method itself (no push, collision,
deposit or field solve): only

* physical constants and the argon-like cross-section shapes, which are the
  method's *input data* (the paper took its cross sections from LXCat, which
  is not available here, so analytic argon-like shapes stand in for them);
* the energy grid of the cross-section table (nodes 2^(lo+o) (1 + m/2^sub) eV:
  equal steps inside each octave), which is the table's storage format;
* run configurations of the workloads, as plain dictionaries of numbers;
* seeded marker states drawn with numpy, in the FP32 storage format.
"""
import math

import numpy as np

# CODATA 2018 (SI)
QE = 1.602176634e-19
ME = 9.1093837015e-31
KB = 1.380649e-23
AMU = 1.66053906660e-27
M_AR = 39.948 * AMU          # Ar+ mass (electron deficit neglected)
TORR = 133.322368            # Pa

E_EXC = 11.55                # excitation threshold [eV]
E_ION = 15.76                # ionization threshold [eV]

ELECTRON, ION = 0, 1


def table_grid(lo_exp2=-7, log2_sub=8, octaves=16):
    """Node energies [eV] of the octave-uniform table."""
    sub = 1 << log2_sub
    j = np.arange(octaves * sub + 1)
    o, m = j // sub, j % sub
    return np.ldexp(1.0 + m / sub, lo_exp2 + o)


def argon_like_xsec(eps):
    """Argon-like analytic cross sections [m^2] at energies eps [eV].

    Elastic: Ramsauer-shaped minimum 1e-21 m^2 at 0.25 eV rising to 1.5e-19
    m^2 at 10 eV, then falling as eps^-1/2.  Excitation (11.55 eV threshold)
    peaks at 1e-20 m^2 at 25 eV; ionization (15.76 eV) peaks at 3e-20 m^2 at
    100 eV, both with the shape 2x/(1+x^2) in x = (eps-th)/(peak-th).
    """
    eps = np.asarray(eps, dtype=np.float64)
    low = 1e-21 + 1.49e-19 * (np.log(eps / 0.25) / np.log(40.0)) ** 2
    high = 1.5e-19 * np.sqrt(10.0 / np.maximum(eps, 1e-300))
    el = np.where(eps <= 10.0, low, high)

    def bump(th, pk, peak):
        x = (eps - th) / (pk - th)
        return np.where(eps > th, peak * 2.0 * x / (1.0 + x * x), 0.0)

    ex = bump(E_EXC, 25.0, 1e-20)
    io = bump(E_ION, 100.0, 3e-20)
    return el, ex, io


# Three argon-like excitation levels (the paper's five processes: elastic,
# three excitations and ionization), as (threshold [eV], peak energy [eV],
# peak cross section [m^2]) with the shape of argon_like_xsec.
EXC_LEVELS = ((E_EXC, 25.0, 0.6e-20), (13.0, 30.0, 0.3e-20), (14.0, 35.0, 0.2e-20))


def make_table(lo_exp2=-7, log2_sub=8, octaves=16, scale=(1.0, 1.0, 1.0), levels=1):
    """Cross-section table of the octave grid.  levels = 1: one excitation
    level at 11.55 eV; levels = 3: the three levels of EXC_LEVELS (keys
    sig_ex/e_ex, sig_ex2/e_ex2, sig_ex3/e_ex3)."""
    e = table_grid(lo_exp2, log2_sub, octaves)
    el, ex, io = argon_like_xsec(e)
    t = {
        "tab_lo_exp2": lo_exp2, "tab_log2_sub": log2_sub, "tab_octaves": octaves,
        "sig_el": (el * scale[0]).astype(np.float32),
        "sig_ex": (ex * scale[1]).astype(np.float32),
        "sig_io": (io * scale[2]).astype(np.float32),
        "e_ex": E_EXC, "e_io": E_ION, "n_exc": 1,
    }
    if levels == 3:
        t["n_exc"] = 3
        for k, (th, pk, peak) in enumerate(EXC_LEVELS):
            x = (e - th) / (pk - th)
            sig = np.where(e > th, peak * 2.0 * x / (1.0 + x * x), 0.0) * scale[1]
            name = "sig_ex" if k == 0 else "sig_ex%d" % (k + 1)
            t[name] = sig.astype(np.float32)
            t["e_ex" if k == 0 else "e_ex%d" % (k + 1)] = th
    return t


def ion_speed(V):
    """Speed of an Ar+ ion after falling through V volts."""
    return math.sqrt(2.0 * QE * V / M_AR)


def gap_spec(*, n_cells, V, pd_torr_cm=1.0, d=0.01, T_K=300.0, dt=None,
             vlim_e=None, vlim_i=math.inf, gamma_se=0.07, field_mode=1,
             area=1.0, charge_shift=32, seed=0, instance=0, table=None):
    """One parallel-plate instance as a plain dict of numbers and arrays."""
    p_Pa = pd_torr_cm / (d * 100.0) * TORR
    if vlim_e is None:
        vlim_e = 4.0 * ion_speed(V)
    dx = d / n_cells
    if dt is None:
        dt = dx / vlim_e
    spec = {
        "n_cells": int(n_cells), "d": d, "V": float(V), "area": area,
        "field_mode": int(field_mode), "p_Pa": p_Pa, "T_K": T_K, "dt": dt,
        "mass_e": ME, "mass_i": M_AR, "charge_e": -QE, "charge_i": QE,
        "vlim_e": float(vlim_e), "vlim_i": float(vlim_i),
        "gamma_se": gamma_se, "charge_shift": int(charge_shift),
        "seed": int(seed), "instance": int(instance),
    }
    spec.update(table if table is not None else make_table())
    return spec


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def small_gap_config(V=300.0, seed=0):
    """Plain small case: 256 cells, 1 Torr cm, 300 V, gamma 0.07,
    v_lim = 4 x the Ar+ speed after falling through V, dt = dx / v_lim;
    2e4 electrons seeded at the cathode at 1 eV, 2000 steps."""
    spec = gap_spec(n_cells=256, V=V, seed=seed)
    return spec, {"n_seed": 20000, "seed_mode": 0, "e0": 1.0, "steps": 2000}


def paschen_point_config(V=300.0, seed=0):
    """Single Paschen point: 4096 cells, 1 Torr cm, V in {250, 300, 350} V,
    1e6 electrons at the cathode at 1 eV, capacity 1.6e7 markers/species."""
    spec = gap_spec(n_cells=4096, V=V, seed=seed)
    return spec, {"n_seed": 1_000_000, "seed_mode": 0, "e0": 1.0,
                  "steps": 100_000, "capacity": 16_000_000}


def microbench_config(n_markers=32_000_000, seed=0, field_mode=1):
    """Push + MCC microbenchmark: 3.2e7 electrons uniform over a 1 cm gap of
    4096 cells at 1 Torr and 300 V, energies log-uniform over 0.1-200 eV,
    isotropic; v_lim = 1/8 of the median electron speed, dt = dx / v_lim;
    4096-bin octave-uniform table over 2^-7..2^9 eV."""
    e_med = math.sqrt(0.1 * 200.0)
    v_med = math.sqrt(2.0 * QE * e_med / ME)
    vlim = v_med / 8.0
    spec = gap_spec(n_cells=4096, V=300.0, vlim_e=vlim, seed=seed,
                    field_mode=field_mode)
    return spec, {"n_seed": int(n_markers), "seed_mode": 2, "e_lo": 0.1,
                  "e_hi": 200.0, "steps": 1000}


def gap_state(n, spec, rng_seed=0, e_lo=0.1, e_hi=200.0, species=ELECTRON,
              wj=1.0, first_id=0, wj_spread=0.0):
    """n markers uniform over the gap with log-uniform energies in
    [e_lo, e_hi] eV and isotropic directions (numpy draws, FP32 storage)."""
    rng = np.random.default_rng(rng_seed)
    N = spec["n_cells"]
    cell = rng.integers(0, N, size=n, dtype=np.int32)
    off = rng.random(n, dtype=np.float32)
    off = np.minimum(off, np.float32(np.nextafter(np.float32(1), np.float32(0))))
    mass = spec["mass_e"] if species == ELECTRON else spec["mass_i"]
    e = e_lo * np.exp(rng.random(n) * math.log(e_hi / e_lo))
    v = np.sqrt(2.0 * QE * e / mass)
    ct = 1.0 - 2.0 * rng.random(n)
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    ph = 2.0 * math.pi * rng.random(n)
    w = np.full(n, wj, dtype=np.float64)
    if wj_spread:
        w = w * (1.0 + wj_spread * rng.random(n))
    return {
        "cell": cell,
        "off": off.astype(np.float32),
        "vx": (v * ct).astype(np.float32),
        "vy": (v * st * np.cos(ph)).astype(np.float32),
        "vz": (v * st * np.sin(ph)).astype(np.float32),
        "wj": w.astype(np.float32),
        "id": (first_id + np.arange(n)).astype(np.uint32),
    }


def beam_state(n, spec, v_x, cell=None, off=0.5, species=ELECTRON, wj=1.0):
    """n identical markers moving along +x with speed v_x (monoenergetic)."""
    N = spec["n_cells"]
    c = N // 2 if cell is None else cell
    return {
        "cell": np.full(n, c, np.int32),
        "off": np.full(n, off, np.float32),
        "vx": np.full(n, v_x, np.float32),
        "vy": np.zeros(n, np.float32),
        "vz": np.zeros(n, np.float32),
        "wj": np.full(n, wj, np.float32),
        "id": np.arange(n, dtype=np.uint32),
    }


def rest_state(n, cell=0, off=0.0, wj=1.0, first_id=0):
    """n markers at rest at one position."""
    return {
        "cell": np.full(n, cell, np.int32),
        "off": np.full(n, off, np.float32),
        "vx": np.zeros(n, np.float32),
        "vy": np.zeros(n, np.float32),
        "vz": np.zeros(n, np.float32),
        "wj": np.full(n, wj, np.float32),
        "id": (first_id + np.arange(n)).astype(np.uint32),
    }
