"""Throughput of the SLPIC-MCC step on GB300: marker-steps per second.

Workload (default): the push + MCC microbenchmark gap -- 3.2e7 electrons
uniform over a 1 cm gap of 4096 cells at 1 Torr and 300 V, energies
log-uniform over 0.1-200 eV, isotropic, v_lim = 1/8 of the median speed,
dt = dx / v_lim, three-process null-collision MCC on a 4096-bin table, ion
births and secondary emission live, fixed-point deposit and the Poisson solve
every step.  A step is one pass of the whole step over every live marker.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own
independent instance (instances do not exchange data), so scaling is weak.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_MARKER_STEP = 48  # read 28 B of state, write the 20 B that change
BYTES_PER_MARKER_STEP_FP64 = 84  # FP64 marker: read 48 B, write the 36 B that change
L2_BYTES = 129 * 2**20
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--markers", type=int, default=32_000_000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--paschen", action="store_true",
                    help="(default) time the batched FP32 breakdown-voltage sweep against the "
                         "plain one-instance FP64 bisection")
    ap.add_argument("--no-paschen", action="store_true",
                    help="leave out the breakdown-voltage sweep")
    ap.add_argument("--paschen-full", action="store_true",
                    help="instead of the benchmark, run the full breakdown search (24 pd points "
                         "over 0.05-200 Torr cm, 8 voltages each, SLPIC at three v_lim and PIC) "
                         "and print one JSON line")
    ap.add_argument("--cpu-config1", action="store_true",
                    help="instead of the benchmark, time config 1 (256 cells, 2e4 electrons, "
                         "2000 steps) in full on the CPU oracle and print one JSON line")
    ap.add_argument("--tab-sims", default=None, metavar="ROWS",
                    help="instead of the benchmark, run the PIC vs SLPIC study shaped like "
                         "Table tab:sims on the rows given (comma-separated indices 0-10, "
                         "or 'all') and print one JSON line")
    ap.add_argument("--batch", action="store_true",
                    help="instead of the benchmark, time the batched sweep workload: 32 uneven "
                         "instances (pd 0.1-100 Torr cm, 1e4-4e6 electrons) in one context")
    ap.add_argument("--dense", action="store_true",
                    help="instead of the benchmark, time one collision-dense instance: the "
                         "batched sweep's instance 26 (about 33 Torr cm, dx = lambda_min / 4, "
                         "6339 cells) with 4e6 electrons, a quarter of them null-collision "
                         "candidates per step")
    ap.add_argument("--small-pop", action="store_true",
                    help="instead of the benchmark, time the paper's breakdown run at 1 Torr cm "
                         "(Table tab:sims row 4) with and without the single-CTA path")
    ap.add_argument("--small-pop-steps", type=int, default=13140)
    ap.add_argument("--tab-sims-pic-max", type=float, default=4.0,
                    help="largest pressure [Torr] with a PIC run (the paper's: 4)")
    ap.add_argument("--tab-sims-pic-full-max", type=float, default=0.4,
                    help="above this pressure [Torr] a PIC run covers its first 3 of 15 "
                         "windows and its wall time is extrapolated")
    ap.add_argument("--tab-sims-slpic-full-max", type=float, default=30.0,
                    help="above this pressure [Torr] an SLPIC run covers its first 3 of 15 "
                         "windows and its wall time is extrapolated")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        v = d.get("hbm_gbs")
        if isinstance(v, dict):
            v = v.get("value")
        if v:
            return float(v), "measured"
    except Exception:
        pass
    return FALLBACK_HBM_GBS, "fallback"


def _code_only(text):
    """C++ source without its comments and whitespace (string literals in
    these kernel files hold no comment markers)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return re.sub(r"\s+", "", text)


def push_source_hash():
    """Hash of the particle kernel's code (the kernel and its headers, with
    comments and whitespace left out): a recorded traffic figure stays valid
    through comment edits and lapses with any change of code."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2103_12194_gb300", "csrc")
    for name in ("push.cu", "device_common.cuh", "slpic_internal.h", "step_ops.cuh"):
        h.update(_code_only(open(os.path.join(csrc, name)).read()).encode())
    return h.hexdigest()[:16]


def push_traffic():
    """DRAM bytes per marker of the particle kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "push_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("push_source_sha256_16") == push_source_hash():
            return float(d["dram_bytes_per_marker"])
    except Exception:
        pass
    return None


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "slpic_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines()]
        except Exception:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 7:
                continue
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except ValueError:
                continue
            for n, v in zip(names, r[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_slice_run(spec, n, first, seconds):
    """One host process: the FP64 oracle on markers first .. first + n - 1 of
    the workload's sample (the same draw as the GPU's), stepped for about
    `seconds`.  Returns (marker-steps, seconds)."""
    import oracle
    from paper_2103_12194_gb300 import inputs
    st = inputs.gap_state(first + n, spec, rng_seed=1, e_lo=0.1, e_hi=200.0)
    st = {k: v[first:first + n] for k, v in st.items()}
    o = oracle.Oracle(spec, precision=64)
    o.load(0, st)
    t0 = time.perf_counter()
    o.step(1)
    per_step = max(time.perf_counter() - t0, 1e-6)
    k = max(1, min(5000, int(seconds / per_step)))
    t0 = time.perf_counter()
    o.step(k)
    dt = time.perf_counter() - t0
    return int(o.history()["marker_steps"][1:].sum()), dt


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the
    machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(spec, n_markers, seconds):
    """The oracle (FP64, as it stands) on a bounded sample of the same
    workload: first one host thread on 2e5 of the workload's electrons, then
    every host core at once, each core's process on its own slice of the same
    2e5 electrons (the oracle is single-threaded; the slices share nothing).
    The all-cores figure is the baseline; the single-thread one is kept."""
    import multiprocessing
    n = min(n_markers, 200_000)
    ms1, dt1 = _oracle_slice_run(spec, n, 0, seconds / 2)
    cores = os.cpu_count() or 1
    per = max(1, n // cores)
    args = [(spec, per, c * per, seconds / 2) for c in range(cores)]
    t0 = time.perf_counter()
    with multiprocessing.get_context("spawn").Pool(cores) as pool:
        res = pool.starmap(_oracle_slice_run, args)
    wall = time.perf_counter() - t0
    ms_all = sum(r[0] for r in res)
    dt_all = max(r[1] for r in res)
    return {"value": ms_all / dt_all, "unit": "marker-steps/s", "cores": cores, "kind": "oracle",
            "stepping_s": dt_all,
            "cpu": cpu_model(),
            "sample": "%d of the workload's electrons (same draw), FP64 oracle: %d processes "
                      "of %d electrons each, %.1f s of stepping (%.1f s with start-up)"
                      % (n, cores, per, dt_all, wall),
            "single_thread": {"value": ms1 / dt1, "cores": 1,
                              "sample": "%d electrons, %.1f s" % (n, dt1)}}


def cpu_config1():
    """Config 1 of the workloads timed in full on the oracle (FP64, one host
    thread): 256 cells, 1 Torr cm, 300 V, gamma 0.07, 2e4 electrons seeded at
    the cathode at 1 eV, 2000 steps, Poisson on."""
    import oracle
    from paper_2103_12194_gb300 import inputs
    spec, run = inputs.small_gap_config()
    o = oracle.Oracle(spec, precision=64)
    o.seed(0, run["n_seed"], run["seed_mode"], e0=run["e0"])
    t0 = time.perf_counter()
    o.step(run["steps"])
    dt = time.perf_counter() - t0
    h = o.history()
    ms = int(h["marker_steps"].sum())
    return {"workload": "config 1: 256 cells, 1 Torr cm, 300 V, gamma 0.07, 2e4 electrons at "
                        "the cathode at 1 eV, 2000 steps, Poisson on, FP64 oracle, 1 thread",
            "seconds": dt, "marker_steps": ms, "value": ms / dt, "unit": "marker-steps/s",
            "live_at_end": [int(x) for x in h["n_live"][-1]], "cores": 1, "cpu": cpu_model()}


def paschen_sweep(slpic, inputs, local, stream, pds=(0.5, 1.0, 2.0, 4.0), n_v=7, rounds=3,
                  n_seed=1000, v_lo=100.0, v_hi=900.0):
    """Breakdown voltages at a few pd points (d = 1 cm, gamma = 0.07, cells
    from dx = lambda_min / 4): the batched FP32 search (all pd points and n_v
    voltages per round in one context) against the plain FP64 bisection (one
    single-instance context per pd point, one voltage per round).  With
    n_v + 1 a power of two the bisection's halvings reach exactly the same
    final bracket width, and both evaluate every gain from n_seed electrons:
    the same breakdown-voltage accuracy."""
    import numpy as np
    import torch
    table = inputs.make_table()
    smax = float(np.max(table["sig_el"].astype(np.float64) + table["sig_ex"] + table["sig_io"]))

    def spec_for(pd, j, inst):
        n_g = pd / 1.0 * inputs.TORR / (inputs.KB * 300.0)
        cells = int(min(16384, max(128, math.ceil(4 * 0.01 * n_g * smax))))
        return inputs.gap_spec(n_cells=cells, V=300.0, pd_torr_cm=pd, gamma_se=0.07,
                               field_mode=0, seed=11 + inst, instance=inst)

    cap = (2 * 16 * n_seed, 32 * n_seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim = slpic.Simulation(len(pds) * n_v, device=local, stream=stream)
    for p, pd in enumerate(pds):
        for j in range(n_v):
            sim.configure(p * n_v + j, spec_for(pd, j, p * n_v + j), capacity=cap)
    lo32, hi32, _ = sim.paschen_bisect([v_lo] * len(pds), [v_hi] * len(pds), n_v=n_v,
                                       rounds=rounds, n_seed=n_seed)
    sim.close()
    t32 = time.perf_counter() - t0
    halvings = int(round(rounds * math.log2(n_v + 1)))
    assert 2 ** halvings == (n_v + 1) ** rounds, "n_v + 1 must be a power of two"
    t0 = time.perf_counter()
    lo64, hi64 = [], []
    for p, pd in enumerate(pds):
        sim = slpic.Simulation(1, device=local, stream=stream, precision=64)
        sim.configure(0, spec_for(pd, 0, 0), capacity=cap)
        lo, hi, _ = sim.paschen_bisect([v_lo], [v_hi], n_v=1, rounds=halvings, n_seed=n_seed)
        sim.close()
        lo64.append(float(lo[0]))
        hi64.append(float(hi[0]))
    t64 = time.perf_counter() - t0
    return {"pd_torr_cm": list(pds), "n_seed": n_seed,
            "fp32_batched": {"s": t32, "instances": len(pds) * n_v, "rounds": rounds,
                             "Vb_lo": [float(x) for x in lo32], "Vb_hi": [float(x) for x in hi32]},
            "fp64_plain": {"s": t64, "instances": 1, "rounds": halvings,
                           "Vb_lo": lo64, "Vb_hi": hi64},
            "bracket_width_V": {"fp32_batched": (v_hi - v_lo) / (n_v + 1) ** rounds,
                                "fp64_plain": (v_hi - v_lo) / 2 ** halvings},
            "Vb_mid_difference_V": [0.5 * (a + b) - 0.5 * (c + d)
                                    for a, b, c, d in zip(lo32, hi32, lo64, hi64)],
            "speedup": t64 / t32}


def paschen_full(slpic, inputs, local, stream, n_pd=24, pd_lo=0.05, pd_hi=200.0, max_cells=2048,
                 n_v=8, rounds=3, n_seed=1000, pic_max=4.0, fp64_points=4):
    """The full breakdown search of the sweep workloads, with the cells capped:
    n_pd pd points log-spaced over [pd_lo, pd_hi] Torr cm (d = 1 cm,
    gamma = 0.07, cells from dx = lambda_min / 4 clamped to 128-max_cells),
    each bracketed by a batched
    section search over n_v voltages per round (n_pd * n_v instances live in
    one context per method).  Methods: SLPIC with v_lim = 1, 4 and 16 times
    v0 = sqrt(2 e V / M), and standard PIC (no limit, dt = dx / v_max) for
    pd <= pic_max (Sec. V ran PIC up to 4 Torr).  Then the plain FP64 form
    (one single-instance context per pd point, bisection at the same final
    bracket width) for SLPIC at 4 v0 on fp64_points of the points."""
    import numpy as np
    import torch
    table = inputs.make_table()
    smax = float(np.max(table["sig_el"].astype(np.float64) + table["sig_ex"] + table["sig_io"]))
    pds = [pd_lo * (pd_hi / pd_lo) ** (k / (n_pd - 1)) for k in range(n_pd)]

    def spec_for(pd, inst):
        n_g = pd * inputs.TORR / (inputs.KB * 300.0)
        cells = int(min(max_cells, max(128, math.ceil(4 * 0.01 * n_g * smax))))
        return inputs.gap_spec(n_cells=cells, V=300.0, pd_torr_cm=pd, gamma_se=0.07,
                               field_mode=0, seed=31 + inst, instance=inst)

    def v_guess(pd):
        # Paschen's law with the Lieberman constants of Sec. V (A = 11.5,
        # B = 176, gamma = 0.07) above its left asymptote, else 1000 V
        if pd <= 0.3:
            return 1000.0
        return 176.0 * pd / (math.log(11.5 * pd) - math.log(math.log(1 + 1 / 0.07)))

    cap = (2 * 16 * n_seed, 32 * n_seed)
    out = {"pd_torr_cm": pds, "n_v": n_v, "rounds": rounds, "n_seed": n_seed,
           "initial_bracket": "[0.5, 3] x Paschen's law (A = 11.5, B = 176, gamma = 0.07), "
                              "1000 V below 0.3 Torr cm",
           "bracket_width_fraction_of_initial": 1.0 / (n_v + 1) ** rounds, "methods": {}}
    for name, f, pmax in (("SLPIC v_lim=1 v0", 1.0, None), ("SLPIC v_lim=4 v0", 4.0, None),
                          ("SLPIC v_lim=16 v0", 16.0, None), ("PIC", 0.0, pic_max)):
        pts = [p for p in pds if pmax is None or p <= pmax * 1.0001]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim = slpic.Simulation(len(pts) * n_v, device=local, stream=stream)
        for a, pd in enumerate(pts):
            for j in range(n_v):
                sim.configure(a * n_v + j, spec_for(pd, a * n_v + j), capacity=cap)
        lo, hi, _ = sim.paschen_bisect([0.5 * v_guess(p) for p in pts],
                                       [3.0 * v_guess(p) for p in pts], n_v=n_v,
                                       rounds=rounds, n_seed=n_seed, vlim_factor=f,
                                       max_steps=2_000_000)
        sim.close()
        out["methods"][name] = {"s": time.perf_counter() - t0, "instances": len(pts) * n_v,
                                "pd_torr_cm": pts, "Vb_lo": [float(x) for x in lo],
                                "Vb_hi": [float(x) for x in hi]}
        print("# " + json.dumps({name: out["methods"][name]}), file=sys.stderr, flush=True)
    # the plain FP64 form on a subset, at the same final bracket width
    # (n_v + 1 = 8 voltages a round, 3 rounds = 9 halvings)
    sub = [pds[k] for k in np.linspace(1, n_pd - 2, fp64_points).round().astype(int)]
    lo32, hi32, t32 = [], [], 0.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim = slpic.Simulation(len(sub) * 7, device=local, stream=stream)
    for a, pd in enumerate(sub):
        for j in range(7):
            sim.configure(a * 7 + j, spec_for(pd, a * 7 + j), capacity=cap)
    lo, hi, _ = sim.paschen_bisect([0.5 * v_guess(p) for p in sub],
                                   [3.0 * v_guess(p) for p in sub], n_v=7, rounds=3,
                                   n_seed=n_seed, vlim_factor=4.0, max_steps=2_000_000)
    sim.close()
    t32 = time.perf_counter() - t0
    t0 = time.perf_counter()
    lo64, hi64 = [], []
    for pd in sub:
        sim = slpic.Simulation(1, device=local, stream=stream, precision=64)
        sim.configure(0, spec_for(pd, 0), capacity=cap)
        l, h, _ = sim.paschen_bisect([0.5 * v_guess(pd)], [3.0 * v_guess(pd)], n_v=1, rounds=9,
                                     n_seed=n_seed, vlim_factor=4.0, max_steps=2_000_000)
        sim.close()
        lo64.append(float(l[0]))
        hi64.append(float(h[0]))
    t64 = time.perf_counter() - t0
    out["fp32_batched_vs_fp64_plain"] = {
        "method": "SLPIC v_lim=4 v0", "pd_torr_cm": sub, "bracket_width_fraction_of_initial": 1 / 512,
        "fp32_batched": {"s": t32, "Vb_lo": [float(x) for x in lo], "Vb_hi": [float(x) for x in hi]},
        "fp64_plain": {"s": t64, "Vb_lo": lo64, "Vb_hi": hi64}, "speedup": t64 / t32}
    return out


# Table tab:sims: pressure [Torr] at d = 1 cm, voltage [V] near the paper's
# breakdown voltage, and cells (dx = a quarter of the mean free path).
TAB_SIMS = ((0.3, 260.0, 66), (0.4, 195.0, 88), (0.6, 175.0, 131), (1.0, 170.0, 219),
            (2.0, 185.0, 437), (4.0, 225.0, 874), (6.0, 262.0, 1310), (10.0, 340.0, 2184),
            (30.0, 620.0, 6550), (100.0, 1400.0, 21832), (300.0, 3100.0, 65494))


def tab_sims_spec(inputs, p, V, cells, pic, seed, instance=0):
    """A Table tab:sims gap set up as in Sec. IV: d = 1 cm, the field V/d
    imposed, the five electron-argon processes, the Eq. sey yield.  SLPIC:
    v_lim = v0 = sqrt(2 e V / M), dt = dx / v0; PIC: no speed limit and
    dt = dx / v_max, v_max = sqrt(2 e V / m_e)."""
    dx = 0.01 / cells
    v0 = inputs.ion_speed(V)
    vmax = math.sqrt(2 * inputs.QE * V / inputs.ME)
    spec = inputs.gap_spec(n_cells=cells, V=V, pd_torr_cm=p, gamma_se=0.07, field_mode=0,
                           vlim_e=math.inf if pic else v0, dt=dx / (vmax if pic else v0),
                           seed=seed, instance=instance, table=inputs.make_table(levels=3))
    spec["emission_model"] = 1
    return spec


def tab_sims_bracket(slpic, inputs, rows, local, stream, n_v=8, rounds=2, n_seed=2000):
    """Breakdown brackets of the synthetic gas at the rows' pressures: the
    batched search on the gain G >= 1 (Sec. II.A) over all rows at once,
    with the SLPIC setup of the runs (v_lim = v0), from [V / 2, 2 V]."""
    import torch
    sim = slpic.Simulation(len(rows) * n_v, device=local, stream=stream)
    for a, r in enumerate(rows):
        p, V, cells = TAB_SIMS[r]
        for j in range(n_v):
            i = a * n_v + j
            sim.configure(i, tab_sims_spec(inputs, p, V, cells, False, 500 + i, i),
                          capacity=(1 << 20, 1 << 20))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lo, hi, _ = sim.paschen_bisect([0.5 * TAB_SIMS[r][1] for r in rows],
                                   [2.0 * TAB_SIMS[r][1] for r in rows], n_v=n_v,
                                   rounds=rounds, n_seed=n_seed, e0=1.0, vlim_factor=1.0)
    wall = time.perf_counter() - t0
    sim.close()
    return [float(x) for x in lo], [float(x) for x in hi], wall


def tab_sims_run(slpic, inputs, p, V, cells, pic, local, stream, seed=1, windows=15,
                 run_windows=None):
    """One breakdown run of Table tab:sims on the GPU (Sec. IV and V): 100
    electrons at rest at the cathode, the ion population tracked over 30 ion
    crossing times in `windows` windows.  SLPIC: 30 crossings (of 2 d / v0
    each) are 60 cells steps of dx / v0; PIC takes sqrt(M / m_e) times more
    steps.  With run_windows < windows only the first run_windows windows
    run and the wall time is extrapolated to the whole run (no
    classification).  An ion population past a third of its store (above
    breakdown for certain) ends the run."""
    import numpy as np
    import torch
    spec = tab_sims_spec(inputs, p, V, cells, pic, seed)
    n_t = 60 * cells * (math.sqrt(inputs.M_AR / inputs.ME) if pic else 1.0)
    spw = int(math.ceil(n_t / windows))
    nw = windows if run_windows is None else run_windows
    sim = slpic.Simulation(1, device=local, stream=stream)
    sim.configure(0, spec, capacity=(1 << 18, 1 << 18))
    sim.seed(0, slpic.ELECTRON, 100, slpic.SEED_REST)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    means, above = sim.ion_trend(spw, max(nw, 2))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    tot = sim.tallies(0)
    sim.close()
    m = means[0]
    steps = int(tot["step"]) + 1  # the step index of the last step run
    rec = {"method": "PIC" if pic else "SLPIC", "dt_s": spec["dt"], "steps_planned": spw * windows,
           "steps_run": steps, "wall_s": wall, "us_per_step": wall / max(steps, 1) * 1e6,
           "marker_steps": int(tot["marker_steps"]), "collisions": int(np.sum(tot["n_coll"])),
           "ion_means": [float(x) for x in m]}
    if nw < windows:
        rec["wall_s_extrapolated"] = wall * windows / max(nw, 2)
        rec["class"] = None
    else:
        rec["class"] = "above" if above[0] else "below"
        rec["saturated"] = bool((m < 0).any())
    return rec


def tab_sims(slpic, inputs, rows, pic_max, pic_full_max, local, stream, margin=0.03,
             slpic_full_max=30.0):
    lo, hi, t_bracket = tab_sims_bracket(slpic, inputs, rows, local, stream)
    out = {"bracket_search_s": t_bracket, "rows": []}
    for a, r in enumerate(rows):
        p, V, cells = TAB_SIMS[r]
        rec = {"row": r, "p_torr": p, "V_paper": V, "cells": cells,
               "Vb_bracket": [lo[a], hi[a]],
               "V_runs": [(1 - margin) * lo[a], (1 + margin) * hi[a]], "runs": []}
        for Vr in rec["V_runs"]:
            run = {"V": Vr, "slpic": tab_sims_run(slpic, inputs, p, Vr, cells, False, local,
                                                  stream,
                                                  run_windows=None if p <= slpic_full_max else 3)}
            if p <= pic_max:
                part = None if p <= pic_full_max else 3
                run["pic"] = tab_sims_run(slpic, inputs, p, Vr, cells, True, local, stream,
                                          run_windows=part)
            rec["runs"].append(run)
        sl = sum(x["slpic"].get("wall_s_extrapolated", x["slpic"]["wall_s"]) for x in rec["runs"])
        rec["slpic_wall_s"] = sl
        rec["slpic_extrapolated"] = p > slpic_full_max
        if p <= pic_max:
            pc = sum(x["pic"].get("wall_s_extrapolated", x["pic"]["wall_s"]) for x in rec["runs"])
            rec["pic_wall_s"] = pc
            rec["pic_extrapolated"] = p > pic_full_max
            rec["speedup"] = pc / sl
            if p <= pic_full_max:
                rec["same_class"] = all(x["pic"]["class"] == x["slpic"]["class"]
                                        for x in rec["runs"])
        print(json.dumps({"tab_sims_row": rec}), file=sys.stderr, flush=True)
        out["rows"].append(rec)
    return out


def batch_specs(inputs, n_inst=32):
    """The batched sweep workload: instance k at pd_k = 0.1 * 1000^(k/31)
    Torr cm (d = 1 cm), cells from dx = lambda_min / 4 clamped to
    128..16384, round(1e4 * 400^(k/31)) electrons log-uniform over
    0.1-200 eV, V_k from Paschen's law (Eq. paschen, A = 11.5 / (cm Torr),
    B = 176 V / (cm Torr), gamma = 0.07) above 0.3 Torr cm, else 1000 V;
    Poisson on, v_lim = 4 sqrt(2 e V / M), dt = dx / v_lim."""
    import numpy as np
    table = inputs.make_table()
    smax = float(np.max(table["sig_el"].astype(np.float64) + table["sig_ex"] + table["sig_io"]))
    out = []
    for k in range(n_inst):
        pd = 0.1 * 1000.0 ** (k / (n_inst - 1))
        n_g = pd * inputs.TORR / (inputs.KB * 300.0)
        cells = int(min(16384, max(128, math.ceil(4 * 0.01 * n_g * smax))))
        n = int(round(1e4 * 400.0 ** (k / (n_inst - 1))))
        if pd > 0.3:
            V = 176.0 * pd / (math.log(11.5 * pd) - math.log(math.log(1.0 + 1.0 / 0.07)))
        else:
            V = 1000.0
        spec = inputs.gap_spec(n_cells=cells, V=V, pd_torr_cm=pd, gamma_se=0.07, field_mode=1,
                               seed=200 + k, instance=k)
        out.append((spec, n))
    return out


def batch_bench(slpic, inputs, steps, warmup, local, stream, world=1, rank=0):
    """All 32 instances of the sweep workload advanced by the same launches:
    aggregate marker-steps/s and the particle kernel's roofline.  With
    several ranks the instances are shared among them by markers x steps
    (ranks.partition) and each rank steps its own in one context; rank 0
    gathers the per-instance marker-steps, and the job's rate is their sum
    over the slowest rank's time."""
    import torch
    from paper_2103_12194_gb300 import ranks
    all_items = batch_specs(inputs)
    mine = ranks.partition([n for _, n in all_items], world)[rank]
    items = [all_items[k] for k in mine]
    for j, (spec, _) in enumerate(items):
        spec["instance"] = j
    sim = slpic.Simulation(len(items), device=local, stream=stream)
    for k, (spec, n) in enumerate(items):
        # avalanches above breakdown grow the ions about 4x in 400 steps
        sim.configure(k, spec, capacity=(4 * n + 65536, 8 * n + 65536))
    for k, (spec, n) in enumerate(items):
        sim.seed(k, slpic.ELECTRON, n, slpic.SEED_GAP, e_lo=0.1, e_hi=200.0)
    shape = sim.autotune(steps_each=4)
    sim.step(warmup)
    sim.synchronize()
    ms0 = sum(int(sim.tallies(k)["marker_steps"]) for k in range(len(items)))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    wall_ms = e0.elapsed_time(e1)
    ms1 = sum(int(sim.tallies(k)["marker_steps"]) for k in range(len(items)))
    # the particle kernel alone, timed launch by launch on the same state
    sim.set_profiling(True)
    ms2 = ms1
    sim.step(steps)
    sim.synchronize()
    push_ms, push_n = sim.profile()
    ms3 = sum(int(sim.tallies(k)["marker_steps"]) for k in range(len(items)))
    sim.set_profiling(False)
    live = [[sim.count(k, 0), sim.count(k, 1)] for k in range(len(items))]
    per_inst = {mine[k]: (int(sim.tallies(k)["marker_steps"]), live[k]) for k in range(len(items))}
    sim.close()
    peak, peak_kind = peaks()
    achieved = BYTES_PER_MARKER_STEP * (ms3 - ms2) / (push_ms / 1e3) / 1e9
    t_job, work_job = combine_ranks(wall_ms, ms1 - ms0, world, "cuda")
    gathered = ranks.gather(per_inst, world, rank)
    if gathered is not None and sorted(gathered) != list(range(len(all_items))):
        raise RuntimeError("the ranks did not cover every instance")
    return {"value": work_job / t_job, "unit": "marker-steps/s", "steps": steps,
            "ms_per_step": t_job * 1e3 / steps, "instances": len(all_items),
            "instances_per_rank": len(items), "ranks": world,
            "markers_seeded": sum(n for _, n in all_items),
            "cells": [spec["n_cells"] for spec, _ in all_items],
            "launch_shape": {"push_warps_per_cta": shape[0], "collide_ctas_per_sm": shape[1]},
            "roofline": {"bound": "hbm", "kernel": "k_push", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                         "push_share_of_step": push_ms / ((ms3 - ms2) / (ms1 - ms0) * wall_ms)},
            "live_at_end": ([gathered[k][1] for k in range(len(all_items))]
                            if gathered is not None else None)}


def dense_bench(slpic, inputs, steps, warmup, local, stream, n=4_000_000):
    """One collision-dense instance (the batched sweep's instance 26: about
    33 Torr cm at the paper's resolution, dx = lambda_min / 4, dt = dx /
    v_lim), n electrons log-uniform over 0.1-200 eV, Poisson on: about a
    quarter of the electrons are null-collision candidates each step, so the
    collision kernel carries a large share of the step.  Whole steps timed
    with CUDA events, then the particle kernel alone on the same state."""
    import torch
    spec, _ = batch_specs(inputs)[26]
    spec["instance"] = 0
    sim = slpic.Simulation(1, device=local, stream=stream)
    sim.configure(0, spec, capacity=(4 * n + 65536, 4 * n + 65536))
    sim.seed(0, slpic.ELECTRON, n, slpic.SEED_GAP, e_lo=0.1, e_hi=200.0)
    sim.step(warmup)
    sim.synchronize()
    t0 = sim.tallies(0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    wall_ms = e0.elapsed_time(e1)
    t1 = sim.tallies(0)
    sim.set_profiling(True)
    sim.step(steps)
    sim.synchronize()
    push_ms, _ = sim.profile()
    t2 = sim.tallies(0)
    sim.set_profiling(False)
    sim.close()
    ms = int(t1["marker_steps"]) - int(t0["marker_steps"])
    cand = int(t1["n_candidates"]) - int(t0["n_candidates"])
    prof_ms = int(t2["marker_steps"]) - int(t1["marker_steps"])
    return {"value": ms / (wall_ms / 1e3), "unit": "marker-steps/s", "steps": steps,
            "warmup": warmup, "ms_per_step": wall_ms / steps, "cells": spec["n_cells"],
            "electrons_seeded": n, "live_at_end": [int(x) for x in t2["n_live"]],
            "candidates_per_marker_step": cand / ms if ms else None,
            "push_share_of_step": (push_ms / (prof_ms / ms * wall_ms)) if ms and prof_ms else None}


def small_pop(slpic, inputs, steps, local, stream, V=171.5):
    """The paper's breakdown run at 1 Torr cm (219 cells, V near this gas's
    V_b, SLPIC with v_lim = v0, 100 electrons at rest, Eq. sey yield, five
    processes), followed for `steps` steps (13140 = 30 ion crossings) with
    the ion-trend protocol: once with the single-CTA path for small
    populations, once with the batched kernels only.  Both give the same
    markers; the wall times differ."""
    import numpy as np
    import torch
    p, _, cells = TAB_SIMS[3]
    out = {}
    for name, limit in (("single_cta", 32), ("batched", 0)):
        spec = tab_sims_spec(inputs, p, V, cells, False, seed=7)
        sim = slpic.Simulation(1, device=local, stream=stream)
        sim.configure(0, spec, capacity=(1 << 18, 1 << 18))
        sim.seed(0, slpic.ELECTRON, 100, slpic.SEED_REST)
        sim.set_small_limit(limit)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        means, _ = sim.ion_trend(max(1, steps // 15), 15)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        tot = sim.tallies(0)
        n = int(tot["step"]) + 1
        out[name] = {"wall_s": wall, "steps": n, "us_per_step": wall / n * 1e6,
                     "marker_steps": int(tot["marker_steps"]),
                     "mean_live_markers": int(tot["marker_steps"]) / n,
                     "final_live": [int(x) for x in tot["n_live"]]}
        sim.close()
    out["same_markers"] = out["single_cta"]["marker_steps"] == out["batched"]["marker_steps"]
    out["speedup"] = out["batched"]["wall_s"] / out["single_cta"]["wall_s"]
    return out


def combine_ranks(elapsed_ms, marker_steps, world, device):
    """Whole-job figures of a weak-scaling run: every rank advances its own
    independent instance, so the job's time is the slowest rank's and its
    work the sum of the ranks' marker-steps.  Returns (seconds, marker-steps).
    With world > 1 the ranks exchange their two numbers (all-gather on
    `device`: "cuda" under NCCL, "cpu" under gloo)."""
    times, counts = [float(elapsed_ms)], [float(marker_steps)]
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([float(elapsed_ms), float(marker_steps)], dtype=torch.float64,
                          device=device)
        allt = [torch.zeros_like(tt) for _ in range(world)]
        dist.all_gather(allt, tt)
        times = [float(x[0]) for x in allt]
        counts = [float(x[1]) for x in allt]
    return max(times) / 1e3, sum(counts)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2103_12194_gb300 import inputs
    spec, _ = inputs.microbench_config(n_markers=args.markers)
    per_step_s = args.cpu_seconds / max(1, args.steps + args.warmup)
    cb = cpu_baseline(spec, args.markers, max(1.0, per_step_s * args.steps))
    line = {"impl": "reference", "metric": "marker-steps/s", "value": cb["value"],
            "unit": "marker-steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "push+MCC microbenchmark gap (CPU oracle sample)",
                       "markers": args.markers, "cells": 4096},
            "cpu_baseline": cb,
            # each of the K steps is a bounded sample of the workload: the
            # all-cores stepping time spread over them
            "ms_per_step": cb["stepping_s"] * 1e3 / max(1, args.steps),
            "e2e": {"value": cb["value"], "unit": "marker-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    from paper_2103_12194_gb300 import build, inputs, slpic

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.current_stream()
    if args.batch:
        res = batch_bench(slpic, inputs, args.steps if args.steps != 1000 else 100,
                          args.warmup, local, stream, world, rank)
        if rank == 0:
            res["study"] = ("32 uneven instances, pd 0.1-100 Torr cm, 1e4-4e6 electrons each, "
                            "Poisson on, one context per rank, instances shared among the "
                            "ranks by markers x steps")
            res["scaling"] = "strong" if world > 1 else None
            print(json.dumps(res), flush=True)
        return
    if args.paschen_full:
        if rank == 0:
            res = paschen_full(slpic, inputs, local, stream)
            res["study"] = ("breakdown-voltage search over a Paschen curve, batched FP32 on one "
                            "GB300, SLPIC at three speed limits and PIC")
            print(json.dumps(res), flush=True)
        return
    if args.dense:
        if rank == 0:
            res = dense_bench(slpic, inputs, args.steps if args.steps != 1000 else 20,
                              args.warmup, local, stream)
            res["study"] = ("one collision-dense instance (the batched sweep's instance 26, "
                            "4e6 electrons, Poisson on)")
            print(json.dumps(res), flush=True)
        return
    if args.small_pop:
        if rank == 0:
            res = small_pop(slpic, inputs, args.small_pop_steps, local, stream)
            res["study"] = ("the paper's breakdown run at 1 Torr cm, 219 cells, 100 electrons at "
                            "rest: single-CTA path against the batched kernels")
            print(json.dumps(res), flush=True)
        return
    if args.tab_sims is not None:
        if rank == 0:
            rows = (range(len(TAB_SIMS)) if args.tab_sims == "all"
                    else [int(x) for x in args.tab_sims.split(",")])
            res = tab_sims(slpic, inputs, rows, args.tab_sims_pic_max,
                           args.tab_sims_pic_full_max, local, stream,
                           slpic_full_max=args.tab_sims_slpic_full_max)
            res.update({"study": "Table tab:sims, PIC vs SLPIC on one GB300",
                        "setup": "d = 1 cm, 100 electrons at rest, E = V/d imposed, five "
                                 "processes, Eq. sey yield, 30 ion crossings in 15 windows; "
                                 "runs at 0.97 x the lower and 1.03 x the upper end of the "
                                 "synthetic gas's breakdown bracket"})
            print(json.dumps(res), flush=True)
        return
    spec, run = inputs.microbench_config(n_markers=args.markers, seed=rank)
    spec["instance"] = 0
    n = args.markers
    cap_e = 4 * n  # the avalanche grows the electrons over 1000 steps
    cap_i = 3 * n

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- device-resident run ------------------------------------------
    sim = slpic.Simulation(1, device=local, stream=stream)
    sim.configure(0, spec, capacity=(cap_e, cap_i))
    sim.seed(0, slpic.ELECTRON, n, slpic.SEED_GAP, e_lo=run["e_lo"], e_hi=run["e_hi"])
    shape = sim.launch_shape()
    if not args.no_autotune:
        # real steps of the run, before the warm-up and the timed region
        shape = sim.autotune(steps_each=16)
    sim.step(args.warmup)
    sim.synchronize()
    sim.set_profiling(True)
    t_before = sim.tallies(0)
    ms_before = int(t_before["marker_steps"])
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    with ClockSampler(local) as clk:
        ev0.record(stream)
        sim.step(args.steps)
        launches += sim.launch_count()
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    sim.synchronize()
    elapsed_ms = ev0.elapsed_time(ev1)
    push_ms, push_launches = sim.profile()
    t_after = sim.tallies(0)
    marker_steps = int(t_after["marker_steps"]) - ms_before
    t_max, total = combine_ranks(elapsed_ms, marker_steps, world, "cuda")
    value = total / t_max
    avg_push_s = push_ms / 1e3 / max(1, push_launches)
    markers_per_launch = marker_steps / max(1, push_launches)
    achieved = BYTES_PER_MARKER_STEP * markers_per_launch / avg_push_s / 1e9
    peak, peak_kind = peaks()
    tr = push_traffic()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_kind,
            "traffic": (tr * markers_per_launch if tr is not None else None),
            "kernel": "k_push", "push_share_of_step": push_ms / elapsed_ms if elapsed_ms else None}
    state_bytes = 28 * n
    sim.set_profiling(False)
    sim.close()
    del sim

    # ---- the same workload on the FP64 marker path (fewer steps) ----------
    fp64 = None
    if not args.no_fp64:
        k64 = max(10, args.steps // 10)
        sim = slpic.Simulation(1, device=local, stream=stream, precision=64)
        sim.configure(0, spec, capacity=(cap_e, cap_i))
        sim.seed(0, slpic.ELECTRON, n, slpic.SEED_GAP, e_lo=run["e_lo"], e_hi=run["e_hi"])
        sim.step(args.warmup)
        sim.synchronize()
        sim.set_profiling(True)
        ms0 = int(sim.tallies(0)["marker_steps"])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(k64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = int(sim.tallies(0)["marker_steps"]) - ms0
        p_ms, p_n = sim.profile()
        t64 = e0.elapsed_time(e1) / 1e3
        ach64 = BYTES_PER_MARKER_STEP_FP64 * (ms64 / max(1, p_n)) / (p_ms / 1e3 / max(1, p_n)) / 1e9
        fp64 = {"value": ms64 / t64, "unit": "marker-steps/s", "steps": k64,
                "ms_per_step": t64 * 1e3 / k64, "dtype": "f64",
                "roofline": {"bound": "hbm", "achieved": ach64, "peak": peak, "unit": "GB/s",
                             "frac": ach64 / peak, "bytes_per_marker_step": BYTES_PER_MARKER_STEP_FP64,
                             "kernel": "k_push<double>"},
                "note": "same workload and seeds on the FP64 marker path; profiled steps "
                        "without graph replay"}
        sim.set_profiling(False)
        sim.close()
        del sim

    # ---- end to end through the C ABI with host buffers -----------------
    e2e = None
    if not args.no_e2e:
        host = inputs.gap_state(n, spec, rng_seed=100 + rank, e_lo=run["e_lo"], e_hi=run["e_hi"])
        pinned = {}
        for k, a in host.items():
            t = torch.empty(a.shape, dtype={np.int32: torch.int32, np.float32: torch.float32,
                                            np.uint32: torch.int32}[a.dtype.type],
                            pin_memory=True)
            t.numpy().view(a.dtype)[:] = a
            pinned[k] = t.numpy().view(a.dtype)
        del host
        sim = slpic.Simulation(1, device=local, stream=stream)
        sim.configure(0, spec, capacity=(cap_e, cap_i))
        sim.load(0, slpic.ELECTRON, pinned)   # build and warm the context
        sim.set_launch_shape(*shape)
        sim.step(args.warmup)
        sim.synchronize()
        dens = np.empty(spec["n_cells"] + 1)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.reset_counters(0)
        # the serial numbers are 0 .. n - 1: the next one is passed, as a
        # caller who knows its markers does (else the binding scans the ids)
        sim.load(0, slpic.ELECTRON, pinned, next_id=n)
        sim.load(0, slpic.ION, {k: v[:0] for k, v in pinned.items()}, next_id=0)
        sim.step(args.steps)
        hist = sim.history(0, capacity=args.steps)
        dens = sim.density(0, slpic.ELECTRON)
        t1 = time.perf_counter()
        barrier()
        ms_e2e = int(hist["marker_steps"].sum())
        d2h = hist.nbytes + dens.nbytes
        e2e = {"value": ms_e2e / (t1 - t0), "unit": "marker-steps/s",
               "h2d_bytes_per_step": state_bytes / args.steps,
               "d2h_bytes_per_step": d2h / args.steps,
               "note": "host SoA in pinned memory loaded through slpic_load_particles, "
                       "K steps, per-step tallies and density read back"}
        sim.close()

    sweep = None
    if not args.no_paschen and rank == 0:
        sweep = paschen_sweep(slpic, inputs, local, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(spec, n, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": "marker-steps/s", "value": value, "unit": "marker-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "push+MCC microbenchmark gap: 3.2e7 electrons log-uniform "
                                   "0.1-200 eV, 4096 cells, 1 Torr, 300 V, Poisson on",
                       "markers": n, "cells": spec["n_cells"], "instances_per_gpu": 1,
                       "live_at_end": [int(x) for x in t_after["n_live"]],
                       "launch_shape": {"push_warps_per_cta": shape[0],
                                        "collide_ctas_per_sm": shape[1],
                                        "autotuned": not args.no_autotune},
                       "parallelism": "independent instance per GPU" if world > 1 else "1 GPU",
                       "l2": "inputs larger than L2 (%.2f GB of markers > %.0f MB)"
                             % (state_bytes / 1e9, L2_BYTES / 2**20)},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "variants": {"fp64": fp64},
            "paschen_sweep": sweep,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.cpu_config1:
        print(json.dumps(cpu_config1()), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
