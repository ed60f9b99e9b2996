"""The measured workloads follow their stated recipes (CPU only): the
batched sweep's 32 instances and the Table tab:sims runs' time steps."""
import math

from paper_2103_12194_gb300 import inputs

import bench


def test_batched_sweep_recipe():
    items = bench.batch_specs(inputs)
    assert len(items) == 32
    pds = [spec["p_Pa"] * 1.0 / inputs.TORR for spec, _ in items]  # d = 1 cm
    assert math.isclose(pds[0], 0.1, rel_tol=1e-12) and math.isclose(pds[-1], 100.0, rel_tol=1e-12)
    assert all(b > a for a, b in zip(pds, pds[1:]))
    ns = [n for _, n in items]
    assert ns[0] == 10_000 and ns[-1] == 4_000_000
    cells = [spec["n_cells"] for spec, _ in items]
    assert min(cells) == 128 and max(cells) == 16384
    for (spec, _), pd in zip(items, pds):
        assert spec["field_mode"] == 1 and spec["gamma_se"] == 0.07
        if pd > 0.3:
            # Eq. paschen with A = 11.5, B = 176, gamma = 0.07
            v_b = 176.0 * pd / (math.log(11.5 * pd) - math.log(math.log(1.0 + 1.0 / 0.07)))
            assert math.isclose(spec["V"], v_b, rel_tol=1e-12)
        else:
            assert spec["V"] == 1000.0


def test_table_sims_time_steps():
    """SLPIC: dt = dx / v0, so 30 ion crossings (2 d / v0 each) are
    60 cells steps; PIC: dt = dx / v_max, sqrt(M / m_e) times shorter."""
    for p, V, cells in bench.TAB_SIMS:
        s = bench.tab_sims_spec(inputs, p, V, cells, False, seed=1)
        q = bench.tab_sims_spec(inputs, p, V, cells, True, seed=1)
        dx = 0.01 / cells
        assert math.isclose(s["dt"], dx / inputs.ion_speed(V), rel_tol=1e-12)
        assert math.isclose(s["vlim_e"], inputs.ion_speed(V), rel_tol=1e-12)
        assert q["vlim_e"] == math.inf
        assert math.isclose(s["dt"] / q["dt"], math.sqrt(inputs.M_AR / inputs.ME), rel_tol=1e-12)
        steps = 30 * (2 * 0.01 / inputs.ion_speed(V)) / s["dt"]
        assert math.isclose(steps, 60 * cells, rel_tol=1e-12)
        assert s["emission_model"] == 1 and s["n_exc"] == 3


def test_table_sims_rows_are_the_papers():
    """The study's rows are Table tab:sims's (p, V, cells), from the golden
    fixture transcribed from the paper."""
    import os
    import numpy as np
    path = os.path.join(os.path.dirname(__file__), "golden", "table_sims.txt")
    rows = np.loadtxt(path, comments="#", usecols=(0, 1, 2))
    assert len(rows) == len(bench.TAB_SIMS)
    for (p, V, cells), r in zip(bench.TAB_SIMS, rows):
        assert (p, V, cells) == (r[0], r[1], int(r[2]))


def test_reference_arm_prints_the_line():
    """`bench.py --impl reference` times the CPU oracle on a bounded sample of
    the benchmark workload (no GPU) and prints one JSON line with the keys a
    reader of the bench expects: the metric and value, the reference marker,
    the CPU baseline's description and an end-to-end entry with no copies."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1", "--cpu-seconds", "3"],
                         capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "marker-steps/s" and d["unit"] == "marker-steps/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]
    assert 0 < d["ms_per_step"] * d["steps"] < 600e3


def test_recorded_push_traffic_matches_the_kernel_source():
    """The bench reports the particle kernel's DRAM traffic only while the
    ncu record in profiles/push_traffic.json was taken on the kernel's
    current code (a digest of its sources without comments and whitespace).
    A change to that code needs a new capture: this fails until it is
    recorded, instead of the bench line silently losing its traffic."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "profiles", "push_traffic.json")
    with open(path) as f:
        rec = json.load(f)
    assert rec["push_source_sha256_16"] == bench.push_source_hash(), (
        "k_push's code changed since the traffic capture: rerun the ncu capture of "
        "profiles/k_push_microbench_8e6.md and update push_traffic.json")
    assert 0 < bench.push_traffic() < 48.0
