"""The C-ABI library loads and exports every symbol that include/slpic.h
declares; host-only helpers agree with the paper's rules.  No GPU needed."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "slpic.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(slpic_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2103_12194_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("slpic_create", "slpic_destroy", "slpic_set_gap", "slpic_set_gas",
                 "slpic_set_cross_sections", "slpic_set_species", "slpic_set_emission",
                 "slpic_seed", "slpic_step", "slpic_read_density", "slpic_read_current",
                 "slpic_read_gain", "slpic_read_tallies"):
        assert must in names


def test_library_exports_every_declared_symbol(built_lib):
    missing = [n for n in declared_functions() if not hasattr(built_lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2103_12194_gb300 import slpic
    L = slpic.lib()
    for n in declared_functions():
        assert getattr(L, n).restype is not None or n == "slpic_destroy"


def test_create_without_gpu_fails_cleanly(built_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2103_12194_gb300 import slpic
    with pytest.raises(slpic.SlpicError) as e:
        slpic.Simulation(1)
    assert e.value.code == slpic.ERR_CUDA


def test_suggest_dt_follows_the_paper_rules(oracle_mod):
    from paper_2103_12194_gb300 import inputs, slpic
    for cells, V in ((66, 260.0), (219, 170.0), (65494, 3100.0)):
        a = slpic.suggest_dt(0.01, cells, V, inputs.M_AR, 0)
        b = oracle_mod.dt_slpic(0.01, cells, V, inputs.M_AR)
        assert a == pytest.approx(b, rel=1e-15)
        a = slpic.suggest_dt(0.01, cells, V, inputs.M_AR, 1)
        b = oracle_mod.dt_pic(0.01, cells, V)
        assert a == pytest.approx(b, rel=1e-15)
    with pytest.raises(slpic.SlpicError):
        slpic.suggest_dt(0.01, 0, 1.0, inputs.M_AR, 0)


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2103_12194_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert "slpic_oracle" not in src, f
