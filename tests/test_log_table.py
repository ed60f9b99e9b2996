"""The particle kernel's logarithm (Tang's table-driven method, used in the
speed-limited kick's solve of Eq. slpicEOMv) reads a table of 64 float pairs
written into the kernel source as literals.  Each entry is pinned here to
its definition: interval j of the reduced argument has centre c_j, the float
at bit pattern 0x3F350000 + 2^17 j + 2^16; r_j is 1 / c_j rounded to float
and n_j = -log(r_j) rounded to the nearest float, evaluated here with 50
digits.  The method's bound is checked on the same reading in numpy: over a
sweep of floats the result is within 3 float ulps of the exact logarithm."""
import pathlib
import re
import struct

import numpy as np
import pytest

SRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2103_12194_gb300" / "csrc" / "device_common.cuh"


def _f32(bits):
    return struct.unpack("<f", struct.pack("<I", bits))[0]


def _kernel_table():
    text = SRC.read_text()
    body = text[text.index("kLogTab[64] = {"):]
    body = body[:body.index("};")]
    pairs = re.findall(r"\{\s*([-+0-9.eE]+)f\s*,\s*([-+0-9.eE]+)f\s*\}", body)
    return np.array([[float(a), float(b)] for a, b in pairs], dtype=np.float32)


def test_table_entries_follow_their_definition():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    tab = _kernel_table()
    assert tab.shape == (64, 2)
    for j in range(64):
        c = np.float32(_f32(0x3F350000 + (j << 17) + (1 << 16)))
        r = np.float32(1.0) / c
        assert tab[j, 0] == r, j
        exact = -mp.log(mp.mpf(float(r)))
        n = np.float32(float(exact))
        # nearest float: no other float is closer to the exact value
        for cand in (np.nextafter(n, np.float32(-1)), np.nextafter(n, np.float32(1))):
            assert abs(mp.mpf(float(n)) - exact) <= abs(mp.mpf(float(cand)) - exact), j
        assert tab[j, 1] == n, j
    assert tab[37, 0] == 1.0 and tab[37, 1] == 0.0


def _tang_log(y, tab):
    """The kernel's steps in numpy float32 (fused multiply-adds taken in
    float64, which rounds them once for these operand sizes)."""
    y = np.asarray(y, np.float32)
    ix = y.view(np.int32).astype(np.int64) - 0x3F350000
    k = ix >> 23
    mb = (ix & 0x7FFFFF).astype(np.uint32)
    m = (mb + np.uint32(0x3F350000)).view(np.float32)
    j = (mb >> 17).astype(np.int64)
    r, n = tab[j, 0], tab[j, 1]

    def fma(a, b, c):
        return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)

    f = fma(m, r, np.float32(-1.0))
    q = fma(f, np.float32(-0.25), np.float32(1.0) / np.float32(3.0))
    q = fma(f, q, np.float32(-0.5))
    lp = fma(f * f, q, f)
    kf = k.astype(np.float32)
    inner = fma(kf, np.float32(1.428606765330187e-06), n + lp)
    return fma(kf, np.float32(0.693145751953125), inner)


def test_table_log_is_within_three_ulps():
    tab = _kernel_table()
    rng = np.random.default_rng(5)
    y = np.concatenate([
        np.float32(10.0) ** rng.uniform(-30, 30, 200_000).astype(np.float32),
        np.float32(1.0) + rng.uniform(-0.3, 0.4, 200_000).astype(np.float32),
        np.nextafter(np.float32(1.0), np.float32(2.0)) * np.ones(1, np.float32),
        np.nextafter(np.float32(1.0), np.float32(0.0)) * np.ones(1, np.float32),
        np.float32([1.0, 2.0, 0.5, 0.70703125, 1.4140625, 3.0e38, 1.2e-38]),
    ]).astype(np.float32)
    got = _tang_log(y, tab).astype(np.float64)
    want = np.log(y.astype(np.float64))
    ulp = np.spacing(np.abs(want).astype(np.float32)).astype(np.float64)
    err = np.abs(got - want) / np.where(want == 0.0, 1.0, ulp)
    assert err.max() <= 3.0, (err.max(), y[np.argmax(err)])
    assert _tang_log(np.float32([1.0]), tab)[0] == 0.0
