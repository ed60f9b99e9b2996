"""Python access to the CPU oracle of the SLPIC-MCC step.

TEST INFRASTRUCTURE ONLY: the tests, the package's smoke check and the CPU
baseline leg of ``bench.py`` may use this module; the product path never does.
It shares no code with the CUDA library.  Configuration arrives as a plain
mapping (the same numbers the tests hand to the library); marker state arrives
as FP32 arrays, the storage format, and is widened exactly in FP64 mode.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None


class OracleConfig(ctypes.Structure):
    _fields_ = [
        ("n_cells", ctypes.c_int),
        ("d", ctypes.c_double),
        ("V", ctypes.c_double),
        ("area", ctypes.c_double),
        ("field_mode", ctypes.c_int),
        ("p_Pa", ctypes.c_double),
        ("T_K", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("mass", ctypes.c_double * 2),
        ("charge", ctypes.c_double * 2),
        ("vlim", ctypes.c_double * 2),
        ("gamma_se", ctypes.c_double),
        ("charge_shift", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("instance", ctypes.c_uint32),
        ("tab_lo_exp2", ctypes.c_int),
        ("tab_log2_sub", ctypes.c_int),
        ("tab_octaves", ctypes.c_int),
        ("sig_el", ctypes.POINTER(ctypes.c_float)),
        ("sig_ex", ctypes.POINTER(ctypes.c_float)),
        ("sig_io", ctypes.POINTER(ctypes.c_float)),
        ("e_ex", ctypes.c_double),
        ("e_io", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("emission_model", ctypes.c_int),
        ("emit", ctypes.c_int),
        ("n_exc", ctypes.c_int),
        ("sig_ex2", ctypes.POINTER(ctypes.c_float)),
        ("sig_ex3", ctypes.POINTER(ctypes.c_float)),
        ("e_ex2", ctypes.c_double),
        ("e_ex3", ctypes.c_double),
        ("kick_scheme", ctypes.c_int),
    ]


TALLY_DTYPE = np.dtype([
    ("step", np.int64),
    ("n_live", np.int64, (2,)),
    ("w_live", np.float64, (2,)),
    ("n_coll", np.int64, (3,)),
    ("n_candidates", np.int64),
    ("n_abs", np.int64, (2, 2)),
    ("w_abs", np.float64, (2, 2)),
    ("n_see", np.int64),
    ("w_see", np.float64),
    ("w_ionz", np.float64),
    ("w_cath_ion", np.float64),
    ("w_cath_ion_gen0", np.float64),
    ("n_clamp", np.int64),
    ("n_majorant", np.int64),
    ("marker_steps", np.int64),
    ("w_gain_gen0", np.float64),
])


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        i64 = ctypes.c_int64
        L.oracle_create.restype = vp
        L.oracle_create.argtypes = [ctypes.POINTER(OracleConfig)]
        L.oracle_destroy.argtypes = [vp]
        L.oracle_load.argtypes = [vp, ctypes.c_int, i64] + [vp] * 7 + [ctypes.c_uint32]
        L.oracle_seed.argtypes = [vp, ctypes.c_int, i64, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double]
        L.oracle_step.argtypes = [vp, i64]
        L.oracle_deposit.argtypes = [vp]
        L.oracle_solve_field.argtypes = [vp]
        L.oracle_count.restype = i64
        L.oracle_count.argtypes = [vp, ctypes.c_int]
        L.oracle_next_id.restype = ctypes.c_uint32
        L.oracle_next_id.argtypes = [vp, ctypes.c_int]
        L.oracle_get.argtypes = [vp, ctypes.c_int] + [vp] * 7
        L.oracle_charge.argtypes = [vp, ctypes.c_int, vp]
        L.oracle_field.argtypes = [vp, vp, vp]
        L.oracle_set_field.argtypes = [vp, vp]
        L.oracle_history_len.restype = i64
        L.oracle_history_len.argtypes = [vp]
        L.oracle_history.argtypes = [vp, vp]
        L.oracle_constants.argtypes = [vp, vp]
        L.oracle_xsec.argtypes = [vp, vp, i64, vp]
        L.oracle_kick.argtypes = [vp, ctypes.c_int, i64, vp, vp, vp, vp, vp]
        L.oracle_philox.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32, vp]
        L.oracle_philox_many.argtypes = [vp, i64, ctypes.c_uint32, ctypes.c_uint32, vp]
        L.oracle_philox2_many.argtypes = [vp, i64, ctypes.c_uint32, vp]
        L.oracle_uniform64.restype = ctypes.c_double
        L.oracle_uniform64.argtypes = [ctypes.c_uint32]
        L.oracle_uniform32.restype = ctypes.c_float
        L.oracle_uniform32.argtypes = [ctypes.c_uint32]
        for name in ("oracle_dt_slpic",):
            getattr(L, name).restype = ctypes.c_double
            getattr(L, name).argtypes = [ctypes.c_double, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_double]
        L.oracle_dt_pic.restype = ctypes.c_double
        L.oracle_dt_pic.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_double]
        L.oracle_ion_crossing_time.restype = ctypes.c_double
        L.oracle_ion_crossing_time.argtypes = [ctypes.c_double] * 3
        _LIB = L
    return _LIB


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox(ctr, seed):
    """Philox4x32-10 blocks for an (n, 4) uint32 counter array."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    lib().oracle_philox_many(_ptr(ctr), ctr.shape[0], seed & 0xFFFFFFFF,
                             (seed >> 32) & 0xFFFFFFFF, _ptr(out))
    return out


def philox2(ctr, key):
    """Philox2x32-10 blocks for an (n, 2) uint32 counter array."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 2)
    out = np.empty_like(ctr)
    lib().oracle_philox2_many(_ptr(ctr), ctr.shape[0], key & 0xFFFFFFFF, _ptr(out))
    return out


def uniform(x, precision=64):
    x = int(x) & 0xFFFFFFFF
    return lib().oracle_uniform64(x) if precision == 64 else lib().oracle_uniform32(x)


def dt_slpic(d, cells, V, M):
    return lib().oracle_dt_slpic(d, cells, V, M)


def dt_pic(d, cells, V):
    return lib().oracle_dt_pic(d, cells, V)


def ion_crossing_time(d, V, M):
    return lib().oracle_ion_crossing_time(d, V, M)


class Oracle:
    """One instance of the oracle.  ``spec`` is a mapping with the keys of
    ``OracleConfig`` except that ``mass``, ``charge`` and ``vlim`` are given as
    ``mass_e``/``mass_i`` etc. and the cross sections as float32 arrays."""

    def __init__(self, spec, precision=64):
        self.spec = dict(spec)
        s = self.spec
        n_exc = int(s.get("n_exc", 1))
        keys = ["sig_el", "sig_ex", "sig_io"] + ["sig_ex%d" % k for k in range(2, n_exc + 1)]
        self._sig = [np.ascontiguousarray(s[k], dtype=np.float32) for k in keys]
        n_nodes = (int(s["tab_octaves"]) << int(s["tab_log2_sub"])) + 1
        for a in self._sig:
            if a.shape != (n_nodes,):
                raise ValueError("cross-section table must have %d nodes" % n_nodes)
        c = OracleConfig()
        c.n_cells = int(s["n_cells"])
        c.d = float(s["d"])
        c.V = float(s["V"])
        c.area = float(s.get("area", 1.0))
        c.field_mode = int(s.get("field_mode", 0))
        c.p_Pa = float(s["p_Pa"])
        c.T_K = float(s["T_K"])
        c.dt = float(s["dt"])
        c.mass[0], c.mass[1] = float(s["mass_e"]), float(s["mass_i"])
        c.charge[0], c.charge[1] = float(s["charge_e"]), float(s["charge_i"])
        c.vlim[0], c.vlim[1] = float(s["vlim_e"]), float(s["vlim_i"])
        c.gamma_se = float(s["gamma_se"])
        c.charge_shift = int(s["charge_shift"])
        c.seed = int(s["seed"]) & 0xFFFFFFFFFFFFFFFF
        c.instance = int(s.get("instance", 0))
        c.tab_lo_exp2 = int(s["tab_lo_exp2"])
        c.tab_log2_sub = int(s["tab_log2_sub"])
        c.tab_octaves = int(s["tab_octaves"])
        fp = ctypes.POINTER(ctypes.c_float)
        c.sig_el = self._sig[0].ctypes.data_as(fp)
        c.sig_ex = self._sig[1].ctypes.data_as(fp)
        c.sig_io = self._sig[2].ctypes.data_as(fp)
        c.e_ex = float(s["e_ex"])
        c.e_io = float(s["e_io"])
        c.precision = int(precision)
        c.emission_model = int(s.get("emission_model", 0))
        c.emit = int(s.get("emit", 1))
        c.n_exc = n_exc
        if n_exc >= 2:
            c.sig_ex2 = self._sig[3].ctypes.data_as(fp)
            c.e_ex2 = float(s["e_ex2"])
        if n_exc >= 3:
            c.sig_ex3 = self._sig[4].ctypes.data_as(fp)
            c.e_ex3 = float(s["e_ex3"])
        c.kick_scheme = int(s.get("kick_scheme", 0))
        self.precision = int(precision)
        self._cfg = c
        self._h = lib().oracle_create(ctypes.byref(c))
        if not self._h:
            raise ValueError("oracle rejected the configuration")
        self.n_cells = c.n_cells

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oracle_destroy(h)
            self._h = None

    def load(self, species, state, next_id=None):
        n = len(state["cell"])
        arrs = [np.ascontiguousarray(state["cell"], dtype=np.int32)]
        arrs += [np.ascontiguousarray(state[k], dtype=np.float32)
                 for k in ("off", "vx", "vy", "vz", "wj")]
        arrs.append(np.ascontiguousarray(state["id"], dtype=np.uint32))
        if next_id is None:
            next_id = int((arrs[-1] & 0x7FFFFFFF).max()) + 1 if n else 0
        rc = lib().oracle_load(self._h, species, n, *[_ptr(a) for a in arrs],
                               int(next_id))
        if rc != 0:
            raise ValueError("oracle_load rejected the state (rc=%d)" % rc)

    def seed(self, species, n, mode, e0=1.0, e_lo=0.1, e_hi=200.0, wj=1.0):
        rc = lib().oracle_seed(self._h, species, int(n), int(mode), float(e0),
                               float(e_lo), float(e_hi), float(wj))
        if rc != 0:
            raise ValueError("oracle_seed failed")

    def step(self, n=1):
        lib().oracle_step(self._h, int(n))

    def deposit(self):
        lib().oracle_deposit(self._h)

    def solve_field(self):
        lib().oracle_solve_field(self._h)

    def count(self, species):
        return int(lib().oracle_count(self._h, species))

    def next_id(self, species):
        return int(lib().oracle_next_id(self._h, species))

    def particles(self, species):
        n = self.count(species)
        out = {"cell": np.empty(n, np.int32)}
        for k in ("off", "vx", "vy", "vz", "wj"):
            out[k] = np.empty(n, np.float64)
        out["id"] = np.empty(n, np.uint32)
        lib().oracle_get(self._h, species, _ptr(out["cell"]), _ptr(out["off"]),
                         _ptr(out["vx"]), _ptr(out["vy"]), _ptr(out["vz"]),
                         _ptr(out["wj"]), _ptr(out["id"]))
        return out

    def charge(self, species):
        out = np.empty(self.n_cells + 1, np.int64)
        lib().oracle_charge(self._h, species, _ptr(out))
        return out

    def field(self):
        phi = np.empty(self.n_cells + 1, np.float64)
        E = np.empty(self.n_cells + 1, np.float64)
        lib().oracle_field(self._h, _ptr(phi), _ptr(E))
        return phi, E

    def set_field(self, E):
        E = np.ascontiguousarray(E, dtype=np.float64)
        lib().oracle_set_field(self._h, _ptr(E))

    def history(self):
        n = int(lib().oracle_history_len(self._h))
        out = np.zeros(n, dtype=TALLY_DTYPE)
        if n:
            lib().oracle_history(self._h, _ptr(out))
        return out

    def constants(self):
        out = np.empty(3, np.float64)
        lib().oracle_constants(self._h, _ptr(out))
        return {"P0": out[0], "vb_cap": out[1], "ndt": out[2]}

    def multiplication(self, steps_per_window, n_windows):
        """Multiplication per ion transit (Sec. V): the flux weight of the
        electrons emitted at the cathode in each of n_windows windows of
        steps_per_window steps, and the ratio of each window's to the one
        before (NaN after a window with no emission).  Steps the oracle."""
        start = len(self.history())
        self.step(int(steps_per_window) * int(n_windows))
        w = self.history()["w_see"][start:].reshape(int(n_windows), int(steps_per_window))
        see = w.sum(axis=1)
        with np.errstate(invalid="ignore", divide="ignore"):
            M = np.where(see[:-1] > 0, see[1:] / np.where(see[:-1] > 0, see[:-1], 1.0), np.nan)
        return see, M

    def kick(self, species, vx, vy, vz, A):
        """New v_x after one step's kick for arrays of velocities and
        unlimited increments A = q E_x dt / m (the oracle's kick, in its
        precision)."""
        arrs = [np.ascontiguousarray(np.broadcast_to(a, np.shape(vx)), dtype=np.float64)
                for a in (vx, vy, vz, A)]
        out = np.empty(arrs[0].size, np.float64)
        lib().oracle_kick(self._h, int(species), out.size, *[_ptr(a) for a in arrs], _ptr(out))
        return out.reshape(np.shape(vx))

    def xsec(self, eps):
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        out = np.empty((eps.size, 3), np.float64)
        lib().oracle_xsec(self._h, _ptr(eps), eps.size, _ptr(out))
        return out
