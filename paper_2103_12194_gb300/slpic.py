"""Thin Python binding of libslpic (include/slpic.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts numpy
arrays and PyTorch streams/tensors to the pointers the C ABI takes.  It fails
loudly when the library has not been built (there is no CPU fallback).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libslpic.so")

OK = 0
ERR_INVALID_ARG, ERR_STATE, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_NUMERIC = -1, -2, -3, -4, -5, -6
ELECTRON, ION = 0, 1
FIELD_FROZEN, FIELD_POISSON = 0, 1
EMISSION_CONSTANT, EMISSION_ENERGY = 0, 1
PHILOX_STATIC_MAX = 32768  # SLPIC_PHILOX_STATIC_MAX
SEED_CATHODE, SEED_REST, SEED_GAP, SEED_THERMAL = 0, 1, 2, 3

_ERRNAMES = {ERR_INVALID_ARG: "INVALID_ARG", ERR_STATE: "STATE", ERR_CAPACITY: "CAPACITY",
             ERR_CUDA: "CUDA", ERR_TIMEOUT: "TIMEOUT", ERR_NUMERIC: "NUMERIC"}


class SlpicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_ERRNAMES.get(code, "?"), code, msg))
        self.code = code


class PaschenSpec(ctypes.Structure):
    _fields_ = [("n_pd", ctypes.c_int), ("n_v", ctypes.c_int), ("rounds", ctypes.c_int),
                ("n_seed", ctypes.c_int64), ("e0", ctypes.c_double),
                ("vlim_factor", ctypes.c_double), ("chunk_steps", ctypes.c_int64),
                ("max_steps", ctypes.c_int64), ("V_lo", ctypes.c_void_p),
                ("V_hi", ctypes.c_void_p)]


class SoA(ctypes.Structure):
    _fields_ = [("cell", ctypes.c_void_p), ("off", ctypes.c_void_p), ("vx", ctypes.c_void_p),
                ("vy", ctypes.c_void_p), ("vz", ctypes.c_void_p), ("wj", ctypes.c_void_p),
                ("id", ctypes.c_void_p)]


TALLY_DTYPE = np.dtype([
    ("step", np.int64), ("n_live", np.int64, (2,)), ("w_live", np.float64, (2,)),
    ("n_coll", np.int64, (3,)), ("n_candidates", np.int64), ("n_abs", np.int64, (2, 2)),
    ("w_abs", np.float64, (2, 2)), ("n_see", np.int64), ("w_see", np.float64),
    ("w_ionz", np.float64), ("w_cath_ion", np.float64), ("w_cath_ion_gen0", np.float64),
    ("n_clamp", np.int64), ("n_majorant", np.int64), ("marker_steps", np.int64),
    ("w_gain_gen0", np.float64),
])

FIELDS = ("cell", "off", "vx", "vy", "vz", "wj", "id")
DTYPES = {"cell": np.int32, "id": np.uint32}

_lib = None


def lib():
    """Load libslpic.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libslpic.so is not built (run python -m paper_2103_12194_gb300.build "
                          "or __graft_entry__.build()); there is no fallback")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, f64, u64, u32 = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                   ctypes.c_uint64, ctypes.c_uint32)
    sig = {
        "slpic_version": ([], i32),
        "slpic_last_error": ([vp], ctypes.c_char_p),
        "slpic_create": ([ctypes.POINTER(vp), i32, i32], i32),
        "slpic_destroy": ([vp], i32),
        "slpic_set_stream": ([vp, vp], i32),
        "slpic_set_gap": ([vp, i32, f64, i32, f64, i32, f64], i32),
        "slpic_set_voltage": ([vp, i32, f64], i32),
        "slpic_set_gas": ([vp, i32, f64, f64], i32),
        "slpic_set_cross_sections": ([vp, i32, i32, i32, i32, vp, vp, f64, vp, f64], i32),
        "slpic_set_species": ([vp, i32, i32, f64, f64, f64, i64], i32),
        "slpic_set_emission": ([vp, i32, f64], i32),
        "slpic_set_dt": ([vp, i32, f64], i32),
        "slpic_set_seed": ([vp, i32, u64], i32),
        "slpic_set_charge_shift": ([vp, i32, i32], i32),
        "slpic_suggest_dt": ([f64, i32, f64, f64, i32, ctypes.POINTER(f64)], i32),
        "slpic_seed": ([vp, i32, i32, i64, i32, f64, f64, f64, f64], i32),
        "slpic_load_particles": ([vp, i32, i32, ctypes.POINTER(SoA), i64, u32], i32),
        "slpic_load_particles_device": ([vp, i32, i32, ctypes.POINTER(SoA), i64, u32], i32),
        "slpic_reset_counters": ([vp, i32], i32),
        "slpic_step": ([vp, i64], i32),
        "slpic_step_small": ([vp, i64, ctypes.POINTER(i64)], i32),
        "slpic_set_small_limit": ([vp, i32], i32),
        "slpic_synchronize": ([vp], i32),
        "slpic_clear_error": ([vp], i32),
        "slpic_count": ([vp, i32, i32, ctypes.POINTER(i64)], i32),
        "slpic_read_particles": ([vp, i32, i32, ctypes.POINTER(SoA), i64, ctypes.POINTER(i64)], i32),
        "slpic_read_charge": ([vp, i32, i32, vp, i64], i32),
        "slpic_read_density": ([vp, i32, i32, vp, i64], i32),
        "slpic_read_field": ([vp, i32, vp, vp, i64], i32),
        "slpic_read_tallies": ([vp, i32, vp], i32),
        "slpic_read_history": ([vp, i32, vp, i64, ctypes.POINTER(i64)], i32),
        "slpic_read_current": ([vp, i32, ctypes.POINTER(f64), ctypes.POINTER(f64)], i32),
        "slpic_read_gain": ([vp, i32, ctypes.POINTER(f64)], i32),
        "slpic_set_profiling": ([vp, i32], i32),
        "slpic_read_profile": ([vp, ctypes.POINTER(f64), ctypes.POINTER(i64)], i32),
        "slpic_launch_count": ([vp, ctypes.POINTER(i64)], i32),
        "slpic_read_wait_stats": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i64)], i32),
        "slpic_philox": ([i32, u64, vp, i64, vp], i32),
        "slpic_philox2x32": ([i32, u32, vp, i64, vp], i32),
        "slpic_philox_static": ([i32, u64, vp, i64, vp], i32),
        "slpic_paschen_bisect": ([vp, ctypes.POINTER(PaschenSpec), vp, vp, vp], i32),
        "slpic_set_precision": ([vp, i32], i32),
        "slpic_set_emission_model": ([vp, i32, i32], i32),
        "slpic_set_cross_sections_levels": ([vp, i32, i32, i32, i32, vp, i32, vp, vp, vp,
                                             f64], i32),
        "slpic_ion_trend": ([vp, i64, i32, vp, vp], i32),
        "slpic_multiplication": ([vp, i64, i32, vp, vp], i32),
        "slpic_set_spin_limit": ([vp, u32], i32),
        "slpic_save": ([vp, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)], i32),
        "slpic_load": ([vp, vp, ctypes.c_size_t], i32),
        "slpic_test_skip_barrier": ([vp, i32, i64], i32),
        "slpic_set_launch_shape": ([vp, i32, i32], i32),
        "slpic_get_launch_shape": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i32)], i32),
        "slpic_autotune": ([vp, i64, ctypes.POINTER(i32), ctypes.POINTER(i32)], i32),
        "slpic_load_particles_f64": ([vp, i32, i32, ctypes.POINTER(SoA), i64, u32], i32),
        "slpic_read_particles_f64": ([vp, i32, i32, ctypes.POINTER(SoA), i64,
                                      ctypes.POINTER(i64)], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def suggest_dt(d, n_cells, V, m_ion, mode=0):
    out = ctypes.c_double()
    rc = lib().slpic_suggest_dt(d, n_cells, V, m_ion, mode, ctypes.byref(out))
    if rc != OK:
        raise SlpicError(rc, "bad arguments")
    return out.value


def philox(ctr, seed, device=0):
    """Philox4x32-10 on the device for an (n, 4) uint32 counter array."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    rc = lib().slpic_philox(device, seed & 0xFFFFFFFFFFFFFFFF, _ptr(ctr), ctr.shape[0], _ptr(out))
    if rc != OK:
        raise SlpicError(rc, "slpic_philox failed")
    return out


def philox_static(ctr, seed, device=0):
    """slpic_philox_static: Philox4x32-10 on the device for an (n, 4) uint32
    counter array, staged in the library's fixed device scratch (no device
    allocation; n <= PHILOX_STATIC_MAX; calls on one device must not overlap)."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    L = lib()
    rc = L.slpic_philox_static(device, seed & 0xFFFFFFFFFFFFFFFF, _ptr(ctr), ctr.shape[0], _ptr(out))
    if rc != OK:
        raise SlpicError(rc, L.slpic_last_error(None).decode())
    return out


def philox2(ctr, key, device=0):
    """Philox2x32-10 on the device for an (n, 2) uint32 counter array."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 2)
    out = np.empty_like(ctr)
    rc = lib().slpic_philox2x32(device, key & 0xFFFFFFFF, _ptr(ctr), ctr.shape[0], _ptr(out))
    if rc != OK:
        raise SlpicError(rc, "slpic_philox2x32 failed")
    return out


class Simulation:
    """A context with ``n_instances`` gaps.  ``configure(i, spec)`` takes the
    mapping produced by :func:`paper_2103_12194_gb300.inputs.gap_spec`."""

    def __init__(self, n_instances=1, device=0, stream=None, precision=32):
        self._L = lib()
        h = ctypes.c_void_p()
        rc = self._L.slpic_create(ctypes.byref(h), device, n_instances)
        if rc != OK:
            raise SlpicError(rc, self._L.slpic_last_error(None).decode())
        self._h = h
        self.n_instances = n_instances
        self.device = device
        self.n_cells = [0] * n_instances
        self.precision = int(precision)
        self._real = np.float64 if self.precision == 64 else np.float32
        if self.precision != 32:
            self._ck(self._L.slpic_set_precision(self._h, self.precision))
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        if getattr(self, "_h", None):
            self._L.slpic_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, rc):
        if rc != OK:
            raise SlpicError(rc, self._L.slpic_last_error(self._h).decode())
        return rc

    # ---- configuration --------------------------------------------------
    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an int handle, or None."""
        handle = getattr(stream, "cuda_stream", stream)
        self._ck(self._L.slpic_set_stream(self._h, ctypes.c_void_p(handle or 0)))

    def configure(self, i, spec, capacity=(1 << 20, 1 << 20)):
        s = spec
        self._ck(self._L.slpic_set_gap(self._h, i, s["d"], s["n_cells"], s["V"],
                                       s.get("field_mode", 1), s.get("area", 1.0)))
        self.n_cells[i] = int(s["n_cells"])
        self._ck(self._L.slpic_set_gas(self._h, i, s["p_Pa"], s["T_K"]))
        el = np.ascontiguousarray(s["sig_el"], np.float32)
        io = np.ascontiguousarray(s["sig_io"], np.float32)
        n_exc = int(s.get("n_exc", 1))
        names = ["sig_ex"] + ["sig_ex%d" % k for k in range(2, n_exc + 1)]
        exs = [np.ascontiguousarray(s[k], np.float32) for k in names]
        ths = np.array([s["e_ex"]] + [s["e_ex%d" % k] for k in range(2, n_exc + 1)], np.float64)
        ptrs = (ctypes.c_void_p * n_exc)(*[a.ctypes.data for a in exs])
        self._ck(self._L.slpic_set_cross_sections_levels(
            self._h, i, s["tab_lo_exp2"], s["tab_log2_sub"], s["tab_octaves"], _ptr(el), n_exc,
            ctypes.cast(ptrs, ctypes.c_void_p), _ptr(ths), _ptr(io), s["e_io"]))
        self._ck(self._L.slpic_set_species(self._h, i, ELECTRON, s["mass_e"], s["charge_e"],
                                           s["vlim_e"], int(capacity[0])))
        self._ck(self._L.slpic_set_species(self._h, i, ION, s["mass_i"], s["charge_i"],
                                           s["vlim_i"], int(capacity[1])))
        self._ck(self._L.slpic_set_emission(self._h, i, s["gamma_se"]))
        self._ck(self._L.slpic_set_emission_model(self._h, i, int(s.get("emission_model", 0))))
        self._ck(self._L.slpic_set_dt(self._h, i, s["dt"]))
        self._ck(self._L.slpic_set_seed(self._h, i, int(s["seed"]) & 0xFFFFFFFFFFFFFFFF))
        self._ck(self._L.slpic_set_charge_shift(self._h, i, int(s["charge_shift"])))

    def set_voltage(self, i, V):
        self._ck(self._L.slpic_set_voltage(self._h, i, float(V)))

    def set_gas(self, i, p_Pa, T_K):
        self._ck(self._L.slpic_set_gas(self._h, i, float(p_Pa), float(T_K)))

    def set_seed(self, i, seed):
        self._ck(self._L.slpic_set_seed(self._h, i, int(seed) & 0xFFFFFFFFFFFFFFFF))

    def set_dt(self, i, dt):
        self._ck(self._L.slpic_set_dt(self._h, i, float(dt)))

    def set_emission(self, i, gamma):
        self._ck(self._L.slpic_set_emission(self._h, i, float(gamma)))

    def set_emission_model(self, i, model):
        """EMISSION_CONSTANT or EMISSION_ENERGY (Eq. sey)."""
        self._ck(self._L.slpic_set_emission_model(self._h, i, int(model)))

    # ---- markers --------------------------------------------------------
    def seed(self, i, species, n, mode, e0=1.0, e_lo=0.1, e_hi=200.0, wj=1.0):
        self._ck(self._L.slpic_seed(self._h, i, species, int(n), int(mode), float(e0),
                                    float(e_lo), float(e_hi), float(wj)))

    def load(self, i, species, state, next_id=None):
        """Load the markers of one species from host arrays (the seven fields;
        pinned memory copies fastest).  next_id is the next serial number the
        instance hands out; left out, it is formed from the ids here, one pass
        over them on the host."""
        n = len(state["cell"])
        arrs = {k: np.ascontiguousarray(state[k], dtype=DTYPES.get(k, self._real))
                for k in FIELDS}
        if next_id is None:
            next_id = int((arrs["id"] & 0x7FFFFFFF).max()) + 1 if n else 0
        soa = SoA(*[arrs[k].ctypes.data for k in FIELDS])
        fn = (self._L.slpic_load_particles_f64 if self.precision == 64
              else self._L.slpic_load_particles)
        self._ck(fn(self._h, i, species, ctypes.byref(soa), n, int(next_id)))

    def load_device(self, i, species, tensors, next_id):
        """tensors: mapping of the seven fields to CUDA tensors (contiguous)."""
        n = int(tensors["cell"].numel())
        soa = SoA(*[int(tensors[k].data_ptr()) for k in FIELDS])
        self._ck(self._L.slpic_load_particles_device(self._h, i, species, ctypes.byref(soa), n,
                                                     int(next_id)))

    def count(self, i, species):
        n = ctypes.c_int64()
        self._ck(self._L.slpic_count(self._h, i, species, ctypes.byref(n)))
        return n.value

    def particles(self, i, species):
        n = self.count(i, species)
        out = {k: np.empty(n, dtype=DTYPES.get(k, self._real)) for k in FIELDS}
        soa = SoA(*[out[k].ctypes.data for k in FIELDS])
        got = ctypes.c_int64()
        fn = (self._L.slpic_read_particles_f64 if self.precision == 64
              else self._L.slpic_read_particles)
        self._ck(fn(self._h, i, species, ctypes.byref(soa), n, ctypes.byref(got)))
        return out

    # ---- stepping -------------------------------------------------------
    def step(self, n=1):
        self._ck(self._L.slpic_step(self._h, int(n)))

    def step_small(self, n):
        """slpic_step_small: up to n steps in the single-CTA path; returns the
        steps run (synchronous)."""
        done = ctypes.c_int64(0)
        self._ck(self._L.slpic_step_small(self._h, int(n), ctypes.byref(done)))
        return int(done.value)

    def step_auto(self, n):
        """n steps: the single-CTA path while the populations are small, the
        batched kernels otherwise (synchronous when the small path runs)."""
        left = int(n)
        while left > 0:
            k = self.step_small(left)
            left -= k
            if left > 0 and k == 0:
                k = min(left, 256)
                self.step(k)
                left -= k

    def set_small_limit(self, max_tiles):
        self._ck(self._L.slpic_set_small_limit(self._h, int(max_tiles)))

    def synchronize(self):
        return self._ck(self._L.slpic_synchronize(self._h))

    def clear_error(self):
        self._ck(self._L.slpic_clear_error(self._h))

    def reset_counters(self, i):
        self._ck(self._L.slpic_reset_counters(self._h, i))

    # ---- reads ----------------------------------------------------------
    def charge(self, i, species):
        out = np.empty(self.n_cells[i] + 1, np.int64)
        self._ck(self._L.slpic_read_charge(self._h, i, species, _ptr(out), out.size))
        return out

    def density(self, i, species):
        out = np.empty(self.n_cells[i] + 1, np.float64)
        self._ck(self._L.slpic_read_density(self._h, i, species, _ptr(out), out.size))
        return out

    def field(self, i):
        phi = np.empty(self.n_cells[i] + 1, np.float64)
        E = np.empty(self.n_cells[i] + 1, np.float64)
        self._ck(self._L.slpic_read_field(self._h, i, _ptr(phi), _ptr(E), phi.size))
        return phi, E

    def tallies(self, i):
        out = np.zeros(1, TALLY_DTYPE)
        self._ck(self._L.slpic_read_tallies(self._h, i, _ptr(out)))
        return out[0]

    def history(self, i, capacity=4096):
        out = np.zeros(capacity, TALLY_DTYPE)
        n = ctypes.c_int64()
        self._ck(self._L.slpic_read_history(self._h, i, _ptr(out), capacity, ctypes.byref(n)))
        return out[: n.value]

    def current(self, i):
        a, c = ctypes.c_double(), ctypes.c_double()
        self._ck(self._L.slpic_read_current(self._h, i, ctypes.byref(a), ctypes.byref(c)))
        return a.value, c.value

    def gain(self, i):
        g = ctypes.c_double()
        self._ck(self._L.slpic_read_gain(self._h, i, ctypes.byref(g)))
        return g.value

    def paschen_bisect(self, V_lo, V_hi, n_v, rounds, n_seed, e0=1.0, vlim_factor=4.0,
                       chunk_steps=256, max_steps=1_000_000):
        """slpic_paschen_bisect over the context's len(V_lo) * n_v instances;
        returns (Vb_lo, Vb_hi, gain[n_pd, n_v] of the last round)."""
        lo = np.ascontiguousarray(V_lo, np.float64)
        hi = np.ascontiguousarray(V_hi, np.float64)
        n_pd = lo.shape[0]
        spec = PaschenSpec(n_pd, int(n_v), int(rounds), int(n_seed), float(e0),
                           float(vlim_factor), int(chunk_steps), int(max_steps),
                           lo.ctypes.data, hi.ctypes.data)
        out_lo, out_hi = np.empty(n_pd), np.empty(n_pd)
        gain = np.empty(n_pd * int(n_v))
        self._ck(self._L.slpic_paschen_bisect(self._h, ctypes.byref(spec), _ptr(out_lo),
                                              _ptr(out_hi), _ptr(gain)))
        return out_lo, out_hi, gain.reshape(n_pd, int(n_v))

    def ion_trend(self, steps_per_window, n_windows):
        """slpic_ion_trend: (means[n_inst, n_windows], above[n_inst])."""
        means = np.empty((self.n_instances, int(n_windows)))
        above = np.empty(self.n_instances, np.int32)
        self._ck(self._L.slpic_ion_trend(self._h, int(steps_per_window), int(n_windows),
                                         _ptr(means), _ptr(above)))
        return means, above.astype(bool)

    def multiplication(self, steps_per_window, n_windows):
        """slpic_multiplication: (see[n_inst, n_windows], M[n_inst, n_windows - 1])."""
        see = np.empty((self.n_instances, int(n_windows)))
        M = np.empty((self.n_instances, max(int(n_windows) - 1, 0)))
        self._ck(self._L.slpic_multiplication(self._h, int(steps_per_window), int(n_windows),
                                              _ptr(see), _ptr(M)))
        return see, M

    def save(self):
        """slpic_save: the context's state as bytes."""
        n = ctypes.c_size_t(0)
        self._ck(self._L.slpic_save(self._h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._ck(self._L.slpic_save(self._h, buf, n.value, ctypes.byref(n)))
        return buf.raw[:n.value]

    def restore(self, snapshot):
        """slpic_load: restore a state saved by save() into this context,
        configured as the saved one was."""
        buf = ctypes.create_string_buffer(bytes(snapshot), len(snapshot))
        self._ck(self._L.slpic_load(self._h, buf, len(snapshot)))

    def set_spin_limit(self, polls):
        self._ck(self._L.slpic_set_spin_limit(self._h, int(polls)))

    def test_skip_barrier(self, inst, barrier):
        self._ck(self._L.slpic_test_skip_barrier(self._h, int(inst), int(barrier)))

    def set_launch_shape(self, push_warps, collide_ctas_per_sm):
        self._ck(self._L.slpic_set_launch_shape(self._h, int(push_warps),
                                                int(collide_ctas_per_sm)))

    def launch_shape(self):
        w, cc = ctypes.c_int32(), ctypes.c_int32()
        self._ck(self._L.slpic_get_launch_shape(self._h, ctypes.byref(w), ctypes.byref(cc)))
        return w.value, cc.value

    def autotune(self, steps_each=32):
        """slpic_autotune: advances the simulation while timing shapes;
        returns the chosen (push warps, collision CTAs per SM)."""
        w, cc = ctypes.c_int32(), ctypes.c_int32()
        self._ck(self._L.slpic_autotune(self._h, int(steps_each), ctypes.byref(w),
                                        ctypes.byref(cc)))
        return w.value, cc.value

    def set_profiling(self, on):
        self._ck(self._L.slpic_set_profiling(self._h, 1 if on else 0))

    def profile(self):
        ms, n = ctypes.c_double(), ctypes.c_int64()
        self._ck(self._L.slpic_read_profile(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def wait_stats(self):
        w, m = ctypes.c_int64(), ctypes.c_int64()
        self._ck(self._L.slpic_read_wait_stats(self._h, ctypes.byref(w), ctypes.byref(m)))
        return w.value, m.value

    def launch_count(self):
        n = ctypes.c_int64()
        self._ck(self._L.slpic_launch_count(self._h, ctypes.byref(n)))
        return n.value
