"""ctypes binding of libnb (include/nb.h): argument marshalling only.

Every step of the method runs inside libnb.so's CUDA kernels; this module
converts numpy arrays (host) or torch tensors (device pointers) into the C
ABI's plain pointers and raises NBError on a negative return code.  There is
no CPU fallback: if libnb.so is missing or cannot be loaded, `lib()` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnb.so")

NB_OK = 0
NB_ERR_ARG = -1
NB_ERR_CUDA = -2
NB_ERR_NOT_SYNC = -3
NB_ERR_DT_UNDERFLOW = -4
NB_ERR_TIMEOUT = -5
NB_ERR_NAN = -6
NB_ERR_NOMEM = -7
NB_FP64 = 0
NB_MIXED = 1

# Every function the header declares, with its C signature.
_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
SIGNATURES = {
    "nb_set_allocator": (C.c_int, [ALLOC_FN, FREE_FN, _P]),
    "nb_create": (C.c_int, [C.POINTER(_P), C.c_int64, C.c_int, C.c_double]),
    "nb_destroy": (None, [_P]),
    "nb_last_error": (C.c_char_p, [_P]),
    "nb_set_stream": (C.c_int, [_P, _P]),
    "nb_set_precision": (C.c_int, [_P, C.c_int]),
    "nb_set_softening": (C.c_int, [_P, _D]),
    "nb_set_params": (C.c_int, [_P, C.c_double, C.c_double, C.c_double, C.c_double]),
    "nb_set_particles": (C.c_int, [_P, _D, _D, _D]),
    "nb_next_block": (C.c_int, [_P, _D, _I32, _I64]),
    "nb_predict": (C.c_int, [_P, C.c_double]),
    "nb_force": (C.c_int, [_P, _P, C.c_int64]),
    "nb_correct": (C.c_int, [_P]),
    "nb_block_step": (C.c_int, [_P, _D, _I64]),
    "nb_step_until": (C.c_int, [_P, C.c_double, _I64, _I64]),
    "nb_energy": (C.c_int, [_P, _D, _D]),
    "nb_get_state": (C.c_int, [_P, _D, _D, _D, _D, _D]),
    "nb_set_state": (C.c_int, [_P, _D, _D, _D, _D, _D]),
    "nb_get_force": (C.c_int, [_P, _D, _D, _D, _D, _D]),
    "nb_get_predicted": (C.c_int, [_P, _D, _D, _D, _D]),
    "nb_get_launch": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "nb_get_pair_warps": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "nb_set_jsplit": (C.c_int, [_P, C.c_int]),
    "nb_set_jrange": (C.c_int, [_P, C.c_int64, C.c_int64]),
    "nb_copy_force": (C.c_int, [_P, _P, _I64, _I64]),
    "nb_reduce_force": (C.c_int, [_P, _P, C.c_int]),
    "nb_version": (C.c_char_p, []),
    "nb_set_block_step": (C.c_int, [_P, C.c_double]),
    "nb_set_profiling": (C.c_int, [_P, C.c_int]),
    "nb_get_profile": (C.c_int, [_P, _D, _I64, _I64]),
    "nb_get_nact_histogram": (C.c_int, [_P, _I64, C.c_int]),
    "nb_set_noise_floor": (C.c_int, [_P, C.c_int, _D]),
    "nb_get_noise_floor": (C.c_int, [_P, C.c_int, _D]),
    "nb_force_static": (C.c_int, [C.c_int, C.c_int, C.c_int64, _P, _P, _P, _P, _P, _P, _P, C.c_int64, _P, _P]),
    "nb_set_graph": (C.c_int, [_P, C.c_int]),
    "nb_fma_peak": (C.c_int, [_P, C.c_int, _D]),
    "nb_selftest_wait": (C.c_int, [_P, C.c_double]),
    "nb_selftest_convert": (C.c_int, [_P, C.c_int64, C.c_uint64, C.POINTER(C.c_int64)]),
    "nb_autotune": (C.c_int, [_P, C.c_int]),
    "nb_get_tuning": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int32), C.POINTER(C.c_int32), _D]),
    "nb_set_tuning": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "nb_batch_create": (C.c_int, [C.POINTER(_P), C.c_int, _I64, C.c_int, C.c_double]),
    "nb_batch_destroy": (None, [_P]),
    "nb_batch_last_error": (C.c_char_p, [_P]),
    "nb_batch_set_stream": (C.c_int, [_P, _P]),
    "nb_batch_set_precision": (C.c_int, [_P, C.c_int]),
    "nb_batch_set_params": (C.c_int, [_P, C.c_double, C.c_double, C.c_double, C.c_double]),
    "nb_batch_set_particles": (C.c_int, [_P, _D, _D, _D]),
    "nb_batch_cycle": (C.c_int, [_P, C.c_double, C.POINTER(C.c_int), _I64]),
    "nb_batch_step_until": (C.c_int, [_P, C.c_double, _I64, _I64]),
    "nb_batch_set_graph": (C.c_int, [_P, C.c_int]),
    "nb_batch_energy": (C.c_int, [_P, _D, _D]),
    "nb_batch_get_state": (C.c_int, [_P, _D, _D, _D, _D]),
    "nb_batch_set_waves": (C.c_int, [_P, C.c_int]),
    "nb_batch_get_waves": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "nb_batch_autotune": (C.c_int, [_P, C.c_int, C.c_int, _D]),
}
NB_STATIC_MAX_N = 16384
NB_JTILE = 128
NB_NPHASES = 6
NB_TUNE_MAX = 32
NB_NACT_CLASSES = 48
PHASES = ("sched", "predict", "force", "reduce", "correct", "other")

_lib = None


class NBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libnb error {code}: {msg}")
        self.code = code


def lib(path: str = LIB_PATH):
    """Load libnb.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"libnb.so not found at {path}; run `python -m paper_1312_1789_b300.build`")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def version() -> str:
    return lib().nb_version().decode()


def _d(a):
    return None if a is None else a.ctypes.data_as(_D)


def _vec(a, n):
    return np.ascontiguousarray(a, dtype=np.float64).reshape(n, 3)


class NBody:
    """One libnb context: n particles, Hermite order 4/6/8, softening eps.

    Host arrays are numpy float64 ([n][3] for vectors).  Device index arrays
    may be passed as torch int32 CUDA tensors.
    """

    def __init__(self, n: int, order: int = 6, eps: float = 0.0, precision: int = NB_MIXED):
        self._L = lib()
        self._h = _P()
        rc = self._L.nb_create(C.byref(self._h), int(n), int(order), float(eps))
        if rc != NB_OK:
            raise NBError(rc, self._L.nb_last_error(None).decode())
        self.n = int(n)
        self.order = int(order)
        self.precision = NB_MIXED
        self.set_precision(precision)

    # -------------------------------------------------------------- plumbing
    def _check(self, rc):
        if rc != NB_OK:
            raise NBError(rc, self._L.nb_last_error(self._h).decode())
        return rc

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            self._L.nb_destroy(self._h)
            self._h = _P()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ parameters
    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
        handle = getattr(stream, "cuda_stream", stream)
        self._check(self._L.nb_set_stream(self._h, _P(handle or 0)))

    def set_precision(self, mode: int):
        self._check(self._L.nb_set_precision(self._h, int(mode)))
        self.precision = int(mode)

    def set_softening(self, eps_i=None):
        e = None if eps_i is None else np.ascontiguousarray(eps_i, dtype=np.float64)
        self._check(self._L.nb_set_softening(self._h, _d(e)))

    def set_params(self, eta=0.2, eta_s=0.01, dt_max=1.0 / 16, dt_min=2.0 ** -40):
        self._check(self._L.nb_set_params(self._h, eta, eta_s, dt_max, dt_min))

    def set_graph(self, cycles: int):
        """cycles > 0: step_until replays a CUDA graph of that many device-driven block cycles."""
        self._check(self._L.nb_set_graph(self._h, int(cycles)))

    def autotune(self, reps: int = 3):
        """Time force launch shapes per active-set size class and use the fastest (reps <= 0: off)."""
        self._check(self._L.nb_autotune(self._h, int(reps)))

    def get_tuning(self):
        """[(class k, ni, js, ms)] of the current precision's autotuned table."""
        n = C.c_int()
        ni = np.zeros(NB_TUNE_MAX, dtype=np.int32)
        js = np.zeros(NB_TUNE_MAX, dtype=np.int32)
        ms = np.zeros(NB_TUNE_MAX)
        self._check(self._L.nb_get_tuning(self._h, C.byref(n), ni.ctypes.data_as(C.POINTER(C.c_int32)),
                                          js.ctypes.data_as(C.POINTER(C.c_int32)), _d(ms)))
        return [(k, int(ni[k]), int(js[k]), float(ms[k])) for k in range(n.value)]

    def set_tuning(self, table):
        """Install [(k, ni, js, ...)] (as get_tuning returns) for the current precision; [] drops it."""
        ni = np.array([e[1] for e in table] or [0], dtype=np.int32)
        js = np.array([e[2] for e in table] or [0], dtype=np.int32)
        self._check(self._L.nb_set_tuning(self._h, len(table), ni.ctypes.data_as(C.POINTER(C.c_int32)),
                                          js.ctypes.data_as(C.POINTER(C.c_int32))))

    def save_tuning(self, path: str):
        """Write the current precision's autotuned table as JSON, keyed by the
        store it was measured on (n, order, precision) and the device."""
        import json
        import torch
        doc = {"n": self.n, "order": self.order, "precision": "mixed" if self.precision == NB_MIXED else "fp64",
               "device": torch.cuda.get_device_name() if torch.cuda.is_available() else None,
               "classes": [{"log2_n_act": k, "ni": ni, "js": js, "ms": ms} for k, ni, js, ms in self.get_tuning()]}
        with open(path, "w") as f:
            json.dump(doc, f, indent=1)

    def load_tuning(self, path: str):
        """Install a table that save_tuning wrote for the same n, order and
        precision (ValueError otherwise)."""
        import json
        with open(path) as f:
            doc = json.load(f)
        want = {"n": self.n, "order": self.order, "precision": "mixed" if self.precision == NB_MIXED else "fp64"}
        got = {k: doc.get(k) for k in want}
        if got != want:
            raise ValueError(f"tuning table for {got}, context is {want}")
        table = [(c["log2_n_act"], int(c["ni"]), int(c["js"])) for c in doc["classes"]]
        if [t[0] for t in table] != list(range(len(table))):
            raise ValueError("tuning classes must be 0, 1, ... in order")
        self.set_tuning(table)

    def selftest_wait(self, seconds: float = 0.2) -> int:
        """Run the bounded-wait probe; returns the code (NB_ERR_TIMEOUT when it works as designed)."""
        return int(self._L.nb_selftest_wait(self._h, float(seconds)))

    def selftest_convert(self, n: int = 1 << 24, seed: int = 1) -> int:
        """Mismatching bits between the integer f64 <-> f32 conversions and the hardware's cvt over n inputs."""
        m = C.c_int64()
        self._check(self._L.nb_selftest_convert(self._h, int(n), int(seed), C.byref(m)))
        return m.value

    def fma_peak(self, fp64: bool = False) -> float:
        """Measured FMA throughput of this GPU in TFLOP/s (FP32, or FP64 when fp64)."""
        t = C.c_double()
        self._check(self._L.nb_fma_peak(self._h, 1 if fp64 else 0, C.byref(t)))
        return t.value

    def set_jsplit(self, js: int):
        self._check(self._L.nb_set_jsplit(self._h, int(js)))

    # ------------------------------------------- j decomposition across ranks
    def set_jrange(self, j_begin: int, j_end: int):
        self._check(self._L.nb_set_jrange(self._h, int(j_begin), int(j_end)))

    def copy_force(self, dst):
        """Copy the last force result into dst (a CUDA float64 tensor or a numpy
        array of ncomp x n_act); returns (ncomp, n_act).  Ordered on the
        context's stream."""
        nc, na = C.c_int64(), C.c_int64()
        ptr = dst.data_ptr() if hasattr(dst, "data_ptr") else np.ascontiguousarray(dst).ctypes.data
        self._check(self._L.nb_copy_force(self._h, _P(ptr), C.byref(nc), C.byref(na)))
        return nc.value, na.value

    def reduce_force(self, parts, n_parts: int):
        """parts: CUDA float64 tensor [n_parts][ncomp][n_act] of force results."""
        self._check(self._L.nb_reduce_force(self._h, _P(parts.data_ptr()), int(n_parts)))

    # ------------------------------------------------------------- the method
    def set_particles(self, m, x, v):
        m = np.ascontiguousarray(m, dtype=np.float64)
        self._check(self._L.nb_set_particles(self._h, _d(m), _d(_vec(x, self.n)), _d(_vec(v, self.n))))

    def next_block(self, want_idx: bool = False):
        tb = C.c_double()
        na = C.c_int64()
        idx = np.zeros(self.n, dtype=np.int32) if want_idx else None
        self._check(self._L.nb_next_block(self._h, C.byref(tb), None if idx is None else idx.ctypes.data_as(_I32),
                                          C.byref(na)))
        if want_idx:
            return tb.value, idx[: na.value].copy()
        return tb.value, na.value

    def predict(self, t: float):
        self._check(self._L.nb_predict(self._h, float(t)))

    def force(self, idx=None, n_act: int = 0):
        """idx: None (scheduler's list), a numpy int array, or a CUDA int32 tensor."""
        if idx is None:
            self._check(self._L.nb_force(self._h, None, int(n_act)))
            return
        if hasattr(idx, "data_ptr"):
            self._check(self._L.nb_force(self._h, _P(idx.data_ptr()), int(idx.numel())))
            return
        a = np.ascontiguousarray(idx, dtype=np.int32)
        self._check(self._L.nb_force(self._h, a.ctypes.data_as(_P), int(a.shape[0])))

    def correct(self):
        self._check(self._L.nb_correct(self._h))

    def block_step(self):
        tb = C.c_double()
        na = C.c_int64()
        self._check(self._L.nb_block_step(self._h, C.byref(tb), C.byref(na)))
        return tb.value, na.value

    def step_until(self, t_end: float):
        nb_ = C.c_int64()
        ni = C.c_int64()
        self._check(self._L.nb_step_until(self._h, float(t_end), C.byref(nb_), C.byref(ni)))
        return nb_.value, ni.value

    def energy(self):
        ek = C.c_double()
        ep = C.c_double()
        self._check(self._L.nb_energy(self._h, C.byref(ek), C.byref(ep)))
        return ek.value, ep.value

    # --------------------------------------------------------- state exchange
    def get_state(self, out=None):
        """State as {x, v, d, t, dt}; out: such a dict of C-contiguous float64 arrays to fill instead."""
        n = self.n
        if out is None:
            out = {"x": np.zeros((n, 3)), "v": np.zeros((n, 3)), "d": np.zeros((n, 6, 3)), "t": np.zeros(n),
                   "dt": np.zeros(n)}
        for k, shape in (("x", (n, 3)), ("v", (n, 3)), ("d", (n, 6, 3)), ("t", (n,)), ("dt", (n,))):
            a = out[k]
            if a.dtype != np.float64 or a.shape != shape or not a.flags["C_CONTIGUOUS"]:
                raise ValueError(f"out[{k!r}] must be a C-contiguous float64 array of shape {shape}")
        self._check(self._L.nb_get_state(self._h, _d(out["x"]), _d(out["v"]), _d(out["d"]), _d(out["t"]),
                                         _d(out["dt"])))
        return out

    def set_state(self, x, v, d, t, dt):
        n = self.n
        self._check(self._L.nb_set_state(self._h, _d(_vec(x, n)), _d(_vec(v, n)),
                                         _d(np.ascontiguousarray(d, dtype=np.float64).reshape(n, 6, 3)),
                                         _d(np.ascontiguousarray(t, dtype=np.float64)),
                                         _d(np.ascontiguousarray(dt, dtype=np.float64))))

    def get_force(self, n_act: int):
        out = {k: np.zeros((n_act, 3)) for k in ("acc", "jerk", "snap", "crackle")}
        out["pot"] = np.zeros(n_act)
        self._check(self._L.nb_get_force(self._h, _d(out["acc"]), _d(out["jerk"]), _d(out["snap"]),
                                         _d(out["crackle"]), _d(out["pot"])))
        return out

    def get_predicted(self):
        n = self.n
        xp, vp, ap, jp = (np.zeros((n, 3)) for _ in range(4))
        self._check(self._L.nb_get_predicted(self._h, _d(xp), _d(vp), _d(ap), _d(jp)))
        return xp, vp, ap, jp

    def set_block_step(self, dt: float):
        self._check(self._L.nb_set_block_step(self._h, float(dt)))

    def set_noise_floor(self, precision: int, eps):
        e = np.ascontiguousarray(eps, dtype=np.float64).reshape(4)
        self._check(self._L.nb_set_noise_floor(self._h, int(precision), _d(e)))

    def get_noise_floor(self, precision: int):
        e = np.zeros(4)
        self._check(self._L.nb_get_noise_floor(self._h, int(precision), _d(e)))
        return e

    def set_profiling(self, enable: bool):
        self._check(self._L.nb_set_profiling(self._h, 1 if enable else 0))

    def get_profile(self):
        """{phase: (ms, launches)} since profiling was enabled, and total launches."""
        ms = np.zeros(NB_NPHASES)
        nl = np.zeros(NB_NPHASES, dtype=np.int64)
        tot = C.c_int64()
        self._check(self._L.nb_get_profile(self._h, _d(ms), nl.ctypes.data_as(_I64), C.byref(tot)))
        return {p: (float(ms[k]), int(nl[k])) for k, p in enumerate(PHASES)}, tot.value

    def get_nact_histogram(self, reset: bool = False):
        """Corrector passes by active-set size class: counts[k] for 2^k .. 2^(k+1) - 1 particles."""
        h = np.zeros(NB_NACT_CLASSES, dtype=np.int64)
        self._check(self._L.nb_get_nact_histogram(self._h, h.ctypes.data_as(_I64), 1 if reset else 0))
        return h

    def get_pair_warps(self) -> int:
        """Warps of the mixed force that took the per-pair softening form since the last call."""
        n = C.c_int64()
        self._check(self._L.nb_get_pair_warps(self._h, C.byref(n)))
        return n.value

    def get_launch(self):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        self._check(self._L.nb_get_launch(self._h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value


class Batch:
    """An ensemble of independent clusters advanced together (nb_batch_*)."""

    def __init__(self, sizes, order: int = 6, eps: float = 0.0, precision: int = NB_MIXED):
        self._L = lib()
        self._h = _P()
        self.sizes = np.ascontiguousarray(sizes, dtype=np.int64)
        rc = self._L.nb_batch_create(C.byref(self._h), len(self.sizes), self.sizes.ctypes.data_as(_I64), int(order),
                                     float(eps))
        if rc != NB_OK:
            raise NBError(rc, "nb_batch_create failed")
        self.n = int(self.sizes.sum())
        self.k = len(self.sizes)
        self._check(self._L.nb_batch_set_precision(self._h, int(precision)))

    def _check(self, rc):
        if rc != NB_OK:
            raise NBError(rc, self._L.nb_batch_last_error(self._h).decode())

    def close(self):
        if self._h:
            self._L.nb_batch_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        handle = getattr(stream, "cuda_stream", stream)
        self._check(self._L.nb_batch_set_stream(self._h, _P(handle or 0)))

    def set_precision(self, mode: int):
        self._check(self._L.nb_batch_set_precision(self._h, int(mode)))

    def set_params(self, eta=0.2, eta_s=0.01, dt_max=1.0 / 16, dt_min=2.0 ** -40):
        self._check(self._L.nb_batch_set_params(self._h, eta, eta_s, dt_max, dt_min))

    def set_particles(self, m, x, v):
        m = np.ascontiguousarray(m, dtype=np.float64)
        self._check(self._L.nb_batch_set_particles(self._h, _d(m), _d(_vec(x, self.n)), _d(_vec(v, self.n))))

    def set_graph(self, cycles: int):
        """cycles > 0: step_until replays a CUDA graph of that many ensemble cycles."""
        self._check(self._L.nb_batch_set_graph(self._h, int(cycles)))

    def cycle(self, t_end: float):
        k = C.c_int()
        ni = C.c_int64()
        self._check(self._L.nb_batch_cycle(self._h, float(t_end), C.byref(k), C.byref(ni)))
        return k.value, ni.value

    def step_until(self, t_end: float):
        nc = C.c_int64()
        ni = C.c_int64()
        self._check(self._L.nb_batch_step_until(self._h, float(t_end), C.byref(nc), C.byref(ni)))
        return nc.value, ni.value

    def set_waves(self, waves: int):
        self._check(self._L.nb_batch_set_waves(self._h, int(waves)))

    def get_waves(self) -> int:
        w = C.c_int()
        self._check(self._L.nb_batch_get_waves(self._h, C.byref(w)))
        return w.value

    def autotune(self, cycles: int = 32, reps: int = 2):
        """Time the force plan with 1, 2, 4, 8 waves on the next `cycles` cycles
        (which the state advances by) and keep the fastest; returns the chosen
        wave count and the total ms of each candidate."""
        ms = np.zeros(4)
        self._check(self._L.nb_batch_autotune(self._h, int(cycles), int(reps), _d(ms)))
        return self.get_waves(), dict(zip((1, 2, 4, 8), ms.tolist()))

    def energy(self):
        ek, ep = np.zeros(self.k), np.zeros(self.k)
        self._check(self._L.nb_batch_energy(self._h, _d(ek), _d(ep)))
        return ek, ep

    def get_state(self):
        x, v = np.zeros((self.n, 3)), np.zeros((self.n, 3))
        t, dt = np.zeros(self.n), np.zeros(self.n)
        self._check(self._L.nb_batch_get_state(self._h, _d(x), _d(v), _d(t), _d(dt)))
        return {"x": x, "v": v, "t": t, "dt": dt}


class TorchAllocator:
    """Routes libnb's device allocations through torch's caching allocator.

    Keep the instance alive while contexts created under it exist.
    """

    def __init__(self, device=None):
        import torch
        self._torch = torch
        self._device = torch.cuda.current_device() if device is None else device
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)

    def _do_alloc(self, nbytes, _user):
        try:
            return int(self._torch.cuda.caching_allocator_alloc(int(nbytes), self._device))
        except Exception:
            return None

    def _do_free(self, ptr, _user):
        self._torch.cuda.caching_allocator_delete(ptr)

    def install(self):
        rc = lib().nb_set_allocator(self._alloc, self._free, None)
        if rc != NB_OK:
            raise NBError(rc, lib().nb_last_error(None).decode())
        return self

    @staticmethod
    def uninstall():
        lib().nb_set_allocator(ALLOC_FN(), FREE_FN(), None)
