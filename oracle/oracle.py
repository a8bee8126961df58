"""ctypes wrapper around liboracle.so (see oracle.c).

TEST INFRASTRUCTURE ONLY.  Arrays are float64, row-major [n][3]; derivative
stacks are [n][6][3] = a, jerk, snap, crackle, a^(4), a^(5).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build

_lib = None

ORC_OK = 0
ORC_ERR_ARG = -1
ORC_ERR_DT_UNDERFLOW = -4
ORC_ERR_CAPACITY = -5


class OracleError(RuntimeError):
    pass


class _Params(C.Structure):
    _fields_ = [("eta", C.c_double), ("eta_s", C.c_double), ("dt_max", C.c_double),
                ("dt_min", C.c_double), ("t_end", C.c_double), ("order", C.c_int),
                ("nthreads", C.c_int), ("init", C.c_int), ("noise", C.c_double * 4)]


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        d, i64, i32 = C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_int32)
        L.orc_force.argtypes = [i64, d, d, d, d, d, d, C.c_int, i64, i32, d, d, d, d, d, d, C.c_int]
        L.orc_energy.argtypes = [i64, d, d, d, d, d, d, C.c_int]
        L.orc_predict.argtypes = [i64, C.c_int, C.c_double, d, d, d, d, d, d, d, d]
        L.orc_correct.argtypes = [C.c_int, C.c_double, d, d, d, d, d, d]
        L.orc_interp.argtypes = [C.c_int, C.c_double, d, d, d]
        L.orc_dt_criterion.argtypes = [C.c_int, C.c_double, d]
        L.orc_dt_criterion.restype = C.c_double
        L.orc_noise_floor.argtypes = [C.c_int, C.c_double, d, d, d, d]
        L.orc_dt_criterion_floored.argtypes = [C.c_int, C.c_double, C.c_double, d, d, d, C.c_double]
        L.orc_dt_criterion_floored.restype = C.c_double
        L.orc_dt_quantise.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, d]
        L.orc_dt_startup.argtypes = [C.c_double, d, d]
        L.orc_dt_startup.restype = C.c_double
        L.orc_next_block.argtypes = [i64, d, d, d, i32, C.POINTER(C.c_int64)]
        L.orc_integrate.argtypes = [i64, d, d, d, d, d, d, d, d, C.POINTER(_Params),
                                    i64, d, C.POINTER(C.c_int64), i64, i32, C.POINTER(C.c_int64)]
        L.orc_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _p(a):
    if a is None:
        return None
    if a.dtype == np.float64:
        return a.ctypes.data_as(C.POINTER(C.c_double))
    if a.dtype == np.int32:
        return a.ctypes.data_as(C.POINTER(C.c_int32))
    if a.dtype == np.int64:
        return a.ctypes.data_as(C.POINTER(C.c_int64))
    raise TypeError(a.dtype)


def _check(rc, what):
    if rc != ORC_OK:
        raise OracleError(f"{what} failed with code {rc}")


def num_threads() -> int:
    return int(lib().orc_num_threads())


def force(m, eps2, x, v, a=None, jk=None, order=6, idx=None, nthreads=1):
    """Direct-sum acc, jerk, snap, crackle and potential on particles idx.

    Also returns "absum" [n_act][6]: sum over j of |A_ij|, |J_ij|, |S_ij|,
    |C_ij| and m_j/R_ij, the magnitude of the terms behind each total, and
    B = sum_j m_j/R_ij^2, the acc scale the noise-floored time step uses.
    """
    m = _f64(m)
    n = m.shape[0]
    eps2 = _f64(np.broadcast_to(eps2, (n,)))
    x = _f64(x, (n, 3))
    v = _f64(v, (n, 3))
    a = None if a is None else _f64(a, (n, 3))
    jk = None if jk is None else _f64(jk, (n, 3))
    idx = np.arange(n, dtype=np.int32) if idx is None else np.ascontiguousarray(idx, dtype=np.int32)
    na = idx.shape[0]
    out = {k: np.zeros((na, 3)) for k in ("acc", "jerk", "snap", "crackle")}
    out["pot"] = np.zeros(na)
    out["absum"] = np.zeros((na, 6))
    rc = lib().orc_force(n, _p(m), _p(eps2), _p(x), _p(v), _p(a), _p(jk), order, na, _p(idx),
                         _p(out["acc"]), _p(out["jerk"]), _p(out["snap"]), _p(out["crackle"]),
                         _p(out["pot"]), _p(out["absum"]), int(nthreads))
    _check(rc, "orc_force")
    return out


def energy(m, eps2, x, v, nthreads=1):
    """(kinetic, potential) energy with pair softening max(eps2_i, eps2_j)."""
    m = _f64(m)
    n = m.shape[0]
    eps2 = _f64(np.broadcast_to(eps2, (n,)))
    ek, ep = C.c_double(), C.c_double()
    rc = lib().orc_energy(n, _p(m), _p(eps2), _p(_f64(x, (n, 3))), _p(_f64(v, (n, 3))),
                          C.byref(ek), C.byref(ep), int(nthreads))
    _check(rc, "orc_energy")
    return ek.value, ep.value


def predict(order, t, ti, x, v, d):
    """Taylor prediction of every particle to time t; returns xp, vp, ap, jp."""
    ti = _f64(ti)
    n = ti.shape[0]
    xp, vp, ap, jp = (np.zeros((n, 3)) for _ in range(4))
    rc = lib().orc_predict(n, order, float(t), _p(ti), _p(_f64(x, (n, 3))), _p(_f64(v, (n, 3))),
                           _p(_f64(d, (n, 6, 3))), _p(xp), _p(vp), _p(ap), _p(jp))
    _check(rc, "orc_predict")
    return xp, vp, ap, jp


def correct(order, h, x0, v0, D0, D1):
    """Hermite corrector for one particle; D0, D1 = [4][3] (a, j, s, c)."""
    x1, v1 = np.zeros(3), np.zeros(3)
    rc = lib().orc_correct(order, float(h), _p(_f64(x0, (3,))), _p(_f64(v0, (3,))),
                           _p(_f64(D0, (4, 3))), _p(_f64(D1, (4, 3))), _p(x1), _p(v1))
    _check(rc, "orc_correct")
    return x1, v1


def interp(mm, h, D0, D1):
    """Derivatives mm..2mm-1 at the step end from the two-point Hermite interpolant."""
    out = np.zeros((mm, 3))
    rc = lib().orc_interp(mm, float(h), _p(_f64(D0, (mm, 3))), _p(_f64(D1, (mm, 3))), _p(out))
    _check(rc, "orc_interp")
    return out


def dt_criterion(order, eta, D):
    """Aarseth-type time step from the acc derivatives a^(0..p-1) ([p][3])."""
    return float(lib().orc_dt_criterion(order, float(eta), _p(_f64(D, (order, 3)))))


def noise_floor(mm, h, D0, D1, eps):
    """Noise floors of the interpolated derivatives mm..2mm-1 ([mm])."""
    out = np.zeros(mm)
    e = np.zeros(4)
    e[: len(eps)] = eps
    rc = lib().orc_noise_floor(mm, float(h), _p(_f64(D0, (mm, 3))), _p(_f64(D1, (mm, 3))), _p(e), _p(out))
    _check(rc, "orc_noise_floor")
    return out


def dt_criterion_floored(order, eta, h, D0, Dfull, eps, bacc=0.0):
    """Step criterion with interpolated norms net of their noise floor
    (precisions eps scaled by max(1, bacc / |a|))."""
    mm = order // 2
    e = np.zeros(4)
    e[: len(eps)] = eps
    D0 = _f64(np.asarray(D0)[:mm], (mm, 3))
    return float(lib().orc_dt_criterion_floored(order, float(eta), float(h), _p(D0),
                                                _p(_f64(Dfull, (2 * mm, 3))), _p(e), float(bacc)))


def dt_quantise(lim, t1, dt_max=1.0 / 16, dt_min=2.0 ** -40):
    """Power-of-two step <= lim commensurate with t1; raises on underflow."""
    out = C.c_double()
    rc = lib().orc_dt_quantise(float(lim), float(t1), float(dt_max), float(dt_min), C.byref(out))
    _check(rc, "orc_dt_quantise")
    return out.value


def dt_startup(eta_s, a, j):
    return float(lib().orc_dt_startup(float(eta_s), _p(_f64(a, (3,))), _p(_f64(j, (3,)))))


def next_block(t, dt):
    t = _f64(t)
    dt = _f64(dt)
    n = t.shape[0]
    idx = np.zeros(n, dtype=np.int32)
    tb = C.c_double()
    na = C.c_int64()
    rc = lib().orc_next_block(n, _p(t), _p(dt), C.byref(tb), _p(idx), C.byref(na))
    _check(rc, "orc_next_block")
    return tb.value, idx[: na.value].copy()


class State:
    """Full integrator state, all float64."""

    def __init__(self, m, eps2, x, v):
        self.m = _f64(m)
        n = self.m.shape[0]
        self.eps2 = _f64(np.broadcast_to(eps2, (n,))).copy()
        self.x = _f64(x, (n, 3)).copy()
        self.v = _f64(v, (n, 3)).copy()
        self.d = np.zeros((n, 6, 3))
        self.t = np.zeros(n)
        self.dt = np.zeros(n)
        self.pot = np.zeros(n)
        self.initialised = False

    @property
    def n(self):
        return self.m.shape[0]


def integrate(state: State, order=6, t_end=0.125, eta=0.2, eta_s=0.01, dt_max=1.0 / 16,
              dt_min=2.0 ** -40, nthreads=1, log=False, log_cap_blocks=1 << 20, log_cap_idx=1 << 26,
              noise=(0.0, 0.0, 0.0, 0.0)):
    """Advance `state` with block steps until the next block would pass t_end.

    noise: relative precision of the force components (acc, jerk, snap,
    crackle) used as the noise floor of interpolated derivatives; zeros give
    the plain criterion.  Returns the block log (list of (t_blk, idx array))
    if log, else the count.
    """
    P = _Params(eta, eta_s, dt_max, dt_min, t_end, order, int(nthreads), 0 if state.initialised else 1,
                (C.c_double * 4)(*noise))
    n = state.n
    nb = C.c_int64()
    if log:
        lt = np.zeros(log_cap_blocks)
        ln = np.zeros(log_cap_blocks, dtype=np.int64)
        li = np.zeros(log_cap_idx, dtype=np.int32)
        args = (log_cap_blocks, _p(lt), _p(ln), log_cap_idx, _p(li))
    else:
        args = (0, None, None, 0, None)
    rc = lib().orc_integrate(n, _p(state.m), _p(state.eps2), _p(state.x), _p(state.v), _p(state.d),
                             _p(state.t), _p(state.dt), _p(state.pot), C.byref(P), *args, C.byref(nb))
    _check(rc, "orc_integrate")
    state.initialised = True
    if not log:
        return nb.value
    out, off = [], 0
    for b in range(nb.value):
        k = int(ln[b])
        out.append((float(lt[b]), li[off: off + k].copy()))
        off += k
    return out


__all__ = ["OracleError", "State", "force", "energy", "predict", "correct", "interp", "dt_criterion",
           "dt_quantise", "dt_startup", "noise_floor", "dt_criterion_floored", "next_block", "integrate", "num_threads", "lib"]
