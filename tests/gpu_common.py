"""Shared helpers of the GPU parity tests: build contexts through the C ABI,
read back what the kernels consumed and produced, and compare with the oracle.

Tolerances (per particle i and derivative X; B_X = sum_j |X_ij| from the oracle):
  FP64 : |X_gpu - X_orc| <= max(1e-12 |X_orc|, 1e-14 B_X) for acc and jerk,
         <= max(1e-10 |X_orc|, 1e-13 B_X) for snap and crackle.
  mixed: |X_gpu - X_orc| <= max(1e-6 |X_orc|, 3e-7 B_X) for acc,
         <= max(1e-5 |X_orc|, 3e-6 B_X) for jerk, snap and crackle.
The relative bounds are the stated targets (FP64 1e-12 in acc and jerk; mixed
acc 1e-6, higher derivatives 1e-5).  The B_X terms admit the particles whose
total is a near-cancellation of much larger pair terms (|X_i| << B_X): there
no implementation in the working precision can hold a relative bound, and the
bound becomes a fixed multiple of the unit roundoff times the term magnitudes
(FP64 u = 1.1e-16, ~90 u; FP32 u = 6e-8, ~5 u per term for acc).
"""
from __future__ import annotations

import numpy as np

import oracle as orc
from paper_1312_1789_b300 import nb

TOL = {
    nb.NB_FP64: {"acc": (1e-12, 1e-14), "jerk": (1e-12, 1e-14), "snap": (1e-10, 1e-13), "crackle": (1e-10, 1e-13),
                 "pot": (1e-12, 1e-14)},
    nb.NB_MIXED: {"acc": (1e-6, 3e-7), "jerk": (1e-5, 3e-6), "snap": (1e-5, 3e-6), "crackle": (1e-5, 3e-6),
                  "pot": (1e-6, 3e-7)},
}
KEYS = {4: ("acc", "jerk"), 6: ("acc", "jerk", "snap"), 8: ("acc", "jerk", "snap", "crackle")}
ABS_COL = {"acc": 0, "jerk": 1, "snap": 2, "crackle": 3, "pot": 4}


def make_ctx(m, x, v, eps2, order, prec, eta=0.2, dt_max=1.0 / 16, pair=False):
    """Context with per-particle softening when eps2 is not one positive value."""
    n = len(m)
    eps2 = np.broadcast_to(np.asarray(eps2, dtype=np.float64), (n,))
    uniform = bool(np.all(eps2 == eps2[0]) and eps2[0] > 0 and not pair)
    ctx = nb.NBody(n, order, float(np.sqrt(eps2[0])) if uniform else 0.0, prec)
    if not uniform:
        ctx.set_softening(np.sqrt(eps2))
    ctx.set_params(eta=eta, eta_s=0.01, dt_max=dt_max, dt_min=2.0 ** -40)
    ctx.set_particles(m, x, v)
    return ctx


def oracle_force_on_predicted(ctx, m, eps2, idx, order):
    """Oracle force computed from exactly the predicted store the kernel read."""
    xp, vp, ap, jp = ctx.get_predicted()
    return orc.force(m, eps2, xp, vp, ap if order >= 6 else None, jp if order >= 8 else None, order=order,
                     idx=idx, nthreads=16)


def force_violations(G, O, order, prec):
    """Per derivative: (max error / allowed, worst particle, its relative error)."""
    res = {}
    for key in KEYS[order] + ("pot",):
        rel, cnd = TOL[prec][key]
        if key == "pot":
            err = np.abs(G[key] - O[key])
            mag = np.abs(O[key])
        else:
            err = np.linalg.norm(G[key] - O[key], axis=1)
            mag = np.linalg.norm(O[key], axis=1)
        allowed = np.maximum(np.maximum(rel * mag, cnd * O["absum"][:, ABS_COL[key]]), 1e-300)
        ratio = err / allowed
        k = int(np.argmax(ratio))
        res[key] = (float(ratio[k]), k, float(err[k] / max(mag[k], 1e-300)))
    return res


def assert_force_close(G, O, order, prec, what=""):
    v = force_violations(G, O, order, prec)
    bad = {k: r for k, r in v.items() if not r[0] <= 1.0}
    assert not bad, f"{what}: error/allowed (worst, particle, rel err) = {bad}"
    return v
