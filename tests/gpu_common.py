"""Shared helpers of the GPU parity tests: build contexts through the C ABI,
read back what the kernels consumed and produced, and compare with the oracle.

The force gate (tolerances per derivative, and the cancellation allowance
above cond = B_X / |X| = 1e3, 1e2 for the mixed snap and crackle) is
oracle/parity.py; assert_force_close returns its statistics, among them the
fraction of particles within the strict relative bound.
"""
from __future__ import annotations

import numpy as np

import oracle as orc
from oracle import parity
from paper_1312_1789_b300 import nb

KEYS = parity.KEYS
ABS_COL = parity.ABS_COL


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


def assert_force_close(G, O, order, prec, what=""):
    return parity.check_force(G, O, order, prec, what)
