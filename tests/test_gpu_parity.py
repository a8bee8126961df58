"""GPU parity: every kernel of the hot path, called through the C ABI, against
the CPU oracle on the same seeded inputs (tolerances: tests/gpu_common.py).

Sizes span several 128-particle j tiles and a ragged tail; the large-N test
runs the 2^20 + 2 nucleus workload in the launch shape the benchmark times and
checks sampled particles one by one.
"""
import math

import numpy as np
import pytest

import oracle as orc
from gpu_common import assert_force_close, make_ctx, oracle_force_on_predicted
from paper_1312_1789_b300 import ics, nb

pytestmark = pytest.mark.gpu

PRECS = [nb.NB_FP64, nb.NB_MIXED]
PNAME = {nb.NB_FP64: "fp64", nb.NB_MIXED: "mixed"}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1312_1789_b300 import build
    build.build()
    nb.lib()


def _system(n, seed, kind):
    """Plummer sphere (uniform eps 1e-4) or stars + two unsoftened holes."""
    if kind == "plummer":
        m, x, v = ics.plummer(n, seed)
        return m, x, v, np.full(n, 1e-8)
    m, x, v = ics.plummer(n - 2, seed)
    mb, xb, vb = ics.bh_circular_pair(0.005, 0.1)
    eps2 = np.concatenate([np.full(n - 2, 1e-8), np.zeros(2)])
    return np.concatenate([m, mb]), np.concatenate([x, xb]), np.concatenate([v, vb]), eps2


def _advanced(m, x, v, eps2, order, prec, t, eta=0.2, pair=False):
    """Context integrated to time t on the FP64 path, then switched to prec.

    Kernel-level parity of the mixed path is tested on states the FP64 path
    reached, so that the comparison does not depend on how the mixed path's
    own integration evolves."""
    ctx = make_ctx(m, x, v, eps2, order, nb.NB_FP64, eta=eta, pair=pair)
    if t > 0:
        ctx.step_until(t)
    ctx.set_precision(prec)
    return ctx


def _idx(kind, n, rng):
    if kind == "all":
        return np.arange(n, dtype=np.int32)
    if kind == "subset":
        return np.sort(rng.choice(n, 37, replace=False)).astype(np.int32)
    return np.array([n // 2], dtype=np.int32)


# ------------------------------------------------------------------ force K2+K3
@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("order", [4, 6, 8])
@pytest.mark.parametrize("kind", ["plummer", "holes"])
def test_force_parity(prec, order, kind):
    n = 3 * 128 + 37
    m, x, v, eps2 = _system(n, 7 + order, kind)
    ctx = _advanced(m, x, v, eps2, order, prec, 1.0 / 128, pair=(kind == "holes"))
    tb, _ = ctx.next_block()
    ctx.predict(tb)
    rng = np.random.default_rng(order)
    for which in ("all", "subset", "one"):
        idx = _idx(which, n, rng)
        O = oracle_force_on_predicted(ctx, m, eps2, idx, order)
        for js in (0, 1, 3, 7):
            ctx.set_jsplit(js)
            ctx.force(idx)
            G = ctx.get_force(len(idx))
            assert_force_close(G, O, order, prec, f"{PNAME[prec]} order {order} {kind} {which} jsplit {js}")
    ctx.close()


@pytest.mark.parametrize("order", [4, 6, 8])
@pytest.mark.parametrize("kind", ["plummer", "holes"])
def test_force_parity_two_particles_per_thread(order, kind):
    # Active sets of >= 512 run the mixed kernel with two i-particles per
    # thread; ragged last i-tile, several split counts.
    n = 2 * 1024 + 77
    m, x, v, eps2 = _system(n, 50 + order, kind)
    ctx = _advanced(m, x, v, eps2, order, nb.NB_MIXED, 1.0 / 256, pair=(kind == "holes"))
    tb, _ = ctx.next_block()
    ctx.predict(tb)
    rng = np.random.default_rng(order + 7)
    for idx in (np.arange(n, dtype=np.int32), np.sort(rng.choice(n, 1500, replace=False)).astype(np.int32)):
        O = oracle_force_on_predicted(ctx, m, eps2, idx, order)
        for js in (0, 1, 5):
            ctx.set_jsplit(js)
            ctx.force(idx)
            G = ctx.get_force(len(idx))
            assert_force_close(G, O, order, nb.NB_MIXED, f"order {order} {kind} n_act {len(idx)} jsplit {js}")
    ctx.close()


def test_uniform_softening_form_on_star_warps():
    # Per-particle softening: a warp whose i-particles all carry the largest
    # eps^2 takes it as the pair value, the others take the per-pair max.
    # Both forms give the same bits, so only the kernel's warp count shows
    # which ran.  Stars at 1e-5 (eps^2 = 1e-10 lies below its nearest float,
    # so a threshold rounded to nearest misses the stored, truncated value),
    # two unsoftened holes listed first: exactly warp 0 of the first i-tile
    # per j-split takes the per-pair form; without the holes none does.
    n = 2 * 1024 + 77
    m, x, v, _ = _system(n, 91, "holes")
    for holes in (True, False):
        eps2 = np.full(n, 1e-10)
        if holes:
            eps2[-2:] = 0.0
        ctx = make_ctx(m, x, v, eps2, 6, nb.NB_MIXED, pair=True)
        tb, _ = ctx.next_block()
        ctx.predict(tb)
        idx = np.concatenate([[n - 2, n - 1], np.arange(n - 2)]).astype(np.int32)
        ctx.get_pair_warps()
        for js in (0, 1, 5):
            ctx.set_jsplit(js)
            ctx.force(idx)
            _, jsplit, ni = ctx.get_launch()
            assert ni == 256
            assert ctx.get_pair_warps() == (jsplit if holes else 0), (holes, js, jsplit)
        ctx.close()


# i-particles per CTA of the mixed force for an active-set size: 4 up to 24
# active, 32 up to 256, 128 below 512, then 256 (two per thread).
def _expected_ni(n_act):
    return 256 if n_act >= 512 else 128 if n_act > 256 else 32 if n_act > 24 else 4


@pytest.mark.parametrize("order", [4, 6, 8])
@pytest.mark.parametrize("kind", ["plummer", "holes"])
def test_force_parity_small_active_sets(order, kind):
    # Active sets of a few particles run the j-parallel variants (32 or 4
    # threads per i-particle, lane sums added in a fixed order); cover each
    # variant's full and ragged i-tiles, a particle with itself in the
    # store, and several split counts.
    n = 5 * 128 + 19
    m, x, v, eps2 = _system(n, 70 + order, kind)
    ctx = _advanced(m, x, v, eps2, order, nb.NB_MIXED, 1.0 / 256, pair=(kind == "holes"))
    tb, _ = ctx.next_block()
    ctx.predict(tb)
    rng = np.random.default_rng(order + 11)
    seen = set()
    for na in (1, 3, 4, 5, 9, 24, 25, 32, 33, 100, 257, 300, 600):
        idx = np.sort(rng.choice(n, na, replace=False)).astype(np.int32)
        if kind == "holes" and na >= 2:
            idx[-1] = n - 1  # an unsoftened hole among the active particles
            idx = np.unique(idx)
        O = oracle_force_on_predicted(ctx, m, eps2, idx, order)
        for js in (0, 1, 6):
            ctx.set_jsplit(js)
            ctx.force(idx)
            it, jsplit, ni = ctx.get_launch()
            assert ni == _expected_ni(len(idx)) and it * ni >= len(idx)
            seen.add(ni)
            G = ctx.get_force(len(idx))
            assert_force_close(G, O, order, nb.NB_MIXED, f"order {order} {kind} n_act {len(idx)} jsplit {js}")
    assert seen >= {4, 32, 128}
    ctx.close()


def test_force_jsplit_changes_only_rounding():
    # FP64 results of different split counts agree to rounding; a given
    # launch shape is bitwise reproducible.
    n = 1000
    m, x, v, eps2 = _system(n, 3, "plummer")
    ctx = make_ctx(m, x, v, eps2, 6, nb.NB_FP64)
    ctx.predict(1.0 / 256)
    idx = np.arange(n, dtype=np.int32)
    ctx.set_jsplit(5)
    ctx.force(idx)
    a = ctx.get_force(n)["acc"]
    ctx.force(idx)
    b = ctx.get_force(n)["acc"]
    assert np.array_equal(a, b)
    ctx.set_jsplit(1)
    ctx.force(idx)
    c = ctx.get_force(n)["acc"]
    assert np.allclose(a, c, rtol=1e-13, atol=0)


# -------------------------------------------------------------------- predictor
@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("order", [4, 6, 8])
def test_predictor_parity(prec, order):
    n = 2 * 128 + 5
    m, x, v, eps2 = _system(n, 21, "plummer")
    ctx = _advanced(m, x, v, eps2, order, prec, 1.0 / 64)
    tb, _ = ctx.next_block()
    ctx.predict(tb)
    S = ctx.get_state()
    assert np.any(S["t"] != S["t"][0]), "want particles at different times"
    xo, vo, ao, jo = orc.predict(order, tb, S["t"], S["x"], S["v"], S["d"])
    xg, vg, ag, jg = ctx.get_predicted()
    if prec == nb.NB_FP64:
        assert np.all(np.abs(xg - xo) <= 2e-15 * np.maximum(np.abs(xo), 1.0))
        assert np.all(np.abs(vg - vo) <= 2e-15 * np.maximum(np.abs(vo), 1.0))
        if order >= 6:
            assert np.all(np.abs(ag - ao) <= 1e-14 * np.maximum(np.abs(ao), 1.0))
        if order >= 8:
            assert np.all(np.abs(jg - jo) <= 1e-13 * np.maximum(np.abs(jo), 1.0))
    else:
        # x = x0 + h (v0 + h T) in FP64, stored double-single (|hi + lo - x| <=
        # 2^-48 |x|); the tail T and the predicted v, a, jerk are FP32 Horner
        # sums: a few float roundings (2^-21) of the magnitudes of their terms.
        h = np.abs(tb - S["t"])[:, None]
        D = np.abs(S["d"])  # [n][6][3]: a, j, s, c, d4a, d5a
        nd = 6 if order == 8 else 4
        fact = [math.factorial(k) for k in range(10)]

        def mag(first, start, kmin):
            # |first| + sum_{k >= kmin} |d_(start + k - kmin)| h^k / k!
            out = np.abs(first).copy() if first is not None else 0.0
            for q in range(start, nd):
                k = kmin + q - start
                out = out + D[:, q, :] * h ** k / fact[k]
            return out

        u = 2.0 ** -21
        tail_x = mag(None, 0, 2)
        assert np.all(np.abs(xg - xo) <= 2e-14 * np.maximum(np.abs(xo), 1e-3) + u * tail_x)
        assert np.all(np.abs(vg - vo) <= u * mag(S["v"], 0, 1) + 1e-15)
        if order >= 6:
            assert np.all(np.abs(ag - ao) <= u * mag(S["d"][:, 0, :], 1, 1) + 1e-14)
        if order >= 8:
            assert np.all(np.abs(jg - jo) <= u * mag(S["d"][:, 1, :], 2, 1) + 1e-13)


def test_mixed_predictor_takes_fp64_series_past_the_float_range():
    # Interpolated high derivatives of a particle just out of a close
    # encounter can exceed the float range: the mixed predictor must then
    # evaluate that particle's series in FP64 (no inf/NaN, the FP64 result),
    # both for h = 0 (the particle is at the block time) and for small h.
    n = 300
    m, x, v, eps2 = _system(n, 33, "plummer")
    ctx = make_ctx(m, x, v, eps2, 8, nb.NB_MIXED)
    S = ctx.get_state()
    d = S["d"].copy()
    t = np.zeros(n)
    dt = np.full(n, 2.0 ** -4)
    d[5, 4, 0] = 1e45    # d4a beyond FLT_MAX; particle 5 predicted with h = 0
    d[7, 4, 1] = -2e45   # particle 7 predicted with h = 2^-24
    d[7, 5, 2] = 3e50
    t[7] = -(2.0 ** -24)
    ctx.set_state(S["x"], S["v"], d, t, dt)
    ctx.predict(0.0)
    xg, vg, ag, jg = ctx.get_predicted()
    assert np.all(np.isfinite(xg)) and np.all(np.isfinite(vg)) and np.all(np.isfinite(ag)) and np.all(np.isfinite(jg))
    xo, vo, ao, jo = orc.predict(8, 0.0, t, S["x"], S["v"], d)
    for i in (5, 7):
        scale = np.abs(xo[i]) + np.abs(S["x"][i]) + 1.0
        assert np.all(np.abs(xg[i] - xo[i]) <= 1e-13 * scale), (i, xg[i], xo[i])
        assert np.all(np.abs(vg[i] - vo[i]) <= 1.2e-7 * (np.abs(vo[i]) + np.abs(S["v"][i])) + 1e-15)
    ctx.close()


# -------------------------------------------------------------------- scheduler
def test_scheduler_parity():
    n = 2048 + 300  # more than one scheduler chunk, ragged
    m, x, v, eps2 = _system(n, 5, "plummer")
    ctx = make_ctx(m, x, v, eps2, 6, nb.NB_FP64)
    for t_stop in (0.0, 1.0 / 512, 1.0 / 128, 1.0 / 32):
        if t_stop > 0:
            ctx.step_until(t_stop)
        S = ctx.get_state()
        tb_o, idx_o = orc.next_block(S["t"], S["dt"])
        tb_g, idx_g = ctx.next_block(want_idx=True)
        assert tb_g == tb_o
        assert np.array_equal(idx_g, idx_o)


# -------------------------------------------------------------------- corrector
@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
@pytest.mark.parametrize("order", [4, 6, 8])
def test_corrector_parity(prec, order):
    n = 3 * 128 + 11
    m, x, v, eps2 = _system(n, 40 + order, "plummer")
    eta = 0.2 if order != 4 else 0.02
    ctx = _advanced(m, x, v, eps2, order, prec, 1.0 / 64, eta=eta)
    tb, idx = ctx.next_block(want_idx=True)
    ctx.predict(tb)
    ctx.force()
    S0 = ctx.get_state()
    F = ctx.get_force(len(idx))
    bacc = oracle_force_on_predicted(ctx, m, eps2, idx, order)["absum"][:, 5]
    ctx.correct()
    S1 = ctx.get_state()
    mm = order // 2
    newd = np.stack([F["acc"], F["jerk"], F["snap"], F["crackle"]], axis=1)  # [n_act][4][3]
    dt_diff = 0
    for p, i in enumerate(idx):
        h = tb - S0["t"][i]
        D0 = S0["d"][i, :4]
        D1 = newd[p, :mm]
        hi = orc.interp(mm, h, D0[:mm], D1)
        Dfull = np.vstack([D1, hi])
        x1, v1 = orc.correct(order, h, S0["x"][i], S0["v"][i], D0, Dfull[:4])
        crit = orc.dt_criterion_floored(order, eta, h, D0, Dfull, ctx.get_noise_floor(prec), bacc[p])
        lim = min(crit, 2 * h)
        dt_o = orc.dt_quantise(lim, tb, 1.0 / 16, 2.0 ** -40)
        assert S1["t"][i] == tb
        # FP64: every step in double.  Mixed: the terms beyond x0 + h/2 (v0 +
        # v1) and v0 + h/2 (a0 + a1), the interpolants and the criterion are
        # evaluated in FP32 from inputs truncated to float (relative error
        # <= 2^-23 each): the bounds are the float rounding of those terms,
        # and the step may move by one level where the criterion sits within
        # float rounding of a power of two.
        tx, tv = _tail_scale(order, h, D0, Dfull)
        if prec == nb.NB_FP64:
            assert S1["dt"][i] == dt_o, (i, S1["dt"][i], dt_o)
            tx = tv = 0.0
        else:
            assert dt_o / 2 <= S1["dt"][i] <= 2 * dt_o, (i, S1["dt"][i], dt_o)
            dt_diff += int(S1["dt"][i] != dt_o)
        assert np.all(np.abs(S1["x"][i] - x1) <= 2e-15 * max(1.0, np.abs(x1).max()) + 2.0 ** -21 * (tx + h / 2 * tv))
        assert np.all(np.abs(S1["v"][i] - v1) <= 2e-15 * max(1.0, np.abs(v1).max()) + 2.0 ** -21 * tv)
        assert np.array_equal(S1["d"][i, :mm], D1)
        for k in range(mm, min(2 * mm, 6)):
            scale = sum((np.linalg.norm(D0[q]) + np.linalg.norm(D1[q])) * h ** (q - k) for q in range(mm))
            tol = 1e-11 if prec == nb.NB_FP64 else _INTERP_COEF_SUM[order][k] * 2.0 ** -22
            assert np.linalg.norm(S1["d"][i, k] - hi[k - mm]) <= tol * scale, (i, k)
    assert dt_diff <= 0.02 * len(idx), dt_diff


# Sum of the absolute coefficients of the closed-form interpolant a^(k) h^k
# in the inputs a^(q) h^q at both ends (order -> k -> sum): the factor by
# which the float rounding of the inputs can grow in it.
_INTERP_COEF_SUM = {
    4: {2: 2 * (3 + 3 + 1 + 2), 3: 6 * (2 + 2 + 1 + 1)},
    6: {3: 3 * (20 + 20 + 3 + 1 + 8 + 12), 4: 12 * (30 + 30 + 3 + 2 + 14 + 16), 5: 60 * (12 + 12 + 1 + 1 + 6 + 6)},
    8: {4: 4 * (210 + 210 + 1 + 4 + 15 + 30 + 90 + 120), 5: 60 * (168 + 168 + 1 + 2 + 14 + 20 + 78 + 90)},
}


def _tail_scale(order, h, D0, D1):
    """Sizes of the corrector terms beyond the leading ones (x, v): the sums of
    the absolute values of every term of h^2 and higher."""
    n = lambda a: np.abs(a)
    if order == 4:
        c = [1 / 12]
    elif order == 6:
        c = [1 / 10, 1 / 120]
    else:
        c = [3 / 28, 1 / 84, 1 / 1680]
    tv = sum(ck * h ** (k + 2) * (n(D0[k + 1]) + n(D1[k + 1])) for k, ck in enumerate(c))
    tx = sum(ck * h ** (k + 2) * (n(D0[k]) + n(D1[k])) for k, ck in enumerate(c))
    return tx, tv


# ---------------------------------------------------------- whole integration
def test_block_sequence_plummer_1k_exact():
    # Plummer N = 1024, order 6, eps 1e-4, eta 0.2, dt_max 1/16 to t = 0.125:
    # FP64 path and oracle take the identical sequence of (t_blk, active set).
    wl = ics.standard_workload(0)
    st = orc.State(wl.m, wl.eps2, wl.x, wl.v)
    log = orc.integrate(st, order=6, t_end=wl.t_end, eta=wl.eta, nthreads=16, log=True)
    ctx = make_ctx(wl.m, wl.x, wl.v, wl.eps2, 6, nb.NB_FP64)
    k = 0
    while True:
        tb, idx = ctx.next_block(want_idx=True)
        if tb > wl.t_end:
            break
        assert k < len(log), "device took more blocks"
        assert tb == log[k][0], f"block {k}: t {tb} vs {log[k][0]}"
        assert np.array_equal(idx, log[k][1]), f"block {k}: active sets differ"
        ctx.predict(tb)
        ctx.force()
        ctx.correct()
        k += 1
    assert k == len(log)
    S = ctx.get_state()
    assert np.all(S["t"] == wl.t_end)
    assert np.max(np.abs(S["x"] - st.x)) < 1e-11
    assert np.max(np.abs(S["v"] - st.v)) < 1e-10
    assert np.array_equal(S["dt"], st.dt)


def test_mixed_integration_block_sequence_close_to_oracle():
    # The mixed path integrates the 1k Plummer sphere without step collapse;
    # the oracle with the same noise floor takes nearly the same blocks.
    wl = ics.standard_workload(0)
    ctx = make_ctx(wl.m, wl.x, wl.v, wl.eps2, 6, nb.NB_MIXED)
    nblk, _ = ctx.step_until(wl.t_end)
    S = ctx.get_state()
    assert np.all(S["t"] == wl.t_end)
    st = orc.State(wl.m, wl.eps2, wl.x, wl.v)
    nblk_o = orc.integrate(st, order=6, t_end=wl.t_end, eta=wl.eta, nthreads=16,
                           noise=ctx.get_noise_floor(nb.NB_MIXED))
    assert abs(nblk - nblk_o) <= 0.1 * nblk_o
    assert np.max(np.abs(S["x"] - st.x)) < 1e-5


def test_mixed_energy_error_close_to_fp64():
    # Same system on both paths to t = 0.125; energies measured in FP64.
    wl = ics.standard_workload(0)
    out = {}
    for prec in PRECS:
        ctx = make_ctx(wl.m, wl.x, wl.v, wl.eps2, 6, prec)
        ctx.set_precision(nb.NB_FP64)
        e0 = sum(ctx.energy())
        ctx.set_precision(prec)
        ctx.step_until(wl.t_end)
        ctx.set_precision(nb.NB_FP64)
        e1 = sum(ctx.energy())
        out[prec] = (e1 - e0) / e0
    print("dE/E fp64 %.3e mixed %.3e" % (out[nb.NB_FP64], out[nb.NB_MIXED]))
    assert abs(out[nb.NB_FP64]) < 1e-9
    assert abs(out[nb.NB_MIXED]) < 1e-8


# ----------------------------------------------------------------------- energy
@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_energy_parity(prec):
    n = 3 * 128 + 7
    m, x, v, eps2 = _system(n, 9, "holes")
    ctx = make_ctx(m, x, v, eps2, 6, prec, pair=True)
    ek, ep = ctx.energy()
    ek_o, ep_o = orc.energy(m, eps2, x, v)
    tol = 1e-13 if prec == nb.NB_FP64 else 1e-6
    assert ek == pytest.approx(ek_o, rel=1e-14)
    assert ep == pytest.approx(ep_o, rel=tol)
    ctx.set_precision(nb.NB_FP64)
    ctx.step_until(1.0 / 16)
    ctx.set_precision(prec)
    S = ctx.get_state()
    assert np.all(S["t"] == 1.0 / 16)
    ek, ep = ctx.energy()
    ek_o, ep_o = orc.energy(m, eps2, S["x"], S["v"])
    assert ek == pytest.approx(ek_o, rel=1e-14)
    assert ep == pytest.approx(ep_o, rel=tol)


# ----------------------------------------------------- 65536 Plummer, sampled
def test_plummer_65536_sampled_blocks_parity_to_t1():
    # The 65536-particle Plummer sphere on the mixed path, integrated to
    # t = 1 as CUDA-graph replays of device-driven block cycles.  At 16
    # times spread over the run, one block is stepped through the C ABI and
    # the force of up to 256 of its active particles is compared with the
    # oracle on the very store the kernel read: alternately the synchronised
    # block at t = k/16 (every particle active) and the first block after
    # it (the particles on the shortest steps), so that early and late
    # blocks (after the core has evolved), large and small, are all checked.
    wl = ics.standard_workload(1)
    ctx = make_ctx(wl.m, wl.x, wl.v, wl.eps2, 6, nb.NB_MIXED)
    ctx.set_graph(64)
    rng = np.random.default_rng(65536)
    checks, sizes, strict = [], [], {}
    for k in range(1, 17):
        t_k = k / 16.0
        ctx.step_until(t_k - 2.0 ** -30 if k % 2 else t_k)
        tb, idx = ctx.next_block(want_idx=True)
        assert (tb == t_k) == bool(k % 2), (k, tb)
        ctx.predict(tb)
        ctx.force()
        pos = np.arange(len(idx)) if len(idx) <= 256 else np.sort(rng.choice(len(idx), 256, replace=False))
        G = ctx.get_force(len(idx))
        O = oracle_force_on_predicted(ctx, wl.m, wl.eps2, idx[pos].astype(np.int32), 6)
        v = assert_force_close({key: G[key][pos] for key in G}, O, 6, nb.NB_MIXED,
                               f"t = {tb} ({len(idx)} active)")
        for key, r in v.items():
            strict.setdefault(key, []).append(r["strict_pass"] * r["n"])
        ctx.correct()
        checks.append(tb)
        sizes.append(len(idx))
    n_checked = sum(min(s, 256) for s in sizes)
    print("65536 Plummer to t = 1: %d blocks checked (t = %.4f .. %.4f, %d .. %d active); strict pass: %s"
          % (len(checks), checks[0], checks[-1], min(sizes), max(sizes),
             ", ".join(f"{k} {sum(v) / n_checked:.4f}" for k, v in strict.items())))
    assert len(checks) == 16 and checks[-1] > 1.0 and max(sizes) == wl.n and min(sizes) < 1024
    ctx.close()


def test_mixed_energy_error_within_twice_fp64_after_one_time_unit():
    # The spec energy target: a 4096-particle Plummer sphere integrated
    # for one time unit on both paths; |dE/E| of the mixed path within twice
    # the FP64 path's (energies measured in FP64 at t = 0 and t = 1).
    wl = ics.plummer_cluster(4096, 1001, 1e-4, 6, 1.0)
    out = {}
    for prec in PRECS:
        ctx = make_ctx(wl.m, wl.x, wl.v, wl.eps2, 6, prec)
        ctx.set_precision(nb.NB_FP64)
        e0 = sum(ctx.energy())
        ctx.set_precision(prec)
        ctx.set_graph(64)
        nblk, _ = ctx.step_until(1.0)
        ctx.set_precision(nb.NB_FP64)
        assert np.all(ctx.get_state()["t"] == 1.0)
        out[prec] = ((sum(ctx.energy()) - e0) / abs(e0), nblk)
        ctx.close()
    print("4096 Plummer to t = 1: dE/E fp64 %.4e (%d blocks), mixed %.4e (%d blocks)"
          % (out[nb.NB_FP64][0], out[nb.NB_FP64][1], out[nb.NB_MIXED][0], out[nb.NB_MIXED][1]))
    assert abs(out[nb.NB_MIXED][0]) <= 2.0 * abs(out[nb.NB_FP64][0])
    assert abs(out[nb.NB_FP64][0]) < 1e-3


# ------------------------------------------------------------ full-size sample
def test_nucleus_2pow20_sampled_parity():
    # 2^20 stars + two holes, every particle active (the benchmarked block),
    # mixed path; sampled particles (both holes among them) against the oracle
    # one by one.  Then the FP64 path on a 64-particle block of the same system.
    wl = ics.standard_workload(2)
    n = wl.n
    ctx = make_ctx(wl.m, wl.x, wl.v, wl.eps2, 6, nb.NB_MIXED, pair=True)
    ctx.predict(2.0 ** -12)
    ctx.force(np.arange(n, dtype=np.int32))
    it, js, per_cta = ctx.get_launch()
    assert it * per_cta >= n > (it - 1) * per_cta and js >= 1
    G = ctx.get_force(n)
    rng = np.random.default_rng(0)
    sample = np.concatenate([rng.choice(n - 2, 22, replace=False), [n - 2, n - 1]]).astype(np.int32)
    O = oracle_force_on_predicted(ctx, wl.m, wl.eps2, sample, 6)
    Gs = {k: G[k][sample] for k in G}
    assert_force_close(Gs, O, 6, nb.NB_MIXED, "nucleus 2^20 mixed, sampled")
    ctx.set_precision(nb.NB_FP64)
    ctx.predict(2.0 ** -12)
    blk = np.sort(rng.choice(n, 64, replace=False)).astype(np.int32)
    ctx.force(blk)
    G = ctx.get_force(len(blk))
    O = oracle_force_on_predicted(ctx, wl.m, wl.eps2, blk, 6)
    assert_force_close(G, O, 6, nb.NB_FP64, "nucleus 2^20 fp64, 64-particle block")
    ctx.close()


# --------------------------------------------------------- checkpoint / restart
@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_checkpoint_restart_is_bitwise(prec):
    n = 700
    m, x, v, eps2 = _system(n, 12, "plummer")
    a = _advanced(m, x, v, eps2, 6, prec, 0.0)
    a.step_until(1.0 / 64)
    S = a.get_state()
    b = _advanced(m, x, v, eps2, 6, prec, 0.0)
    b.set_state(S["x"], S["v"], S["d"], S["t"], S["dt"])
    a.step_until(1.0 / 16)
    b.step_until(1.0 / 16)
    Sa, Sb = a.get_state(), b.get_state()
    for k in Sa:
        assert np.array_equal(Sa[k], Sb[k]), k


# ------------------------------------------------------------------ edge cases
def test_single_particle_moves_in_a_straight_line():
    ctx = nb.NBody(1, 6, 1e-4, nb.NB_FP64)
    ctx.set_particles([1.0], [[0.5, -0.25, 2.0]], [[0.125, 0.5, -1.0]])
    nbk, ni = ctx.step_until(0.5)
    assert nbk == 8 and ni == 8
    S = ctx.get_state()
    assert np.allclose(S["x"][0], [0.5 + 0.0625, -0.25 + 0.25, 2.0 - 0.5], rtol=0, atol=1e-15)
    assert np.all(S["d"] == 0) and S["dt"][0] == 1.0 / 16


@pytest.mark.parametrize("order", [4, 6, 8])
def test_unsoftened_kepler_pair_matches_oracle(order):
    m = np.array([0.5, 0.5])
    e = 0.5
    r = 1 + e
    vrel = math.sqrt((1 - e) / (1 + e))
    x = np.array([[0.5 * r, 0, 0], [-0.5 * r, 0, 0]])
    v = np.array([[0, 0.5 * vrel, 0], [0, -0.5 * vrel, 0]])
    eta = 0.02 if order == 4 else 0.1
    ctx = make_ctx(m, x, v, np.zeros(2), order, nb.NB_FP64, eta=eta, pair=True)
    ctx.step_until(2.0)
    st = orc.State(m, 0.0, x, v)
    orc.integrate(st, order=order, t_end=2.0, eta=eta)
    S = ctx.get_state()
    assert np.max(np.abs(S["x"] - st.x)) < 1e-11
    assert np.array_equal(S["dt"], st.dt)


@pytest.mark.parametrize("prec", PRECS, ids=PNAME.get)
def test_ragged_sizes_force(prec):
    # stores of one particle, of less than one tile, of a tile and one more;
    # an empty active list is an argument error, not a launch
    for n in (1, 2, 127, 128, 129, 255):
        m, x, v, eps2 = _system(max(n, 3), 77, "plummer")
        m, x, v, eps2 = m[:n], x[:n], v[:n], eps2[:n]
        ctx = make_ctx(m, x, v, eps2, 6, prec)
        ctx.predict(1.0 / 1024)
        idx = np.arange(n, dtype=np.int32)
        ctx.force(idx)
        G = ctx.get_force(n)
        O = oracle_force_on_predicted(ctx, m, eps2, idx, 6)
        if n == 1:
            assert np.all(G["acc"] == 0) and G["pot"][0] == 0.0
        else:
            assert_force_close(G, O, 6, prec, f"n={n}")
        with pytest.raises(nb.NBError) as e:
            ctx.force(np.zeros(0, dtype=np.int32))
        assert e.value.code == nb.NB_ERR_ARG
        ctx.close()


# --------------------------------------------------------------- error paths
def test_errors_are_reported_not_faulted():
    n = 300
    m, x, v, eps2 = _system(n, 1, "plummer")
    ctx = make_ctx(m, x, v, eps2, 6, nb.NB_FP64)
    with pytest.raises(nb.NBError) as e:
        ctx.correct()
    assert e.value.code == nb.NB_ERR_ARG
    ctx.predict(1.0 / 64)
    with pytest.raises(nb.NBError) as e:
        ctx.force(np.array([0, n + 3], dtype=np.int32))
    assert e.value.code == nb.NB_ERR_ARG
    ctx.step_until(1.0 / 256)
    S = ctx.get_state()
    if np.all(S["t"] == S["t"][0]):
        ctx.block_step()
    with pytest.raises(nb.NBError) as e:
        ctx.energy()
    assert e.value.code == nb.NB_ERR_NOT_SYNC
    bad = x.copy()
    bad[3, 1] = np.nan
    with pytest.raises(nb.NBError) as e:
        ctx.set_particles(m, bad, v)
    assert e.value.code == nb.NB_ERR_NAN
    # an invalid state is rejected (checked on the device) and leaves the old one
    S = ctx.get_state()
    for key, idx, val, code in (("d", (5, 2, 1), np.inf, nb.NB_ERR_NAN), ("dt", (7,), 0.0, nb.NB_ERR_ARG),
                                ("x", (n - 1, 0), np.nan, nb.NB_ERR_NAN)):
        B = {k: a.copy() for k, a in S.items()}
        B[key][idx] = val
        with pytest.raises(nb.NBError) as e:
            ctx.set_state(B["x"], B["v"], B["d"], B["t"], B["dt"])
        assert e.value.code == code
        after = ctx.get_state()
        for k in S:
            assert np.array_equal(after[k], S[k]), (key, k)
    # a minimum step larger than what the start-up criterion asks for
    c2 = nb.NBody(n, 6, 1e-4, nb.NB_FP64)
    c2.set_params(0.2, 0.01, 1.0 / 16, 1.0 / 32)
    with pytest.raises(nb.NBError) as e:
        c2.set_particles(m, x, v)
    assert e.value.code == nb.NB_ERR_DT_UNDERFLOW


def test_bounded_wait_runs_out_and_reports_a_timeout():
    # Failure detection without a fault: a kernel waits on a barrier nothing
    # completes; its bounded wait gives up after the limit, the host reads
    # NB_ERR_TIMEOUT, and the context computes correct forces afterwards.
    import time
    n = 300
    m, x, v, eps2 = _system(n, 8, "plummer")
    ctx = make_ctx(m, x, v, eps2, 6, nb.NB_MIXED)
    t0 = time.perf_counter()
    rc = ctx.selftest_wait(0.2)
    el = time.perf_counter() - t0
    assert rc == nb.NB_ERR_TIMEOUT
    assert 0.15 < el < 3.0
    ctx.predict(1.0 / 512)
    idx = np.arange(n, dtype=np.int32)
    ctx.force(idx)
    O = oracle_force_on_predicted(ctx, m, eps2, idx, 6)
    assert_force_close(ctx.get_force(n), O, 6, nb.NB_MIXED, "after a timeout")
    ctx.close()


def test_integer_conversions_match_the_hardware_cvt():
    # The mixed predictor and corrector convert f64 <-> f32 in integer
    # arithmetic; it must give the bits of cvt (rz, ftz, inf beyond 2^128).
    m, x, v, eps2 = _system(256, 8, "plummer")
    ctx = make_ctx(m, x, v, eps2, 6, nb.NB_MIXED)
    assert ctx.selftest_convert(1 << 24, 12345) == 0
    ctx.close()


def test_device_index_out_of_range_is_reported():
    torch = pytest.importorskip("torch")
    n = 300
    m, x, v, eps2 = _system(n, 2, "plummer")
    ctx = make_ctx(m, x, v, eps2, 6, nb.NB_FP64)
    ctx.predict(1.0 / 64)
    idx = torch.tensor([1, 2, n + 10], dtype=torch.int32, device="cuda")
    ctx.force(idx)
    with pytest.raises(nb.NBError) as e:
        ctx.get_force(3)
    assert e.value.code == nb.NB_ERR_ARG
    # the context stays usable
    ctx.force(np.array([1, 2], dtype=np.int32))
    assert ctx.get_force(2)["acc"].shape == (2, 3)


# ----------------------------------------------------------- torch plumbing
def test_torch_allocator_stream_and_device_indices():
    torch = pytest.importorskip("torch")
    n = 600
    m, x, v, eps2 = _system(n, 8, "plummer")
    ref = make_ctx(m, x, v, eps2, 6, nb.NB_FP64)
    ref.step_until(1.0 / 64)
    alloc = nb.TorchAllocator().install()
    try:
        ctx = nb.NBody(n, 6, 1e-4, nb.NB_FP64)
        ctx.set_params(0.2, 0.01, 1.0 / 16, 2.0 ** -40)
        s = torch.cuda.Stream()
        ctx.set_stream(s)
        ctx.set_particles(m, x, v)
        ctx.step_until(1.0 / 64)
        A, B = ref.get_state(), ctx.get_state()
        for k in A:
            assert np.array_equal(A[k], B[k]), k
        tb, idx = ctx.next_block(want_idx=True)
        ctx.predict(tb)
        ctx.force(torch.from_numpy(idx).cuda())
        G = ctx.get_force(len(idx))
        ref.next_block()
        ref.predict(tb)
        ref.force(idx)
        assert np.array_equal(G["acc"], ref.get_force(len(idx))["acc"])
        ctx.close()
    finally:
        nb.TorchAllocator.uninstall()
    del alloc
