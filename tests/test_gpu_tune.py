"""Autotuned force launch shapes (nb_autotune): the table, the shapes later
forces take from it, force parity under those shapes, and device-driven
cycles that look the table up on the device."""
from __future__ import annotations

import math

import numpy as np
import pytest

from gpu_common import assert_force_close, make_ctx, oracle_force_on_predicted
from paper_1312_1789_b300 import ics, nb

pytestmark = pytest.mark.gpu


def _tuned_shape(table, n_act):
    """Shape rule of a tuned table, restated: class floor(log2 n_act) (the
    last class serves larger sets), its variant, the split count keeping
    the class's CTA count it * js."""
    k = min(int(math.floor(math.log2(n_act))), len(table) - 1)
    _, ni, js, _ = table[k]
    it_k = -(-(1 << k) // ni)
    it = -(-n_act // ni)
    return ni, it, max(1, (js * it_k + it // 2) // it)


def test_autotune_table_shapes_and_parity():
    n = 3000
    m, x, v = ics.plummer(n, 17)
    eps2 = np.full(n, 1e-8)
    ctx = make_ctx(m, x, v, eps2, 6, nb.NB_MIXED)
    rng = np.random.default_rng(1)
    blocks = [np.sort(rng.choice(n, na, replace=False)).astype(np.int32) for na in (1, 3, 7, 50, 300, 1500, 3000)]
    # the analytic rule's shapes, which classes without a tuned shape keep
    tb, _ = ctx.next_block()
    ctx.predict(tb)
    rule = []
    for idx in blocks:
        ctx.force(idx)
        rule.append(ctx.get_launch())
    ctx.autotune(2)
    table = ctx.get_tuning()
    assert len(table) == 12  # classes 2^0 .. 2^11 <= 3000
    for k, ni, js, ms in table:
        # ni = 0: the class keeps the analytic rule (no candidate beat it by 3 %)
        assert ms > 0 and (ni == 0 or (ni in (4, 32, 128, 256) and js >= 1))
    tb, _ = ctx.next_block()
    ctx.predict(tb)
    for idx, r in zip(blocks, rule):
        na = len(idx)
        ctx.force(idx)
        it, js, ni = ctx.get_launch()
        k = min(int(math.floor(math.log2(na))), len(table) - 1)
        if table[k][1] == 0:
            assert (it, js, ni) == r
        else:
            e_ni, e_it, e_js = _tuned_shape(table, na)
            assert (ni, it) == (e_ni, e_it)
            assert js == min(e_js, n // 128 + 1)  # the split is also capped by the j tiles
        O = oracle_force_on_predicted(ctx, m, eps2, idx, 6)
        assert_force_close(ctx.get_force(na), O, 6, nb.NB_MIXED, f"tuned shape n_act {na}")
    # the table as a JSON file, restored into another context of the same store
    import json
    import os
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.json")
        ctx.save_tuning(path)
        other = make_ctx(m, x, v, eps2, 6, nb.NB_MIXED)
        other.load_tuning(path)
        assert [e[:3] for e in other.get_tuning()] == [e[:3] for e in table]
        other.set_precision(nb.NB_FP64)
        with pytest.raises(ValueError):
            other.load_tuning(path)  # measured in the other precision
        doc = json.load(open(path))
        doc["n"] = n + 1
        json.dump(doc, open(path, "w"))
        other.set_precision(nb.NB_MIXED)
        with pytest.raises(ValueError):
            other.load_tuning(path)  # measured on another store
        other.close()
    ctx.autotune(0)
    assert ctx.get_tuning() == []
    with pytest.raises(nb.NBError):
        ctx.set_tuning([(0, 64, 1, 0.0)])  # no such variant
    ctx.close()


def test_autotune_fp64_table_is_per_precision():
    n = 700
    m, x, v = ics.plummer(n, 4)
    ctx = make_ctx(m, x, v, 1e-8, 6, nb.NB_FP64)
    ctx.autotune(1)
    t64 = ctx.get_tuning()
    assert len(t64) == 10 and all(e[1] in (0, 4, 32, 128) for e in t64)
    ctx.set_precision(nb.NB_MIXED)
    assert ctx.get_tuning() == []  # the mixed table is separate and empty
    ctx.set_precision(nb.NB_FP64)
    assert ctx.get_tuning() == t64
    ctx.close()


@pytest.mark.parametrize("tune_graph", [False, True])
def test_autotuned_graph_cycles_match_host_cycles_bitwise(tune_graph):
    # One measured table, installed in both contexts (a second measurement
    # could pick other shapes, whose rounding differs).  tune_graph: measured
    # with the persistent kernels of graph cycles (nb_set_graph first).
    n = 1800
    m, x, v = ics.plummer(n, 23)
    ctx = make_ctx(m, x, v, 1e-8, 6, nb.NB_MIXED)
    if tune_graph:
        ctx.set_graph(6)
    ctx.autotune(1)
    table = ctx.get_tuning()
    assert len(table) == 11 and all(e[1] in (0, 4, 32, 128, 256) for e in table)
    ctx.close()
    states = []
    for cycles in (0, 6):
        ctx = make_ctx(m, x, v, 1e-8, 6, nb.NB_MIXED)
        ctx.set_tuning(table)
        assert [e[:3] for e in ctx.get_tuning()] == [e[:3] for e in table]
        ctx.set_graph(cycles)
        counts = ctx.step_until(1.0 / 32)
        states.append((counts, ctx.get_state()))
        ctx.close()
    (c0, s0), (c1, s1) = states
    assert c0 == c1
    for key in ("x", "v", "d", "t", "dt"):
        assert np.array_equal(s0[key], s1[key]), key
