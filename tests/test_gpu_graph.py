"""Device-driven block cycles replayed as a CUDA graph (nb_set_graph).

The graph path decides the active set, the block time and the force launch
shape on the device; it must take exactly the blocks the host-driven path
takes, with the same kernels' arithmetic, so the two states agree bit for bit.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1312_1789_b300 import ics, nb
from gpu_common import make_ctx

pytestmark = pytest.mark.gpu


def _run(m, x, v, eps2, order, prec, cycles, t_ends, pair=False, jsplit=0, block_step=None, between=None):
    ctx = make_ctx(m, x, v, eps2, order, prec, pair=pair)
    if jsplit:
        ctx.set_jsplit(jsplit)
    if block_step:
        ctx.set_block_step(block_step)
    ctx.set_graph(cycles)
    counts = []
    for k, te in enumerate(t_ends):
        if between and k > 0:
            between(ctx)
        counts.append(ctx.step_until(te))
    S = ctx.get_state()
    ctx.close()
    return S, counts


def _same(A, B):
    for key in ("x", "v", "d", "t", "dt"):
        assert np.array_equal(A[key], B[key]), f"{key} differs"


@pytest.mark.parametrize("prec", [nb.NB_FP64, nb.NB_MIXED])
@pytest.mark.parametrize("order", [4, 6, 8])
def test_graph_cycles_match_host_cycles_bitwise(prec, order):
    n = 1531
    m, x, v = ics.plummer(n, 11 + order)
    S0, c0 = _run(m, x, v, 1e-4, order, prec, 0, [1.0 / 16])
    S1, c1 = _run(m, x, v, 1e-4, order, prec, 7, [1.0 / 16])
    assert c0 == c1 and c0[0][0] > 20
    _same(S0, S1)


def test_graph_two_particles_per_thread_and_forced_split():
    # every particle active in the first blocks: the mixed force takes the
    # two-particles-per-thread kernel; a forced split must be honoured too
    n = 3000
    m, x, v = ics.plummer(n, 5)
    for js in (0, 3):
        S0, c0 = _run(m, x, v, 1e-4, 6, nb.NB_MIXED, 0, [1.0 / 64], jsplit=js, block_step=2.0 ** -9)
        S1, c1 = _run(m, x, v, 1e-4, 6, nb.NB_MIXED, 5, [1.0 / 64], jsplit=js, block_step=2.0 ** -9)
        assert c0 == c1
        assert c0[0][1] >= n * n  # the first block holds every particle
        _same(S0, S1)


def test_graph_per_particle_softening():
    n = 1100
    m, x, v = ics.plummer(n, 9)
    eps2 = np.linspace(1e-5, 4e-4, n)
    for prec in (nb.NB_FP64, nb.NB_MIXED):
        S0, c0 = _run(m, x, v, eps2, 6, prec, 0, [1.0 / 32])
        S1, c1 = _run(m, x, v, eps2, 6, prec, 16, [1.0 / 32])
        assert c0 == c1
        _same(S0, S1)


def test_graph_recaptured_after_parameter_change():
    n = 700
    m, x, v = ics.plummer(n, 3)

    def change(ctx):
        ctx.set_params(eta=0.1, eta_s=0.01, dt_max=1.0 / 16, dt_min=2.0 ** -40)

    S0, c0 = _run(m, x, v, 1e-4, 6, nb.NB_FP64, 0, [1.0 / 64, 1.0 / 32], between=change)
    S1, c1 = _run(m, x, v, 1e-4, 6, nb.NB_FP64, 3, [1.0 / 64, 1.0 / 32], between=change)
    assert c0 == c1
    _same(S0, S1)


def test_graph_no_block_before_t_end_and_bad_argument():
    n = 300
    m, x, v = ics.plummer(n, 2)
    ctx = make_ctx(m, x, v, 1e-4, 6, nb.NB_MIXED)
    ctx.set_graph(4)
    assert ctx.step_until(0.0) == (0, 0)
    before = ctx.get_state()
    assert ctx.step_until(-1.0) == (0, 0)
    _same(before, ctx.get_state())
    with pytest.raises(nb.NBError):
        ctx.set_graph(-1)
    ctx.set_graph(0)
    nblk, _ = ctx.step_until(1.0 / 128)
    assert nblk > 0
    ctx.close()


def test_nact_histogram_counts_every_block_in_both_modes():
    # host-driven block steps, n_act read per step, against the device count;
    # then graph replays: the same blocks, so the same histogram
    n = 1531
    m, x, v = ics.plummer(n, 29)
    t_end = 1.0 / 32
    hists = []
    for cycles in (0, 7):
        ctx = make_ctx(m, x, v, 1e-4, 6, nb.NB_MIXED)
        ctx.get_nact_histogram(reset=True)
        expect = np.zeros(nb.NB_NACT_CLASSES, dtype=np.int64)
        if cycles == 0:
            while True:
                tb, na = ctx.next_block()
                if tb > t_end:
                    break
                ctx.block_step()
                expect[int(na).bit_length() - 1] += 1
            h = ctx.get_nact_histogram()
            assert np.array_equal(h, expect)
        else:
            ctx.set_graph(cycles)
            blocks, _ = ctx.step_until(t_end)
            h = ctx.get_nact_histogram(reset=True)
            assert h.sum() == blocks
            assert ctx.get_nact_histogram().sum() == 0
        hists.append(h)
        ctx.close()
    assert np.array_equal(hists[0], hists[1]) and hists[0].sum() > 20
