"""Ensembles (nb_batch_*): independent clusters advanced together with one
launch per kernel; each cluster must evolve exactly as if it were alone."""
import numpy as np
import pytest

import oracle as orc
from paper_1312_1789_b300 import ics, nb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1312_1789_b300 import build
    build.build()
    nb.lib()


def _clusters(sizes, eps=1e-4):
    ms, xs, vs = [], [], []
    for k, n in enumerate(sizes):
        m, x, v = ics.plummer(int(n), 500 + k)
        ms.append(m)
        xs.append(x)
        vs.append(v)
    return ms, xs, vs


@pytest.mark.parametrize("graph", [0, 7], ids=["host_cycles", "graph_cycles"])
@pytest.mark.parametrize("order", [4, 6, 8])
def test_batch_fp64_matches_each_cluster_alone(order, graph):
    # Ragged cluster sizes (not multiples of the 128-record tile, one below it);
    # cycles checked on the host one by one, or replayed 7 at a time as a graph.
    sizes = [300, 129, 1000, 64, 700]
    ms, xs, vs = _clusters(sizes)
    eta = 0.02 if order == 4 else 0.2
    b = nb.Batch(sizes, order, 1e-4, nb.NB_FP64)
    b.set_params(eta, 0.01, 1.0 / 16, 2.0 ** -40)
    b.set_graph(graph)
    b.set_particles(np.concatenate(ms), np.concatenate(xs), np.concatenate(vs))
    ncyc, ninter = b.step_until(1.0 / 16)
    assert ncyc > 0 and ninter > 0
    S = b.get_state()
    assert np.all(S["t"] == 1.0 / 16)
    off = 0
    for k, n in enumerate(sizes):
        st = orc.State(ms[k], 1e-8, xs[k], vs[k])
        orc.integrate(st, order=order, t_end=1.0 / 16, eta=eta, nthreads=16)
        sl = slice(off, off + n)
        assert np.array_equal(S["dt"][sl], st.dt), f"cluster {k}: steps differ"
        assert np.max(np.abs(S["x"][sl] - st.x)) < 1e-11, f"cluster {k}"
        assert np.max(np.abs(S["v"][sl] - st.v)) < 1e-10, f"cluster {k}"
        off += n
    b.close()


@pytest.mark.parametrize("prec", [nb.NB_FP64, nb.NB_MIXED])
def test_batch_energy_per_cluster(prec):
    sizes = [500, 257, 900]
    ms, xs, vs = _clusters(sizes)
    b = nb.Batch(sizes, 6, 1e-4, prec)
    b.set_particles(np.concatenate(ms), np.concatenate(xs), np.concatenate(vs))
    ek, ep = b.energy()
    for k in range(len(sizes)):
        ek_o, ep_o = orc.energy(ms[k], 1e-8, xs[k], vs[k])
        assert ek[k] == pytest.approx(ek_o, rel=1e-14)
        assert ep[k] == pytest.approx(ep_o, rel=1e-13 if prec == nb.NB_FP64 else 1e-6)
    e0 = ek + ep
    b.step_until(1.0 / 16)
    ek, ep = b.energy()
    de = (ek + ep - e0) / np.abs(e0)
    assert np.all(np.abs(de) < 1e-6), de
    b.close()


def test_batch_matches_separate_contexts_mixed():
    # The ensemble path and one context per cluster take the same blocks; the
    # mixed forces of both use the same kernels, so states agree to rounding.
    sizes = [640, 384, 1100]
    ms, xs, vs = _clusters(sizes)
    b = nb.Batch(sizes, 6, 1e-4, nb.NB_MIXED)
    b.set_particles(np.concatenate(ms), np.concatenate(xs), np.concatenate(vs))
    b.step_until(1.0 / 32)
    S = b.get_state()
    off = 0
    for k, n in enumerate(sizes):
        c = nb.NBody(n, 6, 1e-4, nb.NB_MIXED)
        c.set_particles(ms[k], xs[k], vs[k])
        c.step_until(1.0 / 32)
        R = c.get_state()
        sl = slice(off, off + n)
        assert np.max(np.abs(S["x"][sl] - R["x"])) < 1e-9
        assert np.mean(S["dt"][sl] == R["dt"]) > 0.99
        c.close()
        off += n
    b.close()


@pytest.mark.parametrize("prec", [nb.NB_FP64, nb.NB_MIXED])
def test_batch_graph_cycles_match_host_cycles_bitwise(prec):
    # The device plans every cycle in both modes, so a graph replay of the
    # cycles reproduces the host-checked cycles bit for bit, including the
    # cycles where only some clusters step and the idle tail past t_end.
    sizes = [2000, 130, 5, 900, 3000, 64]
    ms, xs, vs = _clusters(sizes)
    out = []
    for cycles in (0, 9):
        b = nb.Batch(sizes, 6, 1e-4, prec)
        b.set_graph(cycles)
        b.set_particles(np.concatenate(ms), np.concatenate(xs), np.concatenate(vs))
        first = b.step_until(1.0 / 64)
        second = b.step_until(1.0 / 32)
        out.append(((first, second), b.get_state()))
        b.close()
    (c0, s0), (c1, s1) = out
    assert c0 == c1 and c0[0][0] > 0
    for key in ("x", "v", "t", "dt"):
        assert np.array_equal(s0[key], s1[key]), key


@pytest.mark.parametrize("waves", [1, 8])
def test_batch_fp64_other_wave_counts_match_each_cluster_alone(waves):
    # The plan's wave count changes only how the work is cut into items (and
    # so the split sums' order): the steps stay the oracle's.
    sizes = [300, 129, 1000, 64, 700]
    ms, xs, vs = _clusters(sizes)
    b = nb.Batch(sizes, 6, 1e-4, nb.NB_FP64)
    b.set_waves(waves)
    assert b.get_waves() == waves
    b.set_graph(5)
    b.set_particles(np.concatenate(ms), np.concatenate(xs), np.concatenate(vs))
    b.step_until(1.0 / 16)
    S = b.get_state()
    off = 0
    for k, n in enumerate(sizes):
        st = orc.State(ms[k], 1e-8, xs[k], vs[k])
        orc.integrate(st, order=6, t_end=1.0 / 16, eta=0.2, nthreads=16)
        sl = slice(off, off + n)
        assert np.array_equal(S["dt"][sl], st.dt), f"cluster {k}: steps differ"
        assert np.max(np.abs(S["x"][sl] - st.x)) < 1e-11, f"cluster {k}"
        off += n
    with pytest.raises(nb.NBError):
        b.set_waves(9)
    b.close()


def test_batch_autotune_cycles_are_the_runs_own_cycles():
    # The tuning cycles complete with the wave count in use, so after tuning
    # for k cycles the state is that of k host-checked cycles; the chosen
    # count is one of the candidates and every candidate was timed.
    sizes = [2000, 130, 5, 900, 3000, 64]
    ms, xs, vs = _clusters(sizes)
    states = []
    for tune in (True, False):
        b = nb.Batch(sizes, 6, 1e-4, nb.NB_MIXED)
        b.set_particles(np.concatenate(ms), np.concatenate(xs), np.concatenate(vs))
        if tune:
            w, ms_per = b.autotune(cycles=6, reps=1)
            assert w in (1, 2, 4, 8) and all(v > 0 for v in ms_per.values())
        else:
            for _ in range(6):
                b.cycle(1e9)
        states.append(b.get_state())
        b.close()
    for key in ("x", "v", "t", "dt"):
        assert np.array_equal(states[0][key], states[1][key]), key
