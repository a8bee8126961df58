"""Host logic of the j decomposition across ranks (paper_1312_1789_b300.jdecomp):
the split of the j particles into the ranks' tile ranges, the one exchange per
block (an all-gather over a gloo process group of two CPU ranks), the sum of
the parts in rank order and the replicated corrector.

The ranks drive a stand-in context with the C ABI's call sequence whose
"force" is a tile-ordered sum of simple pair terms in float64 and whose
"corrector" moves the particles with it, so that the test checks the
orchestration, not the physics: both ranks must end in the same state bit for
bit, equal to one rank that sums the same tiles as G j-splits."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1312_1789_b300 import jdecomp

JT = 128


class StandIn:
    """The calls JDecomposedStep makes, on the CPU."""

    def __init__(self, n, seed=3):
        rng = np.random.default_rng(seed)
        self.n, self.order = n, 6
        self.x = rng.uniform(-1, 1, n)
        self.m = rng.uniform(0.5, 1.5, n) / n
        self.t = 0.0
        self.jr = (0, n)
        self.js = 0
        self.F = None
        self.calls = []

    def set_jrange(self, jb, je):
        assert jb % JT == 0 and (je % JT == 0 or je == self.n)
        self.jr = (jb, je)

    def set_jsplit(self, js):
        self.js = js

    def next_block(self):
        return self.t + 0.01, self.n

    def predict(self, t):
        self.calls.append("predict")

    def force(self, n_act=0):
        # tiles of the range, split into js parts as the kernels split them;
        # each split sums its tiles in order, the splits are added in order
        t0, t1 = self.jr[0] // JT, (self.jr[1] + JT - 1) // JT
        nt, js = t1 - t0, max(self.js, 1)
        nc = 11
        total = np.zeros((nc, self.n))
        for s in range(js):
            a, b = t0 + s * nt // js, t0 + (s + 1) * nt // js
            part = np.zeros((nc, self.n))
            for tile in range(a, b):
                j = np.arange(tile * JT, min((tile + 1) * JT, self.n))
                d = self.x[j][None, :] - self.x[:, None]
                term = self.m[j][None, :] * np.tanh(d)
                for c in range(nc):
                    part[c] += (term * (c + 1)).sum(axis=1)
            total = part if s == 0 else total + part
        self.F = total
        self.calls.append("force")

    def copy_force(self, dst):
        dst.copy_(torch.from_numpy(self.F))
        return self.F.shape

    def reduce_force(self, parts, n_parts):
        p = parts.numpy()
        acc = p[0].copy()
        for r in range(1, n_parts):
            acc = acc + p[r]
        self.F = acc
        self.calls.append("reduce")

    def correct(self):
        self.x = self.x + 1e-3 * self.F[0]
        self.t += 0.01
        self.calls.append("correct")


@pytest.mark.parametrize("n", [1, 127, 128, 129, 1000, 4096, 65537])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_jranges_cover_every_tile_once_in_rank_order(n, world):
    r = jdecomp.jranges(n, world)
    assert len(r) == world and r[0][0] == 0 and r[-1][1] == n
    for (a, b), (c, d) in zip(r, r[1:]):
        assert b == c
    for a, b in r:
        assert a % JT == 0 and (b % JT == 0 or b == n) and a <= b
    tiles = (n + JT - 1) // JT
    sizes = [(b - a + JT - 1) // JT for a, b in r]
    assert sum(sizes) == tiles and max(sizes) - min(sizes) <= 1


def test_rank_without_tiles_is_refused():
    with pytest.raises(ValueError):
        jdecomp.JDecomposedStep(StandIn(100), 0, 2, gather=lambda p: p, device="cpu")


def _rank(rank, world, port, q, steps):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ctx = StandIn(1000)
    step = jdecomp.JDecomposedStep(ctx, rank, world, gather=jdecomp.torch_all_gather(), one_split=True,
                                   device="cpu")
    for _ in range(steps):
        step.block_step()
    q.put((rank, ctx.x.copy(), ctx.jr, ctx.calls[:4]))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_equal_one_rank_with_world_splits(world):
    steps = 5
    mpc = mp.get_context("spawn")
    q = mpc.Queue()
    port = 29500 + (os.getpid() * 7 + world) % 1000
    procs = [mpc.Process(target=_rank, args=(r, world, port, q, steps)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[2] for r in res] == jdecomp.jranges(1000, world)
    assert res[0][3] == ["predict", "force", "reduce", "correct"]
    for r in res[1:]:
        assert np.array_equal(r[1], res[0][1])
    # one rank, the same tiles as `world` j-splits: the same bits
    ref = StandIn(1000)
    ref.set_jsplit(world)
    for _ in range(steps):
        ref.predict(0.0)
        ref.force()
        ref.correct()
    assert np.array_equal(res[0][1], ref.x)
