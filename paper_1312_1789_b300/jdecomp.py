"""j decomposition of the block step across ranks (one GPU per rank).

The paper's code runs on many GPUs with MPI ("Codes description"; the
log(N_GPU) communication term of its performance model): every GPU holds all
particles and computes, for the active particles of the block, the force of
its own share of the j particles; the partial forces are summed across the
GPUs once per block, and the corrector runs on the summed force.  Here:

  rank r owns the j tiles [r T / G, (r + 1) T / G) of the store (T tiles of
  NB_JTILE particles, G ranks), via nb_set_jrange;
  every rank schedules the same active set (replicated state, identical
  arithmetic), predicts its own j particles and the active ones, forces the
  active set from its own j particles, copies its partial result
  (nb_copy_force), takes part in ONE all-gather of the G partial results,
  adds them in rank order on the device (nb_reduce_force) and corrects.

Every rank adds the same parts in the same order, so the ranks' states stay
bit for bit identical; with one j-split per rank the summed force is also bit
for bit that of one rank with G j-splits (nb.h, nb_set_jrange).  The exchange
is an all-gather rather than an all-reduce so that the order of the sum is
fixed (an all-reduce may add in any order); it moves G times the bytes of an
all-reduce, N_act x ncomp doubles per rank.

This module only drives the C ABI and the collective: all arithmetic runs in
libnb's kernels.  `gather` is the exchange: by default torch.distributed's
all_gather on the process group; tests on one device pass their own.
"""
from __future__ import annotations

from . import nb


def jranges(n: int, world: int, tile: int = nb.NB_JTILE):
    """Contiguous, tile-aligned j ranges [(j_begin, j_end)] of the G ranks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    tiles = (n + tile - 1) // tile
    out = []
    for r in range(world):
        t0, t1 = r * tiles // world, (r + 1) * tiles // world
        out.append((min(t0 * tile, n), min(t1 * tile, n)))
    return out


def torch_all_gather(group=None):
    """The exchange over a torch.distributed process group: all_gather of one
    [ncomp][n_act] tensor per rank into [world][ncomp][n_act]."""
    import torch
    import torch.distributed as dist

    def gather(part):
        world = dist.get_world_size(group)
        out = torch.empty((world,) + tuple(part.shape), dtype=part.dtype, device=part.device)
        # a list of views into one buffer: every backend (NCCL, and gloo on the
        # CPU) implements the list form
        dist.all_gather(list(out.unbind(0)), part.contiguous(), group=group)
        return out

    return gather


class JDecomposedStep:
    """Block steps of one rank of a j-decomposed run.

    ctx: this rank's nb.NBody, holding every particle (the same state on all
    ranks); rank, world: this rank and the number of ranks; gather: the
    exchange (see torch_all_gather); one_split: one j-split per rank (the
    force is then bitwise that of one rank with `world` splits)."""

    def __init__(self, ctx, rank: int, world: int, gather=None, one_split: bool = False, device=None):
        import torch
        if not 0 <= rank < world:
            raise ValueError("rank must lie in [0, world)")
        self.ctx, self.rank, self.world = ctx, rank, world
        self.range = jranges(ctx.n, world)[rank]
        self.gather = gather or torch_all_gather()
        self.device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        if world > 1:
            if self.range[1] <= self.range[0]:
                raise ValueError(f"rank {rank} of {world} owns no j tile of {ctx.n} particles")
            ctx.set_jrange(*self.range)
        if one_split:
            ctx.set_jsplit(1)
        self._part = None

    def begin_block(self):
        """Schedule, predict and force this rank's share; returns the partial
        result [ncomp][n_act] (a device tensor) to exchange, and (t_blk, n_act)."""
        import torch
        ctx = self.ctx
        tb, na = ctx.next_block()
        ctx.predict(tb)
        ctx.force(n_act=na)
        nc = 3 * (ctx.order // 2) + 2
        self._part = torch.empty((nc, na), dtype=torch.float64, device=self.device)
        ctx.copy_force(self._part)
        return self._part, (tb, na)

    def finish_block(self, parts):
        """Sum the exchanged parts [world][ncomp][n_act] in rank order and correct."""
        if parts.shape[0] != self.world:
            raise ValueError("one part per rank expected")
        self.ctx.reduce_force(parts, self.world)
        self.ctx.correct()
        self._part = None

    def block_step(self):
        part, (tb, na) = self.begin_block()
        self.finish_block(self.gather(part))
        return tb, na

    def step_until(self, t_end: float):
        """Block steps until the next block would pass t_end; returns the block
        count.  Every rank takes the same blocks (their states are identical)."""
        import math
        blocks = 0
        while True:
            tb, _ = self.ctx.next_block()
            if tb > t_end or not math.isfinite(tb):
                return blocks
            self.block_step()
            blocks += 1
