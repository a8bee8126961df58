"""j decomposition through the C ABI on one GPU: G ranks emulated in one
process, in lockstep (each rank forces its j range, the parts are stacked as
the all-gather would deliver them, every rank adds them with nb_reduce_force
and corrects).  With one j-split per rank the summed force and the states
after several block steps equal, bit for bit, those of one context with G
j-splits; and the force agrees with the oracle."""
import numpy as np
import pytest

from gpu_common import assert_force_close, make_ctx, oracle_force_on_predicted
from paper_1312_1789_b300 import ics, jdecomp, nb

pytestmark = pytest.mark.gpu


def _system(n):
    m, x, v = ics.plummer(n - 2, 77)
    mb, xb, vb = ics.bh_circular_pair(0.005, 0.1)
    eps2 = np.concatenate([np.full(n - 2, 1e-8), np.zeros(2)])
    return np.concatenate([m, mb]), np.concatenate([x, xb]), np.concatenate([v, vb]), eps2


@pytest.mark.parametrize("prec", [nb.NB_FP64, nb.NB_MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("world", [2, 3])
def test_lockstep_ranks_equal_one_context_with_world_splits(prec, world):
    import torch
    n = 5 * 128 + 61
    m, x, v, eps2 = _system(n)
    single = make_ctx(m, x, v, eps2, 6, prec, pair=True)
    single.set_jsplit(world)
    ranks = []
    for r in range(world):
        c = make_ctx(m, x, v, eps2, 6, prec, pair=True)
        ranks.append(jdecomp.JDecomposedStep(c, r, world, gather=None, one_split=True))
    assert [s.range for s in ranks] == jdecomp.jranges(n, world)
    for blk in range(6):
        tb, idx = single.next_block(want_idx=True)
        single.predict(tb)
        single.force()
        F1 = single.get_force(len(idx))
        if blk == 0:
            O = oracle_force_on_predicted(single, m, eps2, idx.astype(np.int32), 6)
            assert_force_close(F1, O, 6, prec, f"world {world} reference")
        parts = []
        for s in ranks:
            part, (tb_r, na_r) = s.begin_block()
            assert tb_r == tb and na_r == len(idx)
            parts.append(part)
        stacked = torch.stack(parts)
        for s in ranks:
            s.ctx.reduce_force(stacked, world)
            Fr = s.ctx.get_force(len(idx))
            for key in F1:
                assert np.array_equal(Fr[key], F1[key]), (blk, s.rank, key)
            s.ctx.correct()
        single.correct()
    S1 = single.get_state()
    for s in ranks:
        Sr = s.ctx.get_state()
        for key in ("x", "v", "t", "dt"):
            assert np.array_equal(Sr[key], S1[key]), (s.rank, key)
        s.ctx.close()
    single.close()


def test_ranged_prediction_covers_the_share_and_the_block_only():
    # each rank predicts its own j tiles and the block's active particles;
    # the other records keep the previous prediction, which the restricted
    # force never reads
    n = 4 * 128 + 33
    m, x, v, eps2 = _system(n)
    c = make_ctx(m, x, v, eps2, 6, nb.NB_MIXED, pair=True)
    c.predict(0.0)
    before = c.get_predicted()[0]
    jb, je = 128, 384
    c.set_jrange(jb, je)
    tb, idx = c.next_block(want_idx=True)
    c.predict(tb)
    after = c.get_predicted()[0]
    full = make_ctx(m, x, v, eps2, 6, nb.NB_MIXED, pair=True)
    full.predict(tb)
    ref = full.get_predicted()[0]
    covered = np.zeros(n, bool)
    covered[jb:je] = True
    covered[idx] = True
    assert (~covered).any() and len(idx) < n
    assert np.array_equal(after[covered], ref[covered])
    assert np.array_equal(after[~covered], before[~covered])
    with pytest.raises(nb.NBError) as e:
        c.force(idx.astype(np.int32))
    assert e.value.code == nb.NB_ERR_ARG
    c.force()
    # a new share needs a new prediction
    c.set_jrange(0, 128)
    with pytest.raises(nb.NBError):
        c.force()
    # back to the whole range: a block step predicts every particle again, and
    # an explicit list is accepted afterwards
    c.set_jrange(0, 0)
    c.block_step()
    c.predict(c.next_block()[0])
    c.force(np.arange(n, dtype=np.int32))
    c.close()
    full.close()


def test_jrange_rules():
    n = 3 * 128 + 5
    m, x, v, eps2 = _system(n)
    c = make_ctx(m, x, v, eps2, 6, nb.NB_MIXED, pair=True)
    for bad in ((1, 128), (0, 100), (128, 128), (-128, 128), (256, n + 1)):
        with pytest.raises(nb.NBError):
            c.set_jrange(*bad)
    c.set_jrange(128, n)
    with pytest.raises(nb.NBError):
        c.block_step()
    with pytest.raises(nb.NBError):
        c.step_until(1.0 / 16)
    with pytest.raises(nb.NBError):
        c.set_graph(8)
    with pytest.raises(nb.NBError):
        c.autotune(1)
    # the range restricts the force only: the energy still sums every pair
    ek, ep = c.energy()
    c.set_jrange(0, 0)
    assert c.energy() == (ek, ep)
    c.close()
