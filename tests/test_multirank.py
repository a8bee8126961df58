"""The multi-rank leg of the benchmark (independent replicas, one per rank):
the whole-job number takes the slowest rank's time and every rank's work.
Run as two gloo ranks on the CPU (no GPU, no collective on the data path)."""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value, w = bench.aggregate(100.0 * (rank + 1), steps=4, inter_per_step=1e9, dist=dist, device="cpu")
    q.put((rank, ms, value, w))
    dist.destroy_process_group()


def test_two_rank_aggregate_takes_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29000 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, w in res:
        assert w == 2
        assert ms == pytest.approx(200.0)
        assert value == pytest.approx(2 * 4 * 1e9 / 0.2)


def test_single_process_aggregate_is_local():
    import bench
    ms, value, w = bench.aggregate(50.0, steps=2, inter_per_step=1e6)
    assert (ms, w) == (50.0, 1) and value == pytest.approx(4e7)
