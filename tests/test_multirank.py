"""The bench's multi-process path on CPU: two ranks over gloo (127.0.0.1)
meet at a barrier, reduce their timings to the slowest rank's, and compute
the whole-job rate from it (ranks are independent replicas: no collective on
the data path, so this is the only cross-rank step)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    dist.barrier()
    slowest = bench.max_over_ranks(1.5 + rank, world)
    rate = bench.whole_job_rate(1024, 20, world, slowest)
    dist.barrier()
    q.put((rank, slowest, rate))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_ranks_reduce_to_the_slowest(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    slowest = 1.5 + (world - 1)
    for rank, s, rate in got:
        assert s == slowest
        assert rate == pytest.approx(1024 * 20 * world / slowest)


def test_single_rank_is_its_own_max():
    import bench

    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.whole_job_rate(10, 4, 1, 2.0) == 20.0
