"""Host logic of the multi-GPU bench path (independent replicas) on CPU:
two gloo ranks check the view partition and the max-over-ranks throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        views = bench.rank_views(8, rank, world)
        local_ms = 10.0 * (rank + 1)                 # rank 1 is the slow one
        rate, ms = bench.job_rate(local_ms, 640000, 3, world, "cpu")
        q.put((rank, views, rate, ms))
    finally:
        dist.destroy_process_group()


def test_two_rank_rate_and_views():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time and the whole job's rays
    for rank, views, rate, ms in res:
        assert ms == 20.0
        assert rate == pytest.approx(world * 640000 * 3 / 0.020)
    # each rank's first `steps` views are distinct, and the ranks' first views differ
    v0, v1 = res[0][1], res[1][1]
    assert v0[:4] == [0, 2, 4, 6] and v1[:4] == [1, 3, 5, 7]
    assert not set(v0[:4]) & set(v1[:4])


def test_single_rank_rate():
    import bench
    rate, ms = bench.job_rate(4.0, 1000, 2, 1, "cpu")
    assert ms == 4.0 and rate == pytest.approx(1000 * 2 / 0.004)
