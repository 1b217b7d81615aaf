"""Multi-rank host logic on CPU: two gloo ranks reduce their throughput the
way bench.py does under torchrun (sum of work over the slowest rank)."""
import os
import socket

import pytest

from paper_1603_02421_gb300.replicas import rank_members, reduce_rate


def test_rank_members_partition():
    world, n = 3, 10
    got = sorted(m for r in range(world) for m in rank_members(r, world, n))
    assert got == list(range(n))
    assert rank_members(1, 3, 10) == [1, 4, 7]
    with pytest.raises(ValueError):
        rank_members(3, 3, 10)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = [2.0, 3.0][rank]
    units = [100.0, 50.0][rank]
    out[rank] = reduce_rate(seconds, units, dist)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_rate_two_gloo_ranks():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        rate, tmax, units = out[r]
        assert tmax == 3.0 and units == 150.0 and rate == pytest.approx(50.0)


def test_reduce_rate_single_process():
    assert reduce_rate(2.0, 10.0) == (5.0, 2.0, 10.0)
