"""bench.py with several processes (torchrun, one per GPU): every rank times its own replica
and rank 0 reports the slowest rank's times.  The aggregation is checked here on CPU with two
gloo processes."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: step time 10 + r ms, filter time 5 - r ms
        out[rank] = bench.max_over_ranks([10.0 + rank, 5.0 - rank], dist, "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_two_ranks():
    world = 2
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == [11.0, 5.0]


def test_single_process_passes_values_through():
    import bench

    assert bench.max_over_ranks([3, 4.5], None, "cpu") == [3.0, 4.5]
