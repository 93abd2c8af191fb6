"""The replicas path of bench.py across ranks, on the CPU with gloo (two
ranks): each rank's events are summed and its times maxed, and each rank
runs its own Philox seed."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sums, maxes = bench.reduce_over_ranks([1000 * (rank + 1), rank + 0.5],
                                              [2.0 + rank, 7.0 - rank], "cpu")
        assert sums == [3000.0, 2.0], sums
        assert maxes == [3.0, 7.0], maxes
        seeds = [bench.rank_seed(0xEC0005, r) for r in range(world)]
        assert len(set(seeds)) == world and seeds[rank] == 0xEC0005 + rank
    finally:
        dist.destroy_process_group()


def test_replicas_reduce_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port()), nprocs=2, join=True)
