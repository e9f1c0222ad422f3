"""The replica path of bench.py (N > 1 under torchrun: one independent pair per
rank, max-over-ranks timing, whole-job rate) on two gloo ranks on the CPU."""

import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                       # rank 1 is the slowest
        slowest = bench.max_over_ranks(ms, dist, torch.device("cpu"))
        dist.barrier()
        out[rank] = (bench.pair_seed(rank), slowest, bench.job_rate(world, slowest))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    world = 2
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    seeds = [out[r][0] for r in range(world)]
    assert len(set(seeds)) == world                 # every rank registers its own pair
    for r in range(world):
        assert out[r][1] == pytest.approx(15.0)     # the slowest rank's time on every rank
        assert out[r][2] == pytest.approx(world * 1000.0 / 15.0)


def test_single_process_is_the_identity():
    import bench
    assert bench.max_over_ranks(12.5, None, None) == 12.5
    assert bench.job_rate(1, 100.0) == pytest.approx(10.0)
