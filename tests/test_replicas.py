"""Several ranks (replicas of independent populations): the batch split over
ranks and the whole-job timing, with two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2503_20286_gb300 import workloads as wl
from paper_2503_20286_gb300.replicas import max_over_ranks, shard_populations


def test_shard_populations_covers_and_balances():
    sizes = [p.F.shape[0] for p in wl.config(3)]   # 64 uneven populations
    for world in (1, 2, 3, 8):
        shards = shard_populations(sizes, world)
        assert sorted(i for s in shards for i in s) == list(range(len(sizes)))
        load = [sum(sizes[i] ** 2 for i in s) for s in shards]
        # longest-first greedy: no rank exceeds the mean by more than the largest item
        assert max(load) <= sum(load) / world + max(x ** 2 for x in sizes)
    assert shard_populations(sizes, 4) == shard_populations(sizes, 4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, sizes, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # whole-job time = the slowest rank's time
        out[rank * 2] = max_over_ranks(10.0 + 5.0 * rank)
        # each rank selects its own shard; together the shards cover the batch once
        mine = shard_populations(sizes, world)[rank]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        flat = sorted(i for s in gathered for i in s)
        out[rank * 2 + 1] = float(flat == list(range(len(sizes))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_and_shards():
    sizes = [p.F.shape[0] for p in wl.config(3)]
    out = torch.zeros(4, dtype=torch.float64).share_memory_()
    mp.spawn(_rank_main, args=(2, _free_port(), sizes, out), nprocs=2, join=True)
    assert out.tolist() == [15.0, 1.0, 15.0, 1.0]


def test_single_process_max_is_identity():
    assert max_over_ranks(3.5) == 3.5
