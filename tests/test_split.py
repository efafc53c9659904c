"""The split of one population's dominance columns over ranks
(paper_2503_20286_gb300.split), with two and three gloo ranks on the CPU:
the front exchange gives every rank the oracle's ranks (Deb's sort,
Algorithm S.2) and the oracle's survivors, including a rank that owns no
column block and populations with ties and duplicates."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2503_20286_gb300 import split
from paper_2503_20286_gb300 import workloads as wl


def test_column_ranges_cover_in_blocks():
    for n2, world in [(1, 1), (1024, 2), (2500, 3), (5000, 2), (400000, 8), (1500, 3)]:
        r = split.column_ranges(n2, world)
        assert r[0][0] == 0 and r[-1][1] == n2
        for (a, b), (c, d) in zip(r, r[1:]):
            assert b == c
        assert all(a % 1024 == 0 and a <= b for a, b in r)
    assert split.column_ranges(1500, 3)[0] == (0, 0)  # two blocks, three ranks: one owns none


def test_bit_packing_round_trip():
    rng = np.random.default_rng(0)
    for n in (1, 7, 8, 9, 1000):
        f = torch.from_numpy(rng.integers(0, 2, n).astype(np.uint8))
        assert torch.equal(split.unpack_bits(split.pack_bits(f, torch), n, torch).to(torch.uint8), f)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, case, out):
    from tests._split_numpy import NumpyOps
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        F, R, n_keep, seed, gen = case
        lo, hi = split.column_ranges(F.shape[0], world)[rank]
        surv, _, ranks = split.run(torch.from_numpy(F[lo:hi].copy()), torch.from_numpy(R), n_keep, seed, gen,
                                   NumpyOps(), F.shape[0])
        out[rank]["surv"] = surv.numpy().tolist()
        out[rank]["ranks"] = ranks.numpy().tolist()
    finally:
        dist.destroy_process_group()


def _cases():
    p0 = wl.config(0)
    F1 = wl.population(2500, 5, 14, "linear", seed=61, quantize=8.0)
    F2 = wl.population(1500, 3, 9, "sphere", seed=62)
    return [(p0.F, p0.R, p0.n_keep, p0.seed, 0),
            (F1, wl.das_dennis(5, 5), 1200, 7, 3),
            (F2, wl.das_dennis(12, 3), 750, 9, 1)]


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("ci", range(3))
def test_gloo_ranks_equal_the_oracle(world, ci):
    case = _cases()[ci]
    F, R, n_keep, seed, gen = case
    with mp.Manager() as mgr:
        out = [mgr.dict() for _ in range(world)]
        mp.spawn(_rank_main, args=(world, _free_port(), case, out), nprocs=world, join=True)
        res = [dict(o) for o in out]
    ref_surv, t = oracle.nsga3_select(F, R, n_keep, seed, gen)
    l = t["last_rank"]
    for r in res:
        ranks = np.asarray(r["ranks"])
        assert np.array_equal(ranks[t["rank"] <= l], t["rank"][t["rank"] <= l])
        assert np.all(ranks[t["rank"] > l] == split.NOT_RANKED)
        assert np.array_equal(np.asarray(r["surv"]), ref_surv)
