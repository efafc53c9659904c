"""Several GPUs: independent populations per rank, no collective on the data
path (one population's selection does not shard in this library).

Host helpers for callers that spread a batch of populations over the ranks
of a process group, and for timing a replicated run (the whole-job time is
the slowest rank's).
"""
from __future__ import annotations


def shard_populations(sizes, world: int) -> list[list[int]]:
    """Indices of the populations (``sizes`` = their 2N) each of ``world``
    ranks selects: longest first to the least-loaded rank, the load being the
    dominant cost (2N)^2 of a population (its dominance tiles and peel).
    Every index appears once; each list is ascending."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]) ** 2, i))
    load = [0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += int(sizes[i]) ** 2
        out[r].append(i)
    return [sorted(o) for o in out]


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of ``value`` over the ranks of the default process group
    (``value`` itself when no group of more than one rank is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
