"""One population over several GPUs: the columns of its dominance matrix split
over the ranks of a process group.

Rank r owns a contiguous range of 1024-column blocks of the (caller-order)
dominance matrix, holds D[:, its columns] and their dominator counts, and
peels fronts in step with the others (Algorithm S.3 with the front exchanged
after every step):

1. all-gather of the objectives (each rank brings the rows of its columns);
2. ``emo_dominance_cols``: D for the rank's columns, every row, and the
   dominator count of each column;
3. per front k: the rank's new front members as a bit mask over its columns,
   all-gathered (2N / 8 bytes per front in all) into the front; every rank
   records rank k for its members, and, unless the fronts so far already
   hold n_keep points (then l = k), ``emo_front_counts`` subtracts the
   front's rows from its columns' counts and flags the next front there;
4. ``emo_nsga3_associate_range``: every rank normalises over all of S (the
   same ideal point, extreme points and intercepts everywhere, from the
   gathered objectives) and associates the points of S in its columns;
   the niche counts of its points of P are summed over the ranks (an
   all-reduce of n_r counts) and the references and distances of its
   members of front l are all-gathered (front l is known to every rank, so
   its members' owners are too);
5. ``emo_nsga3_niche_given``: the niching and the survivors from the summed
   counts and front l's association, run by every rank on the same data, so
   every rank returns the same survivors.

The exchange is written once as a generator of collective steps; ``run``
drives it over a torch.distributed process group (NCCL between GPUs, gloo on
CPU tensors), ``run_virtual`` drives several ranks of it in one process (the
collectives become lists and sums), which checks the same exchange on one
device. The per-rank arithmetic comes from an ``ops`` object: ``GpuOps``
calls the library's kernels; nothing here computes on the host.
"""
from __future__ import annotations

import numpy as np

NOT_RANKED = 2147483647
BLOCK = 1024


def column_ranges(n2: int, world: int) -> list[tuple[int, int]]:
    """Columns [lo, hi) of each rank: contiguous runs of 1024-column blocks,
    as equal as the block count allows (every column of the caller-order
    matrix costs the same); a rank may own none when there are more ranks
    than blocks."""
    if world < 1 or n2 < 1:
        raise ValueError("world and n2 must be >= 1")
    ncb = -(-n2 // BLOCK)
    out = []
    for r in range(world):
        b0, b1 = ncb * r // world, ncb * (r + 1) // world
        out.append((min(n2, b0 * BLOCK), min(n2, b1 * BLOCK)))
    return out


def pack_bits(flags, torch):
    """uint8 0/1 flags -> bits (LSB first), padded to whole bytes."""
    n = flags.numel()
    pad = (-n) % 8
    f = torch.cat([flags.to(torch.int32), torch.zeros(pad, dtype=torch.int32, device=flags.device)]) if pad else \
        flags.to(torch.int32)
    w = (1 << torch.arange(8, dtype=torch.int32, device=flags.device))
    return (f.view(-1, 8) * w).sum(dim=1).to(torch.uint8)


def unpack_bits(packed, n: int, torch):
    """Inverse of pack_bits: the first n flags."""
    w = (1 << torch.arange(8, dtype=torch.int32, device=packed.device))
    return ((packed.to(torch.int32).view(-1, 1) & w) != 0).view(-1)[:n]


def steps(rank: int, world: int, F_own, R, n_keep: int, seed: int, generation: int, ops, torch):
    """The exchange of one rank as a generator: it yields ("all_gather", t)
    and receives the list of every rank's t (rank order), or ("all_reduce",
    t) and receives the elementwise sum over the ranks; it returns
    (survivors, info, ranks)."""
    ranges = column_ranges(int(ops.n2), world)
    lo, hi = ranges[rank]
    parts = yield ("all_gather", F_own)
    F = torch.cat(parts)
    n2 = F.shape[0]
    if n2 != ops.n2 or F_own.shape[0] != hi - lo:
        raise ValueError("every rank brings the rows of its own columns")
    max_cols = max(b - a for a, b in ranges)
    ncols = hi - lo
    if ncols:
        D, counts = ops.dominance_cols(F, lo, hi)
        flags = (counts == 0).to(torch.uint8)
    else:
        D = counts = None
        flags = torch.zeros(0, dtype=torch.uint8, device=F.device)
    ranks = torch.full((n2,), NOT_RANKED, dtype=torch.int32, device=F.device)
    total, k = 0, 0
    while True:
        padded = torch.zeros(max_cols, dtype=torch.uint8, device=F.device)
        padded[:ncols] = flags
        masks = yield ("all_gather", pack_bits(padded, torch))
        members = torch.cat([unpack_bits(msk, b - a, torch).nonzero().view(-1) + a
                             for msk, (a, b) in zip(masks, ranges)]).to(torch.int32)
        if members.numel() == 0:
            raise RuntimeError("an empty front before n_keep points: inconsistent dominator counts")
        ranks[members.long()] = k
        total += int(members.numel())
        if total >= n_keep:
            break
        if ncols:
            flags = ops.front_counts(D, ncols, members, counts)
        k += 1
    # members is front l = k, ascending; this rank's share of it
    pi, dist, rho = ops.associate_range(F, R, n_keep, ranks, lo, hi)
    rho_all = yield ("all_reduce", rho)
    own = members[(members >= lo) & (members < hi)].long() - lo
    max_own = max(int(((members >= a) & (members < b)).sum()) for a, b in ranges)
    pi_pad = torch.full((max_own,), -1, dtype=torch.int32, device=F.device)
    d_pad = torch.zeros(max_own, dtype=torch.float64, device=F.device)
    pi_pad[:own.numel()] = pi[own]
    d_pad[:own.numel()] = dist[own]
    pis = yield ("all_gather", pi_pad)
    ds = yield ("all_gather", d_pad)
    counts_l = [int(((members >= a) & (members < b)).sum()) for a, b in ranges]
    last_pi = torch.cat([p[:c] for p, c in zip(pis, counts_l)])
    last_d = torch.cat([x[:c] for x, c in zip(ds, counts_l)])
    survivors, info = ops.niche_given(n2, R.shape[0], n_keep, seed, generation, ranks, rho_all, members, last_pi,
                                      last_d)
    return survivors, info, ranks


def run(F_own, R, n_keep: int, seed: int, generation: int, ops, n2: int, group=None):
    """Selection of one population split over the ranks of a process group.
    F_own: the rows of this rank's columns (column_ranges(n2, world)[rank]);
    every rank returns the same survivors."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    ops.n2 = n2
    ranges = column_ranges(n2, world)
    gen = steps(rank, world, F_own, R, n_keep, seed, generation, ops, torch)
    msg = next(gen)
    while True:
        op, t = msg
        if op == "all_reduce":
            out = t.clone()
            dist.all_reduce(out, op=dist.ReduceOp.SUM, group=group)
            try:
                msg = gen.send(out)
            except StopIteration as e:
                return e.value
            continue
        if op != "all_gather":
            raise RuntimeError(op)
        if t.dim() == 2:  # the objectives: uneven row counts, padded to the largest
            rows = max(b - a for a, b in ranges)
            buf = torch.zeros((rows, t.shape[1]), dtype=t.dtype, device=t.device)
            buf[:t.shape[0]] = t
            out = [torch.empty_like(buf) for _ in range(world)]
            dist.all_gather(out, buf, group=group)
            out = [o[:b - a] for o, (a, b) in zip(out, ranges)]
        else:
            out = [torch.empty_like(t) for _ in range(world)]
            dist.all_gather(out, t.contiguous(), group=group)
        try:
            msg = gen.send(out)
        except StopIteration as e:
            return e.value


def run_virtual(F, R, n_keep: int, seed: int, generation: int, ops, world: int):
    """The same exchange for `world` ranks driven in one process on one
    device (each collective becomes the list of the ranks' tensors)."""
    import torch
    n2 = F.shape[0]
    ops.n2 = n2
    ranges = column_ranges(n2, world)
    gens = [steps(r, world, F[a:b], R, n_keep, seed, generation, ops, torch) for r, (a, b) in enumerate(ranges)]
    msgs = [next(g) for g in gens]
    results = [None] * world
    while True:
        ops_now = {m[0] for m in msgs}
        if len(ops_now) != 1:
            raise RuntimeError(f"ranks at different collectives: {ops_now}")
        payload = [m[1] for m in msgs]
        if ops_now == {"all_reduce"}:
            total = payload[0].clone()
            for t in payload[1:]:
                total += t
        nxt = []
        for r, g in enumerate(gens):
            try:
                nxt.append(g.send(total.clone() if ops_now == {"all_reduce"} else list(payload)))
            except StopIteration as e:
                results[r] = e.value
                nxt.append(None)
        if all(x is None for x in nxt):
            return results
        if any(x is None for x in nxt):
            raise RuntimeError("ranks left the exchange at different steps")
        msgs = nxt


class GpuOps:
    """The per-rank arithmetic of the split on this process's GPU: the
    library's kernels through the C ABI."""

    n2 = 0

    def __init__(self):
        from . import _binding as emo
        self.emo = emo

    def dominance_cols(self, F, lo, hi):
        return self.emo.emo_dominance_cols(F, lo, hi)

    def front_counts(self, D, ncols, members, counts):
        return self.emo.emo_front_counts(D, ncols, members, counts)

    def associate_range(self, F, R, n_keep, ranks, lo, hi):
        return self.emo.emo_nsga3_associate_range(F, R, n_keep, ranks, lo, hi)

    def niche_given(self, n2, n_r, n_keep, seed, generation, ranks, rho, last, last_pi, last_d):
        import torch
        info = torch.zeros(8, dtype=torch.int32, device=ranks.device)
        surv = self.emo.emo_nsga3_niche_given(n2, n_r, n_keep, seed, generation, ranks, rho, last, last_pi, last_d,
                                              info=info)
        return surv, info


def merged_ranks(results) -> np.ndarray:
    """The ranks every rank recorded (identical on every rank)."""
    return results[0][2].cpu().numpy()
