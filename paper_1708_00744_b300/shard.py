"""Walkers across GPUs: one process per GPU, independent walkers per process.

Walkers are independent Markov chains (the paper's walkers never exchange data
during a sweep, Sec. III), so the path shards by walker with no collective in
the data path. A fixed walker population is split across ranks by size class,
balancing the flush and recompute work, which grows as N^3 per walker; a single
walker is never split. Walker i of a class keeps its key walker_seed(base, i)
on whichever rank runs it, so results do not depend on the number of ranks.
The only collective is the end-of-run reduction of counters and timings.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Shard:
    N: int          # electrons of the size class
    first: int      # first walker index within the class
    count: int      # walkers of the class on this rank


def partition_walkers(classes, world):
    """classes: list of (N, walkers). Returns, per rank, a list of Shards.

    Largest-work-first greedy: each class is cut into `world` contiguous
    pieces of near-equal count, and the pieces, heaviest first, go to the rank
    with the least N^3 work so far (ties: lowest rank)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    pieces = []
    for N, n in classes:
        if N < 1 or n < 0:
            raise ValueError("bad class (%r, %r)" % (N, n))
        base, extra = divmod(n, world)
        first = 0
        for r in range(world):
            cnt = base + (1 if r < extra else 0)
            if cnt:
                pieces.append((N, first, cnt))
            first += cnt
    pieces.sort(key=lambda p: (-(p[0] ** 3) * p[2], p[0], p[1]))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for N, first, cnt in pieces:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(Shard(N, first, cnt))
        load[r] += float(N) ** 3 * cnt
    for r in range(world):
        out[r].sort(key=lambda s: (s.N, s.first))
    return out


def work(shards):
    """N^3-weighted walker count of a rank's shards."""
    return sum(float(s.N) ** 3 * s.count for s in shards)


def reduce_counters(counters, group=None):
    """End-of-run reduction over ranks: sums of counts, max of times.

    counters: dict name -> float; names ending in '_s' or '_ms' are times
    (max over ranks), the rest are summed. Without an initialised process
    group the dict is returned unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return dict(counters)
    names = sorted(counters)
    times = [k for k in names if k.endswith("_s") or k.endswith("_ms")]
    sums = [k for k in names if k not in times]
    dev = torch.device("cuda", torch.cuda.current_device()) \
        if dist.get_backend(group) == "nccl" else torch.device("cpu")
    out = {}
    if sums:
        t = torch.tensor([float(counters[k]) for k in sums], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        out.update(zip(sums, t.tolist()))
    if times:
        t = torch.tensor([float(counters[k]) for k in times], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
        out.update(zip(times, t.tolist()))
    return out
