"""The walker partition across ranks and the end-of-run reduction, on CPU
with world_size-2 gloo process groups (the N > 1 path has no collective in the
data path; see paper_1708_00744_b300/shard.py)."""
import os
import socket

import pytest

from paper_1708_00744_b300.shard import Shard, partition_walkers, reduce_counters, work

CONFIG3 = [(512, 256), (1536, 64)]       # the batched workload's two size classes


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_covers_every_walker_once(world):
    parts = partition_walkers(CONFIG3, world)
    assert len(parts) == world
    for N, n in CONFIG3:
        seen = []
        for shards in parts:
            for s in shards:
                if s.N == N:
                    seen += list(range(s.first, s.first + s.count))
        assert sorted(seen) == list(range(n))


@pytest.mark.parametrize("world", [2, 4, 8])
def test_partition_balances_n_cubed_work(world):
    parts = partition_walkers(CONFIG3, world)
    loads = [work(p) for p in parts]
    heaviest_walker = max(N ** 3 for N, _ in CONFIG3)
    # greedy on pieces of near-equal count: within one piece's work of even
    piece = max(N ** 3 * -(-n // world) for N, n in CONFIG3)
    assert max(loads) - min(loads) <= piece
    assert sum(loads) == sum(N ** 3 * n for N, n in CONFIG3)
    assert heaviest_walker <= piece


def test_partition_edge_cases():
    assert partition_walkers([(64, 0)], 2) == [[], []]
    one = partition_walkers([(4096, 1)], 4)            # a walker is never split
    assert sum(len(p) for p in one) == 1 and sum(s.count for p in one for s in p) == 1
    assert partition_walkers([(128, 3)], 1) == [[Shard(128, 0, 3)]]
    with pytest.raises(ValueError):
        partition_walkers([(64, 1)], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        parts = partition_walkers(CONFIG3, world)
        mine = parts[rank]
        # each rank "runs" its walkers: counts and a rank-dependent time
        walkers = sum(s.count for s in mine)
        proposals = sum(s.count * s.N for s in mine)
        out = reduce_counters({"walkers": walkers, "proposals": proposals,
                               "elapsed_s": 1.0 + rank, "kernel_ms": 10.0 * (rank + 1)})
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_reduction_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    total_w = sum(n for _, n in CONFIG3)
    total_p = sum(N * n for N, n in CONFIG3)
    for r in (0, 1):
        assert got[r]["walkers"] == total_w
        assert got[r]["proposals"] == total_p
        assert got[r]["elapsed_s"] == 2.0 and got[r]["kernel_ms"] == 20.0


def test_reduction_without_a_process_group_is_the_identity():
    c = {"walkers": 3, "elapsed_s": 1.5}
    assert reduce_counters(c) == c
