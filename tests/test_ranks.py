"""Multi-process host logic of the benchmark on CPU (gloo, two ranks): the
maximum-over-ranks timing and the split of an ensemble's systems across
ranks (disjoint, complete, balanced, identical on every rank)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, sizes, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.0 + rank, world, torch.device("cpu"))
        own = bench.rank_share(sizes, rank, world)
        # every rank computes the same split independently
        every = [bench.rank_share(sizes, r, world) for r in range(world)]
        gathered = [None] * world
        dist.all_gather_object(gathered, own)
        out.put((rank, t, own, every == gathered))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_ranks_timing_and_split(world):
    sizes = [int(s) for s in np.random.default_rng(1).integers(1000, 60000, size=37)]
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, sizes, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert all(t == float(world) for _, t, _, _ in res)   # max of 1.0, 2.0
    assert all(same for *_, same in res)
    owned = [set(o) for _, _, o, _ in res]
    assert owned[0].isdisjoint(owned[1]) and owned[0] | owned[1] == set(range(len(sizes)))
    loads = [sum(sizes[b] for b in o) for o in owned]
    assert max(loads) - min(loads) <= max(sizes)


def test_rank_share_single_rank_and_greedy():
    import bench
    assert bench.rank_share([5, 3, 8], 0, 1) == [0, 1, 2]
    # largest first to the least loaded rank: 8 -> r0, 5 -> r1, 3 -> r1, 2 -> r0
    assert bench.rank_share([5, 3, 8, 2], 0, 2) == [2, 3]
    assert bench.rank_share([5, 3, 8, 2], 1, 2) == [0, 1]
