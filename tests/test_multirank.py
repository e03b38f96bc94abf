"""The benchmark's multi-rank host logic on CPU with world-size-2 gloo
ranks: each rank takes a disjoint shard of the sources (weak scaling, no
data-path collective) and the timed region is reduced with a max over
ranks."""
import os
import socket

import pytest
import torch.distributed as tdist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sources = list(range(100, 100 + 64 * world))
        mine = bench.shard(sources, 64, rank)
        bench.barrier(world)
        gathered = [None] * world
        tdist.all_gather_object(gathered, mine)
        elapsed = bench.max_over_ranks(0.5 + rank, world)
        q.put((rank, mine, gathered, elapsed, bench.dist_env()))
    finally:
        tdist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_shard_sources_and_take_max_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=90) for _ in range(world))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    shards = [r[1] for r in res]
    assert len(set(shards[0]) & set(shards[1])) == 0 and len(shards[0]) == len(shards[1]) == 64
    assert sorted(shards[0] + shards[1]) == list(range(100, 228))
    assert all(r[3] == 1.5 for r in res)  # max over ranks of 0.5 and 1.5
    assert [r[4][:2] for r in res] == [(2, 0), (2, 1)]
