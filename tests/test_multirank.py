"""Multi-rank host logic of the benchmark on CPU with the gloo backend
(world size 2): independent volumes are sharded across ranks without any
data exchange, and the step time (max) and pair count (sum) are reduced
over ranks."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, sizes, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bench.shard_volumes(sizes, world, rank)
        shards = [None] * world
        dist.all_gather_object(shards, mine)
        pairs, ms = bench.reduce_over_ranks(1000 + rank, 10.0 + 3 * rank, world, "cpu")
        q.put((rank, shards, pairs, ms))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_sharding_and_rank_reduction_gloo(world):
    sizes = [24389, 1000000, 110592, 357911, 42875, 729000, 97336, 15625, 571787, 250047]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, sizes, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, shards, pairs, ms in results:
        assert pairs == sum(1000 + r for r in range(world))
        assert ms == 10.0 + 3 * (world - 1)
        flat = sorted(v for s in shards for v in s)
        assert flat == list(range(len(sizes)))                   # complete and disjoint
        loads = [sum(sizes[v] for v in s) for s in shards]
        assert max(loads) - min(loads) <= max(sizes)             # greedy balance bound


def test_shard_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.shard_volumes([3, 1, 2], 1, 0) == [0, 1, 2]
