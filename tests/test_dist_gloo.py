"""The multi-rank host logic on CPU: world size 2 over gloo."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2402_05193_gb300 import dist as jdist  # noqa: E402
from paper_2402_05193_gb300 import workloads as wl  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, costs, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = jdist.shard_by_cost(costs, world, rank)
    # every rank's shard, gathered: disjoint, complete, balanced
    shards = [None] * world
    dist.all_gather_object(shards, mine)
    slowest = jdist.max_over_ranks(float(sum(costs[k] for k in mine)))
    out.put((rank, shards, slowest))
    dist.destroy_process_group()


def test_drop_batch_sharding_over_two_gloo_ranks():
    costs = [int(c["n"][0] * c["n"][1]) for c in wl.drop_batch()]
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shards = res[0][1]
    assert all(r[1] == shards for r in res)  # every rank computed the same split
    flat = sorted(k for s in shards for k in s)
    assert flat == list(range(len(costs)))
    loads = [sum(costs[k] for k in s) for s in shards]
    assert max(loads) - min(loads) <= max(costs)  # greedy balance bound
    assert all(r[2] == max(loads) for r in res)   # max over ranks


def test_shard_by_cost_single_rank_and_determinism():
    costs = [5, 1, 3, 3, 8, 2]
    assert jdist.shard_by_cost(costs, 1, 0) == list(range(6))
    a = [jdist.shard_by_cost(costs, 3, r) for r in range(3)]
    assert a == [jdist.shard_by_cost(costs, 3, r) for r in range(3)]
    assert sorted(k for s in a for k in s) == list(range(6))
