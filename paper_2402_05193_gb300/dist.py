"""Multi-rank helpers (one process per GPU, torch.distributed).

The batched form's simulations are independent, so N ranks split them with
no collective on the data path: ``shard_by_cost`` assigns simulations to
ranks by their cell counts (largest first, each to the least-loaded rank;
deterministic, identical on every rank).  ``max_over_ranks`` gives the
slowest rank's time for whole-job throughput.
"""
from __future__ import annotations


def shard_by_cost(costs, world: int, rank: int):
    """Indices of the items rank ``rank`` runs, out of ``world`` ranks."""
    order = sorted(range(len(costs)), key=lambda k: (-costs[k], k))
    load = [0] * world
    owner = [0] * len(costs)
    for k in order:
        r = min(range(world), key=lambda j: (load[j], j))
        owner[k] = r
        load[r] += costs[k]
    return [k for k in range(len(costs)) if owner[k] == rank]


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of x over all ranks of the default process group (x itself
    when no group is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
