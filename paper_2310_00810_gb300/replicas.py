"""Independent problems spread over ranks (one GPU each): the replica form of
the batched inversions and of the learned initialiser's training solves.

There is no exchange on the data path: every rank takes its share of the
problems (instances, training seeds), runs them alone, and the per-problem
results are gathered once at the end in the original order.  The split
balances an estimated cost per problem (lattice nodes x time steps) with the
longest-processing-time rule, deterministically, so every rank computes the
same assignment without communicating.
"""
from __future__ import annotations


def shard(costs, world: int) -> list[list[int]]:
    """Indices of the problems each of `world` ranks takes: problems in
    decreasing cost (ties by index) each go to the rank with the least total
    so far (ties to the lower rank); each rank's list is in increasing index."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def run_sharded(items, evaluate, costs=None, group=None) -> list:
    """evaluate(item) for this rank's share of `items` (torch.distributed
    rank / world size; one rank when no process group is initialised), then
    every rank gets every result, in the order of `items`."""
    import torch.distributed as dist

    on = dist.is_available() and dist.is_initialized()
    rank = dist.get_rank(group) if on else 0
    world = dist.get_world_size(group) if on else 1
    parts = shard([1.0] * len(items) if costs is None else costs, world)
    mine = [(i, evaluate(items[i])) for i in parts[rank]]
    if world == 1:
        got = [mine]
    else:
        got = [None] * world
        dist.all_gather_object(got, mine, group=group)
    out = [None] * len(items)
    for part in got:
        for i, r in part:
            out[i] = r
    return out
