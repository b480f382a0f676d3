"""Splitting a batch of independent trees across ranks (one GPU each).

Trees share nothing, so ranks exchange no data while they solve: each rank
builds a Batch of its own trees.  Only per-tree results (final residuals,
cycle counts) are gathered afterwards, on the host.
"""
from __future__ import annotations


def shard_by_cost(costs, world):
    """Tree indices per rank: longest-processing-time greedy on `costs`
    (e.g. unknowns per tree), largest first, ties to the lowest rank.
    Deterministic, so every rank computes the same split."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def gather_tree_values(values, indices, n_trees):
    """All ranks' per-tree values (lists aligned with `indices`) merged into
    one list of n_trees entries, on every rank (host-side all_gather of
    Python objects; call after the solves)."""
    import torch.distributed as dist
    world = dist.get_world_size()
    parts = [None] * world
    dist.all_gather_object(parts, list(zip(indices, values)))
    out = [None] * n_trees
    for part in parts:
        for i, v in part:
            out[i] = v
    return out
