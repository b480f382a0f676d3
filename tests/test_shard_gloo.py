"""Batch split across ranks: every tree on exactly one rank, balanced by
unknowns, per-tree results gathered over gloo (world size 2, CPU)."""
import os
import socket

import pytest

from paper_1901_11370_gb300.shard import shard_by_cost


def test_split_covers_every_tree_once_and_balances():
    costs = [(16 * k) ** 2 for k in [2, 31, 7, 30, 3, 12, 25, 9, 4, 18, 22, 6, 15, 28, 5]]
    for world in (1, 2, 3, 8, 20):
        parts = shard_by_cost(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # greedy bound: no rank exceeds the mean by more than the largest tree
        assert max(loads) <= sum(costs) / world + max(costs)
    assert shard_by_cost(costs, 2) == shard_by_cost(list(costs), 2)  # deterministic


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1901_11370_gb300.shard import gather_tree_values, shard_by_cost
    costs = [5, 1, 9, 3, 7, 2, 8]
    mine = shard_by_cost(costs, world)[rank]
    values = [10.0 * i + rank for i in mine]  # stands for a per-tree residual
    merged = gather_tree_values(values, mine, len(costs))
    q.put((rank, mine, merged))
    dist.barrier()
    dist.destroy_process_group()


def test_gather_over_gloo_two_ranks():
    import torch.multiprocessing as tmp
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    owner = {}
    for rank, mine, merged in res:
        for i in mine:
            owner[i] = rank
    assert sorted(owner) == list(range(7))
    for rank, mine, merged in res:
        assert merged == [10.0 * i + owner[i] for i in range(7)]
