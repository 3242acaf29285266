"""Splitting a batch of independent systems over several GPUs (one process per GPU).

A batch is a set of independent problems, so it shards with no data-path collective: every
rank builds and solves its own share, and only timings are reduced.  The split is the
longest-processing-time rule on a cost per item (its stored entries times its right-hand
sides): items in decreasing cost, each to the rank with the least cost so far, ties to the
lower rank and, among equal costs, to the lower item index -- so every rank computes the same
split from the same list without communicating.
"""
from __future__ import annotations


def item_cost(nnz: int, nrhs: int) -> int:
    return int(nnz) * max(1, int(nrhs))


def shard_batch(costs, world: int) -> list[list[int]]:
    """Item indices of every rank (each list ascending)."""
    if world < 1:
        raise ValueError("world must be at least 1")
    order = sorted(range(len(costs)), key=lambda i: (-int(costs[i]), i))
    load = [0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += int(costs[i])
    return [sorted(p) for p in parts]
