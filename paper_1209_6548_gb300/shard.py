"""Sharding independent solves across ranks (one process per GPU).

Batched and served solves are independent problems, so a multi-GPU run needs
no collective on the data path: each rank takes a share of the instances and
runs them in its own batch.  Shares come from the longest-processing-time
rule: instances in decreasing cost order, each to the rank with the least
work so far (ties to the lowest rank), which keeps the busiest rank within
4/3 of the optimum.  Cost of an instance = nodes x steps x populations.
"""
from __future__ import annotations

import heapq


def instance_cost(problem, steps: int | None = None) -> float:
    n = problem.nroots * problem.nroots
    return float(problem.nx * problem.ny * (steps if steps is not None else problem.steps) * n)


def lpt_partition(costs, world: int):
    """Indices of `costs` per rank (list of lists, each in increasing index order)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(p) for p in parts]


def shard(problems, rank: int, world: int, steps: int | None = None):
    """(indices, problems) of this rank's share."""
    parts = lpt_partition([instance_cost(p, steps) for p in problems], world)
    idx = parts[rank]
    return idx, [problems[i] for i in idx]
