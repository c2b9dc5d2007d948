"""Sharding independent solves across ranks (one process per GPU).

Batched and served solves are independent problems, so a multi-GPU run needs
no collective on the data path: each rank takes a share of the instances and
runs them in its own batch.  Shares come from the longest-processing-time
rule: instances in decreasing cost order, each to the rank with the least
work so far (ties to the lowest rank), which keeps the busiest rank within
4/3 of the optimum.

Cost of an instance = nodes x steps x values stored per node (nroots^2 for
the 2D sets, nroots^3/2 for the D = 3 sets, which store their z-even half).
Solves of a fixed length use that length; solves run to steady state use the
expected number of steps, which grows like the channel's diffusion time over
the time step: the slowest mode of a channel of width 1 decays at the rate
pi^2 nu with a diffusivity nu proportional to Kn (the viscosity mu = Kn T^varpi
of Sec. 2.2, the conductivity (1-b)-weighted), and dt is proportional to the
spacing 1/(ny - 1) at the Courant number of the run.  steps_to_steady returns
that estimate up to a constant factor, which cancels in the partition.
"""
from __future__ import annotations

import heapq


def stored_values(problem) -> int:
    return problem.nroots * problem.nroots * (problem.nroots // 2 if getattr(problem, "dim", 2) == 3 else 1)


def steps_to_steady(problem) -> float:
    """Relative number of steps a channel solve needs to reach steady state:
    (ny - 1) / (Kn min(1, 1 - b)), i.e. diffusion time over time step."""
    return max(problem.ny - 1, 1) / (problem.kn * min(1.0, 1.0 - problem.b))


def instance_cost(problem, steps: int | None = None, to_steady: bool = False) -> float:
    """Work of one instance: nodes x steps x stored values; steps = `steps`,
    problem.steps, or (to_steady) the steady-state estimate."""
    if to_steady:
        n = steps_to_steady(problem)
    else:
        n = steps if steps is not None else problem.steps
    return float(problem.nx * problem.ny * n * stored_values(problem))


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


def shard(problems, rank: int, world: int, steps: int | None = None, to_steady: bool = False):
    """(indices, problems) of this rank's share."""
    parts = lpt_partition([instance_cost(p, steps, to_steady) for p in problems], world)
    idx = parts[rank]
    return idx, [problems[i] for i in idx]
