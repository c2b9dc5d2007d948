"""Multi-rank logic on CPU (gloo, world size 2): the LPT shares of the batched
workload are a disjoint cover with balanced load, every rank derives the same
partition on its own, and the bench's max-over-ranks timing reduction gives
each rank the slowest rank's time."""
from __future__ import annotations

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1209_6548_gb300 import inputs as I
from paper_1209_6548_gb300 import shard as SH


def test_lpt_partition_properties():
    probs = I.batch_mix(n=512, seed=0)
    costs = [SH.instance_cost(p, 2000) for p in probs]
    for world in (1, 2, 3, 8):
        parts = SH.lpt_partition(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(512))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= (4.0 / 3.0) * max(sum(costs) / world, max(costs)) + 1e-6
        assert max(loads) - min(loads) <= max(costs) + 1e-6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    probs = I.batch_mix(n=200, seed=1)
    idx, mine = SH.shard(probs, rank, world, steps=2000)
    t = torch.tensor([len(idx)], dtype=torch.int64)
    counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(counts, t)
    mx = max(int(c.item()) for c in counts)
    padded = torch.full((mx,), -1, dtype=torch.int64)
    padded[: len(idx)] = torch.tensor(idx, dtype=torch.int64)
    gathered = [torch.zeros(mx, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(gathered, padded)
    elapsed = torch.tensor([1.0 + rank], dtype=torch.float64)  # a rank's own timing
    dist.all_reduce(elapsed, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put(([g[g >= 0].tolist() for g in gathered], float(elapsed.item())))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts, slowest = q.get()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert sorted(parts[0] + parts[1]) == list(range(200))
    assert not set(parts[0]) & set(parts[1])
    assert parts == SH.lpt_partition([SH.instance_cost(p, 2000) for p in I.batch_mix(n=200, seed=1)], 2)
    assert slowest == 2.0


def test_costs_count_stored_values_and_steady_state_work():
    """D = 3 instances cost their stored half (nroots^3/2 values per node);
    run-to-steady costs grow with ny and with 1/Kn, as the diffusion time
    over the time step does."""
    from dataclasses import replace
    p = I.Problem(name="c", nx=4, ny=65, kn=0.1, b=0.0)
    assert SH.instance_cost(replace(p, dim=3), 100) == 2 * SH.instance_cost(p, 100)
    assert SH.instance_cost(replace(p, nroots=6, dim=3), 100) == 108 / 16 * SH.instance_cost(p, 100)
    base = SH.instance_cost(p, to_steady=True)
    assert SH.instance_cost(replace(p, kn=0.01), to_steady=True) == 10 * base
    assert SH.instance_cost(replace(p, ny=129), to_steady=True) == pytest.approx(base * 129 * 128 / (65 * 64))
    assert SH.instance_cost(replace(p, b=0.5), to_steady=True) == 2 * base  # slower heat diffusion
