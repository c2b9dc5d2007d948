"""The y-slab decomposition's partition and halo exchange on CPU ranks (gloo).

Each rank holds one slab of a solve as the FP64 oracle running on the slab's
extended grid (own rows plus halo rows, the whole domain's spacing and dt),
and exchanges halos through slab.exchange_dist -- the code the GPU ranks run,
here moving CPU tensors.  The slabs' own rows after several exchanges must
equal the single-domain oracle run exactly (the arithmetic per node is the
same), for periodic and walled domains, two and three ranks, and halos of one
and two steps; the FP64 allreduce of the slabs' conservation totals must give
the whole domain's.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_1209_6548_gb300 import inputs as I
from paper_1209_6548_gb300 import slab as SL
from tests.common import oracle_params, spacing, time_step


class OracleSlab:
    """A slab held by the FP64 oracle; rows travel as float64 CPU tensors of
    the oracle's [a][j][i] populations."""

    def __init__(self, prob, slab, fields, dt):
        self.slab = slab
        sp = SL.slab_problem(prob, slab)
        dx, dy = spacing(prob)
        self.op = oracle_params(sp, dt, nx=prob.nx, ny=slab.ny_ext, bc_y=sp.bc_y)
        self.op.dx, self.op.dy = dx, dy
        self.dt = dt
        self.f = O.init(self.op, None if fields is None else SL.slab_fields(fields, slab))
        self.steps = 0

    def empty_rows(self, nrows):
        return torch.empty((self.f.shape[0], nrows, self.f.shape[2]), dtype=torch.float64)

    def get_rows(self, j0, nrows):
        return torch.from_numpy(np.ascontiguousarray(self.f[:, j0:j0 + nrows]))

    def set_rows(self, j0, nrows, buf):
        self.f[:, j0:j0 + nrows] = buf.numpy()

    def before_comm(self):
        pass

    def step(self, n):
        self.op.time = self.steps * self.dt
        self.f = O.run(self.op, self.f, n)
        self.steps += n

    def own(self):
        s = self.slab
        return self.f[:, s.lo:s.lo + s.rows]


def cases():
    rough = I.Problem(name="rough", nx=9, ny=31, bc_y=I.PERIODIC, kn=0.05, b=-0.5, scheme=I.SPLIT)
    walls = I.Problem(name="walls", nx=7, ny=29, bc_y=I.DIFFUSE, kn=0.1, b=0.5, wall_ux=(-0.05, 0.04),
                      wall_T=(0.97, 1.03), g=(1e-3, 0.0))
    heated = I.Problem(name="heated", nx=4, ny=27, bc_y=I.DIFFUSE, kn=0.2, b=-0.5, wall_specular=0.3,
                       wall_T_amp=0.02, wall_T_freq=0.55536)
    return {"rough": rough, "walls": walls, "heated": heated}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, name, k, nsteps, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    O.set_threads(1)
    prob = cases()[name]
    fields = I.random_fields(prob, seed=5, amp_u=0.03, amp_T=0.03, amp_rho=0.03)
    dt = time_step(prob, fields)
    slab = SL.partition(prob.ny, world, 2 * k, prob.bc_y == I.PERIODIC)[rank]
    st = OracleSlab(prob, slab, fields, dt)
    SL.exchange_dist(st, slab, dist)
    done = 0
    while done < nsteps:
        m = min(k, nsteps - done)
        st.step(m)
        done += m
        if m == k:
            SL.exchange_dist(st, slab, dist)
    own = st.own()
    op_own = oracle_params(prob, dt, ny=slab.rows)  # moments are per node: any params of the set do
    _, sums = O.moments(op_own, np.ascontiguousarray(own))
    tot = torch.tensor(sums, dtype=torch.float64)
    dist.all_reduce(tot)  # the one FP64 reduction of the decomposition
    q.put((rank, slab.y0, slab.y1, own, tot.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def run_ranks(name, world, k, nsteps):
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, name, k, nsteps, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get() for _ in range(world))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    return res


def test_partition_covers_the_rows_and_checks_heights():
    for ny, world, halo, periodic in [(31, 2, 2, True), (29, 3, 4, False), (4096, 8, 16, True), (10, 1, 2, False)]:
        slabs = SL.partition(ny, world, halo, periodic)
        assert [s.y0 for s in slabs] == [0] + [s.y1 for s in slabs[:-1]] and slabs[-1].y1 == ny
        assert max(s.rows for s in slabs) - min(s.rows for s in slabs) <= 1
        for s in slabs:
            if world == 1:
                assert s.lo == s.hi == 0
            else:
                assert s.lo == (0 if (not periodic and s.rank == 0) else halo)
                assert s.hi == (0 if (not periodic and s.rank == world - 1) else halo)
            assert len(s.global_rows()) == s.ny_ext
    with pytest.raises(ValueError):
        SL.partition(12, 4, 4, False)  # 3 rows per slab cannot feed a halo of 4 (and must exceed it at walls)
    with pytest.raises(ValueError):
        SL.partition(12, 2, 3, True)   # halos carry whole steps: an even number of rows


def test_exchange_plans_pair_up():
    """Every send has exactly one receive of the same size and tag at its
    peer, ranges within the extended grids, and the posting order is the same
    on every rank."""
    for ny, world, halo, periodic in [(31, 2, 2, True), (29, 3, 4, False), (40, 4, 2, True), (40, 2, 4, False)]:
        slabs = SL.partition(ny, world, halo, periodic)
        sends, recvs = {}, {}
        for s in slabs:
            plan = SL.exchange_plan(s)
            assert [p[3] for p in plan] == sorted(p[3] for p in plan)  # upward (tag 0) messages first
            for kind, peer, (a, b), tag in plan:
                assert 0 <= a < b <= s.ny_ext
                (sends if kind == "send" else recvs).setdefault((s.rank, peer, tag) if kind == "send"
                                                                else (peer, s.rank, tag), []).append(b - a)
        assert sends == recvs


@pytest.mark.timeout(300)
@pytest.mark.parametrize("name,world,k", [("rough", 2, 1), ("rough", 3, 2), ("walls", 2, 2), ("walls", 3, 1),
                                          ("heated", 2, 1)])
def test_slabs_equal_the_single_domain(name, world, k):
    nsteps = 7  # several exchanges and a partial last chunk
    prob = cases()[name]
    fields = I.random_fields(prob, seed=5, amp_u=0.03, amp_T=0.03, amp_rho=0.03)
    dt = time_step(prob, fields)
    op = oracle_params(prob, dt)
    f = O.run(op, O.init(op, fields), nsteps)
    _, ref_sums = O.moments(op, f)
    res = run_ranks(name, world, k, nsteps)
    whole = np.concatenate([own for _, _, _, own, _ in res], axis=1)
    assert whole.shape == f.shape
    assert np.array_equal(whole, f), np.max(np.abs(whole - f))
    for *_, tot in res:  # every rank holds the allreduced totals
        assert np.allclose(tot, ref_sums, rtol=1e-13, atol=1e-13)
