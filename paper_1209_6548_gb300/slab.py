"""Y-slab decomposition of one large solve over several solvers.

The domain's ny rows are split into contiguous slabs, one per rank (one GPU
per rank), or several slabs in one process.  Each slab runs as an ordinary
solver on an extended grid: its own rows plus `halo` rows below and above
(none at a wall).  The TVD fluxes of Sec. 3.1 reach two rows, so a halo of
2k rows carries k time steps: after step s the outermost 2s halo rows are
stale (their stencils ran off the extended grid, or a wall rule was applied
to the grid's edge row), the rest are exact, and the slab's own rows are
exact throughout.  Every k steps each slab sends its top `halo` own rows to
the slab above, which stores them as its lower halo, and its bottom `halo`
own rows to the slab below (upper halo); with periodic y the ends wrap
around.  The interior arithmetic is that of the single domain node for node,
so the result is bitwise the single-domain result.

Extended grid of a slab: periodic in y where the whole domain is periodic, or
where the slab touches no wall (its edge rows are halo rows, whose own
updates are discarded); with walls where it holds a wall row (the bottom
slab's row 0, the top slab's row ny - 1), the grid's other edge being a halo
edge whose wall rule acts only on a stale row.  Its spacing and time step are
the whole domain's (lesbgk_params dx, dy, dt), its rounding key the global
row (row_offset).  Walls in y stay on the end slabs; the conservation totals
of the whole domain are one sum over the slabs' own rows (FP64; an
allreduce across ranks).

Exchange (every k steps, after the slab's steps, and once before the first):
messages go to the neighbours above and below, posted in the same order on
every rank -- first "send up / receive from below", then "send down / receive
from above" -- so that with two ranks, where both neighbours are one rank,
the pairs still match.

Host logic only; the device work is the library's (lesbgk_step,
lesbgk_get_rows / lesbgk_set_rows, lesbgk_moments_rows).
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

from . import inputs as I


@dataclass(frozen=True)
class Slab:
    """Rank `rank` of `world` owns global rows [y0, y1); its extended grid
    holds rows [y0 - lo, y1 + hi) (wrapping around a periodic domain)."""

    rank: int
    world: int
    ny: int          # rows of the whole domain
    y0: int
    y1: int
    lo: int          # halo rows below (0 at the bottom wall)
    hi: int          # halo rows above (0 at the top wall)
    periodic: bool   # the whole domain is periodic in y

    @property
    def rows(self) -> int:
        return self.y1 - self.y0

    @property
    def ny_ext(self) -> int:
        return self.lo + self.rows + self.hi

    @property
    def up(self):
        """Rank above (None at the top wall)."""
        if self.hi == 0:
            return None
        return (self.rank + 1) % self.world

    @property
    def down(self):
        """Rank below (None at the bottom wall)."""
        if self.lo == 0:
            return None
        return (self.rank - 1) % self.world

    def global_rows(self) -> np.ndarray:
        """Global row of each extended-grid row."""
        return np.arange(self.y0 - self.lo, self.y1 + self.hi) % self.ny

    def grid_walls(self) -> bool:
        """Whether the extended grid has diffuse walls (it holds a wall row)."""
        return not self.periodic and (self.lo == 0 or self.hi == 0)


def partition(ny: int, world: int, halo: int, periodic: bool) -> list[Slab]:
    """Split ny rows into `world` contiguous slabs of nearly equal height (the
    first ny % world slabs get one more row), with `halo` rows of halo at every
    edge between slabs (and around a periodic domain).  Every slab must own at
    least `halo` rows, so that a halo comes from one neighbour, and more than
    `halo` where the domain has walls, so that no halo holds a wall row (whose
    wall rule only its owner applies)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if halo < 2 or halo % 2:
        raise ValueError("halo must be an even number >= 2 (two rows per step)")
    base, extra = divmod(ny, world)
    need = halo if periodic else halo + 1
    if world > 1 and base < need:
        raise ValueError(f"{ny} rows over {world} slabs leave {base} rows per slab; need >= {need}")
    out, y = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        if world == 1:
            lo = hi = 0  # the whole domain: the solver's own y boundary
        else:
            lo = 0 if (not periodic and r == 0) else halo
            hi = 0 if (not periodic and r == world - 1) else halo
        out.append(Slab(r, world, ny, y, y + n, lo, hi, periodic))
        y += n
    return out


def slab_fields(fields: np.ndarray, slab: Slab) -> np.ndarray:
    """The slab's extended-grid share of (4, ny, nx) initial fields."""
    return np.ascontiguousarray(fields[:, slab.global_rows(), :])


def slab_problem(prob: I.Problem, slab: Slab) -> I.Problem:
    """The problem one slab's solver runs (spacing and dt passed separately)."""
    bc = I.DIFFUSE if slab.grid_walls() else I.PERIODIC
    return replace(prob, ny=slab.ny_ext, bc_y=bc, name=f"{prob.name}_slab{slab.rank}of{slab.world}")


def exchange_plan(slab: Slab):
    """The slab's messages of one exchange, in posting order:
    (kind, peer, own-or-halo row range of the extended grid, tag).
    kind 'send' reads the range, 'recv' writes it."""
    n, lo, hi = slab.rows, slab.lo, slab.hi
    plan = []
    if slab.up is not None:  # upward: my top own rows -> the lower halo of the slab above
        plan.append(("send", slab.up, (lo + n - hi, lo + n), 0))
    if slab.down is not None:
        plan.append(("recv", slab.down, (0, lo), 0))
    if slab.down is not None:  # downward: my bottom own rows -> the upper halo of the slab below
        plan.append(("send", slab.down, (lo, lo + lo), 1))
    if slab.up is not None:
        plan.append(("recv", slab.up, (lo + n, lo + n + hi), 1))
    return plan


def exchange_dist(store, slab: Slab, dist) -> None:
    """One halo exchange between ranks (torch.distributed, any backend):
    store.get_rows(j0, nrows) -> tensor, store.empty_rows(nrows) -> tensor,
    store.set_rows(j0, nrows, tensor)."""
    ops, recvs = [], []
    for kind, peer, (a, b), tag in exchange_plan(slab):
        if kind == "send":
            ops.append(dist.P2POp(dist.isend, store.get_rows(a, b - a), peer, tag=tag))
        else:
            buf = store.empty_rows(b - a)
            recvs.append((a, b, buf))
            ops.append(dist.P2POp(dist.irecv, buf, peer, tag=tag))
    if ops:
        store.before_comm()
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for a, b, buf in recvs:
        store.set_rows(a, b - a, buf)


def exchange_local(stores, slabs) -> None:
    """One halo exchange between slabs held in one process: every receive
    takes the matching send's rows directly (all reads before any write)."""
    msgs = {}
    for store, slab in zip(stores, slabs):
        for kind, peer, (a, b), tag in exchange_plan(slab):
            if kind == "send":
                msgs[(slab.rank, peer, tag)] = store.get_rows(a, b - a)
    for store, slab in zip(stores, slabs):
        for kind, peer, (a, b), tag in exchange_plan(slab):
            if kind == "recv":
                store.set_rows(a, b - a, msgs[(peer, slab.rank, tag)])


class GpuSlab:
    """One slab as a library solver (lesbgk_* through the ctypes binding) on
    the current CUDA device; the row buffers are torch uint8 tensors holding
    the library's packed rows."""

    def __init__(self, prob: I.Problem, slab: Slab, fields, dt: float, dx: float, dy: float, storage: int = 0,
                 stream=None):
        import torch
        from . import lesbgk as L
        self._torch, self._L = torch, L
        self.slab = slab
        p = L.params_from_problem(slab_problem(prob, slab), dt=dt)
        p.storage = storage
        if slab.world > 1:
            p.dx, p.dy = dx, dy
            p.row_offset = slab.y0 - slab.lo
            p.row_period = slab.ny if slab.periodic else 0
        self.solver = L.Solver(p, h_init=None if fields is None else slab_fields(fields, slab), stream=stream)

    @property
    def _s(self):
        return self.solver.stream.cuda_stream

    def _nbytes(self, nrows: int) -> int:
        import ctypes as C
        n = C.c_size_t()
        self._L._check(self._L.lib().lesbgk_rows_bytes(C.c_void_p(self.solver.handle), nrows, C.byref(n)))
        return int(n.value)

    def empty_rows(self, nrows: int):
        return self._torch.empty(self._nbytes(nrows), dtype=self._torch.uint8, device="cuda")

    def get_rows(self, j0: int, nrows: int):
        import ctypes as C
        buf = self.empty_rows(nrows)
        self._L._check(self._L.lib().lesbgk_get_rows(C.c_void_p(self.solver.handle), j0, nrows,
                                                     C.c_void_p(buf.data_ptr()), C.c_void_p(self._s)))
        return buf

    def set_rows(self, j0: int, nrows: int, buf) -> None:
        import ctypes as C
        self._L._check(self._L.lib().lesbgk_set_rows(C.c_void_p(self.solver.handle), j0, nrows,
                                                     C.c_void_p(buf.data_ptr()), C.c_void_p(self._s)))

    def before_comm(self) -> None:
        """Communication runs on its own stream: the packed rows must be
        written before it reads them."""
        self.solver.stream.synchronize()

    def step(self, n: int) -> None:
        self.solver.step(n)

    def moments(self, sums: bool = False):
        """The slab's own rows: (9, rows, nx) device tensor (and FP64 totals)."""
        import ctypes as C
        sl = self.slab
        out = self._torch.empty((9, sl.rows, self.solver.params.nx), dtype=self._torch.float32, device="cuda")
        hs = np.zeros(4) if sums else None
        self._L._check(self._L.lib().lesbgk_moments_rows(
            C.c_void_p(self.solver.handle), sl.lo, sl.rows, C.c_void_p(out.data_ptr()),
            C.c_void_p(None if hs is None else hs.ctypes.data), C.c_void_p(self._s)))
        return (out, hs) if sums else out

    def populations(self):
        """The slab's own rows of the populations, public layout (Q, rows, nx)."""
        sl = self.slab
        return self.solver.populations()[:, sl.lo:sl.lo + sl.rows]

    def close(self) -> None:
        self.solver.close()


class SlabRun:
    """Several slabs of one solve in one process (one GPU): created, stepped
    and exchanged together; halo = 2k rows, exchange every k steps."""

    def __init__(self, prob: I.Problem, nslabs: int, steps_per_exchange: int, fields, dt: float, dx: float,
                 dy: float, storage: int = 0):
        self.k = steps_per_exchange
        self.slabs = partition(prob.ny, nslabs, 2 * self.k, prob.bc_y == I.PERIODIC)
        self.stores = [GpuSlab(prob, s, fields, dt, dx, dy, storage) for s in self.slabs]
        self.since = 0
        exchange_local(self.stores, self.slabs)  # halos from their owners (the owners' wall rule included)

    def step(self, n: int) -> None:
        while n > 0:
            m = min(n, self.k - self.since)
            for st in self.stores:
                st.step(m)
            self.since += m
            n -= m
            if self.since == self.k:
                exchange_local(self.stores, self.slabs)
                self.since = 0

    def moments(self):
        """(9, ny, nx) device tensor and the FP64 totals (summed over slabs)."""
        parts = [st.moments(sums=True) for st in self.stores]
        return self.stores[0]._torch.cat([m for m, _ in parts], dim=1), np.sum([s for _, s in parts], axis=0)

    def populations(self):
        return self.stores[0]._torch.cat([st.populations() for st in self.stores], dim=1)

    def close(self) -> None:
        for st in self.stores:
            st.close()
