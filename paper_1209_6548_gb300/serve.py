"""Continuous-batching service for lattice ES-BGK solves.

Requests (a Problem each) arrive over time; each runs until its steady state.
The loop admits waiting requests into free batch slots as soon as the batch's
device pool has room for them (lesbgk_batch_add refusing with LESBGK_ESPACE
is the admission test), advances every admitted solve together in chunks of
`check_every` steps (CUDA-graph replays inside the library), reads the
per-slot residuals, and retires converged solves -- reading their moments and
returning their memory to the pool -- so that solves arriving while others
are on the GPU join them as slots free up.

Convergence (Convergence.verdict), with r the residual of
lesbgk_batch_residuals (max over nodes of |d rho| + |d u| + |d T| per unit
time since the previous check) and m the solve's total mass at each check:
  - converged: r < rtol (1e-8; measured in FP32, force-driven channels
    between isothermal walls at rest reach r = 0 to 2e-11, so the bar is not
    a rounding floor);
  - steady_drift: r has settled on a floor that the wall rule's constant mass
    exchange sets.  With walls hotter or colder than the gas next to them the
    diffuse-wall rule adds or removes a small, constant amount of mass per
    step (the FP64 oracle shows the same), so such solves approach a state
    that drifts at a constant rate, never a fixed point, and r cannot fall
    below 1e-8 in any precision.  Two conditions, over three checks r0, r1, r2
    equally spaced across the latter half of the run so far (so the spacing
    grows with the run): the part of r still decaying,
    estimated by Aitken's delta-squared extrapolation of the three,
    (r2 - r1)^2 / |(r2 - r1) - (r1 - r0)|, is below rtol (a slow exponential
    approach keeps this large until it has run its course); and the mass
    changes linearly in time over the same checks, the drift's signature;
  - diverged: r is infinite (a non-finite node) or not a number after the
    first check -- the slot is freed at once and the request ends with an
    error;
  - max_steps: the cap.

Solves that the batch cannot hold (another width, walls in x such as the
lid-driven cavities of the mix, D3Q216) go to a wide lane: each runs as a single-domain solver on its own CUDA stream,
so they advance concurrently with the batch; the lane admits them in arrival
order while its own device-memory budget has room, and checks them with the
same residual and criterion (lesbgk_residual, one kernel per check).

A request may carry a deadline (seconds after its arrival): one still queued
or running past it ends as "timed_out", its slot or solver freed at the next
check; ServingLoop.cancel(rid) ends one the same way ("cancelled").  A
problem the library refuses ends as "rejected"; a full pool or lane budget
only keeps requests waiting.

Everything on the device runs in the library's kernels; this module is the
scheduler (host bookkeeping only).
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass

import numpy as np

from . import inputs as I
from . import lesbgk as L


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    problem: I.Problem
    admitted: float = float("nan")
    completed: float = float("nan")
    steps: int = 0
    residual: float = float("nan")
    status: str = "pending"  # pending, running, converged, steady_drift, max_steps, diverged, rejected,
    #                          timed_out, cancelled
    error: str = ""          # why a request was rejected or diverged
    moments: object = None   # (9, ny, nx) float32 device tensor when kept
    deadline: float = float("inf")  # seconds after arrival by which it must be done


SOLVED = ("converged", "steady_drift")


@dataclass
class Convergence:
    rtol: float = 1e-8          # the FP32 floor is far below it (force-driven channels reach r = 0)
    min_checks: int = 9         # the drift test's lag is at least 2 check intervals
    mass_linear: float = 0.05   # |m2 - 2 m1 + m0| <= mass_linear |m2 - m1| (+ rounding of m)
    mass_eps: float = 1e-6      # rounding allowance of the mass per node (FP32 per-node values)
    max_steps: int = 400_000

    def verdict(self, hist, steps, mass=None, nodes: int = 1):
        """hist: r at each check (the first is NaN: no previous snapshot);
        mass: the total mass at the same checks (or None: no drift test);
        nodes: the solve's node count (scales the mass rounding allowance)."""
        if not hist:
            return None
        r = hist[-1]
        if np.isinf(r) or (np.isnan(r) and len(hist) > 1):
            return "diverged"
        if np.isfinite(r) and r < self.rtol:
            return "converged"
        if mass is not None and len(hist) >= self.min_checks and self._drift(hist, mass, nodes):
            return "steady_drift"
        if steps >= self.max_steps:
            return "max_steps"
        return None

    def _drift(self, hist, mass, nodes):
        k = (len(hist) - 1) // 4  # lag: r0, r1, r2 span the latter half of the checks so far
        r0, r1, r2 = hist[-1 - 2 * k], hist[-1 - k], hist[-1]
        m0, m1, m2 = mass[-1 - 2 * k], mass[-1 - k], mass[-1]
        if not all(np.isfinite(v) for v in (r0, r1, r2, m0, m1, m2)):
            return False
        d1, d2 = r1 - r0, r2 - r1
        if abs(d2) > abs(d1):  # not contracting
            return False
        den = abs(d2 - d1)
        transient = 0.0 if d2 == 0.0 else (d2 * d2 / den if den > 0.0 else np.inf)
        if not transient < self.rtol:
            return False
        eps = self.mass_eps * nodes
        dm = m2 - m1
        return abs(dm) > eps and abs(m2 - 2.0 * m1 + m0) <= self.mass_linear * abs(dm) + eps


def poisson_trace(n: int, rate: float, problems, seed: int = 0):
    """n requests with exponential inter-arrival times (mean 1/rate s), the
    problem of request k drawn from `problems` in order."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    return [Request(rid=k, arrival=float(t[k]), problem=problems[k % len(problems)]) for k in range(n)]


def serving_mix(n: int, seed: int = 0, q36_share: float = 0.2, ny_hi: int = 512, cavity_share: float = 0.0,
                cavity_n: int = 256):
    """The channel mix of the batched benchmark (nx = 4, Couette / Fourier /
    Poiseuille, Kn log-uniform 0.01-0.5, b in {-1/2, 0, 1/2}) with ny
    log-uniform 16..ny_hi, a share of the requests on D2Q36 (order 4), and a
    share of lid-driven cavities (cavity_n^2, lid 0.05, Kn log-uniform
    0.05-0.5, D2Q16, split scheme)."""
    from dataclasses import replace
    probs = I.batch_mix(n=n, seed=seed, ny_hi=ny_hi)
    rng = np.random.default_rng(seed + 1)
    pick = rng.random(n) < q36_share
    out = [replace(p, nroots=6) if q else p for p, q in zip(probs, pick)]
    rng2 = np.random.default_rng(seed + 2)
    cav = rng2.random(n) < cavity_share
    kn = np.exp(rng2.uniform(np.log(0.05), np.log(0.5), size=n))
    for k in np.flatnonzero(cav):
        out[k] = replace(I.lid_driven_cavity(n=cavity_n, u_lid=0.05, kn=float(kn[k]), b=out[k].b),
                         name=f"cavity{k}")
    return out


def fits_batch(prob, nx: int) -> bool:
    """Whether the batched solver takes this problem (the library's own
    admission checks say the same)."""
    dim = getattr(prob, "dim", 2)
    return (prob.nx == nx and getattr(prob, "bc_x", I.PERIODIC) == I.PERIODIC
            and (dim == 2 or (dim == 3 and prob.nroots == 4)))


class WideLane:
    """Single-domain solvers, one CUDA stream each, for the solves the batch
    cannot hold; admission while the summed workspaces fit budget_bytes."""

    def __init__(self, budget_bytes: int, max_solvers: int = 16):
        import torch
        self._torch = torch
        self.budget = budget_bytes
        self.max_solvers = max_solvers
        self.used = 0
        self.active = {}  # key -> (request, solver, stream, previous fields, residual history)
        self._next = 0

    def try_admit(self, req) -> bool:
        """Admit when the budget has room; raises LesbgkError for a problem
        the library refuses."""
        p = L.params_from_problem(req.problem)
        need = L.workspace_size(p)
        if self.used + need > self.budget or len(self.active) >= self.max_solvers:
            return False
        st = self._torch.cuda.Stream()
        with self._torch.cuda.stream(st):  # the solver's allocations belong to its stream
            s = L.Solver(p, stream=st)
            prev = self._torch.empty((4, p.ny, p.nx), dtype=self._torch.float32, device="cuda")
        r, m = s.residual(prev, 0, mass=True)  # the first snapshot
        self.used += need
        self.active[self._next] = (req, s, st, prev, ([r], [m]))
        self._next += 1
        return True

    def step(self, n: int) -> None:
        for _, s, _, _, _ in self.active.values():
            s.step(n)  # asynchronous on the solver's own stream

    def residuals(self, n: int):
        """key -> residual over the last n steps (max over nodes of
        |d rho| + |d u| + |d T|, per unit time; lesbgk_residual, the same
        quantity as lesbgk_batch_residuals)."""
        out = {}
        for key, (req, s, st, prev, (hist, mass)) in self.active.items():
            r, m = s.residual(prev, n, mass=True)
            hist.append(r)
            mass.append(m)
            out[key] = r
        return out

    def retire(self, key, keep_moments: bool) -> None:
        req, s, st, prev, _ = self.active.pop(key)
        if keep_moments:
            with self._torch.cuda.stream(st):
                req.moments = s.moments()
        st.synchronize()  # nothing of this solve in flight before its memory is released
        self.used -= s.nbytes
        s.close()


class ServingLoop:
    """batch / wide: an L.Batch and a WideLane to serve with (created from
    capacity, pool_bytes, wide_bytes when not given)."""

    def __init__(self, capacity: int, pool_bytes: int, nx: int = 4, check_every: int = 256,
                 conv: Convergence | None = None, keep_moments: bool = False, stream=None,
                 wide_bytes: int | None = None, wide_solvers: int = 16, batch=None, wide=None):
        self.nx = nx
        self.batch = batch if batch is not None else L.Batch(capacity=capacity, nx=nx, pool_bytes=pool_bytes,
                                                             stream=stream)
        self.wide = wide if wide is not None else WideLane(pool_bytes if wide_bytes is None else wide_bytes,
                                                           wide_solvers)
        self.check_every = check_every
        self.conv = conv or Convergence()
        self.keep_moments = keep_moments
        self._cancel = set()

    def cancel(self, rid: int) -> None:
        """End request rid at the loop's next pass (queued: dropped; running:
        its slot or solver freed), with status "cancelled"."""
        self._cancel.add(rid)

    def run(self, requests, clock=time.perf_counter):
        bt, wide = self.batch, self.wide
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()       # for the batch
        waiting_wide = collections.deque()  # for the wide lane
        active = {}  # slot -> (request, residual history, mass history)
        t0 = clock()
        done = []

        def finish(req, v, r, now):
            req.status, req.residual, req.completed = v, r, now
            done.append(req)

        def reject(req, err):  # a problem the library refuses ends alone; the others go on
            req.error = str(err)
            req.admitted = clock() - t0
            finish(req, "rejected", float("nan"), req.admitted)

        def ended(req, now):  # cancelled or past its deadline: the status to end with, else None
            if req.rid in self._cancel:
                return "cancelled"
            return "timed_out" if now > req.arrival + req.deadline else None

        def drop_ended(now):
            for q in (pending, waiting, waiting_wide):
                for req in [r for r in q if r.arrival <= now and ended(r, now)]:
                    q.remove(req)
                    finish(req, ended(req, now), float("nan"), now)
            for slot in list(active):
                req, hist, _ = active[slot]
                v = ended(req, now)
                if v:
                    req.steps = bt.info(slot).steps_done
                    bt.remove(slot)
                    del active[slot]
                    finish(req, v, hist[-1] if hist else float("nan"), now)
            for key in list(wide.active):
                req = wide.active[key][0]
                v = ended(req, now)
                if v:
                    hist = wide.active[key][4][0]
                    wide.retire(key, False)
                    finish(req, v, hist[-1] if hist else float("nan"), now)

        while pending or waiting or waiting_wide or active or wide.active:
            now = clock() - t0
            drop_ended(now)
            while pending and pending[0].arrival <= now:
                req = pending.popleft()
                (waiting if fits_batch(req.problem, self.nx) else waiting_wide).append(req)
            if not (pending or waiting or waiting_wide or active or wide.active):
                break
            while waiting:  # FIFO admission while the pool has room
                req = waiting[0]
                try:
                    slot = bt.try_add(L.params_from_problem(req.problem))
                except L.LesbgkError as err:
                    reject(waiting.popleft(), err)
                    continue
                if slot is None:
                    break
                waiting.popleft()
                req.admitted = clock() - t0
                req.status = "running"
                active[slot] = (req, [], [])
            while waiting_wide:
                try:
                    if not wide.try_admit(waiting_wide[0]):
                        break
                except L.LesbgkError as err:
                    reject(waiting_wide.popleft(), err)
                    continue
                req = waiting_wide.popleft()
                req.admitted = clock() - t0
                req.status = "running"
            if not active and not wide.active:
                if pending:
                    time.sleep(max(0.0, min(pending[0].arrival - (clock() - t0), 0.01)))
                continue
            if wide.active:
                wide.step(self.check_every)  # their own streams: they run beside the batch
            if active:
                bt.step(self.check_every)
                res, mass = bt.residuals(mass=True)
                now = clock() - t0
                for slot in list(active):
                    req, hist, mhist = active[slot]
                    req.steps = bt.info(slot).steps_done
                    hist.append(float(res[slot]))
                    mhist.append(float(mass[slot]))
                    v = self.conv.verdict(hist, req.steps, mhist, req.problem.cells)
                    if v is None:
                        continue
                    if self.keep_moments and v != "diverged":
                        req.moments = bt.moments(slot)
                    if v == "diverged":
                        req.error = "non-finite residual: the solve diverged"
                    bt.remove(slot)  # a diverged slot frees its memory at once
                    del active[slot]
                    finish(req, v, hist[-1], now)
            if wide.active:
                res = wide.residuals(self.check_every)
                now = clock() - t0
                for key in list(wide.active):
                    req, s, _, _, (hist, mhist) = wide.active[key]
                    req.steps = s.info.steps_done
                    v = self.conv.verdict(hist, req.steps, mhist, req.problem.cells)
                    if v is None:
                        continue
                    if v == "diverged":
                        req.error = "non-finite residual: the solve diverged"
                    wide.retire(key, self.keep_moments and v != "diverged")
                    finish(req, v, res[key], now)
        return done


def run_plain_fifo(requests, check_every: int = 256, conv: Convergence | None = None, stream=None,
                   time_budget: float | None = None, clock=time.perf_counter):
    """The baseline: the plain single-domain solver, one request at a time in
    arrival order, with the same residual (lesbgk_residual) and convergence
    test."""
    import torch
    conv = conv or Convergence()
    done = []
    t0 = clock()
    for req in sorted(requests, key=lambda r: r.arrival):
        now = clock() - t0
        if now < req.arrival:
            time.sleep(req.arrival - now)
        if time_budget is not None and clock() - t0 > time_budget:
            break
        req.admitted = clock() - t0
        s = L.Solver(L.params_from_problem(req.problem), stream=stream)
        prev = torch.empty((4, req.problem.ny, req.problem.nx), dtype=torch.float32, device="cuda")
        r, m = s.residual(prev, 0, mass=True)
        hist, mhist = [r], [m]
        while True:
            s.step(check_every)
            r, m = s.residual(prev, check_every, mass=True)
            hist.append(r)
            mhist.append(m)
            v = conv.verdict(hist, s.info.steps_done, mhist, req.problem.cells)
            if v is not None:
                break
        req.status, req.residual, req.steps = v, hist[-1], s.info.steps_done
        req.completed = clock() - t0
        s.close()
        done.append(req)
    return done


def latency_summary(done):
    """Latency percentiles and throughput over the solved requests (converged,
    or settled on the wall-mass drift); every other ending (max_steps,
    diverged, rejected) is counted in `status` and not as a solve."""
    solved = [r for r in done if r.status in SOLVED]
    status = dict(collections.Counter(r.status for r in done))
    lat = np.array([r.completed - r.arrival for r in solved])
    if not len(lat):
        return {"completed": 0, "status": status}
    first = min(r.arrival for r in solved)
    last = max(r.completed for r in solved)
    return {"completed": len(solved), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "solves_per_s": len(solved) / max(last - first, 1e-9),
            "status": status, "not_solved": len(done) - len(solved)}
