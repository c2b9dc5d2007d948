"""Continuous-batching service for lattice ES-BGK solves.

Requests (a Problem each) arrive over time; each runs until its steady state.
The loop admits waiting requests into free batch slots as soon as the batch's
device pool has room for them (lesbgk_batch_add refusing with LESBGK_ESPACE
is the admission test), advances every admitted solve together in chunks of
`check_every` steps (CUDA-graph replays inside the library), reads the
per-slot residuals, and retires converged solves -- reading their moments and
returning their memory to the pool -- so that solves arriving while others
are on the GPU join them as slots free up.

Convergence: with r the residual of lesbgk_batch_residuals (max over nodes of
|d rho| + |d u| + |d T| per unit time since the previous check), a solve is
done when r < rtol, or when r has stopped changing (the last `plateau_checks`
values within `plateau_rel` of each other) -- the state then changes only at a
constant rate.  That second case is real: with walls hotter or colder than the
gas next to them, the diffuse-wall rule exchanges a small, constant amount of
mass per step (the FP64 oracle shows the same), so such solves approach a
constant drift rather than a fixed point.

Everything on the device runs in the library's kernels; this module is the
scheduler (host bookkeeping only).
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

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
    status: str = "pending"  # pending, running, converged, plateau, max_steps
    moments: object = None   # (9, ny, nx) float32 device tensor when kept


@dataclass
class Convergence:
    rtol: float = 1e-6
    plateau_rel: float = 0.02
    plateau_checks: int = 4
    max_steps: int = 400_000

    def verdict(self, hist, steps):
        if not hist:
            return None
        r = hist[-1]
        if np.isfinite(r) and r < self.rtol:
            return "converged"
        if len(hist) >= self.plateau_checks:
            tail = np.array(hist[-self.plateau_checks:])
            if np.all(np.isfinite(tail)) and np.ptp(tail) <= self.plateau_rel * np.max(tail):
                return "plateau"
        if steps >= self.max_steps:
            return "max_steps"
        return None


def poisson_trace(n: int, rate: float, problems, seed: int = 0):
    """n requests with exponential inter-arrival times (mean 1/rate s), the
    problem of request k drawn from `problems` in order."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    return [Request(rid=k, arrival=float(t[k]), problem=problems[k % len(problems)]) for k in range(n)]


def serving_mix(n: int, seed: int = 0, q36_share: float = 0.2, ny_hi: int = 512):
    """The channel mix of the batched benchmark (nx = 4, Couette / Fourier /
    Poiseuille, Kn log-uniform 0.01-0.5, b in {-1/2, 0, 1/2}) with ny
    log-uniform 16..ny_hi, and a share of the requests on D2Q36 (order 4)."""
    from dataclasses import replace
    probs = I.batch_mix(n=n, seed=seed, ny_hi=ny_hi)
    rng = np.random.default_rng(seed + 1)
    pick = rng.random(n) < q36_share
    return [replace(p, nroots=6) if q else p for p, q in zip(probs, pick)]


class ServingLoop:
    def __init__(self, capacity: int, pool_bytes: int, nx: int = 4, check_every: int = 256,
                 conv: Convergence | None = None, keep_moments: bool = False, stream=None):
        self.batch = L.Batch(capacity=capacity, nx=nx, pool_bytes=pool_bytes, stream=stream)
        self.check_every = check_every
        self.conv = conv or Convergence()
        self.keep_moments = keep_moments

    def run(self, requests, clock=time.perf_counter):
        bt = self.batch
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        active = {}  # slot -> (request, residual history)
        t0 = clock()
        done = []
        while pending or waiting or active:
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            while waiting:  # FIFO admission while the pool has room
                req = waiting[0]
                slot = bt.try_add(L.params_from_problem(req.problem))
                if slot is None:
                    break
                waiting.popleft()
                req.admitted = clock() - t0
                req.status = "running"
                active[slot] = (req, [])
            if not active:
                if pending:
                    time.sleep(max(0.0, min(pending[0].arrival - (clock() - t0), 0.01)))
                continue
            bt.step(self.check_every)
            res = bt.residuals()
            now = clock() - t0
            for slot in list(active):
                req, hist = active[slot]
                req.steps = bt.info(slot).steps_done
                hist.append(float(res[slot]))
                v = self.conv.verdict([h for h in hist if np.isfinite(h)], req.steps)
                if v is None:
                    continue
                req.status, req.residual, req.completed = v, hist[-1], now
                if self.keep_moments:
                    req.moments = bt.moments(slot)
                bt.remove(slot)
                del active[slot]
                done.append(req)
        return done


def run_plain_fifo(requests, check_every: int = 256, conv: Convergence | None = None, stream=None,
                   time_budget: float | None = None, clock=time.perf_counter):
    """The baseline: the plain single-domain solver, one request at a time in
    arrival order, with the same residual and convergence test (the residual
    from lesbgk_moments fields of consecutive checks)."""
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
        dt = s.info.dt
        prev = s.moments()[[0, 1, 2, 3]].clone()
        hist = []
        while True:
            s.step(check_every)
            cur = s.moments()[[0, 1, 2, 3]]
            r = float((cur - prev).abs().sum(dim=0).max().item()) / (check_every * dt)
            prev = cur.clone()
            hist.append(r)
            v = conv.verdict(hist, s.info.steps_done)
            if v is not None:
                break
        req.status, req.residual, req.steps = v, hist[-1], s.info.steps_done
        req.completed = clock() - t0
        s.close()
        done.append(req)
    return done


def latency_summary(done):
    lat = np.array([r.completed - r.arrival for r in done])
    if not len(lat):
        return {}
    first = min(r.arrival for r in done)
    last = max(r.completed for r in done)
    return {"completed": len(done), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "solves_per_s": len(done) / max(last - first, 1e-9),
            "status": dict(collections.Counter(r.status for r in done))}
