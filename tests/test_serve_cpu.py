"""Host-side logic of the serving loop (no GPU): the convergence verdict, the
eviction of diverged solves, and faults injected on the host through a fake
batch -- a full pool at admission, a problem the library refuses, a deadline
passed, requests cancelled -- and the seeded arrival trace."""
from __future__ import annotations

import numpy as np

from paper_1209_6548_gb300 import inputs as I
from paper_1209_6548_gb300 import lesbgk as L
from paper_1209_6548_gb300 import serve as S


def test_verdict_threshold_diverged_and_cap():
    c = S.Convergence(rtol=1e-6, max_steps=1000)
    assert c.verdict([], 0) is None
    assert c.verdict([np.nan], 0) is None  # the first check has no residual yet
    assert c.verdict([np.nan, 1e-3, 1e-5, 5e-7], 100) == "converged"
    assert c.verdict([np.nan, 1e-3, 5e-4, 2e-4], 100) is None
    assert c.verdict([np.nan, 1e-3, 5e-4, 2e-4, 1e-4], 1000) == "max_steps"
    assert c.verdict([np.nan, 1e-3, np.inf], 100) == "diverged"
    assert c.verdict([np.nan, 1e-3, np.nan], 100) == "diverged"


def _drifting(t, floor=1.3e-5, amp=1e-3, tau=2000.0, rate=2e-7):
    """A residual decaying exponentially (time constant tau) onto a floor, and
    a mass growing by a transient plus a constant drift."""
    r = floor + amp * np.exp(-t / tau)
    m = 4096.0 + rate * t - 0.05 * np.exp(-t / tau)
    return r, m


def test_steady_drift_needs_the_transient_gone_and_a_linear_mass():
    c = S.Convergence(rtol=1e-8)
    t = np.arange(0, 200_001, 256.0)
    r, m = _drifting(t)
    r[0] = np.nan
    found = None
    for k in range(2, len(t)):
        v = c.verdict(list(r[:k]), int(t[k - 1]), list(m[:k]), nodes=4096)
        if v is not None:
            found = (v, t[k - 1])
            break
    assert found is not None and found[0] == "steady_drift"
    # declared only once the decaying part amp exp(-t/tau) is below 1e-8
    assert 1e-3 * np.exp(-found[1] / 2000.0) < 1e-8
    # the same residual floor without the drift signature -- a constant mass,
    # or one whose rate keeps changing (quadratic) -- gets no verdict
    for m_other in (np.full_like(t, 4096.0), 4096.0 + 1e-9 * t * t):
        assert all(c.verdict(list(r[:k]), int(t[k - 1]), list(m_other[:k]), nodes=4096) is None
                   for k in range(2, len(t)))


def test_slow_exponential_approach_is_not_a_plateau():
    """A residual still decaying with a time constant far beyond the checks
    (the case a fixed-ratio plateau test passed after a few checks) is not
    declared steady: Aitken's estimate of its transient stays large."""
    c = S.Convergence(rtol=1e-8, max_steps=10**9)
    t = np.arange(0, 40_001, 256.0)
    r, m = _drifting(t, floor=1e-6, amp=1e-4, tau=50_000.0)
    r[0] = np.nan
    assert all(c.verdict(list(r[:k]), int(t[k - 1]), list(m[:k]), nodes=4096) is None for k in range(2, len(t)))


class FakeBatch:
    """Stands in for L.Batch: per-problem residual and mass trajectories,
    `capacity` slots."""

    def __init__(self, capacity, traj):
        self.capacity, self.traj = capacity, traj
        self.slots = {}   # slot -> [problem name, steps done, checks]
        self.removed = []

    def try_add(self, p):
        for k in range(self.capacity):
            if k not in self.slots:
                self.slots[k] = [self._names.pop(0), 0, 0]
                return k
        return None

    def step(self, n):
        for v in self.slots.values():
            v[1] += n

    def residuals(self, mass=False):
        res, ms = np.full(self.capacity, np.nan), np.full(self.capacity, np.nan)
        for k, (name, steps, checks) in self.slots.items():
            res[k], ms[k] = self.traj[name](steps, checks)
            self.slots[k][2] += 1
        return (res, ms) if mass else res

    def info(self, slot):
        return type("Info", (), {"steps_done": self.slots[slot][1]})

    def moments(self, slot):
        return None

    def remove(self, slot):
        self.removed.append((self.slots[slot][0], self.slots[slot][1]))
        del self.slots[slot]


class NoWide:
    active = {}

    def try_admit(self, req):
        raise AssertionError("every problem here fits the batch")


def test_diverged_solve_is_evicted_at_once_and_frees_its_slot():
    probs = [I.Problem(name=n, nx=4, ny=32) for n in ("ok0", "boom", "ok1", "ok2")]
    reqs = [S.Request(rid=k, arrival=0.0, problem=p) for k, p in enumerate(probs)]

    def converging(steps, checks):
        return (np.nan if checks == 0 else 1e-3 * np.exp(-steps / 300.0)), 128.0

    def diverging(steps, checks):
        return (np.nan if checks == 0 else (1e-3 if checks < 3 else np.inf)), 128.0

    fb = FakeBatch(2, {"ok0": converging, "ok1": converging, "ok2": converging, "boom": diverging})
    fb._names = [p.name for p in probs]
    loop = S.ServingLoop(capacity=2, pool_bytes=0, check_every=128, batch=fb, wide=NoWide(),
                         conv=S.Convergence(rtol=1e-8, max_steps=100_000))
    done = loop.run(reqs, clock=lambda: 0.0)
    status = {r.problem.name: r.status for r in done}
    assert status == {"ok0": "converged", "boom": "diverged", "ok1": "converged", "ok2": "converged"}
    boom = next(r for r in done if r.problem.name == "boom")
    assert boom.error and boom.steps == 4 * 128  # evicted at the first non-finite residual (4th check)
    assert ("boom", 4 * 128) in fb.removed
    summary = S.latency_summary(done)
    assert summary["completed"] == 3 and summary["status"]["diverged"] == 1


def test_poisson_trace_is_seeded_and_ordered():
    probs = S.serving_mix(10, seed=3)
    a = S.poisson_trace(50, 200.0, probs, seed=3)
    b = S.poisson_trace(50, 200.0, probs, seed=3)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    t = np.array([r.arrival for r in a])
    assert np.all(np.diff(t) > 0)
    assert 0.1 < t[-1] < 0.5  # 50 arrivals at 200/s


def test_serving_mix_share():
    probs = S.serving_mix(1000, seed=0, q36_share=0.2)
    share = np.mean([p.nroots == 6 for p in probs])
    assert 0.15 < share < 0.25
    assert all(p.nx == 4 and 16 <= p.ny <= 512 for p in probs)


def test_serving_mix_cavities_go_to_the_wide_lane():
    probs = S.serving_mix(1000, seed=0, q36_share=0.2, cavity_share=0.1, cavity_n=256)
    cav = [p for p in probs if p.bc_x == 1]
    assert 70 <= len(cav) <= 130
    assert all(p.nx == p.ny == 256 and p.wall_ux == (0.0, 0.05) and 0.05 <= p.kn <= 0.5 for p in cav)
    assert all(not S.fits_batch(p, 4) for p in cav)
    assert all(S.fits_batch(p, 4) for p in probs if p.bc_x == 0)


# ---------------------------------------------------------------- faults injected on the host
def converging(steps, checks):
    return (np.nan if checks == 0 else 1e-3 * np.exp(-steps / 300.0)), 128.0


def never_settling(steps, checks):
    return (np.nan if checks == 0 else 1e-3), 128.0  # r stays at 1e-3 with no mass drift: never steady


class TickClock:
    """A clock that advances `dt` seconds per reading (deterministic time)."""

    def __init__(self, dt):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t


def test_full_pool_keeps_requests_waiting_then_admits_them():
    """A batch that refuses admission (the pool full: try_add returns None)
    for its first calls: requests wait, none is lost or rejected, and they are
    admitted once it has room, in arrival order."""
    probs = [I.Problem(name=f"c{k}", nx=4, ny=32) for k in range(4)]
    reqs = [S.Request(rid=k, arrival=0.0, problem=p) for k, p in enumerate(probs)]

    class FullAtFirst(FakeBatch):
        refusals = 5

        def try_add(self, p):
            if self.refusals:
                self.refusals -= 1
                return None
            return super().try_add(p)

    fb = FullAtFirst(1, {p.name: converging for p in probs})
    fb._names = [p.name for p in probs]
    loop = S.ServingLoop(capacity=1, pool_bytes=0, check_every=128, batch=fb, wide=NoWide(),
                         conv=S.Convergence(rtol=1e-8, max_steps=100_000))
    done = loop.run(reqs, clock=TickClock(1e-3))
    assert [r.problem.name for r in done] == ["c0", "c1", "c2", "c3"]  # one slot: in arrival order
    assert all(r.status == "converged" for r in done)
    assert [n for n, _ in fb.removed] == ["c0", "c1", "c2", "c3"]


def test_a_refused_problem_is_rejected_alone():
    probs = [I.Problem(name=n, nx=4, ny=32) for n in ("a", "bad", "b")]
    reqs = [S.Request(rid=k, arrival=0.0, problem=p) for k, p in enumerate(probs)]

    class Refusing(FakeBatch):
        def try_add(self, p):
            if self._names[0] == "bad":
                self._names.pop(0)
                raise L.LesbgkError(L.EINVAL, "refused")
            return super().try_add(p)

    fb = Refusing(4, {n: converging for n in ("a", "b")})
    fb._names = [p.name for p in probs]
    loop = S.ServingLoop(capacity=4, pool_bytes=0, check_every=128, batch=fb, wide=NoWide(),
                         conv=S.Convergence(rtol=1e-8, max_steps=100_000))
    done = loop.run(reqs, clock=TickClock(1e-3))
    status = {r.problem.name: r.status for r in done}
    assert status == {"a": "converged", "bad": "rejected", "b": "converged"}
    assert next(r for r in done if r.problem.name == "bad").error


def test_deadline_ends_a_running_solve_and_frees_its_slot():
    """A request that cannot settle before its deadline ends as timed_out at
    the next check past it, its slot released; the others finish."""
    probs = [I.Problem(name=n, nx=4, ny=32) for n in ("slow", "ok0", "ok1")]
    reqs = [S.Request(rid=0, arrival=0.0, problem=probs[0], deadline=0.05),
            S.Request(rid=1, arrival=0.0, problem=probs[1]), S.Request(rid=2, arrival=0.0, problem=probs[2])]
    fb = FakeBatch(2, {"slow": never_settling, "ok0": converging, "ok1": converging})
    fb._names = [p.name for p in probs]
    loop = S.ServingLoop(capacity=2, pool_bytes=0, check_every=128, batch=fb, wide=NoWide(),
                         conv=S.Convergence(rtol=1e-8, max_steps=10_000_000))
    done = loop.run(reqs, clock=TickClock(1e-3))
    status = {r.problem.name: r.status for r in done}
    assert status == {"slow": "timed_out", "ok0": "converged", "ok1": "converged"}
    slow = next(r for r in done if r.problem.name == "slow")
    assert 0.05 < slow.completed < 0.2 and slow.steps > 0
    assert any(n == "slow" for n, _ in fb.removed)


def test_cancel_ends_a_running_and_a_queued_request():
    """ServingLoop.cancel(rid): a running solve is removed from the batch at
    the next pass, a queued one never starts; the rest are unaffected."""
    probs = [I.Problem(name=n, nx=4, ny=32) for n in ("run", "queued", "ok")]
    reqs = [S.Request(rid=k, arrival=0.0, problem=p) for k, p in enumerate(probs)]
    fb = FakeBatch(1, {"run": never_settling, "queued": converging, "ok": converging})
    fb._names = [p.name for p in probs]
    loop = S.ServingLoop(capacity=1, pool_bytes=0, check_every=128, batch=fb, wide=NoWide(),
                         conv=S.Convergence(rtol=1e-8, max_steps=10_000_000))
    step0 = fb.step

    def step(n):  # the caller cancels two requests while "run" is on the GPU
        step0(n)
        if fb.slots.get(0, [None])[0] == "run" and fb.slots[0][1] >= 1280:
            loop.cancel(0)
            loop.cancel(1)
    fb.step = step
    fb._names = ["run", "ok"]  # "queued" is dropped before it reaches the batch
    done = loop.run(reqs, clock=TickClock(1e-3))
    status = {r.problem.name: r.status for r in done}
    assert status == {"run": "cancelled", "queued": "cancelled", "ok": "converged"}
    assert [n for n, _ in fb.removed] == ["run", "ok"]
