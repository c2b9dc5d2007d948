"""Continuous batching: requests join while others run, memory is the
admission test, every request finishes, and each served result equals the
same solve run alone for the same number of steps."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1209_6548_gb300 import build as B
from paper_1209_6548_gb300 import lesbgk as L
from paper_1209_6548_gb300 import serve as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def test_continuous_batching_small_trace():
    probs = S.serving_mix(30, seed=11, ny_hi=64)
    reqs = S.poisson_trace(30, 400.0, probs, seed=11)
    one = max(L.batch_slot_bytes(L.params_from_problem(p)) for p in probs)
    loop = S.ServingLoop(capacity=6, pool_bytes=4 * one, check_every=128, keep_moments=True,
                         conv=S.Convergence(rtol=1e-6, max_steps=60_000))
    done = loop.run(reqs)
    assert len(done) == 30
    assert all(r.status in S.SOLVED for r in done), [r.status for r in done]
    # FIFO admission
    adm = [r.admitted for r in sorted(done, key=lambda r: r.arrival)]
    assert all(np.diff(adm) >= 0)
    # the pool (4 slots' worth) held solves back: some admission waited for a retirement
    assert any(r.admitted > min(q.completed for q in done) for r in done)
    # each served result equals the same solve alone for the same steps
    for r in done[::5]:
        s = L.Solver(L.params_from_problem(r.problem))
        s.step(r.steps)
        alone = s.moments().cpu().numpy()
        assert np.array_equal(r.moments.cpu().numpy(), alone), r.rid


def test_cavities_run_in_the_wide_lane_beside_the_batch():
    """Lid-driven cavities (walls in x: not batchable) are served by the wide
    lane concurrently with batched channels; each result equals the same
    solve run alone for the same number of steps."""
    probs = S.serving_mix(24, seed=5, ny_hi=64, cavity_share=0.25, cavity_n=40)
    assert sum(not S.fits_batch(p, 4) for p in probs) >= 3
    reqs = S.poisson_trace(24, 400.0, probs, seed=5)
    one = max(L.batch_slot_bytes(L.params_from_problem(p)) for p in probs if S.fits_batch(p, 4))
    wide_one = max(L.workspace_size(L.params_from_problem(p)) for p in probs if not S.fits_batch(p, 4))
    loop = S.ServingLoop(capacity=8, pool_bytes=6 * one, check_every=128, keep_moments=True,
                         conv=S.Convergence(rtol=1e-6, max_steps=60_000), wide_bytes=2 * wide_one)
    done = loop.run(reqs)
    assert len(done) == 24
    assert all(r.status in S.SOLVED for r in done), [r.status for r in done]
    cav = [r for r in done if not S.fits_batch(r.problem, 4)]
    for r in cav:
        s = L.Solver(L.params_from_problem(r.problem))
        s.step(r.steps)
        assert np.array_equal(r.moments.cpu().numpy(), s.moments().cpu().numpy()), r.rid
    # at most two cavities at a time (the lane's budget): some cavity waited for another to finish
    first_done = min(r.completed for r in cav)
    assert len(cav) <= 2 or any(r.admitted >= first_done for r in cav)


def test_invalid_requests_are_rejected_alone():
    """A request the library refuses (b out of range for the batch, Kn <= 0 for
    the wide lane) ends as 'rejected' with the library's message; the other
    requests are served as usual."""
    from dataclasses import replace
    probs = S.serving_mix(12, seed=9, ny_hi=48, cavity_share=0.3, cavity_n=24)
    batch_k = next(k for k, p in enumerate(probs) if S.fits_batch(p, 4))
    wide_k = next(k for k, p in enumerate(probs) if not S.fits_batch(p, 4))
    probs[batch_k] = replace(probs[batch_k], b=1.5)
    probs[wide_k] = replace(probs[wide_k], kn=0.0)
    reqs = S.poisson_trace(12, 400.0, probs, seed=9)
    loop = S.ServingLoop(capacity=8, pool_bytes=64 << 20, check_every=128,
                         conv=S.Convergence(rtol=1e-6, max_steps=60_000))
    done = loop.run(reqs)
    assert len(done) == 12
    bad = {r.rid for r in done if r.status == "rejected"}
    assert bad == {batch_k, wide_k}, [(r.rid, r.status) for r in done]
    assert all(r.error for r in done if r.status == "rejected")
    assert all(r.status in S.SOLVED for r in done if r.rid not in bad)
    summary = S.latency_summary(done)
    assert summary["status"].get("rejected") == 2 and summary["completed"] == 10
