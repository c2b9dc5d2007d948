"""Host-side logic of the serving loop (no GPU): the convergence verdict and
the seeded arrival trace."""
from __future__ import annotations

import numpy as np

from paper_1209_6548_gb300 import serve as S


def test_verdict_threshold_plateau_and_cap():
    c = S.Convergence(rtol=1e-6, plateau_rel=0.02, plateau_checks=4, max_steps=1000)
    assert c.verdict([], 0) is None
    assert c.verdict([1e-3, 1e-5, 5e-7], 100) == "converged"
    assert c.verdict([1e-3, 5e-4, 2e-4], 100) is None
    assert c.verdict([3e-5, 1.31e-5, 1.32e-5, 1.315e-5, 1.32e-5], 100) == "plateau"
    assert c.verdict([1e-3, 5e-4, 2e-4, 1e-4], 1000) == "max_steps"


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
