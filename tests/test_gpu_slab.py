"""The y-slab decomposition on one GPU: several slabs of one solve in one
process (slab.SlabRun: library solvers on extended grids, halos moved with
lesbgk_get_rows / lesbgk_set_rows every k steps) give bitwise the populations
and moments of the single-domain solve, periodic and walled, for every
storage and velocity set, and the slabs' FP64 totals add up to the whole
domain's."""
from __future__ import annotations

from dataclasses import replace

import numpy as np
import pytest

from paper_1209_6548_gb300 import build as B
from paper_1209_6548_gb300 import inputs as I
from paper_1209_6548_gb300 import lesbgk as L
from paper_1209_6548_gb300 import slab as SL
from tests.common import spacing, time_step

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def compare(prob, fields, nslabs, k, nsteps, storage=L.F32):
    dt = time_step(prob, fields)
    dx, dy = spacing(prob)
    p = L.params_from_problem(prob, dt=dt)
    p.storage = storage
    whole = L.Solver(p, h_init=fields)
    whole.step(nsteps)
    run = SL.SlabRun(prob, nslabs, k, fields, dt, dx, dy, storage)
    run.step(nsteps)
    ref_m, ref_s = whole.moments(sums=True)
    m, s = run.moments()
    assert bool((run.populations() == whole.populations()).all())
    assert bool((m == ref_m).all())
    assert np.allclose(s, ref_s, rtol=1e-12, atol=0.0)
    run.close()
    whole.close()


@pytest.mark.parametrize("nslabs,k", [(2, 1), (3, 2), (4, 4)])
def test_periodic_taylor_green(nslabs, k):
    prob = replace(I.tgv(128), ny=130, name="tgv128x130")
    compare(prob, I.initial_fields(prob), nslabs, k, 21)


@pytest.mark.parametrize("nslabs,k", [(2, 2), (3, 1)])
@pytest.mark.parametrize("scheme", [I.UNSPLIT, I.SPLIT])
def test_walls_force_rough(nslabs, k, scheme):
    prob = I.Problem(name="wf", nx=60, ny=61, bc_y=I.DIFFUSE, kn=0.08, b=0.5, wall_T=(0.96, 1.05),
                     wall_ux=(-0.04, 0.03), g=(2e-3, -1e-3), scheme=scheme)
    compare(prob, I.random_fields(prob, seed=9, amp_u=0.03, amp_T=0.03, amp_rho=0.03), nslabs, k, 13)


@pytest.mark.parametrize("storage,nroots,dim", [(L.F16, 4, 2), (L.BF16, 4, 2), (L.F32C, 4, 2), (L.F16, 6, 3),
                                                (L.BF16, 6, 2)])
def test_16bit_storage_rounds_by_global_row(storage, nroots, dim):
    """Stochastic rounding is keyed by the global row (row_offset), so the
    16-bit slabs are bitwise the single domain too (D3Q216's level warps
    included)."""
    prob = replace(I.tgv(64), ny=66, name="tgv64x66", nroots=nroots, dim=dim)
    compare(prob, I.initial_fields(prob), 3, 2, 10, storage)


@pytest.mark.parametrize("nroots,dim", [(6, 2), (4, 3), (6, 3)])
def test_other_velocity_sets_and_heated_maxwell_walls(nroots, dim):
    prob = I.Problem(name="hm", nroots=nroots, dim=dim, nx=33, ny=40, bc_y=I.DIFFUSE, kn=0.2, b=-0.5,
                     wall_specular=0.3, wall_T_amp=0.02, wall_T_freq=0.55536, wall_ux=(0.0, 0.05))
    compare(prob, I.random_fields(prob, seed=4, amp_u=0.02, amp_T=0.02, amp_rho=0.02), 2, 2, 9)


def test_cavity_walls_in_x():
    prob = replace(I.lid_driven_cavity(n=45, u_lid=0.05, kn=0.1), ny=37)
    compare(prob, None, 3, 1, 12)


def test_rows_round_trip_and_bounds():
    """get_rows / set_rows copy the packed rows exactly, and rows outside
    the grid are refused."""
    import torch
    prob = I.Problem(name="rt", nx=30, ny=20, bc_y=I.PERIODIC, kn=0.1, b=0.0)
    s = L.Solver(L.params_from_problem(prob), h_init=I.random_fields(prob, seed=1))
    slab = SL.Slab(0, 1, 20, 0, 20, 0, 0, True)
    st = SL.GpuSlab.__new__(SL.GpuSlab)
    st._torch, st._L, st.slab, st.solver = torch, L, slab, s
    before = s.populations().clone()
    rows = st.get_rows(3, 5)
    assert rows.numel() == 16 * 5 * 30 * 4
    st.set_rows(11, 5, rows)
    after = s.populations()
    assert bool((after[:, 11:16] == before[:, 3:8]).all())
    assert bool((after[:, :11] == before[:, :11]).all()) and bool((after[:, 16:] == before[:, 16:]).all())
    for j0, n in ((-1, 2), (19, 2), (0, 21)):
        with pytest.raises(L.LesbgkError):
            st.get_rows(j0, n)
