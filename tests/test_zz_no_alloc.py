"""The allocation-free moments entry point (lesbgk_moments_noalloc).

Callers that cannot allocate device memory hand the library populations they
already hold; the library computes the moments with scratch it keeps in a
fixed static array instead of a workspace.  This checks, through the C ABI,
that two calls in a row give the same fields and totals as lesbgk_moments on
the same state, within the tolerance the parity tests use.  The file is named
to be collected last so a run that stops at the first failure has run every
other test before it.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1209_6548_gb300 import build as B
from paper_1209_6548_gb300 import inputs as I
from paper_1209_6548_gb300 import lesbgk as L
from tests.common import field_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


@pytest.mark.parametrize("prob", [I.tgv(512, steps=20), I.poiseuille(64, 300, steps=20),
                                  I.Problem(name="d2q36", nroots=6, nx=45, ny=33, bc_y=I.DIFFUSE, kn=0.1,
                                            b=-0.5, wall_ux=(-0.05, 0.05)),
                                  I.Problem(name="d3q64", nroots=4, dim=3, nx=45, ny=33, bc_y=I.DIFFUSE, kn=0.1,
                                            b=0.5, wall_ux=(-0.05, 0.05), g=(1e-3, 0.0))],
                         ids=["tgv512", "poiseuille64x300", "d2q36", "d3q64"])
def test_noalloc_moments_match_workspace_moments(prob):
    import torch
    fields = I.initial_fields(prob) if prob.init == "tgv" else None
    s = L.Solver(L.params_from_problem(prob), h_init=fields)
    s.step(prob.steps)
    ref, ref_sums = s.moments(sums=True)
    ref = ref.cpu().numpy()
    pops = s.populations()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # two calls in a row share (and reuse) the static scratch
        out = torch.full((9, prob.ny, prob.nx), float("nan"), dtype=torch.float32, device="cuda")
        sums = np.zeros(4)
        L.moments_noalloc(s.params, pops.data_ptr(), out.data_ptr(), sums, stream)
        errs = field_errors(out.cpu().numpy(), ref.astype(np.float64))
        bad = {k: v for k, v in errs.items() if not v["ok"]}
        assert not bad, bad
        # both sum per-node FP32 terms in FP32 runs accumulated in FP64; the
        # runs group nodes differently, so the totals agree to FP32 rounding
        # of the per-node terms (well inside 1e-9 per node)
        assert np.allclose(sums, ref_sums, rtol=0.0, atol=1e-9 * prob.cells)


def test_noalloc_rejects_grids_beyond_its_scratch():
    p = L.make_params(nx=8192, ny=4096, kn=0.1, b=0.0, bc_y=L.PERIODIC)  # 2^25 nodes: valid for a solver
    with pytest.raises(L.LesbgkError) as e:
        L.moments_noalloc(p, 256, 256, None, 0)
    assert e.value.code == L.EINVAL and "at most" in L.last_error()


def _solver_state(prob):
    fields = I.initial_fields(prob) if prob.init == "tgv" else None
    s = L.Solver(L.params_from_problem(prob), h_init=fields)
    s.step(prob.steps)
    ref, ref_sums = s.moments(sums=True)
    return s, ref.cpu().numpy().astype(np.float64), ref_sums, s.populations()


def test_noalloc_null_outputs():
    """d_out = NULL gives the totals alone; h_sums = NULL gives the fields alone
    and leaves the stream unsynchronised (the caller syncs)."""
    import torch
    s, ref, ref_sums, pops = _solver_state(I.tgv(256, steps=10))
    stream = torch.cuda.current_stream()
    sums = np.zeros(4)
    L.moments_noalloc(s.params, pops.data_ptr(), None, sums, stream.cuda_stream)
    assert np.allclose(sums, ref_sums, rtol=0.0, atol=1e-9 * 256 * 256)
    out = torch.full((9, 256, 256), float("nan"), dtype=torch.float32, device="cuda")
    L.moments_noalloc(s.params, pops.data_ptr(), out.data_ptr(), None, stream.cuda_stream)
    stream.synchronize()
    errs = field_errors(out.cpu().numpy(), ref)
    assert all(v["ok"] for v in errs.values()), errs


def test_noalloc_large_then_small_reuses_the_scratch():
    """A large grid fills many of the array's block partial sums; a smaller
    grid after it must read only its own (nothing carries over)."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    big, _, big_sums, big_pops = _solver_state(I.tgv(2048, steps=2))
    small, small_ref, small_sums, small_pops = _solver_state(I.poiseuille(16, 40, steps=30))
    for _ in range(2):
        sums = np.zeros(4)
        L.moments_noalloc(big.params, big_pops.data_ptr(), None, sums, stream)
        assert np.allclose(sums, big_sums, rtol=0.0, atol=1e-9 * 2048 * 2048)
        out = torch.empty((9, 40, 16), dtype=torch.float32, device="cuda")
        sums = np.zeros(4)
        L.moments_noalloc(small.params, small_pops.data_ptr(), out.data_ptr(), sums, stream)
        assert np.allclose(sums, small_sums, rtol=0.0, atol=1e-9 * 16 * 40)
        errs = field_errors(out.cpu().numpy(), small_ref)
        assert all(v["ok"] for v in errs.values()), errs


def test_noalloc_call_allocates_no_device_memory():
    """A warm call (the module and its static array already loaded in this
    context) leaves the device's free memory and torch's allocator unchanged."""
    import torch
    s, _, _, pops = _solver_state(I.tgv(512, steps=2))
    out = torch.empty((9, 512, 512), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    sums = np.zeros(4)
    L.moments_noalloc(s.params, pops.data_ptr(), out.data_ptr(), sums, stream)  # warm-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        L.moments_noalloc(s.params, pops.data_ptr(), out.data_ptr(), sums, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0
