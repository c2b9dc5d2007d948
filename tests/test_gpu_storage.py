"""16-bit population storage (FP32 compute): runs, conserves, round-trips,
and stays within its stated error bound against the FP64 oracle.

The bound is derived, per field and per case, by tests.common.rounding_bound:
the random walk of one stochastic rounding per stored value and step (std at
most 2^-11 |df| in FP16, 2^-8 |df| in BF16), through each moment's
sensitivity to the stored values, evaluated on the oracle's populations.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1209_6548_gb300 import build as B
from paper_1209_6548_gb300 import inputs as I
from paper_1209_6548_gb300 import lesbgk as L
from tests.common import field_errors, oracle_params, record, rounding_bound, time_step

pytestmark = pytest.mark.gpu

STORE = {L.F16: "f16", L.BF16: "bf16", L.F32: "f32"}


def assert_within_bound(gpu_moments, prob, op, states, n, storage, what):
    """Every field within its storage-rounding bound after n steps (states:
    the oracle's populations at the start and at step n)."""
    ref, _ = O.moments(op, states[-1])
    bnd = rounding_bound(states, prob.nroots, prob.dim, n, STORE[storage], prob, op.dt)
    errs = field_errors(gpu_moments, ref, bnd)
    record(what, errs)
    bad = {k: v for k, v in errs.items() if not v["ok"]}
    assert not bad, f"{what}: {bad}"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def solver(prob, storage, fields=None, dt=None):
    p = L.params_from_problem(prob, dt=dt or 0.0)
    p.storage = storage
    return L.Solver(p, h_init=fields)


@pytest.mark.parametrize("storage", [L.F16, L.BF16])
def test_couette_against_oracle(storage):
    prob = I.couette_4x64()
    dt = time_step(prob)
    s = solver(prob, storage, dt=dt)
    s.step(2000)
    op = oracle_params(prob, dt)
    f0 = O.init(op)
    assert_within_bound(s.moments().cpu().numpy(), prob, op, [f0, O.run(op, f0, 2000)], 2000, storage,
                        f"couette {STORE[storage]}")


@pytest.mark.parametrize("storage", [L.F16, L.BF16])
@pytest.mark.parametrize("nroots", [4, 6])
@pytest.mark.parametrize("scheme", [I.UNSPLIT, I.SPLIT])
def test_rough_fields_short_run(storage, nroots, scheme):
    prob = I.Problem(name="r", nroots=nroots, nx=60, ny=33, bc_y=I.PERIODIC, kn=0.05, b=-0.5, scheme=scheme)
    fields = I.random_fields(prob, seed=nroots, amp_u=0.02, amp_T=0.02, amp_rho=0.02)
    dt = time_step(prob, fields)
    s = solver(prob, storage, fields, dt)
    s.step(5)
    op = oracle_params(prob, dt)
    f0 = O.init(op, fields)
    assert_within_bound(s.moments().cpu().numpy(), prob, op, [f0, O.run(op, f0, 5)], 5, storage,
                        f"rough nroots={nroots} scheme={scheme} {STORE[storage]}")


@pytest.mark.parametrize("storage", [L.F16, L.BF16])
def test_populations_round_trip(storage):
    """set then get returns the values rounded to the storage: relative
    deviation (f - w)/w within half an ulp of the 16-bit type."""
    import torch
    prob = I.Problem(name="t", nx=28, ny=9, bc_y=I.PERIODIC, kn=0.1, b=0.0)
    s = solver(prob, storage)
    w = torch.tensor(O.velocity_set(4)[2], dtype=torch.float32, device="cuda")[:, None, None]
    g = torch.Generator(device="cuda").manual_seed(0)
    x = (torch.rand((16, 9, 28), generator=g, device="cuda") - 0.5) * 0.2 * w
    s.set_populations(x, 0)
    y = s.populations()
    rel = ((y - x) / w).abs().max().item()
    half_ulp = {L.F16: 2.0 ** -11, L.BF16: 2.0 ** -8}[storage] * 0.1  # |(f - w)/w| <= 0.1 here
    assert rel <= half_ulp * 1.01


@pytest.mark.parametrize("storage", [L.F16, L.BF16])
def test_periodic_mass_conservation(storage):
    prob = I.tgv(128, steps=100)
    fields = I.initial_fields(prob)
    s = solver(prob, storage, fields)
    _, s0 = s.moments(sums=True)
    s.step(100)
    _, s1 = s.moments(sums=True)
    # flux form conserves exactly; only the 16-bit rounding of the stored values changes mass
    assert abs(s1[0] - s0[0]) < 1e-3 * prob.cells * {L.F16: 1e-3, L.BF16: 1e-2}[storage]


@pytest.mark.parametrize("storage", [L.F16, L.BF16])
def test_wall_heating_16bit(storage):
    """Heated walls (Sec. 4.2) with 16-bit storage: the per-step FP64 wall
    tables serve every storage."""
    prob = I.unsteady_heating(kn=0.1, st=0.5553603672697958, amp=0.02, ny=40)
    dt = time_step(prob)
    s = solver(prob, storage, dt=dt)
    s.step(600)
    op = oracle_params(prob, dt)
    f0 = O.init(op)
    assert_within_bound(s.moments().cpu().numpy(), prob, op, [f0, O.run(op, f0, 600)], 600, storage,
                        f"heated walls {STORE[storage]}")


@pytest.mark.parametrize("storage", [L.F16, L.BF16])
def test_d3q64_16bit(storage):
    """16-bit storage of the D3Q64 set (its z-even half, 3D weights in the
    scale tables): Couette and rough periodic fields against the 64-velocity
    oracle within the storage's bound."""
    from dataclasses import replace
    prob = replace(I.couette_4x64(), dim=3)
    dt = time_step(prob)
    s = solver(prob, storage, dt=dt)
    s.step(1000)
    op = oracle_params(prob, dt)
    f0 = O.init(op)
    assert_within_bound(s.moments().cpu().numpy(), prob, op, [f0, O.run(op, f0, 1000)], 1000, storage,
                        f"d3q64 couette {STORE[storage]}")
    prob = I.Problem(name="r", nroots=4, dim=3, nx=60, ny=33, bc_y=I.PERIODIC, kn=0.05, b=-0.5, scheme=I.SPLIT)
    fields = I.random_fields(prob, seed=3, amp_u=0.02, amp_T=0.02, amp_rho=0.02)
    dt = time_step(prob, fields)
    s = solver(prob, storage, fields, dt)
    s.step(5)
    op = oracle_params(prob, dt)
    f0 = O.init(op, fields)
    assert_within_bound(s.moments().cpu().numpy(), prob, op, [f0, O.run(op, f0, 5)], 5, storage,
                        f"d3q64 rough {STORE[storage]}")


@pytest.mark.parametrize("storage", [L.F16, L.BF16])
def test_d3q216_16bit(storage):
    """16-bit storage of the D3Q216 set (108 stored values per node over three
    level warps, each level's scale factors and random words those of the
    one-thread layout): a Couette channel, rough periodic fields and rough
    fields between moving walls at two temperatures with a body force against
    the 216-velocity oracle within the storage's bound."""
    from dataclasses import replace
    prob = replace(I.couette_4x64(), dim=3, nroots=6)
    dt = time_step(prob)
    s = solver(prob, storage, dt=dt)
    s.step(400)
    op = oracle_params(prob, dt)
    f0 = O.init(op)
    assert_within_bound(s.moments().cpu().numpy(), prob, op, [f0, O.run(op, f0, 400)], 400, storage,
                        f"d3q216 couette {STORE[storage]}")
    for prob in (I.Problem(name="r", nroots=6, dim=3, nx=60, ny=33, bc_y=I.PERIODIC, kn=0.05, b=-0.5,
                           scheme=I.SPLIT),
                 replace(I.unsteady_heating(kn=0.1, amp=0.02, ny=30), nroots=6, dim=3, name="heat"),
                 I.Problem(name="wf", nroots=6, dim=3, nx=40, ny=30, bc_y=I.DIFFUSE, kn=0.1, b=0.5,
                           wall_ux=(-0.05, 0.05), wall_T=(0.97, 1.04), g=(1e-3, 0.0))):
        fields = I.random_fields(prob, seed=3, amp_u=0.02, amp_T=0.02, amp_rho=0.02)
        dt = time_step(prob, fields)
        s = solver(prob, storage, fields, dt)
        s.step(8)
        op = oracle_params(prob, dt)
        f0 = O.init(op, fields)
        assert_within_bound(s.moments().cpu().numpy(), prob, op, [f0, O.run(op, f0, 8)], 8, storage,
                            f"d3q216 {prob.name} {STORE[storage]}")


@pytest.mark.parametrize("storage", [L.F16, L.BF16])
@pytest.mark.parametrize("nroots,dim", [(4, 2), (6, 2), (4, 3), (6, 3)])
def test_walls_in_x_16bit(storage, nroots, dim):
    """16-bit storage with walls in x: a box with heated walls on all sides and
    a lid, and a channel walled in x only, rough fields, every set, against
    the oracle within the storage's bound."""
    for prob in (I.Problem(name="box", nroots=nroots, dim=dim, nx=40, ny=33, bc_y=I.DIFFUSE, bc_x=I.DIFFUSE,
                           kn=0.1, b=0.5, wall_ux=(0.0, 0.05), wall_T=(0.98, 1.02), wall_Tx=(1.03, 0.97),
                           scheme=I.SPLIT),
                 I.Problem(name="xchan", nroots=nroots, dim=dim, nx=29, ny=30, bc_y=I.PERIODIC, bc_x=I.DIFFUSE,
                           kn=0.05, b=-0.5, wall_Tx=(0.97, 1.04), g=(0.0, 1e-3), scheme=I.SPLIT)):
        fields = I.random_fields(prob, seed=prob.nx + 7, amp_u=0.02, amp_T=0.02, amp_rho=0.02)
        dt = time_step(prob, fields)
        s = solver(prob, storage, fields, dt)
        s.step(12)
        op = oracle_params(prob, dt)
        f0 = O.init(op, fields)
        assert_within_bound(s.moments().cpu().numpy(), prob, op, [f0, O.run(op, f0, 12)], 12, storage,
                            f"{prob.name} nroots={nroots} D={dim} {STORE[storage]}")


# ---------------------------------------------------------------- compensated FP32 (hi + lo)
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("scheme", [I.UNSPLIT, I.SPLIT])
def test_compensated_rough_fields_and_walls(scheme, dim):
    """hi + lo storage on rough periodic fields and on rough walled channels
    with moving, heated walls and a force: within the FP32 bound, every field."""
    for prob in (I.Problem(name="r", nroots=4, dim=dim, nx=60, ny=33, bc_y=I.PERIODIC, kn=0.05, b=-0.5,
                           scheme=scheme),
                 I.Problem(name="w", nroots=4, dim=dim, nx=45, ny=37, bc_y=I.DIFFUSE, kn=0.08, b=0.5,
                           wall_T=(0.97, 1.03), wall_ux=(-0.04, 0.03), g=(1e-3, -5e-4), wall_T_amp=0.01,
                           wall_T_freq=0.55536, scheme=scheme)):
        fields = I.random_fields(prob, seed=7, amp_u=0.03, amp_T=0.03, amp_rho=0.03)
        dt = time_step(prob, fields)
        s = solver(prob, L.F32C, fields, dt)
        op = oracle_params(prob, dt)
        f0 = O.init(op, fields)
        done, f = 0, f0
        for n in (1, 10):
            s.step(n - done)
            op.time = done * dt
            f = O.run(op, f, n - done)
            done = n
            ref, _ = O.moments(op, f)
            errs = field_errors(s.moments().cpu().numpy(), ref,
                                rounding_bound([f0, f], prob.nroots, prob.dim, n, "f32c", prob, dt))
            record(f"compensated {prob.name} D={dim} scheme={scheme} step {n}", errs)
            bad = {k: v for k, v in errs.items() if not v["ok"]}
            assert not bad, bad


def test_compensated_couette_is_closer_to_the_oracle_than_fp32():
    """Couette 4x64 over 2000 steps: the remainder plane brings every field at
    least as close to the FP64 oracle as plain FP32 storage, and the stress
    and heat flux closer (at dt/tau = 0.023 the FP32 arithmetic of each
    step's increment, not the storage, sets most of what is left: measured
    2.7 times closer)."""
    prob = I.couette_4x64()
    dt = time_step(prob)
    op = oracle_params(prob, dt)
    ref, _ = O.moments(op, O.run(op, O.init(op), 2000))
    errs = {}
    for st in (L.F32, L.F32C):
        s = solver(prob, st, dt=dt)
        s.step(2000)
        errs[st] = np.max(np.abs(s.moments().cpu().numpy().astype(np.float64) - ref).reshape(9, -1), axis=1)
    assert np.all(errs[L.F32C] <= errs[L.F32] * 1.01 + 1e-12), (errs[L.F32C], errs[L.F32])
    assert np.max(errs[L.F32C][4:]) < 0.5 * np.max(errs[L.F32][4:]), (errs[L.F32C], errs[L.F32])


def test_compensated_populations_round_trip_and_checkpoint():
    """Populations read back as hi + lo; set populations give hi = value,
    lo = 0, so a set-then-get returns the values exactly; a checkpoint of the
    public populations restarts a compensated solve to FP32 resolution."""
    import torch
    prob = I.Problem(name="c", nx=60, ny=30, bc_y=I.DIFFUSE, kn=0.05, b=-0.5, wall_ux=(-0.05, 0.05))
    fields = I.random_fields(prob, seed=3, amp_u=0.02, amp_T=0.02, amp_rho=0.02)
    s = solver(prob, L.F32C, fields)
    s.step(20)
    pops = s.populations().clone()
    s.set_populations(pops, 20)
    assert bool((s.populations() == pops).all())
    assert s.populations().dtype == torch.float32


@pytest.mark.parametrize("storage,nroots,dim", [(L.F16, 4, 2), (L.BF16, 4, 2), (L.F32C, 4, 2), (L.F32, 6, 3),
                                                (L.F16, 6, 3), (L.BF16, 6, 3)])
def test_launch_shape_does_not_change_bits(storage, nroots, dim):
    """Rows per segment change where a warp's prologue loads rows directly and
    where its ring carries them; the result must not depend on it."""
    prob = I.Problem(name="shape", nroots=nroots, dim=dim, nx=64, ny=70, bc_y=I.DIFFUSE, kn=0.05, b=0.5,
                     wall_ux=(-0.05, 0.05), g=(1e-3, 0.0), scheme=I.SPLIT)
    fields = I.random_fields(prob, seed=5, amp_u=0.02, amp_T=0.02, amp_rho=0.02)
    dt = time_step(prob, fields)
    outs = []
    for rows in (32, 1, 7, 33):
        s = solver(prob, storage, fields, dt)
        s.set_launch(0, rows)
        s.step(9)
        outs.append(s.populations().cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
