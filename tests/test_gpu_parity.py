"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerance (FP32 compute, FP32 deviation storage): each of the nine moment
fields is held to max|gpu - ref| <= max(1e-5 S, B), S the largest magnitude of
the quantity the field belongs to and B the field's rounding bound
(tests.common.rounding_bound: one FP32 rounding per stored value and step,
accumulated as the field's errors do, evaluated on the oracle's own
populations) -- the 1e-5 bar, except where FP32 cannot resolve it; raw
populations within tests.common.population_bound (n roundings of the largest
deviation).  Every comparison's e, e_own and e_pert are recorded
(tests.common.record).  Grids span several warp strips (28 nodes each) and row
segments, with a ragged tail in both directions.
"""
from __future__ import annotations

from collections import namedtuple

import numpy as np
import pytest

import oracle as O
from paper_1209_6548_gb300 import build as B
from paper_1209_6548_gb300 import inputs as I
from paper_1209_6548_gb300 import lesbgk as L
from tests.common import field_errors, oracle_params, population_bound, record, rounding_bound, time_step

pytestmark = pytest.mark.gpu

TOL = 1e-5
Check = namedtuple("Check", "n gpu ref gpu_pops ref_pops bound")


class Bound(np.ndarray):
    """The nine fields' rounding bounds, carrying the populations' as .pop."""


def rough_checkpoints(scheme):
    """Checkpoints for rough fields that vary in x and y: to 50 steps with the
    split scheme, to 10 with the printed unsplit update, which amplifies such
    data (its von Neumann factor exceeds 1 in 2D): on the walls-force case a
    1e-9 perturbation of the FP64 oracle's own state grows 17-fold between
    steps 20 and 50 under it and decays 4-fold under the split scheme, so past
    about 20 steps the two sides differ by the growth of their rounding, not
    by rounding alone."""
    return [1, 10, 50] if scheme == I.SPLIT else [1, 10]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def gpu_solver(prob, dt, fields):
    return L.Solver(L.params_from_problem(prob, dt=dt), h_init=fields)


def assert_fields_close(gpu, ref, bound=None, tol=TOL, what=""):
    errs = field_errors(gpu, ref, bound, bar=tol)
    record(what, errs)
    bad = {k: v for k, v in errs.items() if not v["ok"]}
    assert not bad, f"{what}: fields over max({tol} S, bound): {bad}"
    return errs


def run_pair(prob, fields, checkpoints, dt=None, storage="f32"):
    """Run the oracle and the GPU side by side; at each checkpoint n return
    Check(n, gpu moments, oracle moments, gpu populations, oracle populations,
    the storage-rounding bound after n steps over the states so far)."""
    dt = dt or time_step(prob, fields)
    op = oracle_params(prob, dt)
    f = O.init(op, fields)
    states = [f]
    s = gpu_solver(prob, dt, fields)
    done = 0
    out = []
    for n in checkpoints:
        op.time = done * dt  # the oracle's clock follows the steps taken (time-dependent walls)
        f = O.run(op, f, n - done)
        s.step(n - done)
        done = n
        states.append(f)
        ref, _ = O.moments(op, f)
        bnd = rounding_bound(states, prob.nroots, prob.dim, n, storage, prob, dt).view(Bound)
        bnd.pop = population_bound(states, prob.nroots, prob.dim, n, storage, prob, dt)
        out.append(Check(n, s.moments().cpu().numpy(), ref, s.populations().cpu().numpy(), f, bnd))
    return out, s, op


def test_couette_4x64_2000_steps():
    """Planar Couette, D2Q16, N = 3, Kn = 0.1, b = -1/2, walls -/+0.05: the
    nine moment fields after 1, 10, 100 and 2000 steps."""
    prob = I.couette_4x64()
    res, s, _ = run_pair(prob, None, [1, 10, 100, 2000])
    for n, g, r, *_, bnd in res:
        assert_fields_close(g, r, bnd, what=f"step {n}")
    assert s.info.steps_done == 2000


@pytest.mark.parametrize("scheme", [I.UNSPLIT, I.SPLIT])
@pytest.mark.parametrize("nx,ny", [(70, 37), (71, 23), (130, 9), (1, 1), (2, 3), (5, 66)])
def test_rough_periodic_fields(nx, ny, scheme):
    """i.i.d. rough fields exercise every limiter branch; the grids span
    several warp strips and row segments with ragged tails, and the 1x1,
    2x3 and 5x66 grids wrap the stencil onto the node itself."""
    prob = I.Problem(name="rough", nx=nx, ny=ny, bc_y=I.PERIODIC, kn=0.05, b=-0.5, scheme=scheme)
    fields = I.random_fields(prob, seed=nx * 100 + ny)
    res, *_ = run_pair(prob, fields, [1, 6])
    for n, g, r, gp, fp, bnd in res:
        assert_fields_close(g, r, bnd, what=f"{nx}x{ny} step {n}")
        w = O.velocity_set(4)[2][:, None, None]
        dev = fp - w
        err = np.max(np.abs(gp - dev))
        assert err <= bnd.pop, f"populations: {err:.3e} vs bound {bnd.pop:.3e}"


def test_taylor_green_split_128():
    """The 2D Taylor-Green vortex with the split scheme, 300 steps."""
    prob = I.tgv(128, steps=300)
    res, *_ = run_pair(prob, I.initial_fields(prob), [1, 300])
    for n, g, r, *_, bnd in res:
        assert_fields_close(g, r, bnd, what=f"tgv128 step {n}")


@pytest.mark.parametrize("scheme", [I.UNSPLIT, I.SPLIT])
def test_launch_shape_does_not_change_bits(scheme):
    prob = I.Problem(name="shape", nx=128, ny=70, bc_y=I.DIFFUSE, kn=0.05, b=0.5, wall_ux=(-0.05, 0.05),
                     g=(1e-3, 0.0), scheme=scheme)
    fields = I.random_fields(prob, seed=5)
    dt = time_step(prob, fields)
    outs = []
    for rows in [16, 1, 7, 33, 64, 1000]:
        s = gpu_solver(prob, dt, fields)
        s.set_launch(0, rows)
        assert s.info.rows_per_segment == rows
        s.step(9)
        outs.append(s.populations().cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def _sampled_oracle(prob, fields, dt, k, cells):
    """Moments after k steps at the given (j, i) nodes, each computed by the
    oracle on its own periodic (4k+1)^2 patch (x and y periodic) or a
    (4k+1)-wide full-height strip (walls in y): the wrapped-around values do
    not reach the centre within k steps.  Also returns the largest of the
    patches' storage-rounding bounds."""
    r = 2 * k
    out = []
    bound = np.zeros(9)
    for j, i in cells:
        cols = np.arange(i - r, i + r + 1) % prob.nx
        if prob.bc_y == I.PERIODIC:
            rows = np.arange(j - r, j + r + 1) % prob.ny
            jj = r
        else:
            rows = np.arange(prob.ny)
            jj = j
        patch = fields[:, rows][:, :, cols]
        op = oracle_params(prob, dt, nx=len(cols), ny=len(rows))
        f0 = O.init(op, patch)
        f = O.run(op, f0, k)
        m, _ = O.moments(op, f)
        out.append(m[:, jj, r])
        bound = np.maximum(bound, rounding_bound([f0, f], prob.nroots, prob.dim, k, "f32", prob, dt))
    return np.array(out).T, bound  # (9, ncells), (9,)


@pytest.mark.parametrize("which", ["tgv4096", "poiseuille512x1024", "tgv4096_d2q36", "tgv4096_d3q64", "tgv4096_d3q216",
                                   "tgv16384"])
def test_full_size_sampled(which):
    """At the full benchmark sizes and the default launch shape: moments after
    3 steps at 24 seeded nodes against the oracle run node by node."""
    from dataclasses import replace
    prob = {"tgv4096": lambda: I.tgv(4096), "poiseuille512x1024": lambda: I.poiseuille(512, 1024),
            "tgv4096_d2q36": lambda: I.tgv(4096, nroots=6),
            "tgv4096_d3q64": lambda: replace(I.tgv(4096), dim=3),
            "tgv4096_d3q216": lambda: replace(I.tgv(4096, nroots=6), dim=3),
            "tgv16384": lambda: I.tgv(16384)}[which]()  # 268M nodes: 34 GB of populations
    fields = I.initial_fields(prob)
    dt = time_step(prob, fields)
    s = gpu_solver(prob, dt, fields)
    k = 3
    s.step(k)
    mom = s.moments()
    rng = np.random.default_rng(2024)
    cells = [(int(rng.integers(prob.ny)), int(rng.integers(prob.nx))) for _ in range(20)]
    cells += [(0, 5), (prob.ny - 1, 7), (1, 0), (prob.ny - 2, prob.nx - 1)]
    import torch
    jj = torch.tensor([c[0] for c in cells], device="cuda")
    ii = torch.tensor([c[1] for c in cells], device="cuda")
    g = mom[:, jj, ii].cpu().numpy()
    ref, bnd = _sampled_oracle(prob, fields, dt, k, cells)
    assert_fields_close(g[:, :, None], ref[:, :, None], bnd, what=which)


def test_conservation_totals_at_2_to_the_28_nodes():
    """The FP64 totals of lesbgk_moments at 16384^2 = 2^28 nodes (per-node
    sums in FP32, runs of 16 nodes in FP32, the runs in FP64) against FP64
    sums of the stored populations themselves, within the worst case of that
    arithmetic: each total is off by at most 30 FP32 roundings of the absolute
    terms it sums (up to 12 in a node's Hermite moments, 3 combining them, 15
    in a run), i.e. 30 2^-24 sum_nodes sum_a |psi_a| |df_a| with psi = 1, |c_x|,
    |c_y|, c^2 + 4 (the energy's moments m20, m02 and 2 m00)."""
    import torch
    prob = I.tgv(16384)
    fields = I.initial_fields(prob)
    s = gpu_solver(prob, time_step(prob, fields), fields)
    s.step(2)
    _, sums = s.moments(sums=True)
    df = s.populations()  # (16, ny, nx) FP32 deviations f - w, on the device
    cx, cy, w = O.velocity_set(4)
    cells = prob.cells
    col, mag = np.zeros(16), np.zeros(16)  # per population: sum over nodes of df, of |df|
    for a in range(16):
        da = df[a].double()
        col[a] = float(da.sum())
        mag[a] = float(da.abs().sum())
    del df
    psi = [np.ones(16), cx, cy, cx * cx + cy * cy]
    bound_w = [np.ones(16), np.abs(cx), np.abs(cy), cx * cx + cy * cy + 4.0]
    out = {}
    for k, name in enumerate(("mass", "momentum_x", "momentum_y", "energy")):
        scale = 0.5 if k == 3 else 1.0  # energy = 1/2 sum f c^2
        ref = scale * float(np.sum(w * psi[k]) * cells + np.dot(psi[k], col))
        bound = scale * 30 * 2.0 ** -24 * float(np.dot(bound_w[k], mag))
        err = abs(sums[k] - ref)
        out[name] = {"abs": err, "e": err / max(abs(ref), 1e-300), "e_own": None, "e_pert": None, "bound": bound,
                     "tol": bound, "ok": bool(err <= bound)}
    record("totals 16384^2", out)
    assert all(v["ok"] for v in out.values()), out


def test_grid_sizes_near_strip_and_segment_edges():
    """nx around one and two strip widths (60 and 120 nodes), ny not a multiple
    of the segment length, walls."""
    for nx in (58, 60, 62, 120, 122):
        prob = I.Problem(name="edge", nx=nx, ny=35, bc_y=I.DIFFUSE, kn=0.1, b=-0.5, wall_ux=(0.0, 0.05),
                         wall_T=(1.0, 1.02))
        fields = I.random_fields(prob, seed=nx)
        res, *_ = run_pair(prob, fields, [3])
        for n, g, r, *_, bnd in res:
            assert_fields_close(g, r, bnd, what=f"nx={nx}")


@pytest.mark.parametrize("scheme", [I.UNSPLIT, I.SPLIT])
@pytest.mark.parametrize("b", [-0.5, 0.0, 0.5])
def test_walls_force_and_temperature(b, scheme):
    """Walls at different T and u_x, a body force and rough interior fields
    (i.i.d. data: every limiter branch), to 50 steps (split scheme) under the
    derived bound."""
    prob = I.Problem(name="mix", nx=64, ny=45, bc_y=I.DIFFUSE, kn=0.08, b=b, wall_T=(0.96, 1.05),
                     wall_ux=(-0.04, 0.03), g=(2e-3, -1e-3), scheme=scheme)
    fields = I.random_fields(prob, seed=11, amp_u=0.03, amp_T=0.03, amp_rho=0.03)
    res, *_ = run_pair(prob, fields, rough_checkpoints(scheme))
    for n, g, r, *_, bnd in res:
        assert_fields_close(g, r, bnd, what=f"b={b} step {n}")


def test_poiseuille_small():
    prob = I.poiseuille(nx=4, ny=40, steps=300)
    res, *_ = run_pair(prob, None, [300])
    for n, g, r, *_, bnd in res:
        assert_fields_close(g, r, bnd, what=f"poiseuille step {n}")


def test_fourier_small():
    prob = I.fourier(ny=33)
    res, *_ = run_pair(prob, None, [500])
    for n, g, r, *_, bnd in res:
        assert_fields_close(g, r, bnd, what="fourier")


@pytest.mark.parametrize("visc", [0.5, 1.0, 0.75])
def test_viscosity_exponents(visc):
    prob = I.Problem(name="v", nx=8, ny=20, bc_y=I.DIFFUSE, kn=0.1, b=-0.5, visc_exp=visc,
                     wall_T=(0.9, 1.1), wall_ux=(0.0, 0.05))
    res, *_ = run_pair(prob, None, [200])
    for n, g, r, *_, bnd in res:
        assert_fields_close(g, r, bnd, what=f"visc {visc}")


def test_two_row_channel():
    """ny = 2: both rows are walls."""
    prob = I.Problem(name="t", nx=6, ny=2, bc_y=I.DIFFUSE, kn=0.2, b=0.0, wall_T=(0.98, 1.02),
                     wall_ux=(-0.02, 0.02))
    res, *_ = run_pair(prob, None, [1, 20])
    for n, g, r, *_, bnd in res:
        assert_fields_close(g, r, bnd, what=f"two rows step {n}")


def test_default_time_step_rule():
    """dt = 0 asks the library for min(cfl min(dx,dy)/c_max, tau_ref); it must
    agree with the rule restated on the test side."""
    for prob, fields in [(I.couette_4x64(), None), (I.tgv(64), I.initial_fields(I.tgv(64))),
                         (I.Problem(name="s", nx=4, ny=16, kn=0.01, b=0.5), None)]:
        s = L.Solver(L.params_from_problem(prob, dt=0.0), h_init=fields)
        assert abs(s.info.dt - time_step(prob, fields)) <= 1e-15 * time_step(prob, fields)


def test_unstable_dt_rejected():
    prob = I.Problem(name="s", nx=4, ny=16, kn=0.01, b=0.5)
    with pytest.raises(L.LesbgkError) as e:
        L.Solver(L.params_from_problem(prob, dt=0.02))
    assert e.value.code == L.EUNSTABLE


def test_checkpoint_restart_is_bitwise():
    prob = I.Problem(name="c", nx=60, ny=30, bc_y=I.DIFFUSE, kn=0.05, b=-0.5, wall_ux=(-0.05, 0.05))
    fields = I.random_fields(prob, seed=3)
    dt = time_step(prob, fields)
    a = gpu_solver(prob, dt, fields)
    a.step(20)
    ck = a.populations().clone()
    a.step(15)
    b = gpu_solver(prob, dt, fields)
    b.set_populations(ck, 20)
    b.step(15)
    assert b.info.steps_done == 35
    assert bool((a.populations() == b.populations()).all())


def test_deterministic_and_host_moments():
    prob = I.tgv(128, steps=10)
    fields = I.initial_fields(prob)
    dt = time_step(prob, fields)
    a, b = gpu_solver(prob, dt, fields), gpu_solver(prob, dt, fields)
    a.step(7)
    b.step(7)
    ma, sa = a.moments(sums=True)
    mh, sh = b.moments_host()
    assert np.array_equal(ma.cpu().numpy(), mh)
    assert np.array_equal(sa, sh)


def test_conservation_periodic_gpu():
    """Periodic, no force: FP64 totals of mass, momentum and energy drift only
    by FP32 rounding of the stored deviations."""
    prob = I.tgv(256, steps=200)
    fields = I.initial_fields(prob)
    s = gpu_solver(prob, time_step(prob, fields), fields)
    _, s0 = s.moments(sums=True)
    s.step(200)
    _, s1 = s.moments(sums=True)
    cells = prob.cells
    assert abs(s1[0] - s0[0]) < 1e-9 * cells
    assert abs(s1[1] - s0[1]) < 1e-9 * cells
    assert abs(s1[2] - s0[2]) < 1e-9 * cells
    assert abs(s1[3] - s0[3]) < 1e-9 * cells


@pytest.mark.parametrize("nroots", [4, 6])
def test_conservation_sums_match_populations(nroots):
    """The FP64 totals of lesbgk_moments (per-node sums in FP32, the nodes'
    runs accumulated in FP64) agree with FP64 sums of the stored populations
    sum f {1, c_x, c_y, c^2/2}, within the worst case of that arithmetic: 34
    FP32 roundings of the absolute terms (up to 16 in a node's Hermite moments
    on D2Q36, 3 combining them, 15 in a run of 16 nodes)."""
    prob = I.Problem(name="cs", nroots=nroots, nx=70, ny=37, bc_y=I.DIFFUSE, kn=0.1, b=-0.5,
                     wall_ux=(-0.05, 0.05), wall_T=(0.97, 1.03), g=(1e-3, 0.0))
    fields = I.random_fields(prob, seed=21, amp_u=0.05, amp_T=0.05, amp_rho=0.05)
    s = gpu_solver(prob, time_step(prob, fields), fields)
    s.step(13)
    _, sums = s.moments(sums=True)
    df = s.populations().cpu().numpy().astype(np.float64)  # f - w, [a][j][i]
    cx, cy, w = O.velocity_set(nroots)
    phis = [np.ones_like(cx), cx, cy, 0.5 * (cx * cx + cy * cy)]
    absw = [np.ones_like(cx), np.abs(cx), np.abs(cy), 0.5 * (cx * cx + cy * cy + 4.0)]
    cells = prob.cells
    for k, phi in enumerate(phis):
        ref = float(np.sum(w * phi) * cells + np.einsum("a,aji->", phi, df))
        bound = 34 * 2.0 ** -24 * float(np.einsum("a,aji->", absw[k], np.abs(df)))
        assert abs(sums[k] - ref) <= bound, (k, sums[k], ref, bound)


# ---------------------------------------------------------------- other lattices
@pytest.mark.parametrize("scheme", [I.UNSPLIT, I.SPLIT])
def test_d2q36_rough_periodic(scheme):
    """D2Q36 (6 roots of He_6 per axis), Hermite order 4 -- the paper's own
    setting -- on rough periodic fields spanning two strips and segments."""
    prob = I.Problem(name="q36", nroots=6, nx=41, ny=37, bc_y=I.PERIODIC, kn=0.05, b=-0.5, scheme=scheme)
    fields = I.random_fields(prob, seed=36)
    res, *_ = run_pair(prob, fields, [1, 6])
    for n, g, r, gp, fp, bnd in res:
        assert_fields_close(g, r, bnd, what=f"d2q36 step {n}")
        w = O.velocity_set(6)[2][:, None, None]
        dev = fp - w
        assert np.max(np.abs(gp - dev)) <= bnd.pop


def test_d2q36_couette_walls_force():
    prob = I.Problem(name="q36c", nroots=6, nx=4, ny=40, bc_y=I.DIFFUSE, kn=0.1, b=-0.5,
                     wall_ux=(-0.05, 0.05), wall_T=(0.98, 1.02), g=(1e-3, 0.0))
    res, *_ = run_pair(prob, None, [1, 400])
    for n, g, r, *_, bnd in res:
        assert_fields_close(g, r, bnd, what=f"d2q36 couette step {n}")


@pytest.mark.parametrize("scheme", [I.UNSPLIT, I.SPLIT])
def test_d2q16_order4(scheme):
    """N = 4 on D2Q16 (projection not exact, still conservative)."""
    prob = I.Problem(name="q16n4", nroots=4, order=4, nx=30, ny=25, bc_y=I.DIFFUSE, kn=0.1, b=0.5,
                     wall_ux=(0.0, 0.05), g=(0.0, -1e-3), scheme=scheme)
    fields = I.random_fields(prob, seed=4, amp_u=0.02, amp_T=0.02, amp_rho=0.02)
    res, *_ = run_pair(prob, fields, rough_checkpoints(scheme))
    for n, g, r, *_, bnd in res:
        assert_fields_close(g, r, bnd, what=f"d2q16 N=4 step {n}")


@pytest.mark.parametrize("scheme", [I.UNSPLIT, I.SPLIT])
def test_d2q36_order3(scheme):
    prob = I.Problem(name="q36n3", nroots=6, order=3, nx=12, ny=20, bc_y=I.DIFFUSE, kn=0.2, b=0.0,
                     wall_T=(0.95, 1.05), scheme=scheme)
    res, *_ = run_pair(prob, None, [1, 100])
    for n, g, r, *_, bnd in res:
        assert_fields_close(g, r, bnd, what=f"d2q36 N=3 step {n}")


# ---------------------------------------------------------------- wall models
@pytest.mark.parametrize("nroots", [4, 6])
@pytest.mark.parametrize("scheme", [I.UNSPLIT, I.SPLIT])
@pytest.mark.parametrize("spec", [0.3, 1.0])
def test_maxwell_walls(spec, scheme, nroots):
    """Maxwell walls with accommodation 1 - spec (Sec. 3.2's model), moving and
    at two temperatures, rough interior; both update schemes (each its own
    kernel instantiation)."""
    prob = I.Problem(name="mw", nroots=nroots, nx=32, ny=30, bc_y=I.DIFFUSE, kn=0.1, b=-0.5,
                     wall_ux=(-0.05, 0.05), wall_T=(0.97, 1.04), wall_specular=spec, scheme=scheme)
    fields = I.random_fields(prob, seed=12, amp_u=0.02, amp_T=0.02, amp_rho=0.02)
    res, *_ = run_pair(prob, fields, rough_checkpoints(scheme))
    for n, g, r, *_, bnd in res:
        assert_fields_close(g, r, bnd, what=f"nroots {nroots} spec {spec} scheme {scheme} step {n}")


@pytest.mark.parametrize("kn,st", [(0.1, 0.5553603672697958), (0.5, 1.1107207345395915)])
def test_unsteady_wall_heating(kn, st):
    """Both walls heated as T_w = 1 + A sin(St t) (Sec. 4.2), A = 0.02 for a
    clear signal, gas at rest at T = 1 initially; up to t ~ 3 pi / 2 / St."""
    prob = I.unsteady_heating(kn=kn, st=st, amp=0.02, ny=40)
    dt = time_step(prob)
    n_end = int(round(3 * np.pi / 2 / st / dt / 10)) * 10
    res, *_ = run_pair(prob, None, [1, 50, n_end], dt=dt)
    for n, g, r, *_, bnd in res:
        assert_fields_close(g, r, bnd, what=f"heating step {n}")
    assert np.max(np.abs(res[-1][2][3] - 1.0)) > 1e-3  # the walls did heat the gas


# ---------------------------------------------------------------- D = 3 sets
# D3Q64 (N = 3) and D3Q216 (N = 4) on the 2D grid: the library stores the
# z-even half (32 or 108 values per node); the oracle runs all 64 or 216.
def d3(prob, nroots=4):
    from dataclasses import replace
    return replace(prob, dim=3, nroots=nroots, order=0, name=prob.name + f"_d3q{nroots ** 3}")


def z_even_half(fp, nroots=4):
    """Oracle populations (nroots^3, ny, nx) -> deviations at the stored
    velocities (iz, ix, iy), c_z = c[nroots/2 + iz] > 0."""
    *_, w = O.velocity_set_d(nroots, 3)
    h = nroots // 2
    idx = [(ix * nroots + iy) * nroots + h + iz for iz in range(h) for ix in range(nroots) for iy in range(nroots)]
    return (fp - w[:, None, None])[idx]


def assert_d3_populations(gp, fp, what, nroots=4, pop_bound=None):
    dev = z_even_half(fp, nroots)
    err = np.max(np.abs(gp - dev))
    assert err <= pop_bound, f"{what} populations: {err:.3e} vs bound {pop_bound:.3e}"


@pytest.mark.parametrize("nroots", [4, 6])
def test_d3_couette(nroots):
    """Couette 4x64 with the D = 3 sets (the paper's C_p = 5/2 gas)."""
    prob = d3(I.couette_4x64(), nroots)
    res, s, _ = run_pair(prob, None, [1, 10, 100, 2000] if nroots == 4 else [1, 10, 300])
    for n, g, r, gp, fp, bnd in res:
        assert_fields_close(g, r, bnd, what=f"d3q{nroots ** 3} couette step {n}")
        assert_d3_populations(gp, fp, f"d3q{nroots ** 3} couette step {n}", nroots, bnd.pop)
    assert s.info.q == nroots ** 3 // 2


@pytest.mark.parametrize("nroots", [4, 6])
@pytest.mark.parametrize("scheme", [I.UNSPLIT, I.SPLIT])
@pytest.mark.parametrize("nx,ny", [(70, 37), (5, 66), (1, 1)])
def test_d3_rough_periodic_fields(nx, ny, scheme, nroots):
    prob = d3(I.Problem(name="rough", nx=nx, ny=ny, bc_y=I.PERIODIC, kn=0.05, b=-0.5, scheme=scheme), nroots)
    fields = I.random_fields(prob, seed=nx * 100 + ny + 7)
    res, *_ = run_pair(prob, fields, [1, 6])
    for n, g, r, gp, fp, bnd in res:
        assert_fields_close(g, r, bnd, what=f"d3q{nroots ** 3} {nx}x{ny} step {n}")
        assert_d3_populations(gp, fp, f"d3q{nroots ** 3} {nx}x{ny} step {n}", nroots, bnd.pop)


@pytest.mark.parametrize("nroots", [4, 6])
@pytest.mark.parametrize("b,scheme", [(-0.5, I.UNSPLIT), (0.5, I.UNSPLIT), (-0.5, I.SPLIT)])
def test_d3_walls_force_rough(b, scheme, nroots):
    """Moving walls at two temperatures, body force, rough interior."""
    prob = d3(I.Problem(name="wf", nx=60, ny=45, bc_y=I.DIFFUSE, kn=0.1, b=b, wall_ux=(-0.05, 0.05),
                        wall_T=(0.97, 1.03), g=(1e-3, 2e-4), scheme=scheme), nroots)
    fields = I.random_fields(prob, seed=31, amp_u=0.02, amp_T=0.02, amp_rho=0.02)
    res, *_ = run_pair(prob, fields, rough_checkpoints(scheme))
    for n, g, r, gp, fp, bnd in res:
        assert_fields_close(g, r, bnd, what=f"d3q{nroots ** 3} walls b={b} step {n}")
        assert_d3_populations(gp, fp, f"d3q{nroots ** 3} walls b={b} step {n}", nroots, bnd.pop)


@pytest.mark.parametrize("nroots", [4, 6])
@pytest.mark.parametrize("scheme", [I.UNSPLIT, I.SPLIT])
def test_d3_maxwell_walls_and_heating(scheme, nroots):
    """Specular share 0.3 and heated walls (Sec. 3.2, Sec. 4.2) with D = 3,
    both update schemes."""
    prob = d3(I.Problem(name="mh", nx=8, ny=40, bc_y=I.DIFFUSE, kn=0.2, b=-0.5, wall_specular=0.3,
                        wall_T_amp=0.02, wall_T_freq=0.5553603672697958, scheme=scheme), nroots)
    res, *_ = run_pair(prob, None, [1, 50, 300])
    for n, g, r, *_, bnd in res:
        assert_fields_close(g, r, bnd, what=f"d3q{nroots ** 3} maxwell+heating scheme {scheme} step {n}")


@pytest.mark.parametrize("nroots", [4, 6])
def test_d3_conservation_and_totals(nroots):
    """Periodic D = 3: the FP64 totals match the oracle's (energy counts
    c_z^2: 3/2 rho T per node at rest) and are conserved over 200 steps."""
    prob = d3(I.tgv(128, steps=200), nroots)
    fields = I.initial_fields(prob)
    dt = time_step(prob, fields)
    s = gpu_solver(prob, dt, fields)
    op = oracle_params(prob, dt)
    _, ref = O.moments(op, O.init(op, fields))
    _, s0 = s.moments(sums=True)
    cells = prob.cells
    assert np.allclose(s0, ref, rtol=0, atol=1e-9 * cells), (s0, ref)
    s.step(200)
    _, s1 = s.moments(sums=True)
    assert np.allclose(s1, s0, rtol=0, atol=1e-9 * cells)


# ---------------------------------------------------------------- high Mach number (Sec. 4)
@pytest.mark.parametrize("kind", ["couette", "poiseuille", "couette_fourier"])
@pytest.mark.parametrize("nroots,dim", [(6, 2), (4, 3)])
def test_high_mach_workloads(kind, nroots, dim):
    """The paper's nonlinear workloads: Couette at -/+0.2, force-driven
    Poiseuille with g = 0.22, Couette-Fourier with T_w = 1 -/+ 0.15, at
    K_D = 0.1, on D2Q36 (N = 4) and D3Q64 (N = 3)."""
    gen = {"couette": I.couette_high_ma, "poiseuille": I.poiseuille_high_force,
           "couette_fourier": I.couette_fourier}[kind]
    prob = gen(kd=0.1, nroots=nroots, dim=dim, ny=40)
    res, *_ = run_pair(prob, None, [1, 100, 1000])
    for n, g, r, *_, bnd in res:
        assert_fields_close(g, r, bnd, what=f"{prob.name} D={dim} step {n}")
    assert np.max(np.abs(res[-1][2][1])) > 0.1  # a high-speed flow did develop


# ---------------------------------------------------------------- walls in x (cavity)
@pytest.mark.parametrize("nroots,dim", [(4, 2), (6, 2), (4, 3), (6, 3)])
def test_lid_driven_cavity(nroots, dim):
    """Lid-driven cavity (walls on all sides, corners, lid at 0.05), split
    scheme, on a grid that spans two warp strips with a ragged tail."""
    from dataclasses import replace
    prob = replace(I.lid_driven_cavity(n=45, u_lid=0.05, kn=0.1), nroots=nroots, dim=dim, ny=37)
    res, *_ = run_pair(prob, None, [1, 10, 200])
    for n, g, r, *_, bnd in res:
        assert_fields_close(g, r, bnd, what=f"cavity nroots={nroots} D={dim} step {n}")
    assert np.max(np.abs(res[-1][2][2])) > 1e-3  # the lid set up a vortex


@pytest.mark.parametrize("nroots,dim", [(4, 2), (6, 2), (4, 3), (6, 3)])
@pytest.mark.parametrize("scheme", [I.UNSPLIT, I.SPLIT])
def test_walls_in_x_rough(scheme, nroots, dim):
    """Rough fields in a box with heated walls on all sides and a lid, and in
    a channel walled in x only (periodic y); populations element by element,
    on every set with walls in x and in both update schemes."""
    for prob in (I.Problem(name="box", nroots=nroots, dim=dim, nx=60, ny=33, bc_y=I.DIFFUSE, bc_x=I.DIFFUSE,
                           kn=0.1, b=0.5, wall_ux=(0.0, 0.05), wall_T=(0.98, 1.02), wall_Tx=(1.03, 0.97),
                           scheme=scheme),
                 I.Problem(name="xchan", nroots=nroots, dim=dim, nx=29, ny=30, bc_y=I.PERIODIC, bc_x=I.DIFFUSE,
                           kn=0.05, b=-0.5, wall_Tx=(0.97, 1.04), g=(0.0, 1e-3), scheme=scheme)):
        fields = I.random_fields(prob, seed=prob.nx + 3, amp_u=0.02, amp_T=0.02, amp_rho=0.02)
        res, *_ = run_pair(prob, fields, rough_checkpoints(scheme))
        for n, g, r, gp, fp, bnd in res:
            what = f"{prob.name} nroots={nroots} D={dim} step {n}"
            assert_fields_close(g, r, bnd, what=what)
            if dim == 3:
                assert_d3_populations(gp, fp, what, nroots, bnd.pop)
            else:
                w = O.velocity_set(nroots)[2][:, None, None]
                err = np.max(np.abs(gp - (fp - w)))
                assert err <= bnd.pop, f"{what} populations {err:.3e} vs bound {bnd.pop:.3e}"


def test_cavity_of_two_by_two_is_all_corners():
    prob = I.Problem(name="tiny", nx=2, ny=2, bc_y=I.DIFFUSE, bc_x=I.DIFFUSE, kn=0.1, b=0.0,
                     wall_T=(1.0, 1.0), wall_Tx=(1.02, 0.99))
    fields = I.random_fields(prob, seed=2, amp_u=0.02, amp_T=0.02, amp_rho=0.02)
    res, *_ = run_pair(prob, fields, [1, 5])
    for n, g, r, *_, bnd in res:
        assert_fields_close(g, r, bnd, what=f"2x2 step {n}")


# ---------------------------------------------------------------- failure path
def test_diverged_solve_is_reported():
    """The printed (unsplit) update is unstable for flows varying in x and y
    (the oracle pins it); the Taylor-Green vortex then blows up in FP32 too,
    and lesbgk_moments with totals reports LESBGK_EDIVERGED instead of
    returning non-finite sums.  (A data failure, not a GPU fault.)"""
    prob = I.Problem(name="tgv_unsplit", nx=64, ny=64, bc_y=I.PERIODIC, kn=0.05, b=-0.5, init="tgv", scheme=I.UNSPLIT)
    s = gpu_solver(prob, time_step(prob, I.initial_fields(prob)), I.initial_fields(prob))
    for _ in range(200):
        s.step(100)
        m = s.moments()
        if not bool(m.isfinite().all()):
            break
    else:
        pytest.fail("the unsplit 2D update did not diverge")
    with pytest.raises(L.LesbgkError) as e:
        s.moments(sums=True)
    assert e.value.code == L.EDIVERGED


# ---------------------------------------------------------------- initial fields
def test_initial_fields_checked_and_maxima_on_the_device():
    """lesbgk_create checks the initial fields and takes their largest rho and
    T (for tau_ref) on the device: tau_ref equals the host formula, and a
    non-finite or non-positive value is refused with the first bad node."""
    prob = I.Problem(name="f", nx=300, ny=70, bc_y=I.DIFFUSE, kn=0.07, b=0.5, visc_exp=0.7, wall_T=(1.01, 1.05))
    fields = I.random_fields(prob, seed=4, amp_u=0.02, amp_T=0.2, amp_rho=0.2)
    s = L.Solver(L.params_from_problem(prob), h_init=fields)
    tmax = max(1.0, 1.05, float(fields[3].max()))
    ref = (0.07 * (1 - 0.5)) * tmax ** (0.7 - 1.0) / float(fields[0].max())
    assert s.info.tau_ref == pytest.approx(ref, rel=1e-15)
    s.close()
    for field, node, value in ((2, 1234, np.nan), (0, 20000, 0.0), (3, 7, -1.0), (1, 5000, np.inf)):
        bad = fields.copy()
        bad[field].reshape(-1)[node] = value
        bad[field].reshape(-1)[node + 3] = value  # the first one is reported
        with pytest.raises(L.LesbgkError) as e:
            L.Solver(L.params_from_problem(prob), h_init=bad)
        assert e.value.code == L.EINVAL and f"node {node} " in L.last_error(), L.last_error()


# ---------------------------------------------------------------- degenerate cases
def test_collisionless_limit_and_zero_steps():
    """Kn -> infinity (dt/tau ~ 1e-8): pure TVD transport with walls, against
    the oracle; and a zero-step call leaves the state and the clock alone."""
    prob = I.Problem(name="free", nx=61, ny=40, bc_y=I.DIFFUSE, kn=1e6, b=0.0, wall_ux=(-0.05, 0.05),
                     wall_T=(0.97, 1.03), scheme=I.SPLIT)
    fields = I.random_fields(prob, seed=8, amp_u=0.02, amp_T=0.02, amp_rho=0.02)
    res, s, _ = run_pair(prob, fields, [1, 30])
    for n, g, r, *_, bnd in res:
        assert_fields_close(g, r, bnd, what=f"collisionless step {n}")
    before = s.populations().cpu().numpy()
    s.step(0)
    assert s.info.steps_done == 30
    assert np.array_equal(s.populations().cpu().numpy(), before)


# ---------------------------------------------------------------- residual
@pytest.mark.parametrize("nroots,dim", [(4, 2), (6, 2), (4, 3), (6, 3)])
def test_residual_against_the_moment_fields(nroots, dim):
    """lesbgk_residual equals max over nodes of |d rho| + |d u| + |d T| of the
    moment fields, per unit time; the first call only takes the snapshot."""
    import torch
    from dataclasses import replace
    prob = replace(I.Problem(name="res", nx=45, ny=38, bc_y=I.DIFFUSE, kn=0.1, b=0.5, wall_ux=(-0.05, 0.05),
                             wall_T=(0.98, 1.03)), nroots=nroots, dim=dim)
    s = gpu_solver(prob, time_step(prob), None)
    snap = torch.empty((4, prob.ny, prob.nx), dtype=torch.float32, device="cuda")
    assert np.isnan(s.residual(snap, 0))
    m0 = s.moments()[[0, 1, 2, 3]].cpu().numpy().astype(np.float64)
    assert np.allclose(snap.cpu().numpy(), m0, rtol=0, atol=1e-6)
    s.step(37)
    r = s.residual(snap, 37)
    m1 = s.moments()[[0, 1, 2, 3]].cpu().numpy().astype(np.float64)
    ref = np.abs(m1 - m0).sum(axis=0).max() / (37 * s.info.dt)
    assert r == pytest.approx(ref, rel=1e-4, abs=1e-6 / (37 * s.info.dt))
    assert np.allclose(snap.cpu().numpy(), m1, rtol=0, atol=1e-6)
