"""Pins of the FP64 oracle with a three-dimensional velocity set (D = 3, the
paper's thermodynamics: C_p = 5/2) on the two-dimensional grid.

Each test ties a D = 3 code path of the oracle to something other than
itself: numpy's Hermite series, brute-force Gaussian quadrature in three
dimensions, closed forms of the Chapman-Enskog coefficients, or invariants.
The mistakes each one catches are named in its docstring: base-2 instead of
base-3 tensor indexing, D = 2 left in a trace, a 2x2 lambda, a missing c_z in
c^2, or c_z being advected.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import pytest
from numpy.polynomial import hermite_e as HE

import oracle as O
from paper_1209_6548_gb300.inputs import DIFFUSE, PERIODIC, Problem, random_fields
from tests.common import oracle_params, time_step


def he(m, x):
    coef = np.zeros(m + 1)
    coef[m] = 1.0
    return HE.hermeval(x, coef)


def gaussian_moment3(rho, u, lam, m, k, l, npts=12):
    """rho E[He_m(X) He_k(Y) He_l(Z)], (X, Y, Z) ~ N(u, lam), by a 12^3-point
    Gauss-Hermite product rule in the whitened frame (exact to degree 23)."""
    z, wz = HE.hermegauss(npts)
    wz = wz / np.sqrt(2 * np.pi)
    Lc = np.linalg.cholesky(np.asarray(lam).reshape(3, 3))
    Z = np.stack(np.meshgrid(z, z, z, indexing="ij"))
    W = wz[:, None, None] * wz[None, :, None] * wz[None, None, :]
    X = [u[i] + sum(Lc[i, j] * Z[j] for j in range(3)) for i in range(3)]
    return rho * np.sum(W * he(m, X[0]) * he(k, X[1]) * he(l, X[2]))


def moments3(f, cx, cy, cz):
    rho = f.sum()
    c = np.stack([cx, cy, cz])
    u = (c * f).sum(axis=1) / rho
    C = c - u[:, None]
    P = np.einsum("a,ia,ja->ij", f, C, C)
    T = np.trace(P) / (3 * rho)
    q = 0.5 * np.einsum("a,ia,a->i", f, C, (C * C).sum(axis=0))
    return rho, u, P, T, q


def noneq3(nroots, order, seed, amp=0.02, T=1.03, u=(0.04, -0.03), rho=1.1):
    rng = np.random.default_rng(seed)
    f0 = rho * O.feq0(nroots, order, T, *u, dim=3)
    *_, w = O.velocity_set_d(nroots, 3)
    return f0 + amp * w * rng.uniform(-1, 1, size=f0.size)


def params3(nroots=4, order=3, b=-0.5, g=(0.0, 0.0), kn=0.1, visc=0.5, dt=1e-3, **kw):
    return O.make_params(nroots=nroots, order=order, nx=1, ny=1, bc_y=PERIODIC, kn=kn, b=b, visc_exp=visc,
                         dt=dt, dx=1.0, dy=1.0, g=g, dim=3, **kw)


def mirror_z(nroots):
    a = np.arange(nroots ** 3)
    iz = a % nroots
    return a - iz + (nroots - 1 - iz)


# ---------------------------------------------------------------- the set
@pytest.mark.parametrize("nroots", [4, 6])
def test_d3_set_is_the_tensor_product(nroots):
    """alpha = (ix*n + iy)*n + iz, w = w_x w_y w_z; the D = 2 set of the same
    routine equals the 2D set; isotropic moments to degree 2n - 1 per axis."""
    cx, cy, cz, w = O.velocity_set_d(nroots, 3)
    c, w1 = O.gauss_hermite_1d(nroots)
    for ix, iy, iz in itertools.product(range(nroots), repeat=3):
        a = (ix * nroots + iy) * nroots + iz
        assert (cx[a], cy[a], cz[a]) == (c[ix], c[iy], c[iz])
        assert abs(w[a] - w1[ix] * w1[iy] * w1[iz]) < 1e-17
    assert abs(w.sum() - 1) < 1e-15
    assert abs(np.sum(w * cz ** 2) - 1) < 1e-14 and abs(np.sum(w * cz ** 4) - 3) < 1e-13
    assert abs(np.sum(w * cx ** 2 * cz ** 2) - 1) < 1e-14
    assert abs(np.sum(w * (cx ** 2 + cy ** 2 + cz ** 2)) - 3) < 1e-14
    x2, y2, z2, w2 = O.velocity_set_d(nroots, 2)
    rx, ry, rw = O.velocity_set(nroots)
    assert np.array_equal(x2, rx) and np.array_equal(y2, ry) and np.array_equal(w2, rw) and not z2.any()


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4])
def test_chi3_equals_product_of_1d(n):
    """chi^(n) in D = 3 with m x-, k y- and l z-indices equals
    He_m(c_x) He_k(c_y) He_l(c_z).  Catches base-2 index decoding or a
    delta term dropped for the third axis."""
    rng = np.random.default_rng(3)
    for _ in range(4):
        c = rng.normal(size=3) * 1.5
        t = O.chi(n, c)
        for idx in itertools.product((0, 1, 2), repeat=n):
            m, k, l = idx.count(0), idx.count(1), idx.count(2)
            ref = he(m, c[0]) * he(k, c[1]) * he(l, c[2])
            got = t[idx] if n else t[0]
            assert abs(got - ref) < 1e-11 * max(1.0, abs(ref))


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4])
def test_a_es3_is_the_hermite_moment_of_the_es_gaussian(n):
    """The printed a_ES^(n) with 3x3 lambda equal brute-force 3D Gaussian
    Hermite moments (Eq. cfeq).  Catches a 2x2 lambda or index mix-up."""
    rng = np.random.default_rng(9)
    for _ in range(3):
        rho = 1.0 + 0.3 * rng.random()
        u = rng.normal(size=3) * 0.3
        A = rng.normal(size=(3, 3)) * 0.15
        lam = np.eye(3) * (0.8 + 0.4 * rng.random()) + 0.5 * (A + A.T)
        assert np.all(np.linalg.eigvalsh(lam) > 0)
        t = O.a_es(n, rho, u, lam)
        for idx in itertools.product((0, 1, 2), repeat=n):
            ref = gaussian_moment3(rho, u, lam, idx.count(0), idx.count(1), idx.count(2))
            got = t[idx] if n else t[0]
            assert abs(got - ref) < 1e-11 * max(1.0, abs(ref)), (n, idx, got, ref)


@pytest.mark.parametrize("nroots,order", [(4, 3), (6, 4), (4, 2)])
def test_feq0_d3_is_truncated_maxwellian(nroots, order):
    """Eq. (feq0) with D = 3 (c.c, c.u over three components, D in the
    traces) equals the order-N Hermite projection of the 3D Maxwellian."""
    cx, cy, cz, w = O.velocity_set_d(nroots, 3)
    for T, ux, uy in [(1.0, 0.05, 0.0), (1.06, -0.2, 0.13)]:
        got = O.feq0(nroots, order, T, ux, uy, dim=3)
        ref = np.zeros_like(got)
        for m, k, l in itertools.product(range(order + 1), repeat=3):
            if m + k + l > order:
                continue
            a = gaussian_moment3(1.0, (ux, uy, 0.0), np.eye(3) * T, m, k, l)
            ref += w * a * he(m, cx) * he(k, cy) * he(l, cz) / (
                math.factorial(m) * math.factorial(k) * math.factorial(l))
        assert np.allclose(got, ref, atol=1e-14, rtol=0)
        # three translational degrees of freedom: sum S (c - u)^2 = 3 T
        r, u, P, Tm, _ = moments3(got, cx, cy, cz)
        assert abs(r - 1) < 1e-14 and abs(Tm - T) < 1e-13 and abs(np.trace(P) - 3 * T) < 1e-13


# ---------------------------------------------------------------- collision
@pytest.mark.parametrize("nroots,order", [(4, 3), (6, 4)])
@pytest.mark.parametrize("b", [-0.5, 0.0, 0.5])
def test_d3_collision_conserves_and_projects(nroots, order, b):
    """sum (f_ES - f){1, c, c^2} = 0 with c^2 over three axes; P(f_ES) = rho
    lambda (3x3, lambda = (1-b) T I + b P/rho with T = tr P/(3 rho)) and
    q(f_ES) = 0.  Catches T = tr P/(2 rho) or a trace over two axes."""
    p = params3(nroots, order, b)
    cx, cy, cz, _ = O.velocity_set_d(nroots, 3)
    for seed in range(3):
        f = noneq3(nroots, order, seed)
        fes, _, _ = O.cell_terms(p, f)
        d = fes - f
        for phi in (np.ones_like(cx), cx, cy, cz, cx * cx + cy * cy + cz * cz):
            assert abs(np.sum(d * phi)) < 1e-14
        rho, u, P, T, _ = moments3(f, cx, cy, cz)
        lam = (1 - b) * T * np.eye(3) + b * P / rho
        _, _, Pe, _, qe = moments3(fes, cx, cy, cz)
        assert np.allclose(Pe, rho * lam, atol=1e-13)
        assert np.allclose(qe, 0.0, atol=1e-13)


def test_d3_oracle_moments_match_numpy():
    """The oracle's moment routine in D = 3 against numpy (T over three
    degrees of freedom, sigma trace-free in 3D, q with c_z^2 in C^2)."""
    cx, cy, cz, _ = O.velocity_set_d(4, 3)
    f = noneq3(4, 3, 7, amp=0.05)
    out, P, u = O.cell_moments(4, 3, f)
    rho, un, Pn, T, q = moments3(f, cx, cy, cz)
    tr = np.trace(Pn) / 3
    ref = [rho, un[0], un[1], T, Pn[0, 0] - tr, Pn[0, 1], Pn[1, 1] - tr, q[0], q[1]]
    assert np.allclose(out, ref, atol=1e-15, rtol=1e-13)
    assert np.allclose(P, Pn, atol=1e-15) and np.allclose(u, un, atol=1e-16)


@pytest.mark.parametrize("nroots,order", [(4, 3), (6, 4)])
@pytest.mark.parametrize("b", [-0.5, 0.0, 0.5])
def test_d3_b_zero_is_bgk_and_tau(b, nroots, order):
    """tau = (Kn/Pr) T^varpi/(rho T) with the D = 3 temperature; at b = 0,
    f_ES is rho S(T, u) of Eq. (feq0) with D = 3."""
    p = params3(nroots, order, b, kn=0.2, visc=0.7)
    cx, cy, cz, _ = O.velocity_set_d(nroots, 3)
    f = noneq3(nroots, order, 11)
    f = 0.5 * (f + f[mirror_z(nroots)])  # even in c_z: u_z = 0
    fes, _, tau = O.cell_terms(p, f)
    rho, u, _, T, _ = moments3(f, cx, cy, cz)
    assert abs(tau - 0.2 * (1 - b) * T ** 0.7 / (rho * T)) < 1e-15
    if b == 0.0:
        assert abs(u[2]) < 1e-16
        assert np.allclose(fes, rho * O.feq0(nroots, order, T, u[0], u[1], dim=3), atol=1e-15)


@pytest.mark.parametrize("nroots,order", [(4, 3), (6, 4)])
@pytest.mark.parametrize("b", [-0.5, 0.5])
def test_d3_prandtl_number_from_relaxation(b, nroots, order):
    """One homogeneous step at u = 0: (1 - r_q)/(1 - r_sigma) = 1/(1 - b)."""
    dt = 2e-3
    p = params3(nroots, order, b, kn=0.1, dt=dt)
    cx, cy, cz, w = O.velocity_set_d(nroots, 3)
    f = O.feq0(nroots, order, 1.0, 0.0, 0.0, dim=3)
    pert = w * (0.01 * cx * cy + 0.01 * cx * (cx * cx + cy * cy + cz * cz - 5.0))
    f = f + pert - w * np.sum(pert * cx) / np.sum(w * cx * cx) * cx
    _, u0, P0, _, q0 = moments3(f, cx, cy, cz)
    assert np.abs(u0).max() < 1e-15
    f1 = O.run(p, f.reshape(-1, 1, 1), 1).reshape(-1)
    _, _, P1, _, q1 = moments3(f1, cx, cy, cz)
    assert abs((1 - q1[0] / q0[0]) / (1 - P1[0, 1] / P0[0, 1]) - 1.0 / (1.0 - b)) < 1e-9


@pytest.mark.parametrize("nroots,order", [(4, 3), (6, 4)])
def test_d3_force_moments(nroots, order):
    """Projected force with g_z = 0: sum g_a = 0, sum g_a c = rho g (no z
    component), sum g_a c^2 = 2 rho u.g."""
    g = (3e-3, -1e-3)
    p = params3(nroots, order, 0.0, g=g)
    cx, cy, cz, _ = O.velocity_set_d(nroots, 3)
    f = noneq3(nroots, order, 4)
    _, gf, _ = O.cell_terms(p, f)
    rho, u, *_ = moments3(f, cx, cy, cz)
    assert abs(gf.sum()) < 1e-16
    assert abs(np.sum(gf * cx) - rho * g[0]) < 1e-16 and abs(np.sum(gf * cy) - rho * g[1]) < 1e-16
    assert abs(np.sum(gf * cz)) < 1e-16
    assert abs(np.sum(gf * (cx ** 2 + cy ** 2 + cz ** 2)) - 2 * rho * (u[0] * g[0] + u[1] * g[1])) < 1e-16


# ---------------------------------------------------------------- whole steps
@pytest.mark.parametrize("nroots", [4, 6])
def test_d3_uniform_equilibrium_fixed_point_and_conservation(nroots):
    """A uniform rho S(T, u) is a fixed point; rough periodic fields keep mass,
    x/y momentum and energy (1/2 sum f c^2 with c_z^2) to rounding; the energy
    at rest equilibrium is (D/2) rho T per node with D = 3."""
    prob = Problem(name="t", nroots=nroots, dim=3, nx=6, ny=5, bc_y=PERIODIC, kn=0.05, b=-0.5)
    fields = np.zeros((4, 5, 6))
    fields[0], fields[1], fields[2], fields[3] = 1.2, 0.05, -0.03, 1.04
    p = oracle_params(prob, 2e-3)
    f = O.init(p, fields)
    assert np.max(np.abs(O.step(p, f) - f)) < 2e-16
    _, s = O.moments(p, f)
    assert abs(s[3] - 30 * (1.2 * (1.5 * 1.04 + 0.5 * (0.05 ** 2 + 0.03 ** 2)))) < 1e-12
    rough = random_fields(prob, seed=4)
    p = oracle_params(prob, time_step(prob, rough))
    f = O.init(p, rough)
    _, s0 = O.moments(p, f)
    _, s1 = O.moments(p, O.run(p, f, 5))
    assert np.allclose(s1, s0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("nroots", [4, 6])
def test_d3_cz_is_not_advected_and_symmetry_in_cz_is_kept(nroots):
    """The grid is two-dimensional: populations that differ only in c_z have
    the same x/y transport, and a state even in c_z (u_z = 0, g_z = 0, walls
    at rest in z) stays even through steps with walls, force, Maxwell walls
    and heating (to rounding).  Catches c_z entering the advection or a wall
    mirror that also flips c_z."""
    prob = Problem(name="t", nroots=nroots, dim=3, nx=8, ny=12, bc_y=DIFFUSE, kn=0.1, b=-0.5, wall_ux=(-0.05, 0.05),
                   wall_T=(0.97, 1.04), g=(1e-3, 2e-4), wall_specular=0.3, wall_T_amp=0.01, wall_T_freq=0.7)
    fields = random_fields(prob, seed=8, amp_u=0.03, amp_T=0.03, amp_rho=0.03)
    p = oracle_params(prob, time_step(prob, fields))
    f = O.init(p, fields)
    mz = mirror_z(nroots)
    assert np.max(np.abs(f - f[mz])) < 1e-16
    f = O.run(p, f, 20)
    assert np.max(np.abs(f - f[mz])) < 1e-14
    # zero z-momentum and zero normal mass flux at the walls
    *_, cz, _ = O.velocity_set_d(nroots, 3)
    assert np.abs(np.einsum("a,aji->ji", cz, f)).max() < 1e-14
    _, cy, _, _ = O.velocity_set_d(nroots, 3)
    for j in (0, prob.ny - 1):
        assert np.abs(np.einsum("a,ai->i", cy, f[:, j, :])).max() < 1e-15


@pytest.mark.parametrize("kind", ["couette", "fourier"])
def test_d3_navier_stokes_coefficients_cp_five_halves(kind):
    """Near-continuum channel centre with the D = 3 set: sigma_xy = -mu du/dy,
    mu = Kn T^varpi (D-independent), and q_y = -kappa dT/dy with
    kappa = (D + 2)/2 (Kn/Pr) mu = 5/2 (1 - b) Kn T^varpi: the C_p = 5/2 of the
    paper's runs.  (The D = 2 sets give 2 in place of 5/2.)  Gate 0.5%."""
    kn, ny, b = 0.02, 32, -0.5
    if kind == "couette":
        prob = Problem(name="t", nroots=4, dim=3, nx=1, ny=ny, bc_y=DIFFUSE, kn=kn, b=b, wall_ux=(-0.02, 0.02))
    else:
        prob = Problem(name="t", nroots=4, dim=3, nx=1, ny=ny, bc_y=DIFFUSE, kn=kn, b=b, wall_T=(0.98, 1.02))
    dt = time_step(prob)
    p = oracle_params(prob, dt)
    f = O.run(p, O.init(p), int(8 / (np.pi ** 2 * kn) / dt))
    m, _ = O.moments(p, f)
    dy, c = 1.0 / (ny - 1), ny // 2
    T = 0.5 * (m[3, c, 0] + m[3, c - 1, 0])
    if kind == "couette":
        grad = (m[1, c, 0] - m[1, c - 1, 0]) / dy
        flux = 0.5 * (m[5, c, 0] + m[5, c - 1, 0])
        coef = kn * T ** 0.5
    else:
        grad = (m[3, c, 0] - m[3, c - 1, 0]) / dy
        flux = 0.5 * (m[8, c, 0] + m[8, c - 1, 0])
        coef = (3 + 2) / 2 * kn * (1 - b) * T ** 0.5
    assert abs(flux / grad / (-coef) - 1.0) < 5e-3
