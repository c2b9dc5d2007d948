"""Pins of the FP64 oracle's walls in x and cavity corners (not in the paper,
whose flows are uniform in x; the corner rule is a reading).

The x-wall code is pinned against the y-wall code through transposition: with
the printed (unsplit) update on a square grid, exchanging x and y (and c_x
with c_y) maps a channel walled in y onto one walled in x, and a closed box
onto itself, exactly.  Invariants pin the rest: zero normal mass flux at every
wall node, zero flux along the bisector n_x + n_y at corners, a resting gas in
a closed box at the wall temperature stays at rest, and a lid-driven cavity
turns the way the lid drags it.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1209_6548_gb300.inputs import DIFFUSE, PERIODIC, UNSPLIT, Problem, lid_driven_cavity, random_fields
from tests.common import oracle_params, time_step


def transpose_index(nroots, dim):
    """alpha -> alpha' with c_x and c_y exchanged."""
    nz = nroots if dim == 3 else 1
    a = np.arange(nroots * nroots * nz)
    iz, iy, ix = a % nz, (a // nz) % nroots, a // (nz * nroots)
    return (iy * nroots + ix) * nz + iz


def transposed_fields(fields):
    out = np.empty_like(fields.transpose(0, 2, 1))
    out[0], out[3] = fields[0].T, fields[3].T
    out[1], out[2] = fields[2].T, fields[1].T
    return out


def run(prob, fields, steps):
    p = oracle_params(prob, time_step(prob, fields))
    return O.run(p, O.init(p, fields), steps), p


@pytest.mark.parametrize("nroots,dim", [(4, 2), (6, 2), (4, 3)])
def test_x_walled_channel_is_the_transposed_y_walled_channel(nroots, dim):
    """A channel walled in y (periodic x) and the same channel walled in x
    (periodic y), started from transposed fields, stay transposed: the x-wall
    rule, its ghost columns and the spacing follow the y-wall ones exactly.
    Catches c_y left in the x-wall flux, a wrong outgoing half or sign, or
    ghost columns that wrap."""
    n = 12
    py = Problem(name="y", nroots=nroots, dim=dim, nx=n, ny=n, bc_y=DIFFUSE, kn=0.1, b=-0.5, wall_T=(0.97, 1.04),
                 scheme=UNSPLIT)
    px = Problem(name="x", nroots=nroots, dim=dim, nx=n, ny=n, bc_y=PERIODIC, bc_x=DIFFUSE, kn=0.1, b=-0.5,
                 wall_Tx=(0.97, 1.04), scheme=UNSPLIT)
    fy = random_fields(py, seed=3, amp_u=0.03, amp_T=0.03, amp_rho=0.03)
    fx = transposed_fields(fy)
    assert time_step(py, fy) == time_step(px, fx)
    gy, _ = run(py, fy, 12)
    gx, _ = run(px, fx, 12)
    t = transpose_index(nroots, dim)
    assert np.max(np.abs(gx[t] - gy.transpose(0, 2, 1))) < 1e-14


@pytest.mark.parametrize("nroots,dim", [(4, 2), (4, 3)])
def test_closed_box_is_transposition_symmetric(nroots, dim):
    """A closed square box, all walls at one temperature, no lid: transposed
    initial fields give the transposed state (corners included)."""
    n = 10
    prob = Problem(name="box", nroots=nroots, dim=dim, nx=n, ny=n, bc_y=DIFFUSE, bc_x=DIFFUSE, kn=0.1, b=0.5,
                   wall_T=(1.03, 1.03), wall_Tx=(1.03, 1.03), scheme=UNSPLIT)
    f0 = random_fields(prob, seed=5, amp_u=0.03, amp_T=0.03, amp_rho=0.03)
    g0, _ = run(prob, f0, 10)
    g1, _ = run(prob, transposed_fields(f0), 10)
    t = transpose_index(nroots, dim)
    assert np.max(np.abs(g1[t] - g0.transpose(0, 2, 1))) < 1e-14


def test_cavity_wall_fluxes_vanish():
    """After every step: sum c_x f = 0 on x-wall nodes, sum c_y f = 0 on
    y-wall nodes, and sum (c.n_x + c.n_y) f = 0 at the four corners (the
    corner reading's definition of rho_W)."""
    prob = Problem(name="cav", nx=9, ny=11, bc_y=DIFFUSE, bc_x=DIFFUSE, kn=0.1, b=-0.5, wall_ux=(0.0, 0.1),
                   wall_T=(0.98, 1.02), wall_Tx=(1.01, 0.99))
    fields = random_fields(prob, seed=9, amp_u=0.02, amp_T=0.02, amp_rho=0.02)
    p = oracle_params(prob, time_step(prob, fields))
    f = O.init(p, fields)
    cx, cy, _ = O.velocity_set(4)
    for _ in range(4):
        for i in (0, prob.nx - 1):
            assert np.abs(np.einsum("a,aj->j", cx, f[:, 1:-1, i])).max() < 1e-15
        for j in (0, prob.ny - 1):
            assert np.abs(np.einsum("a,ai->i", cy, f[:, j, 1:-1])).max() < 1e-15
        for i, nx_ in ((0, 1.0), (prob.nx - 1, -1.0)):
            for j, ny_ in ((0, 1.0), (prob.ny - 1, -1.0)):
                assert abs(np.sum((cx * nx_ + cy * ny_) * f[:, j, i])) < 1e-15
        f = O.step(p, f)


def test_closed_box_at_rest_stays_at_rest():
    """Rest gas at T = 1 in a box whose walls are at rest at T = 1."""
    prob = Problem(name="box", nx=7, ny=9, bc_y=DIFFUSE, bc_x=DIFFUSE, kn=0.1, b=-0.5)
    p = oracle_params(prob, time_step(prob))
    f = O.init(p)
    assert np.max(np.abs(O.run(p, f, 5) - f)) < 1e-15


def test_lid_driven_cavity_turns_with_the_lid():
    """Lid moving in +x at the top: the gas under the lid moves with it, the
    return flow near the bottom runs in -x, it descends along the right wall
    and rises along the left wall (a clockwise vortex)."""
    prob = lid_driven_cavity(n=24, u_lid=0.05, kn=0.1)
    p = oracle_params(prob, time_step(prob))
    f = O.run(p, O.init(p), 600)
    m, _ = O.moments(p, f)
    ux, uy = m[1], m[2]
    n = prob.nx
    assert ux[-2, n // 2] > 0.01 and ux[2, n // 2] < 0.0
    assert uy[n // 2, -3] < 0.0 and uy[n // 2, 2] > 0.0
    assert np.isfinite(f).all()
