"""Seeded synthetic workloads for the lattice ES-BGK solver.

This module only draws numbers and names problem set-ups; it holds none of the
method's arithmetic (no quadrature, no Hermite algebra, no time-step rule).
Both the CUDA path and the FP64 oracle are fed from it, each computing the
method on its own.

Every workload is a flow of the kind validated in Sec. 4 of the paper
(Couette, Fourier, force-driven Poiseuille, low Mach, Kn 0.01-0.5), plus a
Taylor-Green vortex for a fully periodic throughput case.  Fields are returned
as float64 arrays of shape (4, ny, nx) holding rho, u_x, u_y, T.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

PERIODIC = 0
DIFFUSE = 1
UNSPLIT = 0  # the update of Sec. 3.1 as printed
SPLIT = 1    # y-sweep then x-sweep (for flows varying in x and y)


@dataclass(frozen=True)
class Problem:
    """One solve: lattice, grid, gas and boundary parameters.

    nroots: Gauss-Hermite roots per axis (4 -> D2Q16, 6 -> D2Q36; with dim 3,
            4 -> D3Q64).
    dim:    dimension D of the velocity set (2, or 3 for the paper's D = 3
            thermodynamics on the same two-dimensional grid).
    order:  Hermite truncation order N of f_ES (0 selects the default).
    bc_y:   PERIODIC or DIFFUSE (walls on rows j=0 and j=ny-1).
    bc_x:   PERIODIC or DIFFUSE (walls at rest on columns i=0 and i=nx-1, at
            temperatures wall_Tx; with walls on both axes: a cavity whose lid
            is the top wall, moving at wall_ux[1]).
    kn, b, visc_exp: Knudsen number, ES parameter b, viscosity exponent.
    cfl:    Courant number used when no explicit dt is given.
    wall_T, wall_ux: (bottom, top) wall temperature and x-velocity.
    g:      body force (g_x, g_y).
    init:   'rest', 'tgv' (Taylor-Green vortex with density noise) or 'shear'
            (a shear and temperature wave along y with density noise).
    scheme: UNSPLIT (both flux differences from f^n, as printed) or SPLIT.
    wall_specular, wall_T_amp, wall_T_freq: Maxwell walls (fraction re-emitted
        specularly) and sinusoidal wall heating.
    """

    name: str
    nroots: int = 4
    order: int = 0
    dim: int = 2
    nx: int = 4
    ny: int = 64
    bc_y: int = DIFFUSE
    kn: float = 0.1
    b: float = -0.5
    visc_exp: float = 0.5
    cfl: float = 0.5
    wall_T: tuple = (1.0, 1.0)
    wall_ux: tuple = (0.0, 0.0)
    g: tuple = (0.0, 0.0)
    init: str = "rest"
    tgv_amp: float = 0.05
    tgv_dT: float = 0.01
    rho_noise: float = 1e-4
    seed: int = 0
    steps: int = 1000
    scheme: int = UNSPLIT
    wall_specular: float = 0.0  # 1 - accommodation gamma of the Maxwell wall model
    wall_T_amp: float = 0.0     # wall heating T_w(t) = wall_T + amp sin(freq t)
    wall_T_freq: float = 0.0
    bc_x: int = PERIODIC
    wall_Tx: tuple = (1.0, 1.0)

    @property
    def cells(self) -> int:
        return self.nx * self.ny


def couette_4x64() -> Problem:
    """Planar Couette flow, walls at -/+0.05, T_w = 1, D2Q16, Kn 0.1, b -1/2."""
    return Problem(name="couette_4x64_d2q16", nroots=4, nx=4, ny=64, bc_y=DIFFUSE, kn=0.1,
                   b=-0.5, wall_ux=(-0.05, 0.05), steps=2000)


def tgv(n: int = 4096, steps: int = 1000, nroots: int = 4) -> Problem:
    """Fully periodic Taylor-Green vortex, Ma 0.05, 1% T perturbation, rho noise 1e-4.
    The flow varies in x and y, so it runs with the split scheme."""
    return Problem(name=f"tgv_{n}x{n}_d2q{nroots * nroots}", nroots=nroots, nx=n, ny=n,
                   bc_y=PERIODIC, kn=0.05, b=-0.5, init="tgv", steps=steps, scheme=SPLIT)


def shear_strip(ny: int = 4096, nx: int = 4, kn: float = 0.05, steps: int = 1000, nroots: int = 4,
                dim: int = 2) -> Problem:
    """A periodic strip nx x ny holding a shear wave and a temperature wave
    along y (Taylor-Green amplitudes: u_x = 0.05 sin 2 pi y, T = 1 + 0.01
    cos 2 pi y, density noise 1e-4), Kn 0.05, b = -1/2, split scheme.  With
    ny = 4096 its y-spacing, time step and tau are those of the 4096^2
    Taylor-Green solve (dt/tau ~ 7e-4), on 4 ny nodes instead of ny^2."""
    return Problem(name=f"shear_{nx}x{ny}", nroots=nroots, dim=dim, nx=nx, ny=ny, bc_y=PERIODIC, kn=kn, b=-0.5,
                   init="shear", steps=steps, scheme=SPLIT)


def poiseuille(nx: int = 512, ny: int = 1024, steps: int = 1000) -> Problem:
    """Force-driven Poiseuille channel, g = 1e-4 along +x, Kn 0.2, b = 0."""
    return Problem(name=f"poiseuille_{nx}x{ny}_d2q16", nroots=4, nx=nx, ny=ny, bc_y=DIFFUSE,
                   kn=0.2, b=0.0, g=(1e-4, 0.0), steps=steps)


def fourier(ny: int = 64, kn: float = 0.1, b: float = -0.5) -> Problem:
    """Fourier heat transfer between walls at T = 1 -/+ 0.05."""
    return Problem(name=f"fourier_4x{ny}", nroots=4, nx=4, ny=ny, bc_y=DIFFUSE, kn=kn, b=b,
                   wall_T=(0.95, 1.05))


def unsteady_heating(kn: float = 0.1, b: float = -0.5, st: float = 0.5553603672697958, amp: float = 0.002,
                     ny: int = 64, steps: int = 2000) -> Problem:
    """Both walls heated as T_w = 1 + amp sin(St t), gas initially at rest at
    T = 1 (Sec. 4.2; St = pi sqrt(2)/8 by default)."""
    return Problem(name=f"heating_kn{kn:g}_st{st:.3f}", nroots=4, nx=4, ny=ny, bc_y=DIFFUSE, kn=kn, b=b,
                   wall_T_amp=amp, wall_T_freq=st, steps=steps)


def kn_of_kd(kd: float) -> float:
    """Kn of Sec. 2.2 from the K_D = sqrt(pi/2) Kn that labels the paper's results."""
    return kd / np.sqrt(np.pi / 2.0)


# The high-Mach-number workloads of Sec. 4 (the paper runs them with its
# "11th-order" set, D2Q36 here, or the D = 3 set for its C_p = 5/2 gas).
def couette_high_ma(kd: float = 0.05, nroots: int = 6, dim: int = 2, b: float = -0.5, ny: int = 64,
                    steps: int = 4000) -> Problem:
    """Couette flow with walls at -/+0.2 (viscous heating), T_w = 1."""
    return Problem(name=f"couette_ma_kd{kd:g}", nroots=nroots, dim=dim, nx=4, ny=ny, bc_y=DIFFUSE,
                   kn=kn_of_kd(kd), b=b, wall_ux=(-0.2, 0.2), steps=steps)


def poiseuille_high_force(kd: float = 0.1, nroots: int = 6, dim: int = 2, b: float = -0.5, ny: int = 64,
                          steps: int = 2000) -> Problem:
    """Force-driven Poiseuille flow, g = 0.22 along x, walls at rest, T_w = 1."""
    return Problem(name=f"poiseuille_g0.22_kd{kd:g}", nroots=nroots, dim=dim, nx=4, ny=ny, bc_y=DIFFUSE,
                   kn=kn_of_kd(kd), b=b, g=(0.22, 0.0), steps=steps)


def couette_fourier(kd: float = 0.1, nroots: int = 6, dim: int = 2, b: float = -0.5, ny: int = 64,
                    steps: int = 4000) -> Problem:
    """Combined Couette-Fourier flow: walls at -/+0.2 and T_w = 1 -/+ 0.15."""
    return Problem(name=f"couette_fourier_kd{kd:g}", nroots=nroots, dim=dim, nx=4, ny=ny, bc_y=DIFFUSE,
                   kn=kn_of_kd(kd), b=b, wall_ux=(-0.2, 0.2), wall_T=(0.85, 1.15), steps=steps)


def lid_driven_cavity(n: int = 256, u_lid: float = 0.05, kn: float = 0.1, b: float = -0.5, nroots: int = 4,
                      steps: int = 4000) -> Problem:
    """2D lid-driven cavity on the unit square: n x n nodes, walls on all four
    sides at T_w = 1, the top wall moving at u_lid in x (not in the paper:
    its flows are uniform in x; a standard 2D test of the wall rule)."""
    return Problem(name=f"cavity_{n}_kn{kn:g}", nroots=nroots, nx=n, ny=n, bc_y=DIFFUSE, bc_x=DIFFUSE, kn=kn, b=b,
                   wall_ux=(0.0, u_lid), scheme=SPLIT, steps=steps)


def initial_fields(p: Problem) -> np.ndarray:
    """(4, ny, nx) float64: rho, u_x, u_y, T at the nodes.

    Periodic axes put node i at x = i/n; wall-bounded y puts node j at
    y = j/(ny-1).  'tgv': u_x = A sin(2 pi x) cos(2 pi y),
    u_y = -A cos(2 pi x) sin(2 pi y), T = 1 + dT sin(2 pi x) sin(2 pi y),
    rho = 1 + U(-noise, noise) i.i.d. per node (numpy default_rng(seed)).
    'shear' (periodic in y, node j at y = j/ny): u_x = A sin(2 pi y), u_y = 0,
    T = 1 + dT cos(2 pi y), rho = 1 + U(-noise, noise) i.i.d. per node.
    """
    out = np.zeros((4, p.ny, p.nx))
    out[0] = 1.0
    out[3] = 1.0
    if p.init == "rest":
        return out
    if p.init == "shear":
        y = np.arange(p.ny) / p.ny
        tp = 2.0 * np.pi
        out[1] = p.tgv_amp * np.sin(tp * y)[:, None]
        out[3] = 1.0 + p.tgv_dT * np.cos(tp * y)[:, None]
        rng = np.random.default_rng(p.seed)
        out[0] = 1.0 + rng.uniform(-p.rho_noise, p.rho_noise, size=(p.ny, p.nx))
        return out
    if p.init != "tgv":
        raise ValueError(p.init)
    x = np.arange(p.nx) / p.nx
    y = np.arange(p.ny) / (p.ny if p.bc_y == PERIODIC else (p.ny - 1))
    X, Y = np.meshgrid(x, y)
    tp = 2.0 * np.pi
    out[1] = p.tgv_amp * np.sin(tp * X) * np.cos(tp * Y)
    out[2] = -p.tgv_amp * np.cos(tp * X) * np.sin(tp * Y)
    out[3] = 1.0 + p.tgv_dT * np.sin(tp * X) * np.sin(tp * Y)
    rng = np.random.default_rng(p.seed)
    out[0] = 1.0 + rng.uniform(-p.rho_noise, p.rho_noise, size=(p.ny, p.nx))
    return out


def random_fields(p: Problem, amp_u: float = 0.05, amp_T: float = 0.05, amp_rho: float = 0.05,
                  seed: int = 0) -> np.ndarray:
    """Rough i.i.d. fields (for parity on non-smooth data, every limiter branch)."""
    rng = np.random.default_rng(seed)
    out = np.empty((4, p.ny, p.nx))
    out[0] = 1.0 + rng.uniform(-amp_rho, amp_rho, size=(p.ny, p.nx))
    out[1] = rng.uniform(-amp_u, amp_u, size=(p.ny, p.nx))
    out[2] = rng.uniform(-amp_u, amp_u, size=(p.ny, p.nx))
    out[3] = 1.0 + rng.uniform(-amp_T, amp_T, size=(p.ny, p.nx))
    return out


def batch_mix(n: int = 512, seed: int = 0, ny_lo: int = 16, ny_hi: int = 1024,
              steps: int = 2000) -> list[Problem]:
    """Independent 1D-in-y instances: nx = 4, ny log-uniform on [ny_lo, ny_hi],
    type uniform over Couette (-/+0.05), Fourier (T = 1 -/+ 0.05) and force-driven
    Poiseuille (g = 1e-4); Kn log-uniform on [0.01, 0.5]; b from {-1/2, 0, 1/2}."""
    rng = np.random.default_rng(seed)
    ny = np.rint(np.exp(rng.uniform(np.log(ny_lo), np.log(ny_hi), size=n))).astype(int)
    kind = rng.integers(0, 3, size=n)
    kn = np.exp(rng.uniform(np.log(0.01), np.log(0.5), size=n))
    b = rng.choice(np.array([-0.5, 0.0, 0.5]), size=n)
    out = []
    for k in range(n):
        base = Problem(name=f"batch{k}", nroots=4, nx=4, ny=int(ny[k]), bc_y=DIFFUSE,
                       kn=float(kn[k]), b=float(b[k]), steps=steps)
        if kind[k] == 0:
            base = replace(base, name=f"couette{k}", wall_ux=(-0.05, 0.05))
        elif kind[k] == 1:
            base = replace(base, name=f"fourier{k}", wall_T=(0.95, 1.05))
        else:
            base = replace(base, name=f"poiseuille{k}", g=(1e-4, 0.0))
        out.append(base)
    return out
