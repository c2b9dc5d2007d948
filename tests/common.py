"""Test-side helpers: turn a seeded Problem into oracle parameters.

The grid spacing and time step are fixed here, on the test side, from the
problem statement, and passed explicitly to both the oracle and the CUDA
library, so that neither side's input comes from the other.

Spacing: a periodic axis of n nodes has delta = 1/n; with walls on rows 0 and
ny-1 the channel width is 1, delta_y = 1/(ny-1) and delta_x = delta_y (and
the same with the axes exchanged); with walls on both axes the box is the
unit square, delta_x = 1/(nx-1), delta_y = 1/(ny-1).
Time step: dt = min(cfl * min(dx, dy) / c_max, tau_ref) with
tau_ref = (Kn/Pr) T_max^(varpi-1) / rho_max, T_max over the initial fields and
the walls' peak temperature (forward-Euler relaxation stays at dt/tau <= 1 at
the reference state).
"""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_1209_6548_gb300.inputs import PERIODIC, Problem

DEFAULT_ORDER = {4: 3, 6: 4}


def order_of(p: Problem) -> int:
    return p.order if p.order else DEFAULT_ORDER[p.nroots]


def spacing(p: Problem):
    bc_x = getattr(p, "bc_x", PERIODIC)
    if p.bc_y == PERIODIC and bc_x == PERIODIC:
        return 1.0 / p.nx, 1.0 / p.ny
    if bc_x == PERIODIC:  # walls in y: channel of width 1, square cells
        d = 1.0 / (p.ny - 1)
        return d, d
    if p.bc_y == PERIODIC:  # walls in x only
        d = 1.0 / (p.nx - 1)
        return d, d
    return 1.0 / (p.nx - 1), 1.0 / (p.ny - 1)  # walls on both axes: the unit square


def time_step(p: Problem, fields=None) -> float:
    dx, dy = spacing(p)
    c, _ = O.gauss_hermite_1d(p.nroots)
    dt_cfl = p.cfl * min(dx, dy) / float(np.max(np.abs(c)))
    tmax = max(p.wall_T) + abs(p.wall_T_amp) if p.bc_y != PERIODIC else 1.0
    if getattr(p, "bc_x", PERIODIC) != PERIODIC:
        tmax = max(tmax, max(p.wall_Tx))
    rmax = 1.0
    if fields is not None:
        tmax = max(tmax, float(fields[3].max()))
        rmax = float(fields[0].max())
    pr = 1.0 / (1.0 - p.b)
    tau_ref = (p.kn / pr) * tmax ** (p.visc_exp - 1.0) / rmax
    return min(dt_cfl, tau_ref)


def oracle_params(p: Problem, dt: float, nx=None, ny=None, bc_y=None):
    dx, dy = spacing(p)
    return O.make_params(nroots=p.nroots, order=order_of(p), nx=nx or p.nx, ny=ny or p.ny,
                         bc_y=p.bc_y if bc_y is None else bc_y, kn=p.kn, b=p.b,
                         visc_exp=p.visc_exp, dt=dt, dx=dx, dy=dy, wall_T=tuple(p.wall_T),
                         wall_ux=tuple(p.wall_ux), g=tuple(p.g), scheme=p.scheme,
                         wall_specular=p.wall_specular, wall_T_amp=p.wall_T_amp, wall_T_freq=p.wall_T_freq,
                         dim=p.dim, bc_x=p.bc_x, wall_Tx=tuple(p.wall_Tx))


GROUPS = {"rho": ("rho",), "T": ("T",), "u": ("ux", "uy"), "sigma": ("sxx", "sxy", "syy"),
          "q": ("qx", "qy")}
REST = {"rho": 1.0, "T": 1.0}  # rest-state value of each field (0 for the others)

# Unit roundoff of the stored deviations, per step (std of one rounding is at
# most this times |df|):
#   FP32, round to nearest: the store is the last FMA of the update, whose
#   error is uniform on +-ulp/2 (std ulp/sqrt(12) <= 0.58 * 2^-24 |x|); the
#   increment's other operations round at magnitudes up to |df| on rough data
#   (three FMAs): 2 * 2^-24 covers them.
#   FP16 / BF16, stochastic rounding of df/w: std <= ulp/2 <= 2^-11 (FP16) and
#   2^-8 (BF16) times |df|, plus the same FP32 arithmetic.
#   Compensated FP32 (f32c): the stored remainder makes the storage error
#   2^-11 of half an ulp, but the increment is still formed in FP32, whose
#   rounding is at most that of FP32 storage where the increment is as large
#   as the value (rough data, dt/tau ~ 1): bounded as FP32.
EPS_STEP = {"f32": 2.0 * 2.0 ** -24, "f32c": 2.0 * 2.0 ** -24, "f16": 2.0 ** -11 + 2.0 * 2.0 ** -24,
            "bf16": 2.0 ** -8 + 2.0 * 2.0 ** -24}


def moment_sensitivity(f: np.ndarray, nroots: int, dim: int = 2) -> np.ndarray:
    """First-order sensitivity of the nine moment fields to the stored values.

    f: the oracle's FP64 populations (nvel, ny, nx).  Returns G[k, s, j, i] =
    d(field k)/d(stored value s) at each node, for the nine fields of
    O.MOMENT_NAMES, from the definitions of Eq. (mac):
      rho: 1;  u_i: C_i / rho;  T: (C^2 - D T)/(D rho);
      sigma_ij: C_i C_j - delta_ij C^2 / D  (trace-free: its u-derivative is
        sum f C = 0);
      q_i = 1/2 sum f C_i C^2: 1/2 C_i C^2 - 1/2 [(D rho T + 2 P_ii) C_i
        + 2 P_ij C_j] / rho  (the second term through u).
    For the D = 3 set one stored value stands for the velocities at +c_z and
    -c_z (the z-even half), so their sensitivities add."""
    cx, cy, cz, w = O.velocity_set_d(nroots, dim) if dim == 3 else (*O.velocity_set(nroots)[:2],
                                                                    np.zeros(nroots * nroots),
                                                                    O.velocity_set(nroots)[2])
    e = lambda v: v[:, None, None]  # noqa: E731
    rho = f.sum(0)
    ux = (f * e(cx)).sum(0) / rho
    uy = (f * e(cy)).sum(0) / rho
    Cx, Cy, Cz = e(cx) - ux, e(cy) - uy, e(cz) + 0.0 * ux
    C2 = Cx * Cx + Cy * Cy + Cz * Cz
    T = (f * C2).sum(0) / (dim * rho)
    Pxx, Pxy, Pyy = (f * Cx * Cx).sum(0), (f * Cx * Cy).sum(0), (f * Cy * Cy).sum(0)
    trP = dim * rho * T
    g = np.stack([np.ones_like(Cx), Cx / rho, Cy / rho, (C2 - dim * T) / (dim * rho),
                  Cx * Cx - C2 / dim, Cx * Cy, Cy * Cy - C2 / dim,
                  0.5 * Cx * C2 - 0.5 * ((trP + 2 * Pxx) * Cx + 2 * Pxy * Cy) / rho,
                  0.5 * Cy * C2 - 0.5 * ((trP + 2 * Pyy) * Cy + 2 * Pxy * Cx) / rho])
    if dim != 3:
        return g
    # oracle order alpha = (ix nroots + iy) nroots + iz; stored: iz >= nroots/2
    g = g.reshape(9, nroots * nroots, nroots, *f.shape[1:])
    h = nroots // 2
    return (g[:, :, h:] + g[:, :, h - 1::-1]).reshape(9, -1, *f.shape[1:])


def stored_deviations(f: np.ndarray, nroots: int, dim: int = 2) -> np.ndarray:
    """The values the GPU stores per node, f_a - w_a (the c_z > 0 half for D = 3)."""
    if dim != 3:
        w = O.velocity_set(nroots)[2]
        return f - w[:, None, None]
    w = O.velocity_set_d(nroots, 3)[3]
    d = (f - w[:, None, None]).reshape(nroots * nroots, nroots, *f.shape[1:])
    return d[:, nroots // 2:].reshape(-1, *f.shape[1:])


def rounding_bound(states, nroots: int, dim: int, steps: int, storage: str = "f32", prob=None,
                   dt: float = 0.0) -> np.ndarray:
    """Per-field bound (absolute) on what rounding can do after `steps` time
    steps, evaluated on the oracle's populations.

    states: the oracle's FP64 populations (nvel, ny, nx) along the run (the
    initial state and the checkpoints), or one such array.

    Each step rounds every stored value once, with an error of std at most
    eps |df| (EPS_STEP); a field moves by sum_s G_s delta_s (G from
    moment_sensitivity), so one step adds to its error at a node a term of
    size eps R, R = sqrt(sum_s G_s^2 df_s^2), taken at its largest over the
    nodes and the states given.  How the steps' errors add depends on the
    rounding and on the field:
      - stochastic rounding (16-bit storage) is unbiased: a random walk,
        std <= sqrt(n_eff) eps R, and the largest of N nodes stays below
        sqrt(2 ln 2N) standard deviations;
      - round to nearest (FP32) is a random walk for the conserved fields
        (rho, u, T), as above, but biased for the stress and the heat flux,
        whose slowly varying increments (production by the gradients against
        relaxation) round the same way step after step: there the errors add
        linearly, at most n_eff eps R.
    n_eff = n for the conserved fields; the stress and the heat flux relax
    towards equilibrium at r = (1 - b) dt/tau and dt/tau per step (tau =
    (Kn/Pr) T^(varpi-1)/rho, Pr = 1/(1-b); Sec. 2.1), r at its smallest over
    the nodes, so n_eff = min(n, 1/r) for a sum of biased terms and
    min(n, 1/(2r)) for a random walk's variance.  Once, in addition: the
    initial state and the moments themselves are evaluated in FP32 (and the
    initial populations rounded to the storage), each at most
    eps A with A = sum_s |G_s| |df_s|: 4 * 2^-24 A + eps_store A.  Nothing
    credits the advection's averaging, so the bound is an upper one."""
    if isinstance(states, np.ndarray):
        states = [states]
    Rmax, Amax = np.zeros(9), np.zeros(9)
    omega_min = np.inf
    for f in states:
        G = moment_sensitivity(f, nroots, dim)
        df = stored_deviations(f, nroots, dim)[None]
        R = np.sqrt(np.sum(G * G * df * df, axis=1))  # (9, ny, nx)
        A = np.sum(np.abs(G) * np.abs(df), axis=1)
        Rmax = np.maximum(Rmax, R.reshape(9, -1).max(axis=1))
        Amax = np.maximum(Amax, A.reshape(9, -1).max(axis=1))
        if prob is not None and dt > 0.0:
            m = O.moments(oracle_params(prob, dt, nx=f.shape[2], ny=f.shape[1]), f)[0]
            pr = 1.0 / (1.0 - prob.b)
            tau = (prob.kn / pr) * m[3] ** (prob.visc_exp - 1.0) / m[0]
            omega_min = min(omega_min, float(np.min(dt / tau)))
    nodes = states[0].shape[1] * states[0].shape[2]
    z = np.sqrt(2.0 * np.log(2.0 * nodes))
    n = float(max(steps, 1))
    names = list(O.MOMENT_NAMES)
    relaxing = {"sxx": 1.0 - (prob.b if prob is not None else 0.0), "sxy": 1.0 - (prob.b if prob is not None else 0.0),
                "syy": 1.0 - (prob.b if prob is not None else 0.0), "qx": 1.0, "qy": 1.0}
    eps = EPS_STEP[storage]
    out = np.zeros(9)
    for k, name in enumerate(names):
        rate = relaxing.get(name, 0.0) * omega_min if np.isfinite(omega_min) else 0.0
        if storage in ("f32", "f32c") and name in relaxing:  # biased: linear, damped
            walk = min(n, 1.0 / rate) if rate > 0.0 else n
            per_step = walk * eps * Rmax[k]
        else:  # unbiased: random walk, damped where the field relaxes
            walk = min(n, 1.0 / (2.0 * rate)) if rate > 0.0 else n
            per_step = z * np.sqrt(max(walk, 1.0)) * eps * Rmax[k]
        store = 0.0 if storage in ("f32", "f32c") else eps - 2.0 * 2.0 ** -24
        out[k] = per_step + (4.0 * 2.0 ** -24 + store) * Amax[k]
    return out


def population_bound(states, nroots: int, dim: int, steps: int, storage: str = "f32", prob=None,
                     dt: float = 0.0) -> float:
    """Bound (absolute) on a stored value's accumulated rounding after
    `steps` steps: each step rounds it once by at most eps |df| (EPS_STEP),
    and in the worst case the n errors add (a population's error also feeds
    the conserved moments, which do not relax); plus the initial state's FP32
    evaluation (4 * 2^-24 |df|).  |df| at its largest over the states given."""
    if isinstance(states, np.ndarray):
        states = [states]
    dmax = max(float(np.max(np.abs(stored_deviations(f, nroots, dim)))) for f in states)
    return (max(steps, 1) * EPS_STEP[storage] + 4.0 * 2.0 ** -24) * dmax


def field_errors(gpu: np.ndarray, ref: np.ndarray, bound=None, bar: float = 1e-5):
    """Per-field errors of the GPU moments against the oracle's.

    Returns {name: dict} with
      abs:   max |gpu - ref| over the field;
      e:     abs / S, S the largest magnitude of the quantity the field belongs
             to (rho; T; the velocity vector; the stress tensor; the heat-flux
             vector), so a component near zero by symmetry is measured against
             its vector's scale;
      e_own: abs / max|ref| of the field itself;
      e_pert: abs / max|ref - rest value| (rest: rho = T = 1, the rest 0), or
             None where that perturbation is below 1e-6;
      tol:   max(bar * S, bound) -- the 1e-5 bar, or the field's FP32
             storage-rounding bound (rounding_bound) where that is larger;
      ok:    abs <= tol."""
    names = list(O.MOMENT_NAMES)
    scale = {}
    for members in GROUPS.values():
        s = max(float(np.max(np.abs(ref[names.index(m)]))) for m in members)
        for m in members:
            scale[m] = s
    out = {}
    for k, name in enumerate(names):
        d = float(np.max(np.abs(gpu[k].astype(np.float64) - ref[k])))
        own = float(np.max(np.abs(ref[k])))
        pert = float(np.max(np.abs(ref[k] - REST.get(name, 0.0))))
        b = 0.0 if bound is None else float(bound[k])
        tol = max(bar * scale[name], b)
        out[name] = {"abs": d, "e": d / scale[name] if scale[name] > 0 else d, "e_own": d / own if own > 0 else d,
                     "e_pert": d / pert if pert >= 1e-6 else None, "bound": b, "tol": tol, "ok": d <= tol}
    return out


# Every comparison made through record(): written as JSON at the end of the
# session when LESBGK_PARITY_REPORT names a file (tests/conftest.py).
REPORT = []


def record(what: str, errs: dict) -> None:
    import os
    test = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
    REPORT.append({"test": test, "what": what,
                   "fields": {k: {kk: vv for kk, vv in v.items()} for k, v in errs.items()}})
