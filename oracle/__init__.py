"""FP64 CPU oracle for the lattice ES-BGK step (arXiv 1209.6548).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may load it; the
product library never does.  The arithmetic lives in ``lesbgk_oracle.c``
(plain C, double precision, written from the paper's formulas); this module
only compiles it with gcc and marshals numpy arrays through ctypes.

Functions with no pin beyond agreement with themselves are listed in the
module docstring of ``tests/test_oracle_pins.py``; every other function here
is pinned there against closed forms, library routines or invariants.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lesbgk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblesbgk_oracle.so")
_lock = threading.Lock()
_lib = None


class OrcParams(C.Structure):
    _fields_ = [
        ("nroots", C.c_int32), ("order", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32),
        ("bc_y", C.c_int32), ("scheme", C.c_int32), ("dim", C.c_int32), ("bc_x", C.c_int32),
        ("kn", C.c_double), ("b", C.c_double), ("visc_exp", C.c_double),
        ("dt", C.c_double), ("dx", C.c_double), ("dy", C.c_double),
        ("wall_T", C.c_double * 2), ("wall_ux", C.c_double * 2), ("g", C.c_double * 2),
        ("wall_specular", C.c_double), ("wall_T_amp", C.c_double), ("wall_T_freq", C.c_double),
        ("time", C.c_double), ("wall_Tx", C.c_double * 2),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build (gcc -O2, OpenMP, IEEE math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                               "-fno-fast-math", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.orc_hermite_he.restype = C.c_double
            _lib.orc_hermite_he.argtypes = [C.c_int, C.c_double]
            _lib.orc_get_threads.restype = C.c_int
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def hermite_he(n: int, x: float) -> float:
    return float(lib().orc_hermite_he(int(n), float(x)))


def gauss_hermite_1d(n: int):
    c = np.zeros(n)
    w = np.zeros(n)
    if lib().orc_gauss_hermite_1d(int(n), _dp(c), _dp(w)):
        raise ValueError(f"no {n}-point rule")
    return c, w


def nvel(nroots: int, dim: int = 2) -> int:
    return nroots ** dim


def velocity_set(nroots: int):
    """D = 2 set: (c_x, c_y, w), alpha = ix*nroots + iy."""
    q = nroots * nroots
    cx, cy, w = np.zeros(q), np.zeros(q), np.zeros(q)
    if lib().orc_velocity_set(int(nroots), _dp(cx), _dp(cy), _dp(w)):
        raise ValueError("bad nroots")
    return cx, cy, w


def velocity_set_d(nroots: int, dim: int):
    """(c_x, c_y, c_z, w) of the D-dimensional set (c_z = 0 for D = 2);
    alpha = (ix*nroots + iy)*nroots + iz for D = 3."""
    q = nvel(nroots, dim)
    cx, cy, cz, w = np.zeros(q), np.zeros(q), np.zeros(q), np.zeros(q)
    if lib().orc_velocity_set_d(int(nroots), int(dim), _dp(cx), _dp(cy), _dp(cz), _dp(w)):
        raise ValueError("bad nroots or dim")
    return cx, cy, cz, w


def chi(n: int, c) -> np.ndarray:
    """chi^(n)(c) as a (D,)*n array, D = len(c)."""
    cc = np.ascontiguousarray(c, dtype=np.float64)
    d = cc.size
    out = np.zeros(d ** n)
    lib().orc_chi_d(int(n), int(d), _dp(cc), _dp(out))
    return out.reshape((d,) * n) if n else out


def a_es(n: int, rho: float, u, lam) -> np.ndarray:
    """The printed a_ES^(n) as a (D,)*n array, D = len(u)."""
    uu = np.ascontiguousarray(u, dtype=np.float64)
    d = uu.size
    out = np.zeros(d ** n)
    ll = np.ascontiguousarray(lam, dtype=np.float64).reshape(d * d)
    lib().orc_a_es_d(int(n), int(d), C.c_double(rho), _dp(uu), _dp(ll), _dp(out))
    return out.reshape((d,) * n) if n else out


def cell_moments(nroots: int, dim: int, f):
    """One cell's moments: (the nine fields of moments(), P (D, D), u (D,))."""
    ff = np.ascontiguousarray(f, dtype=np.float64)
    out, P, u = np.zeros(9), np.zeros(dim * dim), np.zeros(dim)
    if lib().orc_cell_moments(int(nroots), int(dim), _dp(ff), _dp(out), _dp(P), _dp(u)):
        raise ValueError("bad nroots or dim")
    return out, P.reshape(dim, dim), u


UNSPLIT, SPLIT = 0, 1


def make_params(*, nroots, order, nx, ny, bc_y, kn, b, visc_exp, dt, dx, dy,
                wall_T=(1.0, 1.0), wall_ux=(0.0, 0.0), g=(0.0, 0.0), scheme=UNSPLIT, wall_specular=0.0,
                wall_T_amp=0.0, wall_T_freq=0.0, time=0.0, dim=2, bc_x=0, wall_Tx=(1.0, 1.0)) -> OrcParams:
    p = OrcParams()
    p.nroots, p.order, p.nx, p.ny, p.bc_y, p.scheme = nroots, order, nx, ny, bc_y, scheme
    p.dim, p.bc_x = dim, bc_x
    p.wall_Tx[0], p.wall_Tx[1] = wall_Tx
    p.kn, p.b, p.visc_exp, p.dt, p.dx, p.dy = kn, b, visc_exp, dt, dx, dy
    p.wall_T[0], p.wall_T[1] = wall_T
    p.wall_ux[0], p.wall_ux[1] = wall_ux
    p.g[0], p.g[1] = g
    p.wall_specular, p.wall_T_amp, p.wall_T_freq, p.time = wall_specular, wall_T_amp, wall_T_freq, time
    return p


def _q(p: OrcParams) -> int:
    return nvel(p.nroots, p.dim or 2)


def cell_terms(p: OrcParams, f):
    q = _q(p)
    ff = np.ascontiguousarray(f, dtype=np.float64)
    fes, gf, tau = np.zeros(q), np.zeros(q), C.c_double()
    if lib().orc_cell_terms(C.byref(p), _dp(ff), _dp(fes), _dp(gf), C.byref(tau)):
        raise ValueError("bad params")
    return fes, gf, tau.value


def feq0(nroots: int, order: int, T: float, ux: float, uy: float, dim: int = 2) -> np.ndarray:
    out = np.zeros(nvel(nroots, dim))
    if lib().orc_feq0_d(int(nroots), int(dim), int(order), C.c_double(T), C.c_double(ux), C.c_double(uy),
                        _dp(out)):
        raise ValueError("bad nroots")
    return out


def advect_1d(c: float, nu: float, f) -> np.ndarray:
    ff = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros_like(ff)
    lib().orc_advect_1d(int(ff.size), C.c_double(c), C.c_double(nu), _dp(ff), _dp(out))
    return out


def init(p: OrcParams, fields=None) -> np.ndarray:
    q = _q(p)
    f = np.zeros((q, p.ny, p.nx))
    if fields is None:
        rc = lib().orc_init(C.byref(p), None, _dp(f))
    else:
        fl = np.ascontiguousarray(fields, dtype=np.float64)
        assert fl.shape == (4, p.ny, p.nx)
        rc = lib().orc_init(C.byref(p), _dp(fl), _dp(f))
    if rc:
        raise ValueError("bad params")
    return f


def step(p: OrcParams, f: np.ndarray) -> np.ndarray:
    fin = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(fin)
    if lib().orc_step(C.byref(p), _dp(fin), _dp(out)):
        raise ValueError("bad params")
    return out


def run(p: OrcParams, f: np.ndarray, nsteps: int) -> np.ndarray:
    ff = np.array(f, dtype=np.float64, order="C", copy=True)
    work = np.empty_like(ff)
    if lib().orc_run(C.byref(p), _dp(ff), _dp(work), C.c_int64(int(nsteps))):
        raise ValueError("bad params")
    return ff


def moments(p: OrcParams, f: np.ndarray):
    ff = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros((9, p.ny, p.nx))
    sums = np.zeros(4)
    if lib().orc_moments(C.byref(p), _dp(ff), _dp(out), _dp(sums)):
        raise ValueError("bad params")
    return out, sums


MOMENT_NAMES = ("rho", "ux", "uy", "T", "sxx", "sxy", "syy", "qx", "qy")
