"""ctypes binding of liblesbgk.so (include/lesbgk.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
PyTorch supplies device memory (the caller-owned workspace and output
buffers) and the CUDA stream handle.  If the library has not been built, the
first call raises; there is no fallback.

The module-level functions keep the C names without the ``lesbgk_`` prefix;
``Solver`` wraps one handle together with its torch-allocated workspace.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np

from .build import LIB

OK, EINVAL, EUNSTABLE, ESPACE, ECUDA, EDIVERGED = 0, -1, -2, -3, -4, -5
PERIODIC, DIFFUSE = 0, 1
F32, F16, BF16, F32C = 0, 1, 2, 3
UNSPLIT, SPLIT = 0, 1
MOMENT_NAMES = ("rho", "ux", "uy", "T", "sxx", "sxy", "syy", "qx", "qy")

# Every entry point declared in include/lesbgk.h.
SYMBOLS = ("lesbgk_workspace_size", "lesbgk_create", "lesbgk_reinit", "lesbgk_step", "lesbgk_moments",
           "lesbgk_moments_host", "lesbgk_get_populations", "lesbgk_set_populations",
           "lesbgk_set_launch", "lesbgk_get_info", "lesbgk_destroy", "lesbgk_moments_noalloc",
           "lesbgk_last_error", "lesbgk_residual", "lesbgk_rows_bytes", "lesbgk_get_rows", "lesbgk_set_rows",
           "lesbgk_moments_rows",
           "lesbgk_batch_workspace_size", "lesbgk_batch_slot_bytes", "lesbgk_batch_create", "lesbgk_batch_add",
           "lesbgk_batch_remove", "lesbgk_batch_step", "lesbgk_batch_residuals", "lesbgk_batch_moments",
           "lesbgk_batch_get_populations", "lesbgk_batch_get_info", "lesbgk_batch_set_rows",
           "lesbgk_batch_autotune", "lesbgk_batch_pool_free", "lesbgk_batch_destroy", "lesbgk_batch_add_many",
           "lesbgk_batch_moments_many", "lesbgk_batch_set_resident", "lesbgk_batch_get_launch",
           "lesbgk_batch_check_guards", "lesbgk_batch_debug_poison", "lesbgk_batch_raw_bytes",
           "lesbgk_batch_get_raw", "lesbgk_batch_set_raw")


class Params(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32), ("nroots", C.c_int32), ("order", C.c_int32),
        ("nx", C.c_int32), ("ny", C.c_int32), ("bc_y", C.c_int32), ("storage", C.c_int32),
        ("scheme", C.c_int32),
        ("kn", C.c_double), ("b", C.c_double), ("visc_exp", C.c_double),
        ("cfl", C.c_double), ("dt", C.c_double),
        ("wall_T", C.c_double * 2), ("wall_ux", C.c_double * 2), ("g", C.c_double * 2),
        ("wall_specular", C.c_double), ("wall_T_amp", C.c_double), ("wall_T_freq", C.c_double),
        ("dim", C.c_int32), ("bc_x", C.c_int32), ("wall_Tx", C.c_double * 2),
        ("dx", C.c_double), ("dy", C.c_double), ("row_offset", C.c_int32), ("row_period", C.c_int32),
    ]


class Info(C.Structure):
    _fields_ = [
        ("dt", C.c_double), ("dx", C.c_double), ("dy", C.c_double), ("c_max", C.c_double),
        ("cfl", C.c_double), ("tau_ref", C.c_double), ("steps_done", C.c_int64),
        ("q", C.c_int32), ("order", C.c_int32),
        ("cells_per_thread", C.c_int32), ("rows_per_segment", C.c_int32),
    ]


class LesbgkError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"liblesbgk error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib():
    """Load liblesbgk.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError(f"{LIB} is missing: build it with "
                                   "`python -m paper_1209_6548_gb300.build` (no CPU fallback exists)")
            L = C.CDLL(LIB)
            vp, i64 = C.c_void_p, C.c_int64
            L.lesbgk_workspace_size.argtypes = [C.POINTER(Params), C.POINTER(C.c_size_t)]
            L.lesbgk_create.argtypes = [C.POINTER(Params), vp, C.c_size_t, vp, vp, C.POINTER(vp)]
            L.lesbgk_reinit.argtypes = [vp, vp, vp]
            L.lesbgk_step.argtypes = [vp, i64, vp]
            L.lesbgk_moments.argtypes = [vp, vp, vp, vp]
            L.lesbgk_moments_host.argtypes = [vp, vp, vp, vp]
            L.lesbgk_get_populations.argtypes = [vp, vp, vp]
            L.lesbgk_set_populations.argtypes = [vp, vp, i64, vp]
            L.lesbgk_set_launch.argtypes = [vp, C.c_int32, C.c_int32]
            L.lesbgk_get_info.argtypes = [vp, C.POINTER(Info)]
            L.lesbgk_destroy.argtypes = [vp]
            L.lesbgk_moments_noalloc.argtypes = [C.POINTER(Params), vp, vp, vp, vp]
            L.lesbgk_rows_bytes.argtypes = [vp, C.c_int32, C.POINTER(C.c_size_t)]
            L.lesbgk_get_rows.argtypes = [vp, C.c_int32, C.c_int32, vp, vp]
            L.lesbgk_set_rows.argtypes = [vp, C.c_int32, C.c_int32, vp, vp]
            L.lesbgk_moments_rows.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp]
            sz, i32 = C.c_size_t, C.c_int32
            L.lesbgk_batch_workspace_size.argtypes = [i32, sz, C.POINTER(sz)]
            L.lesbgk_batch_slot_bytes.argtypes = [C.POINTER(Params), C.POINTER(sz)]
            L.lesbgk_batch_create.argtypes = [i32, i32, vp, sz, vp, C.POINTER(vp)]
            L.lesbgk_batch_add.argtypes = [vp, C.POINTER(Params), vp, vp, C.POINTER(i32)]
            L.lesbgk_batch_remove.argtypes = [vp, i32, vp]
            L.lesbgk_batch_add_many.argtypes = [vp, i32, C.POINTER(Params), vp, vp, vp]
            L.lesbgk_batch_moments_many.argtypes = [vp, i32, vp, vp, vp]
            L.lesbgk_batch_set_resident.argtypes = [vp, i32, i32, i32, vp]
            L.lesbgk_batch_get_launch.argtypes = [vp, vp, vp, vp, vp]
            L.lesbgk_batch_step.argtypes = [vp, i64, vp]
            L.lesbgk_batch_residuals.argtypes = [vp, vp, vp, vp]
            L.lesbgk_residual.argtypes = [vp, vp, i64, vp, vp, vp]
            L.lesbgk_batch_moments.argtypes = [vp, i32, vp, vp, vp]
            L.lesbgk_batch_get_populations.argtypes = [vp, i32, vp, vp]
            L.lesbgk_batch_get_info.argtypes = [vp, i32, C.POINTER(Info)]
            L.lesbgk_batch_set_rows.argtypes = [vp, i32, vp]
            L.lesbgk_batch_autotune.argtypes = [vp, vp, i32, C.POINTER(i32), vp]
            L.lesbgk_batch_pool_free.argtypes = [vp, C.POINTER(sz), C.POINTER(sz)]
            L.lesbgk_batch_check_guards.argtypes = [vp, vp, vp]
            L.lesbgk_batch_raw_bytes.argtypes = [vp, i32, C.POINTER(sz)]
            L.lesbgk_batch_get_raw.argtypes = [vp, i32, vp, vp]
            L.lesbgk_batch_set_raw.argtypes = [vp, i32, vp, i64, vp]
            L.lesbgk_batch_debug_poison.argtypes = [vp, i32, vp]
            L.lesbgk_batch_destroy.argtypes = [vp]
            L.lesbgk_last_error.restype = C.c_char_p
            L.lesbgk_last_error.argtypes = []
            _lib = L
    return _lib


def last_error() -> str:
    return lib().lesbgk_last_error().decode()


def _check(rc: int) -> None:
    if rc != OK:
        raise LesbgkError(rc, last_error())


def make_params(*, nroots=4, order=0, nx, ny, bc_y=DIFFUSE, kn, b, visc_exp=0.5, cfl=0.5, dt=0.0,
                wall_T=(1.0, 1.0), wall_ux=(0.0, 0.0), g=(0.0, 0.0), storage=F32, scheme=UNSPLIT,
                wall_specular=0.0, wall_T_amp=0.0, wall_T_freq=0.0, dim=2, bc_x=PERIODIC,
                wall_Tx=(1.0, 1.0), dx=0.0, dy=0.0, row_offset=0) -> Params:
    p = Params()
    p.struct_size = C.sizeof(Params)
    p.nroots, p.order, p.nx, p.ny, p.bc_y, p.storage = nroots, order, nx, ny, bc_y, storage
    p.scheme = scheme
    p.kn, p.b, p.visc_exp, p.cfl, p.dt = kn, b, visc_exp, cfl, dt
    p.wall_T[0], p.wall_T[1] = wall_T
    p.wall_ux[0], p.wall_ux[1] = wall_ux
    p.g[0], p.g[1] = g
    p.wall_specular, p.wall_T_amp, p.wall_T_freq = wall_specular, wall_T_amp, wall_T_freq
    p.dim = dim
    p.bc_x = bc_x
    p.wall_Tx[0], p.wall_Tx[1] = wall_Tx
    p.dx, p.dy, p.row_offset, p.row_period = dx, dy, row_offset, 0
    return p


def stored_q(p: Params) -> int:
    """Values stored per node: nroots^2 for the 2D sets, nroots^3 / 2 for the
    D = 3 set (its z-even half)."""
    return p.nroots * p.nroots * (p.nroots // 2 if p.dim == 3 else 1)


def params_from_problem(prob, dt: float = 0.0) -> Params:
    return make_params(nroots=prob.nroots, order=prob.order, nx=prob.nx, ny=prob.ny, bc_y=prob.bc_y,
                       kn=prob.kn, b=prob.b, visc_exp=prob.visc_exp, cfl=prob.cfl, dt=dt,
                       wall_T=tuple(prob.wall_T), wall_ux=tuple(prob.wall_ux), g=tuple(prob.g),
                       scheme=prob.scheme, wall_specular=prob.wall_specular, wall_T_amp=prob.wall_T_amp,
                       wall_T_freq=prob.wall_T_freq, dim=getattr(prob, "dim", 2),
                       bc_x=getattr(prob, "bc_x", PERIODIC), wall_Tx=tuple(getattr(prob, "wall_Tx", (1.0, 1.0))))


def workspace_size(p: Params) -> int:
    n = C.c_size_t()
    _check(lib().lesbgk_workspace_size(C.byref(p), C.byref(n)))
    return int(n.value)


def create(p: Params, d_workspace: int, nbytes: int, h_init, stream: int) -> int:
    h = C.c_void_p()
    ptr = None
    if h_init is not None:
        arr = np.ascontiguousarray(h_init, dtype=np.float64)
        if arr.shape != (4, p.ny, p.nx):
            raise ValueError(f"h_init must have shape (4, {p.ny}, {p.nx})")
        ptr = arr.ctypes.data
    _check(lib().lesbgk_create(C.byref(p), C.c_void_p(d_workspace), C.c_size_t(nbytes),
                               C.c_void_p(ptr), C.c_void_p(stream), C.byref(h)))
    return h.value


def reinit(h: int, d_fields, stream: int) -> None:
    _check(lib().lesbgk_reinit(C.c_void_p(h), C.c_void_p(d_fields), C.c_void_p(stream)))


def step(h: int, nsteps: int, stream: int) -> None:
    _check(lib().lesbgk_step(C.c_void_p(h), C.c_int64(nsteps), C.c_void_p(stream)))


def moments(h: int, d_out: int, h_sums, stream: int) -> None:
    sp = None if h_sums is None else h_sums.ctypes.data
    _check(lib().lesbgk_moments(C.c_void_p(h), C.c_void_p(d_out), C.c_void_p(sp), C.c_void_p(stream)))


def moments_host(h: int, h_out: np.ndarray, h_sums, stream: int) -> None:
    assert h_out.dtype == np.float32 and h_out.flags.c_contiguous
    sp = None if h_sums is None else h_sums.ctypes.data
    _check(lib().lesbgk_moments_host(C.c_void_p(h), C.c_void_p(h_out.ctypes.data), C.c_void_p(sp),
                                     C.c_void_p(stream)))


def get_populations(h: int, d_out: int, stream: int) -> None:
    _check(lib().lesbgk_get_populations(C.c_void_p(h), C.c_void_p(d_out), C.c_void_p(stream)))


def set_populations(h: int, d_in: int, steps_done: int, stream: int) -> None:
    _check(lib().lesbgk_set_populations(C.c_void_p(h), C.c_void_p(d_in), C.c_int64(steps_done),
                                        C.c_void_p(stream)))


def set_launch(h: int, cells_per_thread: int = 0, rows_per_segment: int = 0) -> None:
    _check(lib().lesbgk_set_launch(C.c_void_p(h), C.c_int32(cells_per_thread), C.c_int32(rows_per_segment)))


def get_info(h: int) -> Info:
    out = Info()
    _check(lib().lesbgk_get_info(C.c_void_p(h), C.byref(out)))
    return out


def moments_noalloc(p: Params, d_populations: int, d_out, h_sums, stream: int) -> None:
    """lesbgk_moments_noalloc: moments of caller-held populations ([a][j][i]
    deviations on the device) with no device allocation inside the library."""
    sp = None if h_sums is None else h_sums.ctypes.data
    _check(lib().lesbgk_moments_noalloc(C.byref(p), C.c_void_p(d_populations), C.c_void_p(d_out),
                                        C.c_void_p(sp), C.c_void_p(stream)))


def destroy(h: int) -> None:
    lib().lesbgk_destroy(C.c_void_p(h))


@dataclass
class Solver:
    """One solve on the current CUDA device: torch-allocated workspace + handle."""

    params: Params
    h_init: object = None
    stream: object = None

    def __post_init__(self):
        import torch
        self._torch = torch
        if self.stream is None:
            self.stream = torch.cuda.current_stream()
        self.nbytes = workspace_size(self.params)
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        self.handle = create(self.params, self.workspace.data_ptr(), self.nbytes, self.h_init,
                             self.stream.cuda_stream)

    @property
    def q(self) -> int:
        return stored_q(self.params)

    def reinit(self, d_fields=None) -> None:
        """Re-initialise from a (4, ny, nx) float64 CUDA tensor (or rest)."""
        ptr = None
        if d_fields is not None:
            assert d_fields.is_cuda and d_fields.dtype == self._torch.float64 and d_fields.is_contiguous()
            assert tuple(d_fields.shape) == (4, self.params.ny, self.params.nx)
            ptr = d_fields.data_ptr()
        reinit(self.handle, ptr, self.stream.cuda_stream)

    def step(self, n: int) -> None:
        step(self.handle, n, self.stream.cuda_stream)

    def moments(self, sums: bool = False):
        """(9, ny, nx) float32 device tensor; with sums=True also the FP64 totals."""
        out = self._torch.empty((9, self.params.ny, self.params.nx), dtype=self._torch.float32, device="cuda")
        hs = np.zeros(4) if sums else None
        moments(self.handle, out.data_ptr(), hs, self.stream.cuda_stream)
        return (out, hs) if sums else out

    def moments_host(self):
        out = np.empty((9, self.params.ny, self.params.nx), dtype=np.float32)
        hs = np.zeros(4)
        moments_host(self.handle, out, hs, self.stream.cuda_stream)
        return out, hs

    def residual(self, snap, steps: int, mass: bool = False):
        """lesbgk_residual: r over the last `steps` steps against `snap`, a
        (4, ny, nx) float32 CUDA tensor that is overwritten with the current
        fields (steps <= 0 only takes the snapshot and returns NaN); with
        mass=True returns (r, total mass)."""
        assert snap.is_cuda and snap.dtype == self._torch.float32 and snap.is_contiguous()
        assert tuple(snap.shape) == (4, self.params.ny, self.params.nx)
        r, m = C.c_double(), C.c_double()
        _check(lib().lesbgk_residual(C.c_void_p(self.handle), C.c_void_p(snap.data_ptr()), C.c_int64(int(steps)),
                                     C.byref(r), C.byref(m) if mass else None, C.c_void_p(self.stream.cuda_stream)))
        return (r.value, m.value) if mass else r.value

    def populations(self):
        out = self._torch.empty((self.q, self.params.ny, self.params.nx), dtype=self._torch.float32, device="cuda")
        get_populations(self.handle, out.data_ptr(), self.stream.cuda_stream)
        return out

    def set_populations(self, t, steps_done: int) -> None:
        t = t.contiguous()
        set_populations(self.handle, t.data_ptr(), steps_done, self.stream.cuda_stream)

    def set_launch(self, cells_per_thread: int = 0, rows_per_segment: int = 0) -> None:
        set_launch(self.handle, cells_per_thread, rows_per_segment)

    @property
    def info(self) -> Info:
        return get_info(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- batched solver
def batch_workspace_size(capacity: int, pool_bytes: int) -> int:
    n = C.c_size_t()
    _check(lib().lesbgk_batch_workspace_size(C.c_int32(capacity), C.c_size_t(pool_bytes), C.byref(n)))
    return int(n.value)


def batch_slot_bytes(p: Params) -> int:
    n = C.c_size_t()
    _check(lib().lesbgk_batch_slot_bytes(C.byref(p), C.byref(n)))
    return int(n.value)


class Batch:
    """A batch of independent narrow solves (C ABI lesbgk_batch_*) in one
    torch-allocated workspace: `capacity` slots and a pool of `pool_bytes`."""

    def __init__(self, capacity: int, nx: int, pool_bytes: int, stream=None):
        import torch
        self._torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.capacity, self.nx = capacity, nx
        self.nbytes = batch_workspace_size(capacity, pool_bytes)
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        h = C.c_void_p()
        _check(lib().lesbgk_batch_create(C.c_int32(capacity), C.c_int32(nx), C.c_void_p(self.workspace.data_ptr()),
                                         C.c_size_t(self.nbytes), C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.handle = h.value
        self.params = {}

    @property
    def _s(self):
        return C.c_void_p(self.stream.cuda_stream)

    def add(self, p: Params, h_init=None) -> int:
        ptr = None
        if h_init is not None:
            arr = np.ascontiguousarray(h_init, dtype=np.float64)
            assert arr.shape == (4, p.ny, p.nx)
            ptr = arr.ctypes.data
        slot = C.c_int32()
        _check(lib().lesbgk_batch_add(C.c_void_p(self.handle), C.byref(p), C.c_void_p(ptr), self._s, C.byref(slot)))
        self.params[slot.value] = p
        return slot.value

    def add_many(self, params, h_inits=None):
        """lesbgk_batch_add_many: admit every problem of `params` at once
        (all or nothing); h_inits: None or a list of (4, ny, nx) arrays / None."""
        n = len(params)
        arr = (Params * n)(*params)
        keep, ptrs = [], None
        if h_inits is not None:
            ptrs = (C.c_void_p * n)()
            for i, h in enumerate(h_inits):
                if h is not None:
                    a = np.ascontiguousarray(h, dtype=np.float64)
                    keep.append(a)
                    ptrs[i] = a.ctypes.data
        slots = (C.c_int32 * n)()
        _check(lib().lesbgk_batch_add_many(C.c_void_p(self.handle), C.c_int32(n), arr,
                                           None if ptrs is None else C.cast(ptrs, C.c_void_p), self._s,
                                           C.cast(slots, C.c_void_p)))
        out = list(slots)
        for sl, p in zip(out, params):
            self.params[sl] = p
        return out

    def moments_many(self, slots, outs) -> None:
        """lesbgk_batch_moments_many: slot slots[i]'s moment fields into the
        (9, ny, nx) float32 CUDA tensor outs[i], one launch for all."""
        n = len(slots)
        sl = (C.c_int32 * n)(*slots)
        ptrs = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
        _check(lib().lesbgk_batch_moments_many(C.c_void_p(self.handle), C.c_int32(n), C.cast(sl, C.c_void_p),
                                               C.cast(ptrs, C.c_void_p), self._s))

    def try_add(self, p: Params, h_init=None):
        """add(), or None when the pool or the slots are full."""
        try:
            return self.add(p, h_init)
        except LesbgkError as e:
            if e.code == ESPACE:
                return None
            raise

    def remove(self, slot: int) -> None:
        _check(lib().lesbgk_batch_remove(C.c_void_p(self.handle), C.c_int32(slot), self._s))
        self.params.pop(slot, None)

    def step(self, n: int) -> None:
        _check(lib().lesbgk_batch_step(C.c_void_p(self.handle), C.c_int64(n), self._s))

    def residuals(self, mass: bool = False):
        """Per-slot residuals (NaN: empty slot or first call; Inf: diverged);
        with mass=True also the per-slot total mass."""
        out = np.empty(self.capacity)
        m = np.empty(self.capacity) if mass else None
        _check(lib().lesbgk_batch_residuals(C.c_void_p(self.handle), C.c_void_p(out.ctypes.data),
                                            C.c_void_p(None if m is None else m.ctypes.data), self._s))
        return (out, m) if mass else out

    def moments(self, slot: int, sums: bool = False):
        p = self.params[slot]
        out = self._torch.empty((9, p.ny, p.nx), dtype=self._torch.float32, device="cuda")
        hs = np.zeros(4) if sums else None
        _check(lib().lesbgk_batch_moments(C.c_void_p(self.handle), C.c_int32(slot), C.c_void_p(out.data_ptr()),
                                          C.c_void_p(None if hs is None else hs.ctypes.data), self._s))
        return (out, hs) if sums else out

    def populations(self, slot: int):
        p = self.params[slot]
        out = self._torch.empty((stored_q(p), p.ny, p.nx), dtype=self._torch.float32, device="cuda")
        _check(lib().lesbgk_batch_get_populations(C.c_void_p(self.handle), C.c_int32(slot),
                                                  C.c_void_p(out.data_ptr()), self._s))
        return out

    def info(self, slot: int) -> Info:
        out = Info()
        _check(lib().lesbgk_batch_get_info(C.c_void_p(self.handle), C.c_int32(slot), C.byref(out)))
        return out

    def set_rows(self, rows: int) -> None:
        _check(lib().lesbgk_batch_set_rows(C.c_void_p(self.handle), C.c_int32(rows), self._s))

    def autotune(self, candidates=(8, 16, 32, 64, 128)) -> int:
        arr = (C.c_int32 * len(candidates))(*candidates)
        chosen = C.c_int32()
        _check(lib().lesbgk_batch_autotune(C.c_void_p(self.handle), arr, C.c_int32(len(candidates)),
                                           C.byref(chosen), self._s))
        return chosen.value

    def set_resident(self, on: bool, steps_per_launch: int = 0, max_ny: int = 0) -> None:
        _check(lib().lesbgk_batch_set_resident(C.c_void_p(self.handle), C.c_int32(1 if on else 0),
                                               C.c_int32(steps_per_launch), C.c_int32(max_ny), self._s))

    def launch(self) -> dict:
        """rows per item, resident on/off, steps per resident launch, tallest instance the
        resident kernel takes."""
        v = [C.c_int32() for _ in range(4)]
        _check(lib().lesbgk_batch_get_launch(C.c_void_p(self.handle), *[C.byref(x) for x in v]))
        return {"rows_per_item": v[0].value, "resident": bool(v[1].value), "steps_per_launch": v[2].value,
                "resident_max_ny": v[3].value}

    def check_guards(self):
        """Per slot: 1 where the guard words after the slot's memory changed
        (lesbgk_batch_check_guards), numpy int32[capacity]."""
        import numpy as np
        bad = np.zeros(self.capacity, dtype=np.int32)
        _check(lib().lesbgk_batch_check_guards(C.c_void_p(self.handle), C.c_void_p(bad.ctypes.data), self._s))
        return bad

    def checkpoint(self, slot: int):
        """(raw populations as a device uint8 tensor, steps done) of a slot."""
        n = C.c_size_t()
        _check(lib().lesbgk_batch_raw_bytes(C.c_void_p(self.handle), C.c_int32(slot), C.byref(n)))
        buf = self._torch.empty(n.value, dtype=self._torch.uint8, device="cuda")
        _check(lib().lesbgk_batch_get_raw(C.c_void_p(self.handle), C.c_int32(slot), C.c_void_p(buf.data_ptr()),
                                          self._s))
        return buf, self.info(slot).steps_done

    def resume(self, slot: int, raw, steps_done: int) -> None:
        _check(lib().lesbgk_batch_set_raw(C.c_void_p(self.handle), C.c_int32(slot), C.c_void_p(raw.data_ptr()),
                                          C.c_int64(steps_done), self._s))

    def debug_poison(self, slot: int) -> None:
        _check(lib().lesbgk_batch_debug_poison(C.c_void_p(self.handle), C.c_int32(slot), self._s))

    def pool_free(self):
        a, t = C.c_size_t(), C.c_size_t()
        _check(lib().lesbgk_batch_pool_free(C.c_void_p(self.handle), C.byref(a), C.byref(t)))
        return a.value, t.value

    def close(self) -> None:
        if getattr(self, "handle", None):
            lib().lesbgk_batch_destroy(C.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
