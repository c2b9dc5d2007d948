"""Host-side checks of the C ABI that need no GPU: the library builds and loads,
exports every symbol include/lesbgk.h declares, and rejects bad arguments
before touching the device."""
from __future__ import annotations

import ctypes as C
import re
import os

import pytest

from paper_1209_6548_gb300 import build as B
from paper_1209_6548_gb300 import lesbgk as L

HEADER = os.path.join(B.ROOT, "include", "lesbgk.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(lesbgk_[a-z_]+)\s*\(", text)))


def test_header_symbols_exported(lib):
    names = declared_symbols()
    assert set(names) == set(L.SYMBOLS)
    for n in names:
        assert getattr(lib, n) is not None


def test_struct_sizes_match_header(lib):
    # struct_size is checked by the library: a mismatch must be rejected
    p = L.make_params(nx=4, ny=8, kn=0.1, b=0.0)
    assert L.workspace_size(p) > 0
    p.struct_size = C.sizeof(L.Params) - 8
    with pytest.raises(L.LesbgkError) as e:
        L.workspace_size(p)
    assert e.value.code == L.EINVAL


@pytest.mark.parametrize("kw,code", [
    (dict(b=1.0), L.EINVAL),
    (dict(b=-0.6), L.EINVAL),
    (dict(kn=0.0), L.EINVAL),
    (dict(nroots=5), L.EINVAL),
    (dict(order=5), L.EINVAL),
    (dict(ny=1), L.EINVAL),          # walls need two rows
    (dict(nx=0), L.EINVAL),
    (dict(cfl=1.5), L.EINVAL),
    (dict(visc_exp=1.5), L.EINVAL),
    (dict(storage=7), L.EINVAL),
    (dict(wall_specular=1.5), L.EINVAL),
    (dict(wall_specular=-0.1), L.EINVAL),
    (dict(wall_specular=0.5, storage=L.F16), L.EINVAL),  # Maxwell walls: FP32 storage only
    (dict(wall_T_amp=1.0), L.EINVAL),                     # T_w would reach 0
    (dict(wall_T_amp=float("nan")), L.EINVAL),
    (dict(dim=4), L.EINVAL),
    (dict(dim=3, nroots=6, order=3), L.EINVAL),           # D = 3: D3Q64 N = 3, D3Q216 N = 4
    (dict(dim=3, nroots=6, bc_x=L.DIFFUSE, storage=L.F32C), L.EINVAL),  # walls in x: not compensated
    (dict(dim=3, order=4), L.EINVAL),
    (dict(dim=3, nroots=6, storage=L.F32C), L.EINVAL),    # compensated storage: D2Q16 and D3Q64
    (dict(bc_x=2), L.EINVAL),
    (dict(nx=65536, ny=32768, bc_y=L.PERIODIC), L.EINVAL),  # 2^31 nodes
    (dict(bc_x=L.DIFFUSE, nx=1), L.EINVAL),              # walls in x need two columns
    (dict(bc_x=L.DIFFUSE, storage=L.F32C), L.EINVAL),
    (dict(bc_x=L.DIFFUSE, wall_specular=0.2), L.EINVAL),
    (dict(bc_x=L.DIFFUSE, wall_Tx=(1.0, 0.0)), L.EINVAL),
])
def test_invalid_arguments_rejected(lib, kw, code):
    base = dict(nx=4, ny=8, kn=0.1, b=0.0, bc_y=L.DIFFUSE)
    base.update(kw)
    with pytest.raises(L.LesbgkError) as e:
        L.workspace_size(L.make_params(**base))
    assert e.value.code == code


def test_wall_models_accepted(lib):
    for kw in (dict(wall_specular=1.0), dict(wall_T_amp=0.02, wall_T_freq=0.5),
               dict(wall_T_amp=0.02, wall_T_freq=0.5, storage=L.BF16)):
        assert L.workspace_size(L.make_params(nx=4, ny=8, kn=0.1, b=0.0, bc_y=L.DIFFUSE, **kw)) > 0


def test_large_grids_accepted(lib):
    """Grids up to 2^31 - 1 nodes are admissible (a 16384^2 D2Q16 solve needs 34 GB)."""
    p = L.make_params(nx=16384, ny=16384, kn=0.05, b=-0.5, bc_y=L.PERIODIC)
    assert L.workspace_size(p) >= 2 * 16 * 16384 * 16384 * 4
    assert L.workspace_size(L.make_params(nx=65535, ny=32768, kn=0.05, b=0.0, bc_y=L.PERIODIC)) > 0


def test_d3_workspace_holds_the_z_even_half(lib):
    """D3Q64 and D3Q216 store 32 and 108 values per node (their z-even halves)."""
    for nroots, q in ((4, 32), (6, 108)):
        p = L.make_params(nroots=nroots, nx=64, ny=32, kn=0.1, b=0.0, bc_y=L.DIFFUSE, dim=3)
        assert L.stored_q(p) == q
        n = L.workspace_size(p)
        assert 2 * q * 64 * 32 * 4 <= n < 2 * (q + 1) * 64 * 32 * 4 + (1 << 16)


def test_workspace_size_formula(lib):
    p = L.make_params(nx=64, ny=32, kn=0.1, b=0.0)
    n = L.workspace_size(p)
    # two buffers of Q*cells floats + reduction scratch
    assert n >= 2 * 16 * 64 * 32 * 4
    p6 = L.make_params(nroots=6, nx=64, ny=32, kn=0.1, b=0.0)
    assert L.workspace_size(p6) >= 2 * 36 * 64 * 32 * 4


def test_create_rejects_small_workspace_before_device_use(lib):
    p = L.make_params(nx=4, ny=8, kn=0.1, b=0.0)
    h = C.c_void_p()
    rc = lib.lesbgk_create(C.byref(p), C.c_void_p(256), C.c_size_t(16), None, None, C.byref(h))
    assert rc == L.ESPACE and h.value is None
    assert "workspace" in L.last_error()
    rc = lib.lesbgk_create(C.byref(p), C.c_void_p(257), C.c_size_t(1 << 30), None, None, C.byref(h))
    assert rc == L.ESPACE and "aligned" in L.last_error()


def test_null_handles_rejected(lib):
    assert lib.lesbgk_step(None, 1, None) == L.EINVAL
    assert lib.lesbgk_moments(None, None, None, None) == L.EINVAL
    assert lib.lesbgk_destroy(None) == 0
