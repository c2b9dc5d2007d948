"""The heated walls' sine (wall_sin in csrc/setup.h, Cody-Waite reduction and
Taylor series, fused multiply-adds only) against the C library's sin, and the
heated wall tables' polynomial form (Sec. 4.2) against a direct evaluation.

wall_sin is compiled here by the host compiler from the same header the
device code includes; its results must stay within a few ulp of sin(x)."""
from __future__ import annotations

import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1209_6548_gb300", "csrc")
PROGRAM = r'''
#include <cstdio>
#include "setup.h"
int main() {
  double x;
  while (std::scanf("%la", &x) == 1) std::printf("%a\n", lesbgk_setup::wall_sin(x));
  return 0;
}
'''


def cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def wall_sin(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = cuda_include()
    if not cxx or not inc:
        pytest.skip("no host C++ compiler or CUDA headers")
    d = tmp_path_factory.mktemp("wall_sin")
    src, exe = d / "ws.cpp", d / "ws"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-O2", "-std=c++17", f"-I{CSRC}", f"-I{os.path.join(ROOT, 'include')}", f"-I{inc}",
                    str(src), "-o", str(exe)], check=True, capture_output=True)

    def run(x):
        out = subprocess.run([str(exe)], input="\n".join(float(v).hex() for v in x), capture_output=True,
                             text=True, check=True).stdout.split()
        return np.array([float.fromhex(v) for v in out])
    return run


def test_wall_sin_matches_libm(wall_sin):
    rng = np.random.default_rng(0)
    x = np.concatenate([
        np.linspace(-8.0, 8.0, 4001),                      # every quadrant, both signs
        rng.uniform(-2e4, 2e4, 4000),                      # the times of long heated runs
        np.arange(-64, 65) * (np.pi / 2),                  # near the reduction boundaries
        np.arange(1, 2000) * np.pi,                        # near the zeros of sin
        [0.0, 1e-300, -1e-20, 1e-8, np.pi / 4, -np.pi / 4],
    ])
    got = wall_sin(x)
    ref = np.sin(x)
    # a few roundings in the reduction and the series, plus libm's own ulp
    assert np.all(np.abs(got - ref) <= 8 * 2.0 ** -53 * np.abs(ref) + 1e-300), \
        np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300))
    assert wall_sin(np.array([0.0]))[0] == 0.0


def test_wall_sin_is_odd_and_periodic(wall_sin):
    x = np.linspace(0.01, 50.0, 2001)
    s = wall_sin(x)
    assert np.array_equal(wall_sin(-x), -s)  # the reduction and the series are odd exactly
    assert np.max(np.abs(wall_sin(x + 2 * np.pi) - s)) < 1e-14


TABLES = r'''
#include <cmath>
#include <cstdio>
#include <cstring>
#include "setup.h"
using namespace lesbgk_setup;
// heated tables (polynomial in the heating) at time t against the steady
// tables of walls set to T_w + h(t) directly; prints the largest difference
// in units of the FP32 spacing of the value
int main() {
  double worst = 0.0;
  for (int nr : {4, 6})
    for (int dim : {2, 3}) {
      lesbgk_params p; std::memset(&p, 0, sizeof p);
      p.struct_size = sizeof p; p.nroots = nr; p.order = nr == 4 ? 3 : 4; p.nx = 4; p.ny = 32;
      p.bc_y = LESBGK_DIFFUSE; p.kn = 0.1; p.b = 0.0; p.visc_exp = 0.5; p.cfl = 0.5; p.dim = dim;
      p.wall_T[0] = 0.97; p.wall_T[1] = 1.04; p.wall_ux[0] = -0.05; p.wall_ux[1] = 0.03;
      p.wall_Tx[0] = p.wall_Tx[1] = 1.0; p.storage = LESBGK_F32; p.scheme = LESBGK_UNSPLIT;
      p.wall_T_amp = 0.02; p.wall_T_freq = 0.5553603672697958;
      static Setup heated, steady;
      if (build_setup(p, p.order, nullptr, &heated)) return 2;
      const int q = nr * nr * (dim == 3 ? nr / 2 : 1);
      for (int n = 0; n < 400; n += 37) {
        const double t = (n + 1) * heated.dt;
        KArgs A = heated.args;
        set_wall_time(heated, t, &A);
        const double h = heated.wall_T_amp * wall_sin(heated.wall_T_freq * t);
        lesbgk_params ps = p;
        ps.wall_T_amp = 0.0; ps.wall_T[0] = p.wall_T[0] + h; ps.wall_T[1] = p.wall_T[1] + h;
        ps.dt = heated.dt;
        if (build_setup(ps, p.order, nullptr, &steady)) return 3;
        for (int s = 0; s < 2; ++s) {
          for (int a = 0; a < q; ++a) {
            const float x = A.wS[s][a], y = steady.args.wS[s][a];
            const double ulp = std::fabs(std::nextafter(y, 2.0f * y + 1.0f) - y);
            worst = std::fmax(worst, std::fabs(x - y) / ulp);
          }
          const float x = A.wB[s], y = steady.args.wB[s];
          worst = std::fmax(worst, std::fabs(x - y) / std::fabs(std::nextafter(y, 2.0f * y) - y));
        }
      }
    }
  std::printf("%.3f\n", worst);
  return 0;
}
'''


def test_heated_wall_tables_are_the_steady_tables_at_the_heated_temperature(tmp_path):
    """The heated walls' tables (Sec. 4.2), evaluated as polynomials of degree
    2 in the heating, equal the tables built directly for walls at T_w + h(t)
    (the Hermite coefficients of a Gaussian are polynomials of degree <= N/2
    in its temperature), to within one FP32 spacing, on D2Q16, D2Q36, D3Q64
    and D3Q216 with moving walls at two temperatures."""
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = cuda_include()
    if not cxx or not inc:
        pytest.skip("no host C++ compiler or CUDA headers")
    src, exe = tmp_path / "tab.cpp", tmp_path / "tab"
    src.write_text(TABLES)
    lib = os.path.join(os.path.dirname(inc), "lib64")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", f"-I{CSRC}", f"-I{os.path.join(ROOT, 'include')}",
                    f"-I{inc}", str(src), os.path.join(CSRC, "setup.cpp"), os.path.join(CSRC, "tables.cpp"),
                    f"-L{lib}", f"-Wl,-rpath,{lib}", "-lcudart", "-o", str(exe)], check=True, capture_output=True)
    worst = float(subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout)
    assert worst <= 1.0, worst
