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
