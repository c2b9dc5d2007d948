"""Host-side checks of bench.py's roofline bookkeeping (no GPU).

The DRAM traffic in the bench line comes from the committed ncu summaries
under profiles/, keyed by a digest of the step kernels' source: these tests
fail when a kernel's source changed after its counters were taken (the
summaries must then be re-captured), and when a committed figure is far from
the algorithmic bytes it should be close to.
"""
from __future__ import annotations

import pytest

import bench

N = 4096
STORED = {"d2q16": 16, "d2q36": 36, "d3q64": 32, "d3q216": 108}  # values stored per node
CASES = [("d2q16", "f32"), ("d2q16", "f16"), ("d2q16", "bf16"), ("d2q16", "f32c"), ("d2q36", "f32"),
         ("d3q64", "f32"), ("d3q216", "f32")]


@pytest.mark.parametrize("velocity_set,storage", CASES)
def test_profiles_were_taken_on_the_current_kernel_source(velocity_set, storage):
    assert bench.committed_traffic(bench.source_digest(), velocity_set, storage) is not None


@pytest.mark.parametrize("velocity_set,storage", CASES)
def test_committed_traffic_is_near_the_algorithmic_bytes(velocity_set, storage):
    """Each population is read and written once per launch: 2 Q s bytes per
    lattice update; halo re-reads and data still in L2 at the end of a launch
    keep the measured traffic within a few per cent to ~15% of it."""
    traffic = bench.committed_traffic(bench.source_digest(), velocity_set, storage)
    algorithmic = 2 * STORED[velocity_set] * bench.STORE_BYTES[storage] * N * N
    assert 0.8 < traffic / algorithmic < 1.1


def test_a_different_digest_gets_no_traffic():
    assert bench.committed_traffic("0" * 16, "d2q16", "f32") is None


def test_digest_ignores_code_outside_the_step_kernels(tmp_path, monkeypatch):
    """The digest hashes device.cuh, the step-kernel section of lesbgk.cu and
    its launch functions: an edit elsewhere in lesbgk.cu leaves it unchanged,
    an edit inside the section changes it."""
    import os
    import shutil

    csrc = tmp_path / "paper_1209_6548_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = os.path.join(bench.ROOT, "paper_1209_6548_gb300", "csrc")
    for name in ("device.cuh", "lesbgk.cu"):
        shutil.copy(os.path.join(src, name), csrc / name)
    real = bench.source_digest()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.source_digest()
    assert d0 == real  # only these two files enter the digest
    text = (csrc / "lesbgk.cu").read_text()
    (csrc / "lesbgk.cu").write_text(text.replace("// Host side", "// Host side (edited)", 1))
    assert bench.source_digest() == d0
    a = text.index("// The fused time step")
    (csrc / "lesbgk.cu").write_text(text[:a] + text[a:].replace("const int lane", "const int lane ", 1))
    assert bench.source_digest() != d0


INSTR_CASES = [("d2q16", "f32"), ("d2q16", "f16"), ("d2q16", "bf16"), ("d2q16", "f32c"), ("d2q36", "f32"),
               ("d2q36", "f16"),
               ("d3q64", "f32"), ("d3q64", "f16"), ("d3q64", "bf16"), ("d3q216", "f32")]


@pytest.mark.parametrize("velocity_set,storage", INSTR_CASES)
def test_instruction_counts_were_taken_on_the_current_kernel_source(velocity_set, storage):
    n = bench.committed_instructions(bench.source_digest(), velocity_set, storage)
    assert n is not None and 500 < n < 6000


def test_issue_view_arithmetic():
    """674.2 instructions per update over 4096^2 updates in 356.3 us is
    674.2/32 * 4096^2 / 356.3e-6 warp-instructions/s; the issue peak of 152
    SMs at 2070 MHz is 152 * 4 * 2.07e9."""
    v = bench.issue_view(674.2, 4096 * 4096, 0.3563, 152, 2070.0)
    assert abs(v["achieved"] - 674.2 / 32 * 4096 ** 2 / 356.3e-6) < 1e-3 * v["achieved"]
    assert v["peak"] == 152 * 4 * 2070e6
    assert abs(v["frac"] - v["achieved"] / v["peak"]) < 1e-15
    assert bench.issue_view(None, 1, 1.0, 152, 2070.0) is None


def test_precision_record_backs_the_compensated_claim():
    """The bench line's precision object quotes the committed 4096^2 record:
    it holds every storage, compensated FP32 within the 1e-5 bar and plain
    FP32 above it (the reason the compensated storage exists), and the 16-bit
    storages far above both."""
    rec = bench.precision_record()
    assert rec is not None and set(rec) == {"f32", "f16", "bf16", "f32c"}
    assert rec["f32c"] < 1e-5 < rec["f32"]
    assert rec["f32"] < rec["f16"] and rec["f32"] < rec["bf16"]
