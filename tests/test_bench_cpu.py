"""The measurement arithmetic of bench.py (no GPU): algorithmic bytes and operation counts against
the data layouts they describe, the derived ALU peaks, the per-kernel traffic records and the
parsing of the clock samples."""
import os

import pytest

import bench


def test_algorithmic_bytes_per_site():
    # FP64 operator and spinors: 4 links of 18 reals + 72 clover reals, 2 (apply) or 3 (Jacobi
    # sweep) spinors of 24 reals per RHS, 8 bytes each
    assert bench.algorithmic_bytes("dslash_apply", 1) == (4 * 18 + 72) * 8 + 2 * 24 * 8
    assert bench.algorithmic_bytes("dslash_apply", 12) == 1152 + 384 * 12
    assert bench.algorithmic_bytes("dslash_jacobi", 12) == 1152 + 576 * 12
    # the double-float sweep: FP32 12-real links and inverse blocks, spinors as FP32 pairs
    assert bench.algorithmic_bytes("dslash_jacobi", 12, 8, 12, 4) == 480 + 576 * 12
    # FP32 and BF16 sweeps
    assert bench.algorithmic_bytes("dslash_jacobi", 12, 4, 12, 4) == 480 + 288 * 12
    assert bench.algorithmic_bytes("dslash_jacobi", 12, 2, 12, 4) == 480 + 144 * 12
    with pytest.raises(ValueError):
        bench.algorithmic_bytes("gram", 12)


def test_operation_counts():
    # the grid-sum double-float sweep and the FP32-lane FP64 stencil, as their derivations state
    assert bench.DF_OPS_GRID == 7598
    assert bench.X3_FP64_OPS == 96 + 48 + 24 + 264
    assert bench.X3_FP32_OPS == 288 * 48 + 48 * 38 + 96 * 15 + 360
    assert bench.FLOP_APPLY == 1320 + 504


def test_network_flop_count():
    # one 1 -> 1 layer: one input channel transported along 8 hops (4 spins x 9 complex
    # multiply-adds x 8 flop) and one channel pair mixed in 9 directions (4 x 4 spin entries x 3
    # colours x 8 flop)
    assert bench.net_flop(1, 1) == 8 * 4 * 9 * 8 + 9 * 16 * 3 * 8
    # 1 -> 4 -> 4 -> 4 -> 1: 13 transported input channels, 40 channel pairs
    assert bench.net_flop(4, 4) == 13 * 8 * 288 + 40 * 9 * 384


def test_derived_alu_peaks():
    p = bench.alu_peaks(152, 2070.0)
    assert p["fp32_lane_tops"] == pytest.approx(152 * 128 * 2.07e9 / 1e12)
    assert p["fp64_tflops"] == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)   # 2 DFMA/clk/SM
    assert p["fp32_lane_tops"] / p["fp64_tflops"] == pytest.approx(32.0)


def test_solve_flop_counts_the_papers_mvm():
    cfg = bench.SMALL_CONFIGS["c2"]
    # #MVM per column x L x V x 1824 flop
    assert bench.solve_flop(cfg, 391) == 391 * 12 * 8 * 8 * 8 * 16 * 1824


def test_traffic_records_follow_the_kernel_sources(tmp_path, monkeypatch):
    """A bench-traffic line counts only while the kernel's own sources hash to its tag."""
    sha = bench.csrc_sha(bench.KERNEL_SOURCES[("dslash_jacobi_lp", "df")])
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "a.md").write_text(f"text\nbench-traffic: dslash_jacobi_lp df 123456 {sha}\n"
                               "bench-traffic: dslash_apply fp64 777 0000000000000000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = tmp_path / "paper_0907_3261_gb300" / "csrc"
    csrc.mkdir(parents=True)
    real = os.path.join(os.path.dirname(bench.__file__), "paper_0907_3261_gb300", "csrc")
    for name in os.listdir(real):
        if name.endswith((".cu", ".cuh", ".h")):
            (csrc / name).write_bytes(open(os.path.join(real, name), "rb").read())
    assert bench.ncu_traffic("dslash_jacobi_lp", "df") == 123456
    assert bench.ncu_traffic("dslash_apply", "fp64") is None          # stale tag
    assert bench.ncu_traffic("dslash_jacobi_lp", "fp32") is None      # no record
    # editing a file of another kernel keeps the record; editing one of its own drops it
    (csrc / "blas.cu").write_text("// edited\n")
    assert bench.ncu_traffic("dslash_jacobi_lp", "df") == 123456
    (csrc / "sweep_df.cu").write_text("// edited\n")
    assert bench.ncu_traffic("dslash_jacobi_lp", "df") is None


def test_committed_traffic_records_name_known_kernel_classes():
    pdir = os.path.join(os.path.dirname(bench.__file__), "profiles")
    for name in os.listdir(pdir):
        for line in open(os.path.join(pdir, name)):
            if line.startswith("bench-traffic:"):
                cls, prec = line.split()[1:3]
                assert (cls, prec) in bench.KERNEL_SOURCES, line


def test_clock_samples_are_parsed(monkeypatch):
    """The nvidia-smi CSV rows of the timed region: median SM clock, maximum, throttle reasons."""
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    import tempfile
    s.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    s.p = None
    s.f.write("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
              "0, 1995, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active\n"
              "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    out = s.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3}
