"""Host-side logic of bench.py, on CPU: the algorithmic bytes per node that the roofline divides by,
the rule that ncu figures count only when taken on the current kernel sources, and the parsing
of the nvidia-smi clock samples taken during the timed region."""
import os
import tempfile

import pytest

import bench


def test_collide_bytes_per_node():
    """Every population read and written once, plus the (rho, phi) field (two-pass) or the two
    fixed-point accumulators (fused pass), plus the colour record (compact storage)."""
    assert bench.collide_bytes("f16", 5) == 2 * 27 * 4 + 8 == 224
    assert bench.collide_bytes("bf16", 1) == 224
    assert bench.collide_bytes("f32", 3) == 2 * 54 * 4 + 16 == 448
    assert bench.collide_bytes("f32", 1) == 2 * 54 * 4 + 8 == 440
    assert bench.collide_bytes("f64", 1) == 2 * 54 * 8 + 16 == 880
    assert bench.collide_bytes("c16", 1) == 2 * (26 * 2 + 4) + 8 + 16 == 136


def test_profile_names():
    assert bench.profile_name("f16", 5) == "collide_stream_tma_pipelined_jet_f16.md"
    assert bench.profile_name("f32", 3) == "collide_stream_fused_jet_f32.md"
    assert bench.profile_name("c16", 1) == "collide_stream_jet_c16.md"


def test_profiled_figures_count_only_on_the_current_kernel_sources(monkeypatch, tmp_path):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / bench.profile_name("f16", 5)).write_text(
        "# summary\nkernel_sources_sha: 0123456789abcdef\ndram_bytes_per_launch: 1.5e+09\n"
        "fp32_flop_per_node: 1070.5\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0123456789abcdef")
    assert bench.profiled_traffic("f16", 5) == 1.5e9
    assert bench.profiled("f16", "fp32_flop_per_node", 5) == 1070.5
    assert bench.profiled_traffic("f32", 3) is None  # no summary for it
    monkeypatch.setattr(bench, "kernel_hash", lambda: "fedcba9876543210")  # sources changed since
    assert bench.profiled_traffic("f16", 5) is None


def test_kernel_hash_covers_every_kernel_source():
    csrc = os.path.join(bench.ROOT, "paper_1705_03141_gb300", "csrc")
    device = sorted(f for f in os.listdir(csrc) if f.endswith((".cu", ".cuh")))
    host_only = {"lbm_capi.cu", "lbm_mlp.cu", "lbm_peak.cu", "lbm_static_diag.cu"}
    assert sorted(set(device) - host_only) == sorted(bench.KERNEL_SOURCES)
    assert len(bench.kernel_hash()) == 16


def _summary(rows):
    s = bench.ClockSampler(0)
    s.proc = object()  # stands for a running nvidia-smi
    s.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    s.f.write("\n".join(rows) + "\n")
    return s.summary()


def test_clock_samples_median_max_and_reasons():
    rows = ["0, 2070, 2070, 950.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1010.7, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 990.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"]
    out = _summary(rows)
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    out = _summary([rows[0], "0, 1500, 2070, 700.0, 0x0000000000000008, Active, Not Active, Active, Not Active"])
    assert out["sm_mhz"] == pytest.approx(1785.0)
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_samples_missing():
    assert _summary(["garbage"])["reasons"] == ["no samples"]
    s = bench.ClockSampler(0)
    assert s.summary()["reasons"] == ["nvidia-smi unavailable"]
