"""Host-side arithmetic of bench.py (no GPU): the workload's unit count, the
roofline fractions, the traffic record's source check and the clock summary."""
import json
import os
import shutil

import pytest

import bench


def test_workload_units():
    # 2048 DOS steps of K - 1 = 17 sweeps and ceil(4096 / 2) KPM passes per state
    n = 2 * 1024 * 1024
    assert bench.workload_units(n, 18) == n * (2048 * 17 + 2048)
    assert bench.workload_units(10, 3, n_steps=5, M=7) == 10 * (5 * 2 + 4)


def test_roofline_fractions(monkeypatch):
    peak = bench.measured_hbm()[0]
    r = bench.hbm_roof(1e9, 100.0, "basis")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(100.0) and r["frac"] == pytest.approx(100.0 / peak, abs=1e-4)
    monkeypatch.setattr(bench, "PEAK64", {"tflops": 1.25, "source": "test"})
    a = bench.alu_roof(1e10, 16)
    # 16 FP64 operations of 2 flops each per unit, against the measured peak
    assert a["achieved"] == pytest.approx(0.32) and a["peak"] == pytest.approx(1.25)
    assert a["frac"] == pytest.approx(0.32 / 1.25, abs=1e-4)


def test_survey_bytes_per_orbital_term():
    # FP64 CSR: 4 entries x (16 B value + 4 B column) + 4 B row pointer + 5 vectors x 16 B
    assert bench.SURVEY_B_PER_TERM == 164


def test_stored_matrix_and_blocked_stencil_byte_bases():
    """Per orbital-term bytes of the FP32 forms: plain SELL (3 x (int32 column +
    FP32 value) + FP32 diagonal + slice offset), packed per entry (16-bit offset
    + 8-bit index), packed per row (one 64-bit word + diagonal); the blocked
    stencil's step (first, middle and final blocks over 17 sweeps, without and
    with the 96 x 32 / 90 x 26 region's halo re-reads) and one middle block of 6
    sweeps with its halo (8.8 B)."""
    assert bench.B_SELL32 == pytest.approx(28.25)
    assert bench.B_SELL32_PACKED == pytest.approx(13.25)
    assert bench.B_SELL32_ROWS == 12
    assert bench.B_TBLOCK_STEP / 17 == pytest.approx(116 / 17)
    region = (96 * 32) / (90 * 26)
    assert bench.B_TBLOCK_STEP_HALO == pytest.approx(68 * region + 48)
    assert bench.B_TBLOCK_MIDDLE_HALO / 6 == pytest.approx(8.79, abs=0.01)


def test_traffic_record_follows_the_kernel_source(tmp_path, monkeypatch):
    """The recorded DRAM bytes are reported only while the sweep sources are the
    ones they were measured on."""
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    csrc = root / "paper_2509_26309_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.TRAFFIC_SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_2509_26309_gb300", "csrc", f), csrc / f)
    monkeypatch.setattr(bench, "ROOT", str(root))
    rec = {"kernel_sources_sha256_16": bench.sources_hash(), "sweep_traffic_bytes": 123456789}
    json.dump(rec, open(root / "profiles" / "traffic.json", "w"))
    assert bench.profile_traffic() == rec["sweep_traffic_bytes"]
    with open(csrc / "sweep_ops.cuh", "a") as f:
        f.write("\n// edited\n")
    assert bench.profile_traffic() is None


def test_clock_summary_reasons():
    c = bench.ClockSampler(0)
    c.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1300.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1310.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
    ]
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    c.lines.append("0, 1500, 2070, 1000.0, 0x8, Not Active, Active, Not Active, Not Active")
    assert "hw_thermal_slowdown" in c.summary()["reasons"]
