"""Host-side helpers of bench.py, without a GPU: the clock record summarised
into the JSON line, the DRAM-traffic guard that drops a capture once the
kernel's source changes, and the algorithmic byte counts of the roofline."""
import hashlib
import json
import os

import pytest

import bench


def test_clock_summary():
    lines = [
        "0, 1965, 2070, 1010.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",     # skipped
        "garbage",
        "0, 2010, 2070, 1200.2, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
    ]
    s = bench.clock_summary(lines)
    assert s == {"sm_mhz": 1980.0, "sm_max_mhz": 2070.0, "reasons": ["hw_slowdown", "sw_power_cap"],
                 "samples": 3}
    assert bench.clock_summary(["garbage"]) is None
    assert bench.clock_summary([]) is None


def test_traffic_guard_follows_the_kernel_source(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    body = "__global__ void k_a() {}\n// --- k_b begins\n__global__ void k_b() { int x = 1; }\n// --- k_b ends\n"
    src.write_text(body)
    region = body[body.index("// --- k_b begins"):body.index("// --- k_b ends")]
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps({"k_b": {
        "source": "k.cu", "source_region": ["// --- k_b begins", "// --- k_b ends"],
        "source_sha256": hashlib.sha256(region.encode()).hexdigest(), "dram_bytes_per_launch": 12345}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.dram_traffic("k_b") == 12345
    assert bench.dram_traffic("k_c") is None                              # never captured
    src.write_text(body.replace("void k_a() {}", "void k_a() { return; }"))
    assert bench.dram_traffic("k_b") == 12345                             # an edit outside the region
    src.write_text(body.replace("int x = 1;", "int x = 2;"))
    assert bench.dram_traffic("k_b") is None                              # the kernel changed
    src.write_text(body.replace("// --- k_b ends", ""))
    assert bench.dram_traffic("k_b") is None                              # region markers gone


def test_committed_traffic_record_is_well_formed():
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for name, r in rec.items():
        assert os.path.exists(os.path.join(bench.ROOT, r["source"])), name
        assert r["dram_bytes_per_launch"] > 0 and len(r["source_sha256"]) == 64
        assert "--clock-control none" in r.get("command", "--clock-control none")


def test_algorithmic_bytes_of_the_subdivision_write():
    # 10 output rows of which 8 are the children of one split parent: 2 survivors read and written,
    # 8 children written, the parent's row read once
    assert bench.algorithmic_bytes("subdivide_apply", n=5, pairs=0, slots=0, npix=0, n_new=10, split=1, row=694,
                                   parent_row=241) == 2 * 2 * 694 + 8 * 694 + 241
    assert bench.algorithmic_bytes("unknown", 1, 1, 1, 1) == 0


def test_alu_peak():
    # 152 SMs x 128 FP32 lanes x 2 (FMA) at 2070 MHz
    assert bench.alu_peak_tflops(2070.0) == pytest.approx(80.54, abs=0.01)
