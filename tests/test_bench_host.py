"""Host-side helpers of bench.py, without a GPU: the clock record summarised
into the JSON line, the DRAM-traffic guard that drops a capture once the
kernel's source changes, the algorithmic byte counts of the roofline, and the
batches whose step is timed after the autotuner."""
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


def test_stage_work_and_step_roofline():
    w = bench.stage_work(n=10, slots=4, pairs=6, npix=3, tiles=2, samples=5, split=1, pruned=2, row=694,
                         parent_row=241)
    # per pair the slot index and the 64-byte record, per pixel the 24 output bytes, one w_max word per pair
    assert w["a5_forward_composite"] == {"bytes": 6 * 68 + 3 * 24 + 6 * 8, "flops": 5 * 68}
    assert w["a6_backward_composite"] == {"bytes": 6 * 68 + 3 * 40 + 6 * 88, "flops": 5 * 102}
    # in place: the split parent's row read once, its 8 children written, the mask and the hole list
    assert w["subdivide_inplace"]["bytes"] == 241 + 8 * 694 + 10 + 4 * 2
    r = bench.step_roofline({"x": {"bytes": 2e9, "flops": 0}, "y": {"bytes": 1e6, "flops": 1e12}}, ms_step=24.0,
                            hbm_gbs=1000.0, fp32_tflops=100.0)
    # x: 2 ms of HBM; y: 10 ms of FP32 against 0.001 ms of HBM
    assert r["stages"]["x"]["bound"] == "hbm" and r["stages"]["y"]["bound"] == "alu"
    assert r["sum_bound_ms"] == pytest.approx(12.0) and r["frac"] == pytest.approx(0.5)


def test_alu_peak():
    # 152 SMs x 128 FP32 lanes x 2 (FMA) at 2070 MHz
    assert bench.alu_peak_tflops(2070.0) == pytest.approx(80.54, abs=0.01)


def test_step_batch_candidates_follow_the_tuner_layout():
    # lv_autotune's ms_out: index 6 t + 3 p + b, tiles (8, 16, 32), schedules (block, persistent),
    # batches (32, 64, 128); -1 for a skipped candidate
    ms = [-1.0] * 18
    ms[6 * 2 + 3 + 0] = 0.5838   # tile 32, persistent, batch 32
    ms[6 * 2 + 3 + 1] = 0.5776   # tile 32, persistent, batch 64 (the tuner's pick)
    ms[6 * 2 + 0 + 0] = 0.40     # other schedules never enter
    assert bench.step_batch_candidates(32, True, 64, ms) == [64, 32]
    ms[6 * 2 + 3 + 0] = 0.60     # 3.9 % slower: left out
    assert bench.step_batch_candidates(32, True, 64, ms) == [64]
    ms = [-1.0] * 18
    ms[6 * 1 + 0 + 0], ms[6 * 1 + 0 + 1], ms[6 * 1 + 0 + 2] = 0.71, 0.70, 0.72   # tile 16, block per tile
    assert bench.step_batch_candidates(16, False, 64, ms) == [64, 32, 128]
    assert bench.step_batch_candidates(16, False, 64, None) == [64]
    assert bench.step_batch_candidates(16, False, 64, [-1.0] * 18) == [64]
