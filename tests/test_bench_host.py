"""Host-side helpers of bench.py, on CPU: the DRAM traffic lookup of the dominant
kernel, the kernel each variant name launches, and the parsing of the clock
samples taken during the timed region."""
import json
import os
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _traffic_file(tmp_path, entries):
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(entries))
    return str(p)


def test_traffic_is_scaled_by_nodes_and_tied_to_the_kernel_sources(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    entry = {"dram_bytes_per_launch": 1000.0, "cells": 10, "source_hash": h}
    monkeypatch.setattr(bench, "TRAFFIC_FILE", _traffic_file(tmp_path, {"v": entry}))
    t, why = bench.ncu_traffic("v", 25)
    assert t == 2500.0 and "scaled by nodes" in why
    t, why = bench.ncu_traffic("v", 10)            # the captured grid itself: as captured
    assert t == 1000.0 and "this grid" in why
    # a variant without a capture, and a capture taken on other sources, give None
    assert bench.ncu_traffic("w", 25)[0] is None
    stale = dict(entry, source_hash="0" * 16)
    monkeypatch.setattr(bench, "TRAFFIC_FILE", _traffic_file(tmp_path, {"v": stale}))
    t, why = bench.ncu_traffic("v", 25)
    assert t is None and "changed" in why


def test_missing_traffic_file_gives_none(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "absent.json"))
    assert bench.ncu_traffic("v", 1)[0] is None


def test_clock_summary_median_and_throttle_reasons():
    s = bench.ClockSampler(0)
    s.out = tempfile.TemporaryFile(mode="w+")
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    s.out.write("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                "0, 1995, 2070, 1380.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                "0, 2055, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                "garbage line\n")
    s.proc = object()   # a sampler that ran
    got = s.summary()
    assert got["sm_mhz"] == 2055 and got["sm_max_mhz"] == 2070
    assert got["reasons"] == ["sw_power_cap"] and got["samples"] == 3
    s.out.close()


def test_clock_summary_without_sampler_says_unavailable():
    assert bench.ClockSampler(0).summary()["reasons"] == ["unavailable"]


def test_kernel_named_for_each_variant_family():
    """The roofline line names the CUDA kernel a variant launches (its name in ncu
    launch lists): rolling-slot layouts, split barriers included, run the slim
    kernel, tensor-memory and producer-warp layouts the tensor-memory kernel, and
    the register-window variants the plain fused kernel."""
    cases = {
        "k32_t2_split_r32x1_pf3": "fused_step_slim_kernel",
        "f32_t2_split_w72_r32x1_pf2": "fused_step_slim_kernel",
        "k32_t2_roll_w32_r32x1_pf2_b2": "fused_step_slim_kernel",
        "k32_t2_hyb_w32_r32x1_pf2_b2": "fused_step_slim_kernel",
        "k32_t2_slim_w32_r32x1_pf2_b2": "fused_step_slim_kernel",
        "k32_t2_tmem_w32_r32x1_pf2_b2": "fused_step_tmem_kernel",
        "f32_t3_ws_r32x1_pf2": "fused_step_tmem_kernel",
        "k32_t1_w64_r32x2_pf2": "fused_step_kernel",
        "f64_t1_w64_r16x2_pf1_b2": "fused_step_kernel",
    }
    for variant, kernel in cases.items():
        assert bench.kernel_function(variant) == kernel, variant
