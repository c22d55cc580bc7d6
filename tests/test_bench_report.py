"""The bench line's roofline arithmetic, on CPU: from the per-kernel counters
(launches, device milliseconds, algorithmic bytes) the dominant kernel's
achieved bandwidth is its bytes over its time, its fraction is that over the
measured copy peak, the per-kernel table is per step, and the DRAM traffic
figure appears only for a kernel whose source still hashes to the captured one.
"""
import json
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def peak():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"], "measured"
    except (OSError, ValueError, KeyError):
        return 6400.0, "fallback"


def test_roofline_of_the_dominant_kernel():
    stats = {
        "check_flood_sp_f32": {"launches": 300, "ms": 600.0, "bytes": 1.5e12, "units": 1.25e11},
        "var_flood_f32": {"launches": 300, "ms": 200.0, "bytes": 0.9e12, "units": 4.5e10},
        "slice_llr": {"launches": 6, "ms": 100.0, "bytes": 1.0e9, "units": 1.0e8},
    }
    roof, kernels, launches = bench.roofline(stats, steps=3)
    p, src = peak()
    assert roof["kernel"] == "check_flood_sp_f32" and roof["peak_source"] == src
    assert roof["achieved"] == pytest.approx(1.5e12 / 0.6 / 1e9, rel=1e-4)
    assert roof["frac"] == pytest.approx(roof["achieved"] / p, abs=1e-4)
    assert roof["avg_launch_ms"] == pytest.approx(2.0)
    assert roof["algorithmic_bytes_per_launch"] == pytest.approx(5e9)
    assert roof["share"] == pytest.approx(600 / 900, abs=1e-4)
    assert list(kernels) == ["check_flood_sp_f32", "var_flood_f32", "slice_llr"]
    assert kernels["var_flood_f32"]["ms_per_step"] == pytest.approx(200 / 3, abs=1e-3)
    assert kernels["var_flood_f32"]["GB/s"] == pytest.approx(0.9e12 / 0.2 / 1e9, rel=1e-3)
    assert launches == 202
    assert roof["traffic"] == pytest.approx(bench.load_traffic("check_flood_sp_f32", stats["check_flood_sp_f32"]))
    # the traffic figure: DRAM bytes per unit from the committed capture, scaled
    # by this run's units per launch, present while the kernel source matches
    units = 1e9
    t = bench.load_traffic("check_flood_sp_f32", {"units": units, "launches": 10})
    ref = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["check_flood_sp_f32"]
    src = os.path.join(ROOT, "paper_2108_08418_b300", "csrc", ref["source"])
    if bench.source_region_sha(src, *ref["region"]) == ref["source_sha"]:
        assert t == pytest.approx(ref["dram_bytes_per_unit"] * units / 10)
    else:
        assert t is None            # the kernel changed since the capture: no traffic figure
    assert bench.load_traffic("no_such_kernel", {"units": 1, "launches": 1}) is None


def test_traffic_key_follows_the_kernel_source(tmp_path):
    src = tmp_path / "k.cu"
    src.write_text("head\n// start\nkernel body\n// end\ntail\n")
    a = bench.source_region_sha(str(src), "// start", "// end")
    src.write_text("head changed\n// start\nkernel body\n// end\ntail changed\n")
    assert bench.source_region_sha(str(src), "// start", "// end") == a      # outside the region: same key
    src.write_text("head\n// start\nkernel body, edited\n// end\ntail\n")
    assert bench.source_region_sha(str(src), "// start", "// end") != a      # inside: a new key


def test_sweep_workload_names_its_rate_rule():
    assert "back-off rates" in bench.sweep_workload("backoff")
    assert "codes at 0.95 x slice capacity" not in bench.sweep_workload("backoff")
    assert "codes at 0.95 x slice capacity" in bench.sweep_workload("capacity")


def test_block_work_model():
    import numpy as np
    t = np.array([1, 2, 3, 40, 5] * 10)            # 50 frames: two 32-frame blocks
    assert bench.block_work(t, ()) == 32 * 40 + 32 * 40
    # re-packed after iteration 16: one frame of the 10 with 40 passes per block
    # row ... all ten long frames share one block from pass 17 on
    assert bench.block_work(t, (16,)) == 32 * 16 * 2 + 32 * (40 - 16)
    assert bench.block_work(np.array([3] * 64), (1, 2)) == 64 * 3
