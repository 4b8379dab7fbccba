"""Host-side checks of bench.py's roofline bookkeeping (no GPU): the per-unit algorithmic cost
formulas at the realistic size, and the committed ncu summary that supplies the measured DRAM
traffic per launch."""

import os
import re

import bench


def test_algorithmic_cost_per_unit_at_512():
    # 2 FFTs at 5 N log2 N + Phi and D multiplies (6 N each) + imaging / scatter (4 N)
    assert bench.flops_per_unit(512) == 2 * 5 * 512 * 9 + 16 * 512 == 54272
    # source row 8 N + Phi, D rows shared by K = 16 shots + the item's data row over nz = 256 depths
    assert bench.bytes_per_unit(512, 512, 256, 16) == 8 * 512 + 16 * 512 / 16 + 8 * 512 / 256 == 4624


def test_profile_summary_is_present_and_parses():
    assert os.path.exists(bench.PROFILE_SUMMARY), bench.PROFILE_SUMMARY
    text = open(bench.PROFILE_SUMMARY).read()
    assert re.search(r"kernel_source_hash:\s*[0-9a-f]{16}", text)
    for kclass in ("adjoint", "forward", "source"):
        m = re.search(rf"{kclass}_dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
        assert m and 1e9 < float(m.group(1)) < 1e10, kclass
    assert "--clock-control none" in text


def test_kernel_source_hash_is_stable():
    assert bench.kernel_source_hash() == bench.kernel_source_hash()
    assert re.fullmatch(r"[0-9a-f]{16}", bench.kernel_source_hash())


def test_peaks_fall_back_when_unmeasured():
    peaks, kind = bench.measured_peaks()
    assert kind in ("measured", "fallback")
    if kind == "fallback":
        assert peaks["hbm_gbs"] == 6800.0
