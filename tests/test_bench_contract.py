"""Host-side pieces of bench.py's JSON contract: the roofline object of the dominant
kernel (bound, achieved = algorithmic work / average launch time, peak, frac = achieved /
peak, traffic only while the kernel's source matches the ncu capture)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_df_roofline_is_hbm_bound_with_measured_traffic():
    prof = (1.0, 8, 8 * 1e9, 8 * 385.6e6)  # 8 launches in 1 ms, 385.6 MB each
    r = bench.roofline("band_mass", "assembled_df", "k", prof, 6800.0, "measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6800.0
    assert r["achieved"] == pytest.approx(8 * 385.6e6 / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6800.0)
    assert r["avg_launch_ms"] == pytest.approx(1.0 / 8)
    key_sha = bench.source_sha(bench.KERNEL_SOURCE["band_mass_df"])
    assert r["traffic"] == bench.NCU_TRAFFIC.get(("band_mass_df", key_sha))


def test_fp64_roofline_is_alu_bound():
    prof = (2.0, 4, 4 * 0.17e9, 4 * 400e6)
    r = bench.roofline("band_mass", "assembled", "k", prof, 6800.0, "measured")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(4 * 0.17e9 / 2e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_traffic_is_null_when_the_source_changed(monkeypatch):
    monkeypatch.setattr(bench, "source_sha", lambda name: "0000000000000000")
    r = bench.roofline("band_mass", "assembled_df", "k", (1.0, 1, 1.0, 1.0), 6800.0, "measured")
    assert r["traffic"] is None


def test_recorded_traffic_keys_name_existing_sources():
    for (key, sha), val in bench.NCU_TRAFFIC.items():
        assert key in bench.KERNEL_SOURCE and len(sha) == 16 and val > 0
