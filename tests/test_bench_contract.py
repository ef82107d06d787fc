"""Host-side pieces of bench.py's JSON contract: the roofline object of the dominant
kernel (bound, achieved = algorithmic work / average launch time, peak, frac = achieved /
peak, traffic only while the kernel's source matches the ncu capture), the algorithmic
bytes of the method's matrix-free operators, the arithmetic labels and the bounded
sample the oracle is timed on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads as W  # noqa: E402

DF = dict(op_form="assembled_df", precond="banded32", guess="zero")
C2 = W.config("cube64_p3")


def _band_prof(w, launches, vectors, ms):
    """(ms, launches, flops, band bytes) as the library's profiler reports a band product."""
    H = bench.band_slots(w)
    return (ms, launches, 1.0, launches * 8.0 * (H * w.ndof + 2 * vectors * w.ndof))


def test_method_bytes_of_the_mass_product():
    # 64^3 elements, p = 3: 256^3 Gauss points, W in FP64 (134 MB), 16 B per dof and vector
    fac, per_vec = bench.method_bytes(C2, mass=True)
    assert fac == 256 ** 3 * 8 and per_vec == 16 * C2.ndof
    fac_k, _ = bench.method_bytes(C2, mass=False)
    assert fac_k == 6 * fac
    assert bench.band_slots(C2) == (7 ** 3 + 1) // 2 == 172


def test_band_roofline_counts_the_methods_bytes():
    prof = _band_prof(C2, 8, 2, 1.0)  # 8 two-vector launches in 1 ms
    r = bench.roofline("band_mass", DF, "k", prof, 6800.0, "measured", C2)
    fac, per_vec = bench.method_bytes(C2)
    alg = fac + 2 * per_vec
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6800.0
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(alg)
    assert r["achieved"] == pytest.approx(8 * alg / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6800.0)
    assert r["avg_launch_ms"] == pytest.approx(1.0 / 8)
    band = prof[3] / 8
    assert r["band_view"]["bytes_per_launch"] == pytest.approx(band)
    assert r["band_view"]["frac"] == pytest.approx(8 * band / 1e-3 / 1e9 / 6800.0)


def test_alu_view_counts_the_tiny_slots_terms():
    """The double-FP32 view counts 12 FP32 operations per exact term and 1 per tiny slot's
    term (the profiler's flops count 2 per term)."""
    prof = (2.0, 4, 4 * 1.0e9, 4 * 400e6)  # 4 launches of 0.5 G terms in 2 ms
    r0 = bench.roofline("band_mass", DF, "k", prof, 6800.0, "measured", C2)
    r = bench.roofline("band_mass", DF, "k", prof, 6800.0, "measured", C2, tiny=0.25)
    assert r0["alu_view"]["fp32_ops_per_term"] == 12.0
    assert r["alu_view"]["fp32_ops_per_term"] == pytest.approx(12.0 * 0.75 + 0.25)
    assert r["alu_view"]["achieved_tops"] == pytest.approx((12.0 * 0.75 + 0.25) * 2.0e9 / 2e-3 / 1e12)
    assert r["alu_view"]["frac"] == pytest.approx(r["alu_view"]["achieved_tops"] / r["alu_view"]["peak_tops"])
    assert r["frac"] == pytest.approx(r0["frac"])  # the HBM view does not depend on the arithmetic


def test_traffic_scaled_from_the_capture_while_the_source_matches(monkeypatch):
    monkeypatch.setattr(bench, "source_sha", lambda name: "feedfacefeedface")
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("band_mass_df", "feedfacefeedface", C2.name, 2), 400e6)
    r = bench.roofline("band_mass", DF, "k", _band_prof(C2, 4, 2, 1.0), 6800.0, "measured", C2)
    assert r["traffic"] == pytest.approx(400e6)  # same vectors per launch as the capture
    r1 = bench.roofline("band_mass", DF, "k", _band_prof(C2, 4, 1, 1.0), 6800.0, "measured", C2)
    assert r1["traffic"] < 400e6


def test_traffic_is_null_when_the_source_changed(monkeypatch):
    monkeypatch.setattr(bench, "source_sha", lambda name: "0000000000000000")
    r = bench.roofline("band_mass", DF, "k", _band_prof(C2, 1, 2, 1.0), 6800.0, "measured", C2)
    assert r["traffic"] is None


def test_matrix_free_roofline_is_alu_bound():
    prof = (2.0, 4, 4 * 0.17e9, 4 * 400e6)
    opts = dict(op_form="matrix_free", precond="fp64", guess="zero")
    r = bench.roofline("mass", opts, "k", prof, 6800.0, "measured", C2)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(4 * 0.17e9 / 2e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_recorded_traffic_keys_name_existing_sources():
    for (key, sha, workload, nvec), val in bench.NCU_TRAFFIC.items():
        assert key in bench.KERNEL_SOURCE and len(sha) == 16 and val > 0
        W.config(workload)
        assert 1 <= nvec <= 8


def test_arithmetic_labels():
    assert bench.arithmetic(dict(op_form="matrix_free", precond="fp64")) == "f64"
    assert bench.arithmetic(dict(op_form="assembled", precond="banded")) == "f64"
    lab = bench.arithmetic(DF)
    assert "df32" in lab and "f32 band-Cholesky" in lab and lab.startswith("f64 state")
    assert "tcgen05" in bench.arithmetic(dict(op_form="assembled", precond="bf16"))


def test_bounded_sample_keeps_the_discretisation():
    w = W.config("cube128_p4")
    ws = bench.sample_workload(w, 24)
    assert ws.nel == (24, 24, 24) and ws.p == w.p and ws.k == w.k and ws.amp == w.amp and ws.init == w.init
    assert ws.ndof == 26 ** 3 and w.nel == (128, 128, 128)
    assert bench.sample_workload(W.config("square32_p2"), 64).nel == (32, 32)
