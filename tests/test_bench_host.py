"""Host logic of bench.py's roofline object, on synthetic step statistics (no GPU): the dominant
step class is chosen by device time; FP64 classes are reported against the FP64 FMA rate, the
FP32 sweeps of the mixed form against HBM bandwidth with their algorithmic bytes."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def stats(**kw):
    st = {"t_matvec_ms": 30.0, "t_resid_ms": 10.0, "t_precond_ms": 100.0, "t_local_ms": 240.0,
          "t_gram_ms": 60.0, "t_rr_ms": 150.0, "t_update_ms": 65.0, "nnz_L": 48_621_362,
          "precond_cols": 6000, "precond_calls": 125, "matvec_cols": 8000, "minres_spmm_cols": 9000,
          "local_calls": 110}
    st.update(kw)
    return st


def test_minres_dominant_is_an_fp64_alu_roofline():
    st = stats()
    r = bench.roofline_object(st, 2_951_752, 0, 1.25e12, "mixed", "medium")
    assert r["kernel"] == "minres" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    flops = 4.0 * 2_951_752 * st["minres_spmm_cols"]
    assert r["achieved"] == pytest.approx(flops / 0.240 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1.25)
    assert r["traffic"] == pytest.approx(bench.MINRES_DRAM_BYTES_PER_COLUMN_PRODUCT * 9000 / 110)


def test_fp32_sweeps_dominant_is_an_hbm_roofline(monkeypatch):
    monkeypatch.setattr(bench, "hbm_peak_gbs", lambda: (6761.9, "measured"))
    st = stats(t_precond_ms=300.0)
    r = bench.roofline_object(st, 2_951_752, 0, 1.25e12, "mixed", "medium")
    assert r["kernel"] == "precond" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(8.0 * st["nnz_L"] * st["precond_calls"] / 0.300 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6761.9) and r["traffic"] is None


def test_fp64_sweeps_dominant_stay_an_alu_roofline():
    r = bench.roofline_object(stats(t_precond_ms=300.0), 2_951_752, 0, 1.25e12, "fp64", "medium")
    assert r["kernel"] == "precond" and r["bound"] == "alu"


def test_hbm_peak_falls_back_without_the_peaks_file(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peak, source = bench.hbm_peak_gbs()
    assert peak == 6800.0 and "fallback" in source
