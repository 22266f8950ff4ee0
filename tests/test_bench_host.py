"""Host logic of bench.py's roofline object, on synthetic step statistics (no GPU): the dominant
step class is chosen by device time; FP64 classes are reported against the FP64 FMA rate, the
FP32 sweeps of the mixed form against HBM bandwidth with their algorithmic bytes."""
import json
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
    r = bench.roofline_object(st, 2_951_752, 0, 1.25e12, "fp64", "medium")
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


def test_double_float_update_dominant_is_an_fp32_issue_roofline():
    st = stats(t_update_ms=2500.0, update_fma=3.0 * 334_272 * 538 * 282 * 46)
    r = bench.roofline_object(st, 17_220_448, 0, 1.25e12, "mixed", "large", peak32=80e12)
    assert r["kernel"] == "update" and r["bound"] == "alu"
    instr = bench.DF_FP32_OPS * st["update_fma"]
    assert r["achieved"] == pytest.approx(instr / 2.5 / 1e12)
    assert r["peak"] == pytest.approx(40.0) and r["frac"] == pytest.approx(r["achieved"] / 40.0)
    # the same step in the FP64 form is bound by the FP64 FMA rate
    r64 = bench.roofline_object(st, 17_220_448, 0, 1.25e12, "fp64", "large", peak32=80e12)
    assert r64["unit"] == "TFLOP/s" and r64["achieved"] == pytest.approx(2.0 * st["update_fma"] / 2.5 / 1e12)


def test_oracle_sample_of_the_large_workload_scales_by_the_stored_runs(monkeypatch):
    runs = {("medium", -1): {"nev": 64, "iters": 114, "oracle_seconds": 228.0},
            ("large", -1): {"nev": 256, "iters": 46, "oracle_seconds": 4600.0}}
    monkeypatch.setattr(bench, "golden", lambda w="medium", m0=-1, required=True: runs.get((w, m0)))
    swl, snev, scale, its, how = bench.oracle_sample_plan("large", -1)
    assert swl == "medium" and snev == 64 and its == 46
    assert scale == pytest.approx((4600.0 / 46) / (228.0 / 114))
    del runs[("large", -1)]
    swl, snev, scale, its, how = bench.oracle_sample_plan("large", -1)
    assert scale is None and "unscaled" in how


def test_angles_at_gaps_sees_a_small_rotation():
    import numpy as np
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((200, 12)))
    Xa = Q[:, :6]
    Xb = Xa.copy()
    Xb[:, 2] = np.cos(1e-7) * Xa[:, 2] + np.sin(1e-7) * Q[:, 8]
    lam = np.array([1.0, 2.0, 3.0, 3.0000001, 5.0, 6.0])
    got = bench.angles_at_gaps(Xa.T @ Xa, Xb.T @ Xb, Xa.T @ Xb, lam, 6)
    assert abs(got - 1e-7) <= 2e-8


def test_mixed_form_products_are_fp32_pipe_rooflines():
    # double-float SpMM of steps 3/7 and FP32 MINRES products in the mixed form
    st = stats(t_matvec_ms=900.0)
    r = bench.roofline_object(st, 2_951_752, 0, 1.25e12, "mixed", "medium", peak32=80e12)
    assert r["kernel"] == "matvec" and r["unit"] == "T FP32 instr/s"
    assert r["achieved"] == pytest.approx(bench.DF_FP32_OPS * 2.0 * 2_951_752 * st["matvec_cols"] / 0.9 / 1e12)
    r = bench.roofline_object(stats(), 2_951_752, 0, 1.25e12, "mixed", "medium", peak32=80e12)
    assert r["kernel"] == "minres" and r["unit"] == "TFLOP/s" and r["peak"] == pytest.approx(80.0)


def test_batched_workload_is_a_bench_choice_and_has_no_reference_arm(capsys):
    import bench
    a = bench.parse(["--workload", "batched", "--impl", "reference"])
    assert a.workload == "batched" and a.batch_count == 64 and a.batch_concurrent == 8
    bench.run_reference(a)
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and "unavailable" in line
