#!/usr/bin/env python
"""Benchmark: converged eigenpairs per second (Res_max <= 1e-8) of the LABPSD solve on GB300,
mixed precision against plain FP64 on the same GPU.

Workload (default, `large`): 64^3 periodic Q1 elements, 32 atoms (Z = 4), 4 Gaussian enrichment
dofs per node within r_c = 0.08 (n = 334,272), nev = 256 with the default m0 = 26, tol = 1e-8,
hybrid preconditioner.  `medium` is the 32^3 workload (8 atoms, r_c = 0.15, n = 47,620, nev = 64),
`medium-nonlocal` the same with the nonlocal term F G F^T.  A step is one solve (Sec. 3 outline,
steps 1-12) from the same seed-normal start block on a session whose global factor was computed at
creation (Sec. 4: once per SCF run).  `value` is device-timed (CUDA events on the session stream,
inputs resident in HBM) for the form given by --precision (mixed by default); the line also
carries the plain FP64 form on the same problem (`config.fp64`) and the accuracy of both against
the stored oracle run and against each other (`accuracy`).  `e2e` times the public host API end to
end per step: hbsd_create (H2D of H, S, factorisation) + hbsd_solve (H2D of X0, D2H of lambda, X).

Multi-GPU: replicas only -- every rank solves its own instance, no collective on the data
path; value = eigenpairs of all ranks / max-over-ranks time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload large|medium|...]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TOL = 1e-8
# DRAM bytes (read + write) per column product of the fused MINRES kernel, from one ncu capture of a
# 57-column, 99-step launch on the 32^3 workload; the roofline's traffic scales it by the column
# products of the average launch of the timed solve (32^3 workload only)
MINRES_DRAM_BYTES_PER_COLUMN_PRODUCT = (1212.506368e6 + 438.241536e6) / 156
# FP32 instructions of one double-float multiply-add (TwoProd by FMA with both cross terms,
# TwoSum into the running pair, the low-part add): 1 mul + 3 fma + 8 add/sub
DF_FP32_OPS = 12
METRIC = "eigenpairs/s to 1e-8 residual (LABPSD, hybrid preconditioner)"
WORKLOADS = {
    "large": "64^3 periodic Q1 elements, 32 atoms Z=4, 4 Gaussian enrichment dofs/node within r_c=0.08, nev=256, "
             "tol=1e-8",
    "medium": "32^3 periodic Q1 elements, 8 atoms Z=4, 4 Gaussian enrichment dofs/node within r_c=0.15, nev=64, "
              "tol=1e-8",
}
WORKLOADS["medium-nonlocal"] = WORKLOADS["medium"] + ", nonlocal F G F^T with s+p projectors per atom (k=32, r_p=0.2)"
WORKLOADS["batched"] = ("independent instances solved by hbsd_solve_batch: mesh from {16^3, 24^3, 32^3, 40^3}, 4-16 "
                        "atoms Z=4, 2-4 enrichment dofs/node within r_c=0.15, nev from {32, 64, 128} (seeded draws), "
                        "mixed form, tol=1e-8")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"],
                    help="mixed: step 6(a) in FP32 on the scaled pencil, Gram and update in double-float, "
                         "the rest in FP64 (default); fp64: FP64 throughout")
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="timed solves of the plain FP64 form on the same problem (0: leave it out)")
    ap.add_argument("--fp64-warmup", type=int, default=1)
    ap.add_argument("--local-solver", default="minres", choices=["minres", "onestep"],
                    help="step 6(b): MINRES (default) or the first-order one-step refinement (Sec. 6)")
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS),
                    help="large: 64^3, nev 256 (default); medium: 32^3, nev 64; medium-nonlocal: with the "
                         "nonlocal term H_nl = F G F^T (Sec. 4)")
    ap.add_argument("--batch-count", type=int, default=64, help="batched workload: instances per batch")
    ap.add_argument("--batch-concurrent", type=int, default=8, help="batched workload: sessions solved at once")
    ap.add_argument("--m0", type=int, default=-1,
                    help="guard columns (remark 1; default max(3, ceil(nev/10))); the medium workloads "
                         "have stored oracle runs for m0 = 21")
    return ap.parse_args(argv)


def aggregate_replicas(ms, converged, device):
    """Replicas-only aggregation: the slowest rank's time and the eigenpairs of all ranks (the job's
    value is all ranks' eigenpairs over the slowest rank's time).  One process: unchanged."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(ms), float(converged)
    t = torch.tensor([ms, converged], dtype=torch.float64, device=device)
    mx = t.clone()
    tdist.all_reduce(mx, op=tdist.ReduceOp.MAX)
    sm = t.clone()
    tdist.all_reduce(sm, op=tdist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling during the timed region (SM clock, max clock, throttle reasons)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def golden_path(workload="medium", m0=-1):
    base = workload.replace("-", "_")
    name = f"{base}_seed1.json" if m0 < 0 else f"{base}_m0_{m0}_seed1.json"
    return os.path.join(ROOT, "tests", "golden", name)


def golden(workload="medium", m0=-1, required=True):
    """The stored oracle run of the workload (tests/golden/make_golden.py writes them)."""
    path = golden_path(workload, m0)
    if not os.path.exists(path):
        if required:
            raise SystemExit(f"no stored oracle run for workload {workload} with m0 = {m0} "
                             f"(tests/golden/make_golden.py writes one)")
        return None
    with open(path) as f:
        return json.load(f)


def m0_of(nev, m0):
    return m0 if m0 >= 0 else max(3, -(-nev // 10))


def problem(workload):
    from paper_1308_2445_gb300 import pufe_inputs as pi
    if workload == "large":
        return pi.large_case(1), pi.LARGE_NEV
    if workload == "medium-nonlocal":
        return pi.medium_nonlocal_case(1), pi.MEDIUM_NEV
    return pi.medium_case(1), pi.MEDIUM_NEV


def oracle_iteration_times(workload, nev, m0, iters):
    """Wall times of the CPU oracle's outer iterations on `workload` (its library factorisation
    first, untimed); returns (factor seconds, per-iteration seconds)."""
    from oracle import labpsd as L
    from paper_1308_2445_gb300 import pufe_inputs as pi
    p, _ = problem(workload)
    X0 = pi.seed_normal_block(1, p.n, nev + m0_of(nev, m0))
    t0 = time.perf_counter()
    Hs, S, s0 = L.make_shifted(p)
    K = L.GlobalPreconditioner(Hs, p.dof_node, p.grid)
    t_factor = time.perf_counter() - t0
    marks = [time.perf_counter()]
    L.labpsd(p, nev, TOL, X0=X0, precond=K, opts=L.Options(max_outer=iters, m0=m0_of(nev, m0)),
             on_iteration=lambda it, res: marks.append(time.perf_counter()))
    return t_factor, [marks[i + 1] - marks[i] for i in range(len(marks) - 1)]


def oracle_sample_plan(workload, m0):
    """Which workload the oracle is timed on and how its iteration time scales to `workload`.

    The 64^3 workload's library sparse LU takes the oracle tens of minutes, so a bounded sample
    cannot run there: its iterations are timed on the 32^3 workload and scaled by the ratio of
    the oracle's own per-iteration times on the two workloads, both from the stored oracle runs
    (written on one host by tests/golden/make_golden.py), times the 64^3 run's iteration count.
    Returns (sample workload, sample nev, scale, target iterations, description)."""
    if workload != "large":
        g = golden(workload, m0)
        return workload, g["nev"], 1.0, g["iters"], f"the {workload} workload itself"
    gl = golden("large", -1, required=False)
    gm = golden("medium", -1)
    per_m = gm["oracle_seconds"] / max(1, gm["iters"])
    if gl is None:
        return "medium", gm["nev"], None, None, "no stored 64^3 oracle run: unscaled 32^3 sample"
    per_l = gl["oracle_seconds"] / max(1, gl["iters"])
    scale = per_l / per_m
    return ("medium", gm["nev"], scale, gl["iters"],
            f"oracle iterations on the 32^3 workload, scaled by {scale:.1f} (the stored oracle runs' per-iteration "
            f"times, 64^3: {per_l:.1f} s, 32^3: {per_m:.2f} s, on one host) and by the 64^3 run's {gl['iters']} "
            f"iterations")


def cpu_baseline(workload="large", m0=-1, iters=2):
    """Time the CPU oracle, as it stands, on a bounded sample (factorisation excluded like value's)."""
    nev_target = problem_nev(workload)
    swl, snev, scale, target_iters, how = oracle_sample_plan(workload, m0)
    t_factor, d = oracle_iteration_times(swl, snev, m0 if swl == workload else -1, iters)
    per_iter = sum(d[1:]) / len(d[1:]) if len(d) > 1 else d[0]
    if scale is None:
        value, nev_used, its = snev / (per_iter * golden(swl)["iters"]), snev, golden(swl)["iters"]
    else:
        value, nev_used, its = nev_target / (per_iter * scale * target_iters), nev_target, target_iters
    return {"value": value, "unit": "eigenpairs/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"{how}: library factorisation ({t_factor:.1f} s, excluded like value's) + initial "
                       f"Rayleigh-Ritz + {iters} BPSD iterations ({per_iter:.2f} s each after the first) of the "
                       f"oracle, solve time = per-iteration time x {its} iterations for {nev_used} eigenpairs; "
                       f"numpy/scipy threads = all host cores, the sparse triangular solves single-threaded"),
            "t_factor_s": t_factor, "t_iter_s": per_iter}


def problem_nev(workload):
    from paper_1308_2445_gb300 import pufe_inputs as pi
    return pi.LARGE_NEV if workload == "large" else pi.MEDIUM_NEV


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of the GB300s when the peaks file is present, else the
    profiling recipe's fallback figure (said so in the result)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured HBM copy bandwidth (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback HBM figure (6.8 TB/s; no measured peaks file)"


def roofline_object(st, nnz, nl_nnz, peak64, precision, workload, peak32=None):
    """Roofline of the dominant step class, from the solve's CUDA-event step times and the
    algorithmic work per unit.  FP64 classes are bound by the FP64 FMA rate (measured in the same
    run, peak64 in FLOP/s); the FP32 sweeps of the mixed form by HBM (their panels, 4 bytes per
    entry, read once per sweep: 8 nnz(L) bytes per call); the double-float Gram and update of the
    mixed form by the FP32 pipes: DF_FP32_OPS FP32 instructions per double-float multiply-add
    against the measured FP32 FMA instruction rate (peak32 / 2)."""
    mixed = precision == "mixed"
    # in the mixed form the products of steps 3/7 run in double-float and MINRES's operator products
    # in FP32 (the library's defaults spmm_df64 = 1, minres_f32 = 1)
    classes = {
        "precond": (st["t_precond_ms"], 4.0 * st["nnz_L"] * st["precond_cols"],
                    "supernodal triangular solves of step 6(a): 2 FMA per factor entry per column"),
        "matvec": (st["t_matvec_ms"], (4.0 * nnz + 4.0 * nl_nnz) * st["matvec_cols"],
                   "fused SpMM of steps 3/7: 2 FMA (h and s) per nonzero per column"
                   + (" + 2 FMA per F entry (F^T X and F Z)" if nl_nnz else "")),
        "minres": (st["t_local_ms"], (4.0 * nnz + 4.0 * nl_nnz) * st["minres_spmm_cols"],
                   "MINRES of step 6(b): shifted fused SpMM, 2 FMA per nonzero per column"
                   + (" + 2 FMA per F entry" if nl_nnz else "")),
        "update": (st["t_update_ms"], 2.0 * st.get("update_fma", 0.0),
                   "steps 10-11: [Psi P] W for Psi, Psi_H, Psi_S, 3 n q w multiply-adds per iteration"
                   + (" in double-float" if mixed else "")),
        "gram": (st["t_gram_ms"], 2.0 * st.get("gram_fma", 0.0),
                 "step 8: both reduced matrices, n q (q+1) multiply-adds per iteration"
                 + (" in double-float" if mixed else "")),
    }
    dom = max(classes, key=lambda k: classes[k][0])
    t_ms, flops, what = classes[dom]
    step_ms = {k: st[f"t_{k}_ms"] for k in ("matvec", "resid", "precond", "local", "gram", "rr", "update")}
    if dom == "precond" and mixed:
        peak, source = hbm_peak_gbs()
        achieved = 8.0 * st["nnz_L"] * st["precond_calls"] / (t_ms * 1e-3) / 1e9 if t_ms > 0 else 0.0
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": dom,
                "what": "FP32 supernodal sweeps of step 6(a): the FP32 panels read once per sweep, 8 nnz(L) bytes per call",
                "peak_source": source, "step_ms": step_ms}
    if dom == "matvec" and mixed and peak32:
        # 2 double-float multiply-adds per stored nonzero per column, DF_FP32_OPS FP32 instructions each
        dfma = (2.0 * nnz) * st["matvec_cols"]
        achieved = DF_FP32_OPS * dfma / (t_ms * 1e-3) / 1e12 if t_ms > 0 else 0.0
        peak = peak32 / 2.0 / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP32 instr/s",
                "frac": achieved / peak, "traffic": None, "kernel": dom,
                "what": "steps 3/7 and the Psi_H, Psi_S recomputation: fused SpMM in double-float on the scaled pencil, "
                        f"2 double-float multiply-adds (h and s) per stored nonzero per column, {DF_FP32_OPS} FP32 "
                        "instructions each (the FP64 products of the convergence check counted alike)",
                "peak_source": "FP32 FMA probe (hbsd_probe_peak) measured in this run, one instruction per FMA",
                "step_ms": step_ms}
    if dom == "minres" and mixed and peak32:
        achieved = flops / (t_ms * 1e-3) / 1e12 if t_ms > 0 else 0.0
        return {"bound": "alu", "achieved": achieved, "peak": peak32 / 1e12, "unit": "TFLOP/s",
                "frac": achieved / (peak32 / 1e12), "traffic": None, "kernel": dom,
                "what": what + " (FP32 products on the scaled pencil, FP64 recurrences)",
                "peak_source": "FP32 FMA probe (hbsd_probe_peak) measured in this run", "step_ms": step_ms}
    if dom in ("update", "gram") and mixed and peak32:
        # FP32 instructions per second of the double-float products against the FP32 FMA issue rate
        achieved = DF_FP32_OPS * (flops / 2.0) / (t_ms * 1e-3) / 1e12 if t_ms > 0 else 0.0
        peak = peak32 / 2.0 / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP32 instr/s",
                "frac": achieved / peak, "traffic": None, "kernel": dom,
                "what": what + f" ({DF_FP32_OPS} FP32 instructions per double-float multiply-add)",
                "fp64_equivalent_tflops": flops / (t_ms * 1e-3) / 1e12 if t_ms > 0 else 0.0,
                "peak_source": "FP32 FMA probe (hbsd_probe_peak) measured in this run, one instruction per FMA",
                "step_ms": step_ms}
    achieved = flops / (t_ms * 1e-3) / 1e12 if t_ms > 0 else 0.0
    traffic = None
    if dom == "minres" and st["local_calls"] > 0 and workload == "medium":
        traffic = MINRES_DRAM_BYTES_PER_COLUMN_PRODUCT * st["minres_spmm_cols"] / st["local_calls"]
    return {"bound": "alu", "achieved": achieved, "peak": peak64 / 1e12, "unit": "TFLOP/s",
            "frac": achieved / (peak64 / 1e12) if peak64 > 0 else None, "traffic": traffic,
            "traffic_note": "DRAM bytes per launch: ncu bytes per column product of one capture on the 32^3 "
                            "workload x the average launch's column products" if traffic is not None else None,
            "kernel": dom, "what": what, "peak_source": "FP64 FMA probe (hbsd_probe_peak) measured in this run",
            "step_ms": step_ms}


def angles_at_gaps(Ga, Gb, C, lam, nev):
    """Largest S-principal angle between span Xa(:, :j) and span Xb(:, :j) over the gaps
    lam[j] - lam[j-1] > 1e-2 max|lam|, from Ga = Xa^T S Xa, Gb = Xb^T S Xb and C = Xa^T S Xb
    (nev x nev): each leading block is whitened by the Cholesky factors of its Grams, and the
    sine of the largest angle is sqrt(1 - sigma_min^2) of the whitened block."""
    import numpy as np
    lam = np.asarray(lam)
    scale = np.abs(lam).max()
    worst = 0.0
    for j in range(1, nev):
        if lam[j] - lam[j - 1] > 1e-2 * scale:
            La = np.linalg.cholesky(0.5 * (Ga[:j, :j] + Ga[:j, :j].T))
            Lb = np.linalg.cholesky(0.5 * (Gb[:j, :j] + Gb[:j, :j].T))
            W = np.linalg.solve(La, np.linalg.solve(Lb, C[:j, :j].T).T)
            smin = float(np.linalg.svd(W, compute_uv=False).min())
            worst = max(worst, float(np.sqrt(max(0.0, 1.0 - min(1.0, smin) ** 2))))
    return worst


def run_reference(args):
    ws, rank, _ = dist()
    if rank != 0:
        return
    if args.workload == "batched":
        print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no reference arm of its own; "
                          "the gb300 line's cpu_baseline times the oracle on its smallest instance"}), flush=True)
        return
    nev = problem_nev(args.workload)
    swl, snev, scale, target_iters, how = oracle_sample_plan(args.workload, args.m0)
    t_factor, d = oracle_iteration_times(swl, snev, args.m0 if swl == args.workload else -1,
                                         args.warmup + args.steps)
    timed = d[args.warmup:] or d
    per_iter = sum(timed) / len(timed)
    if scale is None:
        its = golden(swl)["iters"]
        value = snev / (per_iter * its)
        ms_step = per_iter * 1e3
    else:
        value = nev / (per_iter * scale * target_iters)
        ms_step = per_iter * scale * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "eigenpairs/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "nev": nev, "m0": m0_of(nev, args.m0),
                       "arithmetic": "fp64 (the CPU oracle)",
                       "step": "one BPSD iteration of the CPU oracle; value scaled to the oracle's full solve"},
            "cpu_baseline": {"value": value, "unit": "eigenpairs/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{how}; {len(timed)} timed BPSD iterations after {args.warmup} warm-up "
                                       f"(library factorisation {t_factor:.1f} s untimed)"},
            "e2e": {"value": value, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_solves(sess, nev, X0, lam, X, warmup, steps, stream, ws, clocks=None):
    import torch
    for _ in range(warmup):
        sess.solve_device(nev, TOL, X0, lam, X)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    converged = 0
    stats = []
    for _ in range(steps):
        it, rc, st = sess.solve_device(nev, TOL, X0, lam, X)
        stats.append(st)
        if rc == 0 and st["res_max"] <= TOL:
            converged += nev
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop() if clocks else None
    return e0.elapsed_time(e1), converged, stats, ck


def batched_cpu_baseline(inst, iters_gpu, iters=2):
    """The oracle, as it stands, on the batch's smallest instance: its library factorisation
    (excluded, as the sessions' are), the initial Rayleigh-Ritz and `iters` BPSD iterations;
    eigenpairs/s = nev / (per-iteration time x the GPU's iteration count for that instance)."""
    from oracle import labpsd as L
    from paper_1308_2445_gb300 import pufe_inputs as pi
    i = min(range(len(inst)), key=lambda j: inst[j][0].n * inst[j][1])
    p, nev, _ = inst[i]
    m0 = m0_of(nev, -1)
    X0 = pi.seed_normal_block(1, p.n, nev + m0)
    t0 = time.perf_counter()
    Hs, S, s0 = L.make_shifted(p)
    K = L.GlobalPreconditioner(Hs, p.dof_node, p.grid)
    t_factor = time.perf_counter() - t0
    marks = [time.perf_counter()]
    L.labpsd(p, nev, TOL, X0=X0, precond=K, opts=L.Options(max_outer=iters, m0=m0),
             on_iteration=lambda it, res: marks.append(time.perf_counter()))
    d = [marks[k + 1] - marks[k] for k in range(len(marks) - 1)]
    per_iter = sum(d[1:]) / len(d[1:]) if len(d) > 1 else d[0]
    its = max(1, iters_gpu[i])
    return {"value": nev / (per_iter * its), "unit": "eigenpairs/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"instance {i} of the batch (n = {p.n}, nev = {nev}, the smallest): library factorisation "
                       f"({t_factor:.1f} s, excluded) + initial Rayleigh-Ritz + {iters} BPSD iterations "
                       f"({per_iter:.2f} s each after the first); solve time = per-iteration time x the GPU's "
                       f"{its} iterations on that instance"),
            "t_factor_s": t_factor, "t_iter_s": per_iter}


def run_batched(args):
    """The batched workload: hbsd_solve_batch over seeded uneven instances (one GPU, replicas
    only under torchrun: each rank its own batch)."""
    import torch
    from paper_1308_2445_gb300 import batch_bench
    ws, rank, local = dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    a = argparse.Namespace(count=args.batch_count, seed=1 + rank, concurrent=args.batch_concurrent,
                           arms="batched,one_at_a_time,fp64" if args.fp64_steps > 0 else "batched,one_at_a_time",
                           meshes="16,24,32,40", tol=TOL)
    inst_holder = {}
    res = batch_bench.run(a, args.steps, args.warmup, clocks=Clocks(local), keep=inst_holder)
    b = res["batched"]
    wall_ms, conv = aggregate_replicas(b["wall_s"] * 1e3, b["converged_eigenpairs"], "cuda")
    line = {"metric": METRIC + ", batched form", "value": conv / (wall_ms * 1e-3), "unit": "eigenpairs/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS["batched"], "instances": res["count"], "concurrent": res["concurrent"],
                       "total_nev": res["total_nev"], "n": res["instances"]["n"], "nev": res["instances"]["nev"],
                       "mesh": res["instances"]["mesh"], "iters": b["iters"], "run_ms": b["run_ms"],
                       "tune": res.get("tune"), "t_create_s": res.get("t_create_mixed_s"),
                       "t_autotune_s": res.get("t_autotune_s"),
                       "timing": "host wall clock between device synchronisations around each batch call (the "
                                 "solves run on one stream per session); median of the timed calls",
                       "l2": "working set > L2 (all sessions' factors and blocks resident)",
                       "one_at_a_time": res.get("one_at_a_time"), "fp64": res.get("fp64"),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "roofline": None,
            "roofline_note": "a batch mixes every kernel of many problem sizes; the per-kernel roofs are those of "
                             "the 64^3 and 32^3 lines",
            "e2e": res.get("e2e"), "gpu_launches": int(b["gpu_launches_per_call"] * args.steps),
            "clocks": res.get("clocks")}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = batched_cpu_baseline(inst_holder["inst"], b["iters"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    import numpy as np
    import torch
    ws, rank, local = dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_1308_2445_gb300 import build_lib
    if not os.path.exists(build_lib.LIB):
        build_lib.build()
    from paper_1308_2445_gb300 import hbsd, pufe_inputs as pi

    p, nev = problem(args.workload)
    nl_nnz = int(np.count_nonzero(p.F)) if p.F is not None else 0
    w = nev + m0_of(nev, args.m0)
    stream = torch.cuda.Stream()
    prec = hbsd.PRECISION_MIXED if args.precision == "mixed" else hbsd.PRECISION_FP64
    lsol = hbsd.LOCAL_ONESTEP if args.local_solver == "onestep" else hbsd.LOCAL_MINRES
    sess = hbsd.Session.from_problem(p, stream=stream.cuda_stream, precision=prec, local_solver=lsol, m0=args.m0)
    torch.cuda.synchronize()
    X0h = torch.from_numpy(pi.seed_normal_block(1, p.n, w)).pin_memory()
    X0 = torch.zeros(p.n, w + (w % 2), dtype=torch.float64, device="cuda")[:, :w]
    X0.copy_(X0h)
    lam = torch.zeros(nev, dtype=torch.float64, device="cuda")
    X = torch.zeros(p.n, nev, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()

    # ---- timed region: K solves of the benchmarked form --------------------------------
    clocks = Clocks(local)
    ms, converged, stats, ck = timed_solves(sess, nev, X0, lam, X, args.warmup, args.steps, stream, ws, clocks)
    ms, converged = aggregate_replicas(ms, converged, "cuda")
    value = converged / (ms * 1e-3)
    st = stats[-1]
    lam_main = lam.cpu().numpy()

    # ---- roofline of the dominant step class (device time from the solve's CUDA events) ----
    peak64 = hbsd.probe_peak(0, stream.cuda_stream)
    peak32 = hbsd.probe_peak(1, stream.cuda_stream)
    roof = roofline_object(st, p.nnz, nl_nnz, peak64, args.precision, args.workload, peak32)

    # ---- the plain FP64 form on the same problem and GPU ----------------------------------
    fp64 = None
    X64 = None
    if args.precision == "mixed" and args.fp64_steps > 0:
        s64 = hbsd.Session.from_problem(p, stream=stream.cuda_stream, precision=hbsd.PRECISION_FP64,
                                        local_solver=lsol, m0=args.m0)
        lam64 = torch.zeros(nev, dtype=torch.float64, device="cuda")
        X64 = torch.zeros(p.n, nev, dtype=torch.float64, device="cuda")
        ms64, conv64, stats64, _ = timed_solves(s64, nev, X0, lam64, X64, args.fp64_warmup, args.fp64_steps,
                                                stream, ws)
        ms64, conv64 = aggregate_replicas(ms64, conv64, "cuda")
        st64 = stats64[-1]
        fp64 = {"value": conv64 / (ms64 * 1e-3), "unit": "eigenpairs/s", "ms_per_solve": ms64 / args.fp64_steps,
                "steps": args.fp64_steps, "warmup": args.fp64_warmup, "iters": st64["iters"],
                "res_max": st64["res_max"],
                "step_ms": {k: st64[f"t_{k}_ms"] for k in ("matvec", "resid", "precond", "local", "gram", "rr",
                                                           "update")}}
        # S X for both blocks (the session's own product of steps 3/7), then the S-Grams
        HX = torch.zeros_like(X64)
        SXa = torch.zeros_like(X64)
        SXb = torch.zeros_like(X64)
        s64.spmm_pair(X, HX, SXa)
        s64.spmm_pair(X64, HX, SXb)
        torch.cuda.synchronize()
        Ga, Gb, Cab = [(A.T @ B).cpu().numpy() for A, B in ((X, SXa), (X64, SXb), (X, SXb))]
        lam64_h = lam64.cpu().numpy()
        fp64["max_rel_eig_diff_vs_mixed"] = float(np.abs(lam64_h - lam_main).max() / np.abs(lam64_h).max())
        fp64["max_angle_vs_mixed"] = angles_at_gaps(Ga, Gb, Cab, lam64_h, nev)
        fp64["lam"] = lam64_h
        s64.close()
        del HX, SXa, SXb

    # ---- accuracy against the stored oracle run -------------------------------------------
    acc = {}
    g = golden(args.workload, args.m0, required=False)
    if g is not None:
        ref = np.array(g["lam"])
        acc["oracle_iters"] = g["iters"]
        acc["max_rel_eig_err_vs_oracle"] = float(np.abs(lam_main - ref).max() / np.abs(ref).max())
        acc["per_eig_abs_err_vs_oracle_max"] = float(np.abs(lam_main - ref).max())
        if fp64 is not None:
            acc["fp64_max_rel_eig_err_vs_oracle"] = float(np.abs(fp64["lam"] - ref).max() / np.abs(ref).max())
    else:
        acc["oracle"] = "no stored oracle run for this workload"
    if fp64 is not None:
        acc["max_rel_eig_diff_mixed_vs_fp64"] = fp64.pop("max_rel_eig_diff_vs_mixed")
        acc["max_s_angle_mixed_vs_fp64_at_gaps"] = fp64.pop("max_angle_vs_mixed")
        fp64.pop("lam")
    acc["res_max"] = st["res_max"]

    # ---- end to end through the public host API ----------------------------------------
    rp = np.ascontiguousarray(p.row_ptr)
    h2d = rp.nbytes + p.col_idx.nbytes + p.h_val.nbytes + p.s_val.nbytes + p.dof_node.nbytes + p.n * w * 8
    if p.F is not None:
        h2d += p.F.nbytes + p.G.nbytes
    d2h = nev * 8 + p.n * nev * 8
    X0n = pi.seed_normal_block(1, p.n, w)
    e2e_t = []
    e2e_conv = 0
    st2 = None
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        ta = time.perf_counter()
        s2 = hbsd.Session.from_problem(p, precision=prec, local_solver=lsol, m0=args.m0)
        lam_h, X_h, it2, rc2, st2 = s2.solve(nev, TOL, X0=X0n)
        s2.close()
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - ta)
        if rc2 == 0 and st2["res_max"] <= TOL:
            e2e_conv += nev
    e2e = None
    if e2e_t:
        e2e_ms, e2e_all = aggregate_replicas(sum(e2e_t) * 1e3, e2e_conv, "cuda")
        e2e = {"value": e2e_all / (e2e_ms * 1e-3), "unit": "eigenpairs/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "t_create_s": statistics.mean(e2e_t) - st2["t_solve_ms"] * 1e-3}

    line = {"metric": METRIC, "value": value,
            "unit": "eigenpairs/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "n": p.n,
                       "nnz": p.nnz, "nev": nev, "m0": m0_of(nev, args.m0), "precision": args.precision,
                       "nonlocal_nnz": nl_nnz,
                       "local_solver": args.local_solver,
                       "iters": st["iters"], "iters_fp64": st["iters_fp64"], "t_factor_ms": st["t_factor_ms"],
                       "nnz_L": st["nnz_L"], "res_max": st["res_max"], "rr_fallbacks": st["rr_fallbacks"],
                       "minres_steps": st["minres_steps"],
                       "l2": "working set > L2 (factor %.0f MB + matrix %.0f MB)" % (st["nnz_L"] * 8e-6, p.nnz * 20e-6),
                       "kappa_S": {"large": 2.2e12, "medium": 1.6e11,
                                   "what": "kappa(D S D), D = diag(S)^-1/2: lambda_max by Lanczos (scipy), lambda_min "
                                           "by an FP64 solve of (D S D) x = lambda x with the library (its factor of D "
                                           "S D as the preconditioner; the 32^3 value matches shift-invert Lanczos)"},
                       "fp64": fp64,
                       "parallelism": "replicas" if ws > 1 else "single"},
            "accuracy": acc,
            "roofline": roof, "e2e": e2e, "gpu_launches": int(sum(s["gpu_launches"] for s in stats)),
            "clocks": ck}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.m0)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
