#!/usr/bin/env python
"""Benchmark: converged eigenpairs per second (Res_max <= 1e-8) of the LABPSD solve on GB300.

Workload (default): 32^3 periodic Q1 elements, 8 atoms (Z = 4), 4 Gaussian enrichment dofs per
node within r_c = 0.15 (~47.6k dofs), nev = 64, tol = 1e-8, FP64 throughout, hybrid
preconditioner.  A step is one solve (Sec. 3 outline, steps 1-12) from the same seed-normal
start block on a session whose global factor was computed at creation (Sec. 4: once per SCF
run).  `value` is device-timed (CUDA events on the session stream, inputs resident in HBM);
`e2e` times the public host API end to end per step: hbsd_create (H2D of H, S, factorisation)
+ hbsd_solve (H2D of X0, D2H of lambda and X).

Multi-GPU: replicas only -- every rank solves its own instance, no collective on the data
path; value = eigenpairs of all ranks / max-over-ranks time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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
# products of the average launch of the timed solve
MINRES_DRAM_BYTES_PER_COLUMN_PRODUCT = (1212.506368e6 + 438.241536e6) / 156
METRIC = "eigenpairs/s to 1e-8 residual (LABPSD, hybrid preconditioner)"
WORKLOAD = "32^3 periodic Q1 elements, 8 atoms Z=4, 4 Gaussian enrichment dofs/node within r_c=0.15, nev=64, tol=1e-8"
WORKLOAD_NL = WORKLOAD + ", nonlocal F G F^T with s+p projectors per atom (k=32, r_p=0.2)"


def parse():
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
    ap.add_argument("--local-solver", default="minres", choices=["minres", "onestep"],
                    help="step 6(b): MINRES (default) or the first-order one-step refinement (Sec. 6)")
    ap.add_argument("--workload", default="medium", choices=["medium", "medium-nonlocal"],
                    help="medium-nonlocal: the same problem with the nonlocal term H_nl = F G F^T (Sec. 4)")
    ap.add_argument("--m0", type=int, default=-1,
                    help="guard columns (remark 1; default max(3, ceil(nev/10))); the medium workload "
                         "has a stored oracle run for m0 = 21")
    return ap.parse_args()


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


def golden(workload="medium", m0=-1):
    name = "medium_nonlocal_seed1.json" if workload == "medium-nonlocal" else "medium_seed1.json"
    if m0 >= 0:
        name = f"{workload.replace('-', '_')}_m0_{m0}_seed1.json"
    path = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(path):
        raise SystemExit(f"no stored oracle run for workload {workload} with m0 = {m0} "
                         f"(tests/golden/make_golden.py writes one)")
    with open(path) as f:
        return json.load(f)


def m0_of(nev, m0):
    return m0 if m0 >= 0 else max(3, -(-nev // 10))


def problem(workload):
    from paper_1308_2445_gb300 import pufe_inputs as pi
    return pi.medium_nonlocal_case(1) if workload == "medium-nonlocal" else pi.medium_case(1)


def cpu_baseline(nev, W_iters=2, workload="medium", m0=-1):
    """Time the CPU oracle, as it stands, on a bounded sample of the same workload."""
    import numpy as np
    from oracle import labpsd as L
    from paper_1308_2445_gb300 import pufe_inputs as pi
    p = problem(workload)
    g = golden(workload, m0)
    w = nev + m0_of(nev, m0)
    X0 = pi.seed_normal_block(1, p.n, w)
    t0 = time.perf_counter()
    Hs, S, s0 = L.make_shifted(p)
    K = L.GlobalPreconditioner(Hs, p.dof_node, p.grid)
    t_factor = time.perf_counter() - t0
    marks = []
    t1 = time.perf_counter()
    L.labpsd(p, nev, TOL, X0=X0, precond=K, opts=L.Options(max_outer=W_iters, m0=m0_of(nev, m0)),
             on_iteration=lambda it, res: marks.append(time.perf_counter()))
    per_iter = (marks[-1] - marks[0]) / max(1, len(marks) - 1) if len(marks) > 1 else marks[0] - t1
    t_solve = per_iter * g["iters"]
    return {"value": nev / t_solve, "unit": "eigenpairs/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"medium workload: library factorisation ({t_factor:.1f} s, excluded like value's) + initial "
                       f"Rayleigh-Ritz + {W_iters} BPSD iterations ({per_iter:.2f} s each), solve time extrapolated "
                       f"to the oracle's {g['iters']} iterations; numpy/scipy threads = all host cores, the "
                       f"sparse triangular solves single-threaded"),
            "t_factor_s": t_factor, "t_iter_s": per_iter}


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of the GB300s when the peaks file is present, else the
    profiling recipe's fallback figure (said so in the result)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured HBM copy bandwidth (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback HBM figure (6.8 TB/s; no measured peaks file)"


def roofline_object(st, nnz, nl_nnz, peak64, precision, workload):
    """Roofline of the dominant step class, from the solve's CUDA-event step times and the
    algorithmic work per unit.  FP64 classes are bound by the FP64 FMA rate (measured in the same
    run, peak64 in FLOP/s); the FP32 sweeps of the mixed form by HBM (their panels, 4 bytes per
    entry, read once per sweep: 8 nnz(L) bytes per call)."""
    classes = {
        "precond": (st["t_precond_ms"], 4.0 * st["nnz_L"] * st["precond_cols"], st["precond_calls"],
                    "supernodal triangular solves of step 6(a): 2 FMA per factor entry per column"),
        "matvec": (st["t_matvec_ms"], (4.0 * nnz + 4.0 * nl_nnz) * st["matvec_cols"], None,
                   "fused SpMM of steps 3/7: 2 FMA (h and s) per nonzero per column"
                   + (" + 2 FMA per F entry (F^T X and F Z)" if nl_nnz else "")),
        "minres": (st["t_local_ms"], (4.0 * nnz + 4.0 * nl_nnz) * st["minres_spmm_cols"], None,
                   "MINRES of step 6(b): shifted fused SpMM, 2 FMA per nonzero per column"
                   + (" + 2 FMA per F entry" if nl_nnz else "")),
    }
    dom = max(classes, key=lambda k: classes[k][0])
    t_ms, flops, _, what = classes[dom]
    step_ms = {k: st[f"t_{k}_ms"] for k in ("matvec", "resid", "precond", "local", "gram", "rr", "update")}
    if dom == "precond" and precision == "mixed":
        peak, source = hbm_peak_gbs()
        achieved = 8.0 * st["nnz_L"] * st["precond_calls"] / (t_ms * 1e-3) / 1e9 if t_ms > 0 else 0.0
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": dom,
                "what": "FP32 supernodal sweeps of step 6(a): the FP32 panels read once per sweep, 8 nnz(L) bytes per call",
                "peak_source": source, "step_ms": step_ms}
    achieved = flops / (t_ms * 1e-3) / 1e12 if t_ms > 0 else 0.0
    traffic = None
    if dom == "minres" and st["local_calls"] > 0 and workload == "medium":
        traffic = MINRES_DRAM_BYTES_PER_COLUMN_PRODUCT * st["minres_spmm_cols"] / st["local_calls"]
    return {"bound": "alu", "achieved": achieved, "peak": peak64 / 1e12, "unit": "TFLOP/s",
            "frac": achieved / (peak64 / 1e12) if peak64 > 0 else None, "traffic": traffic,
            "traffic_note": "DRAM bytes per launch: ncu bytes per column product x the average launch's column products"
            if traffic is not None else None,
            "kernel": dom, "what": what, "peak_source": "FP64 FMA probe (hbsd_probe_peak) measured in this run",
            "step_ms": step_ms}


def run_reference(args):
    ws, rank, _ = dist()
    if rank != 0:
        return
    from oracle import labpsd as L
    from paper_1308_2445_gb300 import pufe_inputs as pi
    nev = pi.MEDIUM_NEV
    p = problem(args.workload)
    g = golden(args.workload, args.m0)
    m0 = m0_of(nev, args.m0)
    X0 = pi.seed_normal_block(1, p.n, nev + m0)
    Hs, S, s0 = L.make_shifted(p)
    K = L.GlobalPreconditioner(Hs, p.dof_node, p.grid)
    marks = [time.perf_counter()]
    L.labpsd(p, nev, TOL, X0=X0, precond=K, opts=L.Options(max_outer=args.warmup + args.steps, m0=m0),
             on_iteration=lambda it, res: marks.append(time.perf_counter()))
    d = [marks[i + 1] - marks[i] for i in range(len(marks) - 1)]
    timed = d[args.warmup:] or d
    per_iter = sum(timed) / len(timed)
    value = nev / (per_iter * g["iters"])
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "eigenpairs/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_iter * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NL if args.workload == "medium-nonlocal" else WORKLOAD, "n": p.n,
                       "nnz": p.nnz, "nev": nev, "m0": m0, "arithmetic": "fp64 (the CPU oracle)",
                       "step": "one BPSD iteration of the CPU oracle; value scaled to the oracle's full solve"},
            "cpu_baseline": {"value": value, "unit": "eigenpairs/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{len(timed)} timed BPSD iterations after {args.warmup} warm-up, "
                                       f"solve extrapolated to {g['iters']} iterations"},
            "e2e": {"value": value, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
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

    nev = pi.MEDIUM_NEV
    p = problem(args.workload)
    nl_nnz = int(np.count_nonzero(p.F)) if p.F is not None else 0
    w = nev + m0_of(nev, args.m0)
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    prec = hbsd.PRECISION_MIXED if args.precision == "mixed" else hbsd.PRECISION_FP64
    lsol = hbsd.LOCAL_ONESTEP if args.local_solver == "onestep" else hbsd.LOCAL_MINRES
    sess = hbsd.Session.from_problem(p, stream=stream.cuda_stream, precision=prec, local_solver=lsol, m0=args.m0)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    X0h = torch.from_numpy(pi.seed_normal_block(1, p.n, w)).pin_memory()
    X0 = torch.zeros(p.n, w + (w % 2), dtype=torch.float64, device="cuda")[:, :w]
    X0.copy_(X0h)
    lam = torch.zeros(nev, dtype=torch.float64, device="cuda")
    X = torch.zeros(p.n, nev, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        it, rc, st = sess.solve_device(nev, TOL, X0, lam, X)
    # timed region
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    converged = 0
    stats = []
    for _ in range(args.steps):
        it, rc, st = sess.solve_device(nev, TOL, X0, lam, X)
        stats.append(st)
        if rc == 0 and st["res_max"] <= TOL:
            converged += nev
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms, converged = aggregate_replicas(ms, converged, "cuda")
    value = converged / (ms * 1e-3)
    st = stats[-1]

    # ---- end to end through the public host API ----------------------------------------
    rp = np.ascontiguousarray(p.row_ptr)
    h2d = rp.nbytes + p.col_idx.nbytes + p.h_val.nbytes + p.s_val.nbytes + p.dof_node.nbytes + p.n * w * 8
    if p.F is not None:
        h2d += p.F.nbytes + p.G.nbytes
    d2h = nev * 8 + p.n * nev * 8
    X0n = pi.seed_normal_block(1, p.n, w)
    e2e_t = []
    e2e_conv = 0
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

    # ---- roofline of the dominant step class (device time from the solve's CUDA events) ----
    peak64 = hbsd.probe_peak(0, stream.cuda_stream)
    roof = roofline_object(st, p.nnz, nl_nnz, peak64, args.precision, args.workload)

    line = {"metric": METRIC, "value": value,
            "unit": "eigenpairs/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NL if args.workload == "medium-nonlocal" else WORKLOAD, "n": p.n,
                       "nnz": p.nnz, "nev": nev, "m0": m0_of(nev, args.m0), "precision": args.precision,
                       "nonlocal_nnz": nl_nnz,
                       "local_solver": args.local_solver,
                       "iters": st["iters"], "iters_fp64": st["iters_fp64"], "t_factor_ms": st["t_factor_ms"],
                       "nnz_L": st["nnz_L"], "res_max": st["res_max"], "rr_fallbacks": st["rr_fallbacks"],
                       "minres_steps": st["minres_steps"],
                       "l2": "working set > L2 (factor %.0f MB + matrix %.0f MB)" % (st["nnz_L"] * 8e-6, p.nnz * 20e-6),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "roofline": roof, "e2e": e2e, "gpu_launches": int(sum(s["gpu_launches"] for s in stats)),
            "clocks": ck}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(nev, workload=args.workload, m0=args.m0)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
