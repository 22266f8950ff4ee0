"""Batched-form benchmark: many independent instances of uneven size solved by hbsd_solve_batch.

  python -m paper_1308_2445_gb300.batch_bench [--count 64] [--seed 1] [--concurrent 8]
         [--steps 1] [--warmup 1] [--arms batched,one_at_a_time,fp64] [--meshes 16,24,32,40]

Workload (synthetic, seeded): pufe_inputs.batch_spec(seed, count) -- per instance a periodic
mesh from {16^3, 24^3, 32^3, 40^3}, 4-16 atoms (Z = 4) at seed positions, 2-4 enrichment dofs per
node within r_c = 0.15, nev from {32, 64, 128}; real FP64 matrices on input, solved in the mixed
form to Res_max <= 1e-8 from seed-normal start blocks.

Not timed: generating the instances (a spawn process pool), one session per instance (upload,
SELL-C-sigma, factorisation: hbsd_create), start blocks on the device, and the autotuner (timed on
its own and reported).  Timed: K batch calls after W warm-up calls, each solving every instance
from its start block; wall clock between two device synchronisations, since the solves run on
many streams.  Arms:
  batched        hbsd_solve_batch, `concurrent` sessions at a time, tuned launch shapes
  one_at_a_time  the same tuned sessions, one at a time (results checked bit for bit against the
                 batched arm)
  untuned        fresh mixed sessions with the built-in launch shapes (no autotuner), batched
  fp64           FP64 sessions of the same instances (plain FP64 BSD), batched the same way
e2e: the batched arm with each instance's start block copied from pinned host memory and its
eigenvalues read back inside the timed region.

Prints one JSON line (value: converged eigenpairs per second of the batched arm).
"""
import argparse
import concurrent.futures as cf
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _instance(spec):
    from paper_1308_2445_gb300 import pufe_inputs as pi
    return pi.batch_instance(spec)


def generate(specs, workers=None):
    """The instances of `specs`, generated in a spawn process pool (no CUDA in the children)."""
    workers = workers or min(len(specs), os.cpu_count() or 1, 16)
    if workers <= 1:
        return [_instance(s) for s in specs]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_instance, specs))


def add_args(ap):
    ap.add_argument("--count", type=int, default=64)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--concurrent", type=int, default=8)
    ap.add_argument("--arms", default="batched,one_at_a_time,fp64")
    ap.add_argument("--meshes", default="16,24,32,40")
    ap.add_argument("--tol", type=float, default=1e-8)


def run(a, steps=1, warmup=1, log=None, clocks=None, keep=None):
    """Runs the arms; returns the result dict.  clocks: an object with start() and stop() -> dict,
    sampled around the batched arm's timed calls."""
    import torch
    from paper_1308_2445_gb300 import build_lib, hbsd, pufe_inputs as pi
    if not os.path.exists(build_lib.LIB):
        build_lib.build()
    say = log or (lambda *x: None)
    meshes = tuple(int(x) for x in a.meshes.split(","))
    specs = pi.batch_spec(a.seed, a.count, meshes=meshes)
    t = time.perf_counter()
    inst = generate(specs)
    t_gen = time.perf_counter() - t
    if keep is not None:
        keep["inst"] = inst
    say(f"generated {len(inst)} instances in {t_gen:.1f} s")
    arms = [x for x in a.arms.split(",") if x]
    out = {"count": len(inst), "concurrent": a.concurrent, "t_generate_s": t_gen,
           "instances": {"n": [p.n for p, _, _ in inst], "nnz": [p.nnz for p, _, _ in inst],
                         "nev": [nev for _, nev, _ in inst], "mesh": [s[0] for s in specs],
                         "atoms": [at for _, _, at in inst]}}
    total_nev = sum(nev for _, nev, _ in inst)

    def sessions(precision):
        t0 = time.perf_counter()
        ss = [hbsd.Session.from_problem(p, precision=precision) for p, _, _ in inst]
        torch.cuda.synchronize()
        return ss, time.perf_counter() - t0

    def blocks(ss):
        X0, lam = [], []
        for i, ((p, nev, _), s) in enumerate(zip(inst, ss)):
            X0.append(torch.from_numpy(pi.seed_normal_block(a.seed * 1000 + i, p.n, nev + s.m0(nev))).cuda())
            lam.append(torch.zeros(nev, dtype=torch.float64, device="cuda"))
        return X0, lam

    def timed(ss, X0, lam, concurrent, tune, k, w, ck=None):
        entries = [(s, nev, a.tol, x, l, None) for (p, nev, _), s, x, l in zip(inst, ss, X0, lam)]
        for _ in range(w):
            hbsd.solve_batch(entries, max_concurrent=concurrent, autotune=tune)
        walls, items = [], None
        if ck is not None:
            ck.start()
        for _ in range(k):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, items = hbsd.solve_batch(entries, max_concurrent=concurrent, autotune=tune)
            torch.cuda.synchronize()
            walls.append(time.perf_counter() - t0)
        if ck is not None:
            out["clocks"] = ck.stop()
        conv = sum(nev for (p, nev, _), it in zip(inst, items) if it["status"] == 0 and it["res_max"] <= a.tol)
        return walls, items, conv

    def summary(walls, items, conv):
        wall = float(np.median(walls))
        return {"eigenpairs_per_s": conv / wall, "wall_s": wall, "walls_s": walls, "converged_eigenpairs": conv,
                "failed": int(sum(1 for it in items if it["status"] != 0)),
                "iters": [it["iters"] for it in items], "run_ms": [round(it["run_ms"], 2) for it in items]}

    if "batched" in arms or "one_at_a_time" in arms:
        ss, t_create = sessions(hbsd.PRECISION_MIXED)
        say(f"created {len(ss)} mixed sessions in {t_create:.1f} s")
        out["t_create_mixed_s"] = t_create
        t0 = time.perf_counter()
        tunes = [s.autotune(nev) for (p, nev, _), s in zip(inst, ss)]
        torch.cuda.synchronize()
        out["t_autotune_s"] = time.perf_counter() - t0
        out["tune"] = {"spmm_lanes": [t["spmm_lanes"] for t in tunes], "minres_ctas": [t["minres_ctas"] for t in tunes],
                       "minres_ctas_full": tunes[0]["minres_ctas_full"],
                       "timed_classes": int(sum(1 for t in tunes if not t["from_table"]))}
        X0, lam = blocks(ss)
        lam_b = None
        if "batched" in arms:
            walls, items, conv = timed(ss, X0, lam, a.concurrent, True, steps, warmup, clocks)
            out["batched"] = summary(walls, items, conv)
            # kernels of the last timed call (each session's own count of its last solve)
            out["batched"]["gpu_launches_per_call"] = int(sum(s.stats()["gpu_launches"] for s in ss))
            lam_b = [l.cpu().numpy().copy() for l in lam]
            say(f"batched: {out['batched']['eigenpairs_per_s']:.1f} eigenpairs/s, {out['batched']['wall_s']:.2f} s")
            # e2e: start blocks from pinned host memory in, eigenvalues out, inside the timed region
            hX0 = [x.cpu().pin_memory() for x in X0]
            hlam = [torch.empty(l.shape, dtype=torch.float64).pin_memory() for l in lam]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for h, d in zip(hX0, X0):
                d.copy_(h, non_blocking=True)
            torch.cuda.synchronize()
            entries = [(s, nev, a.tol, x, l, None) for (p, nev, _), s, x, l in zip(inst, ss, X0, lam)]
            rc, items_e = hbsd.solve_batch(entries, max_concurrent=a.concurrent)
            for h, d in zip(hlam, lam):
                h.copy_(d, non_blocking=True)
            torch.cuda.synchronize()
            we = time.perf_counter() - t0
            conv_e = sum(nev for (p, nev, _), it in zip(inst, items_e) if it["status"] == 0 and it["res_max"] <= a.tol)
            out["e2e"] = {"value": conv_e / we, "unit": "eigenpairs/s",
                          "h2d_bytes_per_step": int(sum(x.numel() * 8 for x in X0)),
                          "d2h_bytes_per_step": int(sum(l.numel() * 8 for l in lam))}
        if "one_at_a_time" in arms:
            walls, items, conv = timed(ss, X0, lam, 1, True, 1, 0)
            out["one_at_a_time"] = summary(walls, items, conv)
            if lam_b is not None:
                out["one_at_a_time"]["bitwise_equal_to_batched"] = bool(
                    all(np.array_equal(x, l.cpu().numpy()) for x, l in zip(lam_b, lam)))
            say(f"one at a time: {out['one_at_a_time']['eigenpairs_per_s']:.1f} eigenpairs/s")
        for s in ss:
            s.close()
        del ss, X0, lam
        torch.cuda.empty_cache()
    if "untuned" in arms:
        # fresh sessions, built-in launch shapes (no autotuner), batched the same way
        ss, t_create = sessions(hbsd.PRECISION_MIXED)
        X0, lam = blocks(ss)
        walls, items, conv = timed(ss, X0, lam, a.concurrent, False, 1, 0)
        out["untuned"] = summary(walls, items, conv)
        say(f"untuned batched: {out['untuned']['eigenpairs_per_s']:.1f} eigenpairs/s")
        for s in ss:
            s.close()
        del ss, X0, lam
        torch.cuda.empty_cache()
    if "fp64" in arms:
        ss, t_create = sessions(hbsd.PRECISION_FP64)
        out["t_create_fp64_s"] = t_create
        X0, lam = blocks(ss)
        walls, items, conv = timed(ss, X0, lam, a.concurrent, True, 1, 0)
        out["fp64"] = summary(walls, items, conv)
        say(f"fp64 batched: {out['fp64']['eigenpairs_per_s']:.1f} eigenpairs/s")
        for s in ss:
            s.close()
    out["total_nev"] = total_nev
    return out


def main():
    ap = argparse.ArgumentParser()
    add_args(ap)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=1)
    a = ap.parse_args()
    res = run(a, a.steps, a.warmup, log=lambda *x: print(*x, file=sys.stderr, flush=True))
    res["metric"] = "converged eigenpairs/s, batched form (independent uneven instances, one GPU)"
    res["data"] = "synthetic"
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
