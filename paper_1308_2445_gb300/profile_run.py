"""Run one LABPSD solve of a named workload through the C ABI, for profilers (ncu).

  python -m paper_1308_2445_gb300.profile_run --workload small|medium|medium-nonlocal [--precision fp64|mixed]
         [--max-outer K] [--solves S]
  python -m paper_1308_2445_gb300.profile_run --update-df64 Q K N

--max-outer is the library's own outer-iteration cap (hbsd_options.max_outer): with a small
value the run is a bounded, representative slice of the solve (factorisation, initial
Rayleigh-Ritz and K full BPSD iterations) that a profiler can capture quickly.

--update-df64 runs only the double-float update of steps 10-11 (hbsd_update_df64) three times on
a seeded N x Q block Z with a Q x K block W scaled by 1/sqrt(Q) (Z(:, 0:K) <- Z W), and prints the
CUDA-event time of each launch (the 64^3 workload reaches Q = 538, K = 282, N = 334,272).
"""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="small", choices=["small", "medium", "medium-nonlocal"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--max-outer", type=int, default=1000)
    ap.add_argument("--solves", type=int, default=1)
    ap.add_argument("--update-df64", type=int, nargs=3, metavar=("Q", "K", "N"))
    a = ap.parse_args()
    if a.update_df64:
        return update_only(*a.update_df64)
    import numpy as np
    from paper_1308_2445_gb300 import build_lib, hbsd, pufe_inputs as pi
    if not os.path.exists(build_lib.LIB):
        build_lib.build()
    p = {"small": pi.small_case, "medium": pi.medium_case, "medium-nonlocal": pi.medium_nonlocal_case}[a.workload](1)
    nev = pi.SMALL_NEV if a.workload == "small" else pi.MEDIUM_NEV
    prec = hbsd.PRECISION_MIXED if a.precision == "mixed" else hbsd.PRECISION_FP64
    s = hbsd.Session.from_problem(p, precision=prec, max_outer=a.max_outer)
    w = nev + s.m0(nev)
    X0 = pi.seed_normal_block(1, p.n, w)
    for _ in range(a.solves):
        lam, X, it, rc, st = s.solve(nev, 1e-8, X0=X0, want_vectors=False)
    print(json.dumps({"workload": a.workload, "n": p.n, "iters": it, "rc": rc, "res_max": st["res_max"],
                      "t_solve_ms": st["t_solve_ms"], "launches": st["gpu_launches"]}))


def update_only(q, k, n):
    import torch
    from paper_1308_2445_gb300 import build_lib, hbsd
    if not os.path.exists(build_lib.LIB):
        build_lib.build()
    g = torch.Generator(device="cuda").manual_seed(1)
    Z = torch.randn(n, q, dtype=torch.float64, device="cuda", generator=g)
    W = torch.randn(q, k, dtype=torch.float64, device="cuda", generator=g) / q ** 0.5
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    for i in range(3):
        ev[i].record()
        hbsd.update_df64(Z, W, k)
        ev[i + 1].record()
    torch.cuda.synchronize()
    ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(3)]
    print(json.dumps({"update_df64": [q, k, n], "ms": ms, "df_fma_per_s": n * q * k / (ms[-1] * 1e-3),
                      "finite": bool(torch.isfinite(Z[:, :k]).all())}))


if __name__ == "__main__":
    main()
