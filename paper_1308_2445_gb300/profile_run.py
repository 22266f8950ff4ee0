"""Run one LABPSD solve of a named workload through the C ABI, for profilers (ncu).

  python -m paper_1308_2445_gb300.profile_run --workload small|medium|medium-nonlocal [--precision fp64|mixed]
         [--max-outer K] [--solves S]
  python -m paper_1308_2445_gb300.profile_run --update-df64 Q K N
  python -m paper_1308_2445_gb300.profile_run --update-oz Q0 Q1 K N
  python -m paper_1308_2445_gb300.profile_run --workload medium --sweep32 K
  python -m paper_1308_2445_gb300.profile_run --workload medium --spmm K

--max-outer is the library's own outer-iteration cap (hbsd_options.max_outer): with a small
value the run is a bounded, representative slice of the solve (factorisation, initial
Rayleigh-Ritz and K full BPSD iterations) that a profiler can capture quickly.

--update-df64 runs only the double-float update of steps 10-11 (hbsd_update_df64) three times on
a seeded N x Q block Z with a Q x K block W scaled by 1/sqrt(Q) (Z(:, 0:K) <- Z W), and prints the
CUDA-event time of each launch (the 64^3 workload reaches Q = 538, K = 282, N = 334,272).

--update-oz does the same for the tensor-core update (hbsd_update_oz) with blocks of Q0 and Q1
columns (the Psi and P blocks of the solve).

--sweep32 K runs step 6(a) of the mixed form (hbsd_precond_apply_f32, the FP32 supernodal sweeps)
three times on a seeded K-column block of the workload's scaled pencil; --spmm K runs the fused SpMM
of steps 3/7 three times in FP64 (hbsd_spmm_pair), then three times in double-float on the scaled
pencil (hbsd_spmm_pair_df64), on K columns.  Both print the CUDA-event times.
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
    ap.add_argument("--workload", default="small", choices=["small", "medium", "medium-nonlocal", "large"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--max-outer", type=int, default=1000)
    ap.add_argument("--solves", type=int, default=1)
    ap.add_argument("--update-df64", type=int, nargs=3, metavar=("Q", "K", "N"))
    ap.add_argument("--update-oz", type=int, nargs=4, metavar=("Q0", "Q1", "K", "N"))
    ap.add_argument("--sweep32", type=int, metavar="K")
    ap.add_argument("--spmm", type=int, metavar="K")
    a = ap.parse_args()
    if a.update_df64:
        return update_only(*a.update_df64)
    if a.update_oz:
        return update_oz_only(*a.update_oz)
    if a.sweep32 or a.spmm:
        return step_only(a.workload, a.sweep32, a.spmm)
    import numpy as np
    from paper_1308_2445_gb300 import build_lib, hbsd, pufe_inputs as pi
    if not os.path.exists(build_lib.LIB):
        build_lib.build()
    p = {"small": pi.small_case, "medium": pi.medium_case, "medium-nonlocal": pi.medium_nonlocal_case,
         "large": pi.large_case}[a.workload](1)
    nev = {"small": pi.SMALL_NEV, "large": pi.LARGE_NEV}.get(a.workload, pi.MEDIUM_NEV)
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


def timed(fn, reps=3):
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    torch.cuda.synchronize()
    for i in range(reps):
        ev[i].record()
        fn()
        ev[i + 1].record()
    torch.cuda.synchronize()
    return [ev[i].elapsed_time(ev[i + 1]) for i in range(reps)]


def update_oz_only(q0, q1, k, n):
    import torch
    from paper_1308_2445_gb300 import build_lib, hbsd
    if not os.path.exists(build_lib.LIB):
        build_lib.build()
    g = torch.Generator(device="cuda").manual_seed(1)
    Z0 = torch.randn(n, q0 + q0 % 2, dtype=torch.float64, device="cuda", generator=g)[:, :q0]
    Z1 = torch.randn(n, max(q1, 1) + q1 % 2, dtype=torch.float64, device="cuda", generator=g)[:, :q1]
    W = torch.randn(q0 + q1, k, dtype=torch.float64, device="cuda", generator=g) / (q0 + q1) ** 0.5
    Y = torch.zeros(n, k + k % 2, dtype=torch.float64, device="cuda")[:, :k]

    def run():
        hbsd.check(hbsd.lib().hbsd_update_oz(Z0.data_ptr(), Z0.stride(0), q0, Z1.data_ptr(), Z1.stride(0), q1, n,
                                             W.data_ptr(), k, Y.data_ptr(), Y.stride(0), None), "hbsd_update_oz")
    ms = timed(run)
    print(json.dumps({"update_oz": [q0, q1, k, n], "ms": ms, "fma_per_s": n * (q0 + q1) * k / (ms[-1] * 1e-3)}))


def step_only(workload, k_sweep, k_spmm):
    import torch
    from paper_1308_2445_gb300 import build_lib, hbsd, pufe_inputs as pi
    if not os.path.exists(build_lib.LIB):
        build_lib.build()
    p = {"small": pi.small_case, "medium": pi.medium_case, "medium-nonlocal": pi.medium_nonlocal_case,
         "large": pi.large_case}[workload](1)
    s = hbsd.Session.from_problem(p, precision=hbsd.PRECISION_MIXED)
    out = {"workload": workload, "n": p.n, "nnz": p.nnz}
    if k_sweep:
        R = torch.randn(p.n, (k_sweep + 3) // 4 * 4, dtype=torch.float32, device="cuda")[:, :k_sweep]
        P = torch.zeros(p.n, (k_sweep + 3) // 4 * 4, dtype=torch.float32, device="cuda")[:, :k_sweep]
        out["sweep32_k"] = k_sweep
        out["sweep32_ms"] = timed(lambda: s.precond_apply_f32(R, P))
        out["nnz_L"] = s.stats()["nnz_L"]
    if k_spmm:
        X = torch.randn(p.n, k_spmm + k_spmm % 2, dtype=torch.float64, device="cuda")[:, :k_spmm]
        HX, SX = [torch.zeros(p.n, k_spmm + k_spmm % 2, dtype=torch.float64, device="cuda")[:, :k_spmm]
                  for _ in range(2)]
        out["spmm_k"] = k_spmm
        out["spmm_ms"] = timed(lambda: s.spmm_pair(X, HX, SX))
        out["spmm_df64_ms"] = timed(lambda: s.spmm_pair_df64(X, HX, SX))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
