"""Write the stored expected values of the GPU parity tests by running the CPU oracle only.

  python tests/golden/make_golden.py medium            -> tests/golden/medium_seed1.json
  python tests/golden/make_golden.py medium_nonlocal   -> tests/golden/medium_nonlocal_seed1.json
  python tests/golden/make_golden.py medium_m0 21      -> tests/golden/medium_m0_21_seed1.json
                                                          (the same solve with m0 = 21 guard columns)
  python tests/golden/make_golden.py medium_nonlocal_m0 21
                                                       -> tests/golden/medium_nonlocal_m0_21_seed1.json
  python tests/golden/make_golden.py large             -> tests/golden/large_seed1.json
                                                          (64^3, 32 atoms, nev = 256: hours of host time,
                                                          most of it the library sparse LU)

The medium workload (32^3 Q1 elements, 8 atoms, 4 enrichment dofs per node, nev = 64) takes the
oracle a few minutes, too long to rerun inside the test suite; every value in the file comes
from oracle/labpsd.py on inputs of paper_1308_2445_gb300/pufe_inputs.py.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import labpsd as L  # noqa: E402
from paper_1308_2445_gb300 import pufe_inputs as pi  # noqa: E402


def medium(seed=1, nonlocal_term=False, m0=-1):
    p = pi.medium_nonlocal_case(seed) if nonlocal_term else pi.medium_case(seed)
    t0 = time.time()
    r = L.labpsd(p, pi.MEDIUM_NEV, 1e-8, seed=seed, opts=L.Options(m0=None if m0 < 0 else m0))
    name = "32^3 Q1, 8 atoms, 4 enrichment dofs/node, r_c 0.15"
    if nonlocal_term:
        name += ", s+p projectors per atom (k = 32)"
    return dict(workload=name, seed=seed, n=p.n, nnz=p.nnz,
                nev=pi.MEDIUM_NEV, tol=1e-8, eps_bar=p.eps_bar, lam=[float(x) for x in r.lam],
                E_all=[float(x) for x in r.E_all], iters=r.iters, converged=bool(r.converged),
                res_history=[float(x) for x in r.res_history], minres_total=int(sum(int(s.sum()) for s in r.minres_steps)),
                rr_fallbacks=r.rr_fallbacks, m0=m0 if m0 >= 0 else L.default_m0(pi.MEDIUM_NEV),
                oracle_seconds=time.time() - t0)


def large(seed=1):
    """The 64^3 workload (32 atoms, 4 enrichment dofs per node, r_c 0.08, nev = 256) with the
    default m0; progress to stderr after every outer iteration."""
    p = pi.large_case(seed)
    nev = pi.LARGE_NEV
    t0 = time.time()
    Hs, S, s0 = L.make_shifted(p)
    K = L.GlobalPreconditioner(Hs, p.dof_node, p.grid)
    t_factor = time.time() - t0
    sys.stderr.write(f"factorisation {t_factor:.0f} s\n")
    sys.stderr.flush()
    t1 = time.time()

    def progress(it, res):
        sys.stderr.write(f"iteration {it}: Res_max {res.max():.3e} at {time.time() - t1:.0f} s\n")
        sys.stderr.flush()
    r = L.labpsd(p, nev, 1e-8, seed=seed, precond=K, on_iteration=progress)
    return dict(workload="64^3 Q1, 32 atoms, 4 enrichment dofs/node, r_c 0.08", seed=seed, n=p.n, nnz=p.nnz,
                nev=nev, tol=1e-8, eps_bar=p.eps_bar, lam=[float(x) for x in r.lam],
                E_all=[float(x) for x in r.E_all], iters=r.iters, converged=bool(r.converged),
                res_history=[float(x) for x in r.res_history],
                minres_total=int(sum(int(s.sum()) for s in r.minres_steps)), rr_fallbacks=r.rr_fallbacks,
                m0=L.default_m0(nev), oracle_seconds=time.time() - t1, factor_seconds=t_factor,
                nnz_L=int(K.lu.L.nnz))


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "medium"
    if which in ("medium", "medium_nonlocal"):
        out = medium(1, nonlocal_term=which == "medium_nonlocal")
        with open(os.path.join(HERE, f"{which}_seed1.json"), "w") as f:
            json.dump(out, f, indent=1)
        print("iters", out["iters"], "seconds", out["oracle_seconds"])
    elif which == "large":
        out = large(1)
        with open(os.path.join(HERE, "large_seed1.json"), "w") as f:
            json.dump(out, f, indent=1)
        print("iters", out["iters"], "seconds", out["oracle_seconds"])
    elif which in ("medium_m0", "medium_nonlocal_m0"):
        m0 = int(sys.argv[2])
        out = medium(1, nonlocal_term=which == "medium_nonlocal_m0", m0=m0)
        with open(os.path.join(HERE, f"{which}_{m0}_seed1.json"), "w") as f:
            json.dump(out, f, indent=1)
        print("iters", out["iters"], "seconds", out["oracle_seconds"])
