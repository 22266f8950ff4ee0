"""GPU parity of the first-order one-step refinement of step 6(b) (Sec. 6, reading R18) against
the CPU oracle, through the C ABI: the kernel on its own (hbsd_onestep) and whole solves with
local_solver = HBSD_LOCAL_ONESTEP.  Bars as for MINRES: iterates to 1e-6 (the systems have
kappa up to ~1e9), steps within +-1, eigenvalues to 1e-9, outer iterations within +-1.
"""
import json
import os

import numpy as np
import pytest

from oracle import labpsd as L
from paper_1308_2445_gb300 import pufe_inputs as pi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1308_2445_gb300 import build_lib
    if not os.path.exists(build_lib.LIB):
        build_lib.build()


def hb():
    from paper_1308_2445_gb300 import hbsd
    return hbsd


def dbuf(n, k):
    t = torch.zeros(n, k + (k % 2), dtype=torch.float64, device="cuda")
    return t[:, :k]


def dev(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim == 1:
        return torch.from_numpy(a).cuda()
    t = dbuf(a.shape[0], a.shape[1])
    t.copy_(torch.from_numpy(a))
    return t


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def cases():
    return {"mid": pi.generate(12, 2, 4, 0.15, 3), "mid_nl": pi.generate(12, 2, 4, 0.15, 3, n_proj=4),
            "small": pi.small_case(1), "small_nl": pi.generate(8, 2, 2, 0.25, 1, n_proj=4)}


@pytest.mark.parametrize("case", ["mid", "mid_nl"])
def test_onestep_against_oracle(cases, case):
    p = cases[case]
    s = hb().Session.from_problem(p)
    Hs, S, _ = L.make_shifted(p)
    r = L.labpsd(p, 10, 1e-8, seed=3, opts=L.Options(max_outer=6))
    K = L.GlobalPreconditioner(Hs, p.dof_node, p.grid)
    E = r.E_all - r.sigma0
    PH, PS = L.spmm_pair(Hs, S, r.X)
    R, res = L.residual(PH, PS, E, 10)
    P0 = K.apply(R)
    e = E[:10]
    steps = torch.zeros(10, dtype=torch.int32, device="cuda")
    Pd = dbuf(p.n, 10)
    Pd.copy_(dev(P0))
    s.onestep(dev(R), dev(e), Pd, 0.25, 20, steps)
    Pg, sg = host(Pd), host(steps)
    same = 0
    for j in range(10):
        xo, ko, _ = L.refine_one_step(Hs, S, e[j], R[:, j], P0[:, j], 0.25, 20)
        assert abs(int(sg[j]) - ko) <= 1, (j, sg[j], ko)
        if int(sg[j]) == ko:
            same += 1
            assert np.abs(Pg[:, j] - xo).max() <= 1e-6 * np.abs(xo).max()
        rr = np.linalg.norm(Hs @ Pg[:, j] - e[j] * (S @ Pg[:, j]) + R[:, j])
        if int(sg[j]) < 20:
            assert rr <= 0.25 * np.linalg.norm(R[:, j]) * (1 + 1e-6)
    assert same >= 8 and int(sg.sum()) > 0


def test_onestep_full_run_and_ragged_columns(cases):
    """Tight tolerance: every column takes all 20 steps; 37 columns (a ragged pass)."""
    p = cases["mid_nl"]
    s = hb().Session.from_problem(p)
    Hs, S, _ = L.make_shifted(p)
    k = 37
    R = pi.seed_normal_block(12, p.n, k)
    e = np.linspace(0.1, 3.0, k)
    P0 = pi.seed_normal_block(13, p.n, k) * 1e-3
    steps = torch.zeros(k, dtype=torch.int32, device="cuda")
    Pd = dbuf(p.n, k)
    Pd.copy_(dev(P0))
    s.onestep(dev(R), dev(e), Pd, 1e-14, 20, steps)
    Pg = host(Pd)
    assert (host(steps) == 20).all()
    for j in range(k):
        xo, ko, hist = L.refine_one_step(Hs, S, e[j], R[:, j], P0[:, j], 1e-14, 20)
        assert ko == 20
        assert np.abs(Pg[:, j] - xo).max() <= 1e-8 * np.abs(xo).max()


def test_onestep_zero_steps_when_start_meets_tolerance(cases):
    p = cases["mid"]
    s = hb().Session.from_problem(p)
    Hs, S, _ = L.make_shifted(p)
    X = pi.seed_normal_block(3, p.n, 4)
    e = np.array([0.2, 0.5, 1.0, 2.0])
    R = -(Hs @ X - (S @ X) * e[None, :])          # X solves the system exactly
    steps = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    Pd = dbuf(p.n, 4)
    Pd.copy_(dev(X))
    s.onestep(dev(R), dev(e), Pd, 0.25, 20, steps)
    assert (host(steps) == 0).all()
    assert np.array_equal(host(Pd), X)


@pytest.mark.parametrize("case", ["small", "small_nl", "mid"])
def test_solve_with_onestep_refinement(cases, case):
    p = cases[case]
    nev = 16
    X0 = pi.seed_normal_block(4, p.n, nev + L.default_m0(nev))
    s = hb().Session.from_problem(p, local_solver=hb().LOCAL_ONESTEP)
    lam, X, it, rc, st = s.solve(nev, 1e-8, X0=X0)
    ro = L.labpsd(p, nev, 1e-8, X0=X0, opts=L.Options(local_solver="one_step"))
    assert rc == 0 and ro.converged
    assert np.abs(lam - ro.lam).max() <= 1e-9 * np.abs(ro.lam).max()
    assert abs(it - ro.iters) <= 1, (it, ro.iters)
    assert st["local_cols"] > 0 and st["minres_steps"] > 0
    # the trajectories agree to rounding until the refinement (kappa up to ~1e9) amplifies it
    hist = s.res_history()
    assert np.abs(hist[:5] / np.array(ro.res_history[:5]) - 1).max() <= 1e-6


def test_medium_solve_with_onestep_refinement():
    """32^3 workload, mixed form: the eigenpairs of the stored oracle solve (which used MINRES;
    the local solver changes the path, not the answer)."""
    g = json.load(open(os.path.join(HERE, "golden", "medium_seed1.json")))
    p = pi.medium_case(1)
    nev = g["nev"]
    X0 = pi.seed_normal_block(1, p.n, nev + L.default_m0(nev))
    s = hb().Session.from_problem(p, precision=hb().PRECISION_MIXED, local_solver=hb().LOCAL_ONESTEP)
    lam, X, it, rc, st = s.solve(nev, 1e-8, X0=X0)
    ref = np.array(g["lam"])
    assert rc == 0
    assert np.abs(lam - ref).max() <= 1e-9 * np.abs(ref).max()


def test_unknown_local_solver_is_refused(cases):
    with pytest.raises(hb().HbsdError) as e:
        hb().Session.from_problem(cases["small"], local_solver=7)
    assert e.value.code == hb().HBSD_ERR_ARG
