"""Batched form (hbsd_solve_batch) and the autotuner (hbsd_autotune).

A batch solves independent sessions concurrently, each on its own stream.  The kernels are
deterministic, and tuning fixes a session's launch shapes before its solves, so every result in a
batch must equal, bit for bit, the same tuned session solved alone; one instance is also checked
against the FP64 oracle at the solver's bar (|dlambda| <= 1e-9 max|lambda|, angles at the gaps).
"""
import numpy as np
import pytest

from paper_1308_2445_gb300 import pufe_inputs as pi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1308_2445_gb300 import build_lib
    import os
    if not os.path.exists(build_lib.LIB):
        build_lib.build()


def hb():
    from paper_1308_2445_gb300 import hbsd
    return hbsd


# uneven instances: three mesh sizes, both precision forms, one complex (Bloch) problem
INSTANCES = [
    (lambda: pi.small_case(1), 16, "mixed"),
    (lambda: pi.generate(10, 3, 2, 0.2, 3), 24, "mixed"),
    (lambda: pi.generate(12, 4, 3, 0.15, 5), 32, "mixed"),
    (lambda: pi.generate(8, 2, 2, 0.25, 2), 12, "fp64"),
    (lambda: pi.generate(10, 2, 2, 0.2, 7), 8, "fp64"),
    (lambda: pi.generate(8, 2, 2, 0.25, 4, kpt=(0.5 * np.pi, -0.5 * np.pi, 0.5 * np.pi)), 8, "mixed"),
]


def make_sessions():
    out = []
    for make, nev, form in INSTANCES:
        p = make()
        prec = hb().PRECISION_MIXED if form == "mixed" else hb().PRECISION_FP64
        s = hb().Session.from_problem(p, precision=prec)
        out.append((p, s, nev))
    return out


def start_block(p, s, nev, seed):
    w = nev + s.m0(nev)
    if s.is_complex:   # complex128 tensors: leading dimensions count complex entries
        return torch.from_numpy(np.ascontiguousarray(pi.seed_normal_block_complex(seed, p.n, w))).cuda()
    return torch.from_numpy(pi.seed_normal_block(seed, p.n, w)).cuda()


def buffers(p, s, nev):
    lam = torch.zeros(nev, dtype=torch.float64, device="cuda")
    X = torch.zeros(p.n, nev, dtype=torch.complex128 if s.is_complex else torch.float64, device="cuda")
    return lam, X


@pytest.fixture(scope="module")
def batch_results():
    """Each instance tuned, solved alone, then all solved again in one batch of 3 at a time."""
    sess = make_sessions()
    tunes = [s.autotune(nev) for _, s, nev in sess]
    alone = []
    for i, (p, s, nev) in enumerate(sess):
        X0 = start_block(p, s, nev, 11 + i)
        lam, X = buffers(p, s, nev)
        it, rc, st = s.solve_device(nev, 1e-8, X0, lam, X)
        alone.append((rc, it, lam.cpu().numpy(), X.cpu().numpy()))
    entries, outs = [], []
    for i, (p, s, nev) in enumerate(sess):
        X0 = start_block(p, s, nev, 11 + i)
        lam, X = buffers(p, s, nev)
        entries.append((s, nev, 1e-8, X0, lam, X))
        outs.append((lam, X))
    rc, items = hb().solve_batch(entries, max_concurrent=3)
    torch.cuda.synchronize()
    batched = [(it["status"], it["iters"], lam.cpu().numpy(), X.cpu().numpy()) for it, (lam, X) in zip(items, outs)]
    return sess, tunes, alone, rc, items, batched


def test_batch_equals_alone_bit_for_bit(batch_results):
    sess, tunes, alone, rc, items, batched = batch_results
    assert rc == 0
    for (rca, ita, la, Xa), (rcb, itb, lb, Xb), it in zip(alone, batched, items):
        assert rca == 0 and rcb == 0
        assert ita == itb
        assert np.array_equal(la, lb)
        assert np.array_equal(Xa, Xb)
        assert it["res_max"] <= 1e-8 and it["run_ms"] > 0


def test_batch_instance_against_the_oracle(batch_results):
    """The first instance (the 8^3 small case, mixed form, nev 16) against the FP64 oracle."""
    from oracle import labpsd as L
    sess, tunes, alone, rc, items, batched = batch_results
    p, s, nev = sess[0]
    _, _, lam, X = batched[0]
    X0 = pi.seed_normal_block(11, p.n, nev + s.m0(nev))
    ro = L.labpsd(p, nev, 1e-8, X0=X0)
    assert ro.converged
    scale = np.abs(ro.lam).max()
    assert np.abs(lam - ro.lam).max() <= 1e-9 * scale
    H, S = p.scipy_pair()
    Sd = S.toarray()
    assert np.abs(X.T @ (S @ X) - np.eye(nev)).max() <= 1e-10
    C = np.linalg.cholesky(Sd)
    for j in range(1, nev):
        if ro.lam[j] - ro.lam[j - 1] > 1e-2 * scale:
            qa, _ = np.linalg.qr(C.T @ X[:, :j])
            qb, _ = np.linalg.qr(C.T @ ro.X[:, :j])
            sv = np.linalg.svd(qa.T @ qb, compute_uv=False)
            assert np.arccos(np.clip(sv.min(), -1, 1)) <= 1e-6, j


def test_complex_instance_in_the_batch_is_s_orthonormal(batch_results):
    sess, tunes, alone, rc, items, batched = batch_results
    p, s, nev = sess[5]
    _, _, lam, X = batched[5]
    assert X.dtype == np.complex128
    H, S = p.scipy_pair()
    assert np.abs(X.conj().T @ (S @ X) - np.eye(nev)).max() <= 1e-10
    R = H @ X - (S @ X) * lam[None, :]
    assert (np.linalg.norm(R, axis=0) / np.linalg.norm(H @ X, axis=0)).max() <= 2e-8
    assert np.all(np.diff(lam) >= 0)


def test_autotune_choices(batch_results):
    sess, tunes, alone, rc, items, batched = batch_results
    for (p, s, nev), t in zip(sess, tunes):
        assert t["width"] == s.block_width(nev)
        assert t["spmm_lanes"] in (4, 8, 16, 32)
        assert 1 <= t["minres_ctas"] <= t["minres_ctas_full"]
        if not t["from_table"]:
            assert all(x > 0 for x in t["spmm_ms"])
            assert t["minres_ms"][0] > 0
            fastest = min(x for x in t["minres_ms"] if x > 0)
            k = [i for i in range(6) if t["minres_ms"][i] > 0 and (t["minres_ctas_full"] >> i) == t["minres_ctas"]]
            assert k and t["minres_ms"][k[0]] <= 1.10 * fastest
    # a second session of the same size class takes the table's entry without timing
    p0, s0, nev0 = sess[0]
    s2 = hb().Session.from_problem(p0, precision=hb().PRECISION_MIXED)
    t2 = s2.autotune(nev0)
    assert t2["from_table"] == 1
    assert (t2["spmm_lanes"], t2["minres_ctas"]) == (tunes[0]["spmm_lanes"], tunes[0]["minres_ctas"])


def test_batch_argument_errors():
    hbsd = hb()
    p = pi.small_case(2)
    s = hbsd.Session.from_problem(p)
    lam = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(hbsd.HbsdError) as e:
        hbsd.solve_batch([(s, 16, 1e-8, None, lam, None), (s, 16, 1e-8, None, lam, None)])
    assert e.value.code == hbsd.HBSD_ERR_ARG
    with pytest.raises(hbsd.HbsdError) as e:
        hbsd.solve_batch([(s, 16, 1e-8, None, lam, None)], max_concurrent=0)
    assert e.value.code == hbsd.HBSD_ERR_ARG
    with pytest.raises(hbsd.HbsdError) as e:
        hbsd.check(hbsd.lib().hbsd_autotune(s.h, 0, None), "hbsd_autotune")
    assert e.value.code == hbsd.HBSD_ERR_ARG
    rc, items = hbsd.solve_batch([])
    assert rc == 0 and items == []


def test_mixed_form_escalates_a_stalled_solve_to_fp64_and_converges():
    """An instance of the batched workload (16^3 mesh, 9 atoms, four enrichment functions per node
    within r_c = 0.15, nev 32) on which the double-float products of the mixed form stall near
    Res_max 1e-6 while the FP64 form converges in 23 iterations: the stall rule switches the
    products to FP64 (and, if it stalls again, the Gram and the update), and the solve converges
    to the FP64 form's eigenvalues."""
    hbsd = hb()
    p, nev, _ = pi.batch_instance(pi.batch_spec(1, 64)[14])
    X0 = pi.seed_normal_block(1014, p.n, nev + max(3, -(-nev // 10)))
    sm = hbsd.Session.from_problem(p, precision=hbsd.PRECISION_MIXED)
    lam_m, X, it_m, rc_m, st_m = sm.solve(nev, 1e-8, X0=X0)
    sd = hbsd.Session.from_problem(p, precision=hbsd.PRECISION_FP64)
    lam_d, _, it_d, rc_d, st_d = sd.solve(nev, 1e-8, X0=X0, want_vectors=False)
    assert rc_m == 0 and rc_d == 0
    assert st_m["fp64_from_iter"] >= 10 and st_d["fp64_from_iter"] == -1 and st_d["fp64_gram_from_iter"] == -1
    assert st_m["fp64_gram_from_iter"] == -1 or st_m["fp64_gram_from_iter"] > st_m["fp64_from_iter"]
    assert it_m <= it_d + 30
    assert np.abs(lam_m - lam_d).max() <= 1e-9 * np.abs(lam_d).max()
    H, S = p.scipy_pair()
    R = (H - sm.sigma0 * S) @ X - (S @ X) * (lam_m - sm.sigma0)[None, :]
    assert (np.linalg.norm(R, axis=0) / np.linalg.norm((H - sm.sigma0 * S) @ X, axis=0)).max() <= 1e-8 * 1.001
