"""Served form (hbsd_server_*): requests of different problems in flight at once on one GPU.

The kernels are deterministic (fixed reduction orders, no atomics in the arithmetic), so a
result computed in the mix must equal, bit for bit, the same solve run alone on a session of
its own; SCF-style follow-ups (new H values on the same pattern, warm start) must equal the
same sequence on a plain session.
"""
import numpy as np
import pytest

from paper_1308_2445_gb300 import pufe_inputs as pi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NEV = 16


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


@pytest.fixture(scope="module")
def problems():
    return [pi.generate(8, 2, 2, 0.25, 1), pi.generate(8, 2, 2, 0.25, 2), pi.generate(10, 3, 2, 0.2, 3),
            pi.generate(8, 2, 2, 0.25, 4)]


def alone(p, nev, X0=None, **opts):
    s = hb().Session.from_problem(p, **opts)
    lam, X, it, rc, st = s.solve(nev, 1e-8, X0=X0)
    s.close()
    return lam, X, it, rc


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_results_same_alone_and_in_the_mix(problems, precision):
    prec = hb().PRECISION_MIXED if precision == "mixed" else hb().PRECISION_FP64
    ref = []
    for i, p in enumerate(problems):
        w = NEV + max(3, -(-NEV // 10))
        X0 = pi.seed_normal_block(10 + i, p.n, w)
        ref.append((X0, alone(p, NEV, X0=X0, precision=prec)))
    sv = hb().Server(max_slots=3)
    # submitted together (and twice each): all in flight on the GPU at once
    tickets = []
    for rep in range(2):
        for p, (X0, _) in zip(problems, ref):
            tickets.append(sv.submit(NEV, 1e-8, problem=p, X0=X0, precision=prec))
    outs = [sv.wait(t) for t in tickets]
    sv.close()
    for k, (res, lam, X) in enumerate(outs):
        lam0, X0v, it0, rc0 = ref[k % len(problems)][1]
        assert res["status"] == 0 and rc0 == 0
        assert res["iters"] == it0
        assert np.array_equal(lam, lam0), (k, np.abs(lam - lam0).max())
        assert np.array_equal(X, X0v)
        assert res["latency_ms"] >= res["run_ms"] >= 0.0 and res["queue_ms"] >= 0.0


def test_scf_follow_ups_match_a_plain_session(problems):
    p = problems[0]
    q1 = pi.generate(8, 2, 2, 0.25, 1, v_noise=0.01, noise_seed=7)
    q2 = pi.generate(8, 2, 2, 0.25, 1, v_noise=0.01, noise_seed=8)
    assert np.array_equal(q1.row_ptr, p.row_ptr) and np.array_equal(q1.col_idx, p.col_idx)
    # plain session: solve, then two follow-ups warm-started with the first factor
    s = hb().Session.from_problem(p)
    lam0, X0v, _, _, _ = s.solve(NEV, 1e-8)
    s.update_H(q1.h_val)
    lam1, X1, _, _, _ = s.solve(NEV, 1e-8, warm=True)
    s.update_H(q2.h_val)
    lam2, X2, _, _, _ = s.solve(NEV, 1e-8, warm=True)
    s.close()
    sv = hb().Server(max_slots=2)
    res, lam, X = sv.wait(sv.submit(NEV, 1e-8, problem=p))
    sid = res["session_id"]
    assert sid >= 0 and np.array_equal(lam, lam0) and np.array_equal(X, X0v)
    res1, la1, Xa1 = sv.wait(sv.submit(NEV, 1e-8, session_id=sid, H_val=q1.h_val, warm=True,
                                       X0=None, want_vectors=False))
    assert res1["status"] == 0 and res1["session_id"] == sid and np.array_equal(la1, lam1)
    res2, la2, _ = sv.wait(sv.submit(NEV, 1e-8, session_id=sid, H_val=q2.h_val, warm=True, want_vectors=False))
    assert res2["status"] == 0 and np.array_equal(la2, lam2)
    sv.release(sid)
    with pytest.raises(hb().HbsdError):
        sv.submit(NEV, 1e-8, session_id=sid, warm=True, want_vectors=False)
    sv.close()


def test_admission_and_errors(problems):
    p = problems[0]
    # a budget smaller than one problem's estimate refuses it at submission
    sv = hb().Server(max_slots=2, hbm_budget_bytes=1 << 20)
    with pytest.raises(hb().HbsdError) as e:
        sv.submit(NEV, 1e-8, problem=p)
    assert e.value.code == hb().HBSD_ERR_OOM
    sv.close()
    # a budget for about one problem at a time: the others wait, then run after eviction
    sv = hb().Server(max_slots=3, hbm_budget_bytes=200 << 20)
    tickets = [sv.submit(NEV, 1e-8, problem=q, want_vectors=False) for q in problems]
    outs = [sv.wait(t) for t in tickets]
    assert all(r["status"] == 0 for r, _, _ in outs)
    with pytest.raises(hb().HbsdError):
        sv.poll(tickets[0])   # a polled ticket is forgotten
    with pytest.raises(hb().HbsdError):
        sv.submit(NEV, 1e-8, session_id=12345, want_vectors=False)
    sv.close()


def test_bloch_requests_in_the_mix():
    """Complex (Bloch) requests at several k-points of the 2 x 2 x 2 grid, in flight together
    with a real one: each result equals, bit for bit, its solve alone on a complex session, and
    a complex SCF follow-up (new H values, warm start) equals the same sequence on a session."""
    kgrid = [(a * 0.5 * np.pi, b * 0.5 * np.pi, c * 0.5 * np.pi) for a in (1, -1) for b in (1, -1) for c in (1, -1)]
    probs = [pi.generate(8, 2, 2, 0.25, 1, kpt=kgrid[0]), pi.generate(8, 2, 2, 0.25, 2, kpt=kgrid[3]),
             pi.generate(8, 2, 2, 0.25, 1), pi.generate(10, 3, 2, 0.2, 3, kpt=kgrid[6])]
    w = NEV + max(3, -(-NEV // 10))
    starts, ref = [], []
    for i, p in enumerate(probs):
        X0 = (pi.seed_normal_block_complex(20 + i, p.n, w) if np.iscomplexobj(p.h_val)
              else pi.seed_normal_block(20 + i, p.n, w))
        starts.append(X0)
        ref.append(alone(p, NEV, X0=X0))
    sv = hb().Server(max_slots=4)
    tickets = [sv.submit(NEV, 1e-8, problem=p, X0=X0) for p, X0 in zip(probs, starts)]
    outs = [sv.wait(t) for t in tickets]
    for k, (res, lam, X) in enumerate(outs):
        lam0, X0v, it0, rc0 = ref[k]
        assert res["status"] == 0 and rc0 == 0 and res["iters"] == it0
        assert np.iscomplexobj(X) == np.iscomplexobj(probs[k].h_val)
        assert np.array_equal(lam, lam0) and np.array_equal(X, X0v)
    # complex follow-up of request 0
    q1 = pi.generate(8, 2, 2, 0.25, 1, kpt=kgrid[0], v_noise=0.01, noise_seed=5)
    sid = outs[0][0]["session_id"]
    t = sv.submit(NEV, 1e-8, session_id=sid, H_val=q1.h_val, warm=True, n=probs[0].n, is_complex=True)
    res, lam_f, X_f = sv.wait(t)
    sv.close()
    s = hb().Session.from_problem(probs[0])
    s.solve(NEV, 1e-8, X0=starts[0])
    s.update_H(q1.h_val)
    lam_s, X_s, it_s, rc_s, _ = s.solve(NEV, 1e-8, warm=True)
    s.close()
    assert res["status"] == 0 and rc_s == 0 and res["iters"] == it_s
    assert np.array_equal(lam_f, lam_s) and np.array_equal(X_f, X_s)
