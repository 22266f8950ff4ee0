"""Pins of the CPU oracle to facts that do not come from the oracle itself:
closed forms, brute-force dense solves, invariants, special cases.  Planted-mistake
tests at the end show that plausible slips in the oracle fail one of these pins."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import labpsd as L
from paper_1308_2445_gb300 import pufe_inputs as pi


def _angles(A, B, M=None):
    """Largest principal angle between span(A) and span(B) (M-inner product if given)."""
    if M is not None:
        C = np.linalg.cholesky(M)
        A, B = C.T @ A, C.T @ B
    qa, _ = np.linalg.qr(A)
    qb, _ = np.linalg.qr(B)
    s = np.linalg.svd(qa.conj().T @ qb, compute_uv=False)
    return float(np.arccos(np.clip(s.min(), -1.0, 1.0)))


# ------------------------------------------------------------------ closed form
@pytest.mark.parametrize("nev", [7, 19, 27])
def test_closed_form_eigenvalues(nev):
    # unenriched periodic Q1, constant V = 0.3: lambda = 0.3 + sum_d 3(1-cos t)/(h^2(2+cos t))
    q = pi.generate(6, 0, 0, 0.1, 1, v0=0.3)
    r = L.labpsd(q, nev, 1e-10, seed=2)
    ref = pi.closed_form_eigenvalues(6, 0.3)[:nev]
    assert r.converged
    assert np.abs(r.lam - ref).max() <= 1e-10 * np.abs(ref).max()


def test_spmm_pair_on_fourier_modes():
    # Steps 3 and 7 on the unenriched pair with V = v0: a discrete Fourier mode
    # x(i, j, k) = c_a(i) c_b(j) c_c(k) with c_a(i) = cos(2 pi a i / N) is an exact eigenvector, so
    # the two products of spmm_pair satisfy Hs x = (lambda - sigma0) S x, lambda = v0 plus the
    # 1-D linear-element symbol 3 (1 - cos t) / (h^2 (2 + cos t)) summed over the three wavenumbers
    N, v0 = 6, 0.3
    q = pi.generate(N, 0, 0, 0.1, 1, v0=v0)
    Hs, S, sigma0 = L.make_shifted(q)
    i = np.arange(N ** 3)
    ijk = (i % N, (i // N) % N, i // (N * N))
    h = 1.0 / N
    sym = lambda a: 3.0 * (1.0 - math.cos(2 * math.pi * a / N)) / (h * h * (2.0 + math.cos(2 * math.pi * a / N)))
    waves = [(1, 1, 1), (1, 2, 0), (3, 0, 2), (0, 0, 0)]
    X = np.stack([np.prod([np.cos(2 * math.pi * w[d] * ijk[d] / N) for d in range(3)], axis=0) for w in waves], 1)
    lam = np.array([v0 + sum(sym(a) for a in w) for w in waves])
    HX, SX = L.spmm_pair(Hs, S, X)
    assert np.abs(SX).max() > 0.0
    for j in range(len(waves)):
        assert np.abs(HX[:, j] - (lam[j] - sigma0) * SX[:, j]).max() <= 1e-12 * np.abs(HX[:, j]).max() + 1e-13
    # the shift: sigma0 = eps_bar, and the constant mode carries only the potential
    assert sigma0 == q.eps_bar
    assert np.allclose(HX[:, 3], (v0 - sigma0) * SX[:, 3], rtol=1e-10, atol=0)   # row sums of K round


def test_closed_form_cluster_subspace():
    # the 6-fold cluster of the 6^3 mesh is spanned by the sampled cos/sin(2 pi x_d) modes
    N = 6
    q = pi.generate(N, 0, 0, 0.1, 1, v0=0.3)
    r = L.labpsd(q, 7, 1e-10, seed=3)
    i = np.arange(N ** 3)
    x = np.stack([i % N, (i // N) % N, i // (N * N)], axis=1) / N
    modes = np.concatenate([np.cos(2 * np.pi * x), np.sin(2 * np.pi * x)], axis=1)
    assert _angles(r.X[:, 1:7], modes) < 1e-6
    assert _angles(r.X[:, :1], np.ones((N ** 3, 1))) < 1e-6


def test_closed_form_bloch_complex():
    k = (0.5 * np.pi, -0.5 * np.pi, 0.5 * np.pi)
    q = pi.generate(5, 0, 0, 0.1, 1, v0=0.3, kpt=k)
    X0 = pi.seed_normal_block(4, q.n, 8) + 1j * pi.seed_normal_block(5, q.n, 8)
    r = L.labpsd(q, 5, 1e-10, X0=X0)
    ref = pi.closed_form_eigenvalues(5, 0.3, k)[:5]
    assert r.converged and np.iscomplexobj(r.X)
    assert np.abs(r.lam - ref).max() <= 1e-10 * np.abs(ref).max()


def test_complex_oracle_agrees_with_the_real_equivalent_pencil():
    # H = Hr + i Hi, S = Sr + i Si Hermitian is equivalent to the real symmetric pencil
    # ([Hr, -Hi; Hi, Hr], [Sr, -Si; Si, Sr]) of size 2n, every eigenvalue twice (x and i x): the
    # oracle's complex solve must agree with its real solve of that pencil (a missing conjugate
    # anywhere in the complex path breaks it), and the complex span of V[:n] + i V[n:] over the
    # 2 nev real vectors must have dimension nev and hold the complex eigenvectors
    import dataclasses
    import scipy.sparse as sp
    k = (0.5 * np.pi, -0.5 * np.pi, 0.5 * np.pi)
    q = pi.generate(8, 2, 2, 0.25, 1, kpt=k)
    nev = 16
    w = nev + L.default_m0(nev)
    rc = L.labpsd(q, nev, 1e-8, X0=pi.seed_normal_block(4, q.n, w) + 1j * pi.seed_normal_block(5, q.n, w))
    H, S = q.scipy_pair()

    def blocks(A):
        Ar = sp.csr_matrix((A.data.real.copy(), A.indices, A.indptr), shape=A.shape)
        Ai = sp.csr_matrix((A.data.imag.copy(), A.indices, A.indptr), shape=A.shape)
        B = sp.bmat([[Ar, -Ai], [Ai, Ar]], format="csr")
        B.sort_indices()
        return B
    Hb, Sb = blocks(H.tocsr()), blocks(S.tocsr())
    assert np.array_equal(Hb.indices, Sb.indices) and abs(Hb - Hb.T).max() == 0.0
    qr = dataclasses.replace(q, n=2 * q.n, row_ptr=Hb.indptr.astype(np.int64), col_idx=Hb.indices.astype(np.int32),
                             h_val=Hb.data, s_val=Sb.data, kpt=None,
                             dof_node=np.concatenate([q.dof_node, q.dof_node]).astype(np.int32),
                             dof_cluster=np.concatenate([q.dof_cluster, q.dof_cluster]).astype(np.int32))
    w2 = 2 * nev + L.default_m0(2 * nev)
    rr = L.labpsd(qr, 2 * nev, 1e-8, X0=pi.seed_normal_block(6, qr.n, w2))
    assert rc.converged and rr.converged
    scale = np.abs(rc.lam).max()
    assert np.abs(rr.lam[0::2] - rc.lam).max() <= 1e-12 * scale
    assert np.abs(rr.lam[1::2] - rc.lam).max() <= 1e-12 * scale
    Z = rr.X[:q.n] + 1j * rr.X[q.n:]
    g = np.sort(np.linalg.eigvalsh(Z.conj().T @ (S @ Z)))[::-1]
    assert g[nev - 1] > 1.0 and g[nev] < 1e-10                        # complex rank nev
    # each complex eigenvector of the native solve lies in that span (S-projection residual)
    Q = Z @ np.linalg.pinv(Z.conj().T @ (S @ Z), rcond=1e-10) @ (Z.conj().T @ (S @ rc.X))
    assert np.abs(Q - rc.X).max() <= 1e-6 * np.abs(rc.X).max()


# ------------------------------------------------------------------ brute force
def _brute(p):
    H, S = p.scipy_pair()
    return sla.eigh(H.toarray(), S.toarray())


@pytest.mark.parametrize("case", [(4, 1, 2, 0.3, 1, 6), (6, 2, 2, 0.2, 3, 10), (8, 2, 2, 0.25, 1, 16)])
def test_brute_force_dense(case):
    N, na, ne, rc, seed, nev = case
    p = pi.generate(N, na, ne, rc, seed)
    w, V = _brute(p)
    r = L.labpsd(p, nev, 1e-9, seed=seed)
    assert r.converged
    scale = np.abs(w[:nev]).max()
    assert np.abs(r.lam - w[:nev]).max() <= 1e-9 * scale
    # compare subspaces at every gap g = 1e-2 max|lambda| that ends at or before nev
    H, S = p.scipy_pair()
    Sd = S.toarray()
    gaps = [j for j in range(1, nev) if w[j] - w[j - 1] > 1e-2 * scale]
    for j in gaps:
        assert _angles(r.X[:, :j], V[:, :j], Sd) < 1e-6


def test_brute_force_extended_precision_at_kappa_3e10():
    """A tiny case whose S is far worse conditioned than the 8^3 case (4^3 mesh, four enrichment
    functions per node within r_c = 0.3: n = 92, kappa(D S D) = 2.6e10), where FP64 dense solvers
    themselves err near 1e-10 relative.  Reference: the generalized eigenvalues in 40-digit
    arithmetic (Cholesky S = L L^T, then the symmetric eigenvalues of L^-1 H L^-T, both in mpmath).
    The oracle at Res <= 1e-8 meets the solver's bar, |dlambda| <= 1e-9 max|lambda|."""
    mp = pytest.importorskip("mpmath")
    p = pi.generate(4, 1, 4, 0.3, 1)
    H, S = p.scipy_pair()
    Hd, Sd = H.toarray(), S.toarray()
    d = np.diag(Sd) ** -0.5
    ks = np.linalg.eigvalsh(Sd * d[:, None] * d[None, :])
    assert ks[-1] / ks[0] > 1e10
    with mp.workdps(40):
        Li = mp.inverse(mp.cholesky(mp.matrix(Sd.tolist())))
        C = Li * mp.matrix(Hd.tolist()) * Li.T
        ref = np.array(sorted(float(x) for x in mp.eigsy((C + C.T) / 2, eigvals_only=True)))
    nev = 8
    r = L.labpsd(p, nev, 1e-8, seed=1)
    assert r.converged
    assert np.abs(r.lam - ref[:nev]).max() <= 1e-9 * np.abs(ref[:nev]).max()


def test_inertia_count_small(small_problem):
    # Sylvester: #eigenvalues below sigma = #negative eigenvalues of H - sigma S
    p = small_problem
    r = L.labpsd(p, 16, 1e-8, seed=1)
    H, S = p.scipy_pair()
    Hd, Sd = H.toarray(), S.toarray()
    sigma = r.lam[0] + 0.5 * (r.E_all[1] - r.E_all[0])
    neg = np.count_nonzero(np.linalg.eigvalsh(Hd - sigma * Sd) < 0)
    assert neg == 1
    sigma = 0.5 * (r.lam[6] + r.lam[7])
    neg = np.count_nonzero(np.linalg.eigvalsh(Hd - sigma * Sd) < 0)
    assert neg == 7


# ------------------------------------------------------------------ invariants
def test_invariants_small(small_problem):
    p = small_problem
    r = L.labpsd(p, 16, 1e-8, seed=1)
    H, S = p.scipy_pair()
    # S-orthonormal Ritz vectors
    assert np.abs(r.X.T @ (S @ r.X) - np.eye(16)).max() <= 1e-10
    # Courant-Fischer: span(Z_l) contains span(Psi_{l-1}), so Ritz values never increase
    hist = np.array(r.ritz_history)
    scale = np.abs(hist).max()
    assert np.all(np.diff(hist, axis=0) <= 1e-12 * scale)
    # Ritz values lie above the exact eigenvalues
    w, _ = _brute(p)
    assert np.all(hist + r.sigma0 >= w[None, : hist.shape[1]] - 1e-10 * scale)
    # stopping claim re-checked in extended precision, unshifted definition of Eq. res1
    Hs = (H - r.sigma0 * S).tocsr()
    Xl = r.X.astype(np.longdouble)
    HX = np.stack([_spmv_ld(Hs, Xl[:, j]) for j in range(16)], axis=1)
    SX = np.stack([_spmv_ld(S.tocsr(), Xl[:, j]) for j in range(16)], axis=1)
    E = (r.lam - r.sigma0).astype(np.longdouble)
    res = np.linalg.norm((HX - SX * E).astype(np.float64), axis=0) / np.linalg.norm(HX.astype(np.float64), axis=0)
    assert res.max() <= 1e-8 * 1.01
    # La within the paper's reported range (0..4 MINRES steps per column per iteration)
    steps = np.concatenate([s for s in r.minres_steps if s.size])
    assert steps.max() <= 20 and steps.mean() <= 4


def _spmv_ld(A, x):
    out = np.zeros(A.shape[0], dtype=np.longdouble)
    data = A.data.astype(np.longdouble)
    for i in range(A.shape[0]):
        s, e = A.indptr[i], A.indptr[i + 1]
        out[i] = np.dot(data[s:e], x[A.indices[s:e]])
    return out


def test_krylov_bogoliubov_bound_against_brute_force(small_problem):
    # every computed pair (lam, x) has an exact eigenvalue within ||r||_{S^-1} / ||x||_S,
    # r = H x - lam S x (the bound for the pencil (H, S)); the computed ones are the lowest
    p = small_problem
    nev = 16
    r = L.labpsd(p, nev, 1e-8, seed=2)
    H, S = p.scipy_pair()
    Hd, Sd = H.toarray(), S.toarray()
    w, _ = _brute(p)
    Sinv_R = np.linalg.solve(Sd, Hd @ r.X - (Sd @ r.X) * r.lam[None, :])
    R = Hd @ r.X - (Sd @ r.X) * r.lam[None, :]
    bound = np.sqrt(np.einsum("ij,ij->j", R, Sinv_R)) / np.sqrt(np.einsum("ij,ij->j", r.X, Sd @ r.X))
    for j in range(nev):
        assert np.abs(w - r.lam[j]).min() <= bound[j] * (1 + 1e-6) + 1e-12 * np.abs(w).max()
    assert np.abs(r.lam - w[:nev]).max() <= 1e-8 * np.abs(w[:nev]).max()


def test_locking_and_localisation_bookkeeping(small_problem):
    # remarks 3-4: only unconverged columns among the first m get a direction (soft locking,
    # R9); of those, the localized ones are refined, at most max_minres steps each; nothing is
    # localized at the first iteration (R10, no previous Ritz value)
    p = small_problem
    m = 16
    r = L.labpsd(p, m, 1e-8, seed=4)
    assert r.converged and len(r.n_precond) == len(r.n_local) == len(r.minres_steps) == r.iters
    assert r.n_local[0] == 0
    for npc, nloc, st in zip(r.n_precond, r.n_local, r.minres_steps):
        assert 0 < npc <= m and 0 <= nloc <= npc and st.size == nloc
        assert np.all((st >= 0) & (st <= 20))
    assert r.n_precond[-1] < m                      # converged columns left the block of directions
    assert sum(r.n_local) > 0


def test_exact_invariant_subspace_zero_iterations(small_problem):
    p = small_problem
    w, V = _brute(p)
    r = L.labpsd(p, 16, 1e-8, X0=V[:, :19])
    assert r.converged and r.iters == 0


def test_hybrid_beats_global_only(small_problem):
    p = small_problem
    rh = L.labpsd(p, 16, 1e-8, seed=1)
    rg = L.labpsd(p, 16, 1e-8, seed=1, opts=L.Options(local=False))
    assert rh.converged and rg.converged
    assert rh.iters < rg.iters
    assert np.abs(rh.lam - rg.lam).max() <= 1e-9 * np.abs(rh.lam).max()


def test_local_only_without_localization_is_textbook_block_sd():
    # the local-only mode (Sec. 5, reading R16) with no localized column (tau1 = 0) is plain
    # block steepest descent: P = -R on the unconverged columns, Rayleigh-Ritz on [Psi P];
    # written out here with scipy's generalized eigh and compared iteration by iteration
    p = pi.generate(4, 1, 1, 0.3, 5)
    Hs, S, _ = L.make_shifted(p)
    Hd, Sd = Hs.toarray(), S.toarray()
    m, w = 3, 6
    X0 = pi.seed_normal_block(4, p.n, w)
    r = L.labpsd(p, m, 1e-10, X0=X0, opts=L.Options(use_global=False, tau1=0.0, m0=w - m, max_outer=6))
    ev, V = sla.eigh(X0.T @ Hd @ X0, X0.T @ Sd @ X0)
    Psi, E = X0 @ V[:, :w], ev[:w]
    hist = [E.copy()]
    for _ in range(6):
        R = Hd @ Psi[:, :m] - Sd @ Psi[:, :m] * E[:m]
        res = np.linalg.norm(R, axis=0) / np.linalg.norm(Hd @ Psi[:, :m], axis=0)
        U = np.nonzero(res > 1e-10)[0]
        Z = np.hstack([Psi, -R[:, U]])
        ev, V = sla.eigh(Z.T @ Hd @ Z, Z.T @ Sd @ Z)
        Psi, E = Z @ V[:, :w], ev[:w]
        hist.append(E.copy())
    assert len(r.ritz_history) == len(hist)
    for a, b in zip(r.ritz_history, hist):
        assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()   # both held shifted by sigma0


def test_local_only_is_slower_than_hybrid(small_problem):
    # Sec. 5 (Fig. 9 comparison): without the global step, the same eigenpairs need more outer
    # iterations than the hybrid scheme
    p = small_problem
    rh = L.labpsd(p, 16, 1e-8, seed=1)
    rl = L.labpsd(p, 16, 1e-8, seed=1, opts=L.Options(use_global=False, max_outer=400))
    assert rh.converged
    assert rl.iters > rh.iters


# ------------------------------------------------------------------ MINRES
def _indefinite(n, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.concatenate([-np.linspace(0.5, 3, n // 3), np.linspace(0.2, 5, n - n // 3)])
    return (Q * ev) @ Q.T


def test_minres_equals_direct_solve():
    A = _indefinite(40, 1)
    b = np.random.default_rng(2).standard_normal(40)
    x0 = np.random.default_rng(3).standard_normal(40)
    x, k, hist = L.minres(lambda v: A @ v, b, x0, 1e-13 * np.linalg.norm(b), 200)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-10)
    # the recurrence estimate is the true residual norm and never increases
    assert np.all(np.diff(hist) <= 1e-12 * hist[0])


def test_minres_recurrence_residual_is_true_residual():
    A = _indefinite(30, 4)
    b = np.random.default_rng(5).standard_normal(30)
    for maxit in range(1, 8):
        x, k, hist = L.minres(lambda v: A @ v, b, np.zeros(30), 0.0, maxit)
        assert k == maxit
        assert abs(np.linalg.norm(b - A @ x) - hist[-1]) <= 1e-10 * np.linalg.norm(b)


def test_minres_minimises_over_krylov_space():
    # x_k minimises ||b - A x|| over x0 + K_k(A, r0): compare with a least-squares solve
    A = _indefinite(25, 6)
    b = np.random.default_rng(7).standard_normal(25)
    x0 = np.random.default_rng(8).standard_normal(25)
    r0 = b - A @ x0
    for k in (1, 2, 3, 5):
        K = np.stack([np.linalg.matrix_power(A, j) @ r0 for j in range(k)], axis=1)
        c, *_ = np.linalg.lstsq(A @ K, r0, rcond=None)
        best = np.linalg.norm(r0 - A @ K @ c)
        x, _, hist = L.minres(lambda v: A @ v, b, x0, 0.0, k)
        assert abs(np.linalg.norm(b - A @ x) - best) <= 1e-9 * np.linalg.norm(r0)


def test_minres_residual_history_never_grows():
    # the iterates minimise the residual over nested Krylov spaces, so the recurrence estimate
    # is non-increasing (here for an indefinite operator, as in step 6(b))
    A = _indefinite(40, 11)
    b = np.random.default_rng(12).standard_normal(40)
    _, k, hist = L.minres(lambda v: A @ v, b, np.zeros(40), 0.0, 30)
    assert k == 30
    assert all(q <= p_ * (1 + 1e-12) for p_, q in zip(hist, hist[1:]))
    assert hist[-1] < 0.05 * hist[0]


def test_minres_zero_steps_when_start_meets_eta():
    A = _indefinite(20, 9)
    xs = np.random.default_rng(10).standard_normal(20)
    b = A @ xs
    x, k, _ = L.minres(lambda v: A @ v, b, xs + 1e-9, 1e-3, 20)
    assert k == 0 and np.array_equal(x, xs + 1e-9)


# ------------------------------------------------------------------ global preconditioner and RR
def test_global_preconditioner_solves(small_problem):
    p = small_problem
    Hs, S, s0 = L.make_shifted(p)
    K = L.GlobalPreconditioner(Hs, p.dof_node, p.grid)
    R = np.random.default_rng(1).standard_normal((p.n, 5))
    P = K.apply(R)
    Ad = Hs.toarray()
    assert np.allclose(Ad @ P, -R, rtol=0, atol=1e-9 * np.abs(R).max())
    assert np.allclose(P, -np.linalg.solve(Ad, R), rtol=1e-6, atol=0)


def test_nested_dissection_is_permutation():
    for N in (4, 6, 8, 9):
        o = L.nested_dissection_nodes(N)
        assert np.array_equal(np.sort(o), np.arange(N ** 3))


def test_rayleigh_ritz_against_generalized_eigh():
    rng = np.random.default_rng(11)
    q = 12
    B = rng.standard_normal((q, q))
    SR = B @ B.T + 0.1 * np.eye(q)
    HR = rng.standard_normal((q, q))
    HR = HR + HR.T
    g, W, fb = L.rayleigh_ritz(HR, SR, 5)
    ref = sla.eigh(HR, SR, eigvals_only=True)[:5]
    assert not fb
    assert np.allclose(g, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert np.allclose(W.T @ SR @ W, np.eye(5), atol=1e-12)
    assert np.allclose(W.T @ HR @ W, np.diag(g), atol=1e-11)


def test_rayleigh_ritz_rank_deficient_fallback():
    rng = np.random.default_rng(12)
    n, q = 30, 8
    Bm = rng.standard_normal((n, n))
    Sf = Bm @ Bm.T + n * np.eye(n)
    Hf = rng.standard_normal((n, n))
    Hf = Hf + Hf.T
    Z = rng.standard_normal((n, q))
    Z[:, -1] = Z[:, 0] * 2.0 - Z[:, 1]            # exactly dependent column
    HR, SR = Z.T @ Hf @ Z, Z.T @ Sf @ Z
    HR, SR = 0.5 * (HR + HR.T), 0.5 * (SR + SR.T)
    g, W, fb = L.rayleigh_ritz(HR, SR, 4)
    assert fb
    # reference on an independent basis of the same space
    Zi = Z[:, :-1]
    ref = sla.eigh(Zi.T @ Hf @ Zi, Zi.T @ Sf @ Zi, eigvals_only=True)[:4]
    assert np.allclose(g, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_residual_by_hand():
    # steps 4-5 (Eq. res1): r_i = H psi_i - eps_i S psi_i and Res_i = ||r_i|| / ||H psi_i||, the
    # columns beyond m ignored.  PsiH = [[3, 1, 9], [4, 0, 9]], PsiS = [[1, 1, 9], [0, 2, 9]],
    # E = (2, 0.5, 7): r_1 = (3 - 2, 4 - 0) = (1, 4), r_2 = (1 - 0.5, 0 - 1) = (0.5, -1);
    # ||H psi_1|| = 5, ||H psi_2|| = 1
    PH = np.array([[3.0, 1.0, 9.0], [4.0, 0.0, 9.0]])
    PS = np.array([[1.0, 1.0, 9.0], [0.0, 2.0, 9.0]])
    R, res = L.residual(PH, PS, np.array([2.0, 0.5, 7.0]), 2)
    assert R.shape == (2, 2)
    assert np.array_equal(R, [[1.0, 0.5], [4.0, -1.0]])
    assert res == pytest.approx([math.sqrt(17.0) / 5.0, math.sqrt(1.25)], rel=1e-15)


def test_localized_by_hand():
    # remark 4: a column is refined locally when Res_i <= tau1 and the Ritz value moved by at
    # most tau2 of its previous value; nothing is localized without a previous value (l = 1)
    res = np.array([0.05, 0.05, 0.2, 0.1])
    E = np.array([1.0, 2.0, 3.0, -1.05])
    E_prev = np.array([1.05, 2.5, 3.0, -1.0])
    got = L.localized(res, E, E_prev, 0.1, 0.1)
    # col 0: 0.05 <= 0.1 and |1 - 1.05| = 0.05 <= 0.105; col 1: moved 0.5 > 0.25;
    # col 2: Res 0.2 > 0.1; col 3: Res at the bound, moved 0.05 <= 0.1 (|E_prev| taken)
    assert got.tolist() == [True, False, False, True]
    assert not L.localized(res, E, None, 0.1, 0.1).any()


def test_default_m0():
    assert [L.default_m0(m) for m in (1, 16, 30, 31, 64, 256)] == [3, 3, 3, 4, 7, 26]


# ------------------------------------------------------------------ planted mistakes
def test_planted_mistakes_are_caught(monkeypatch):
    """Each plausible slip below, planted in the oracle, fails a pin used above."""
    p = pi.generate(6, 2, 2, 0.2, 3)
    w, V = _brute(p)
    nev = 10

    def pinned():
        try:
            r = L.labpsd(p, nev, 1e-9, seed=3, opts=L.Options(max_outer=200))
        except (np.linalg.LinAlgError, ValueError, FloatingPointError):
            return False
        return bool(r.converged and np.abs(r.lam - w[:nev]).max() <= 1e-9 * np.abs(w[:nev]).max())

    assert pinned()
    orig_res, orig_rr, orig_ref, orig_red = L.residual, L.rayleigh_ritz, L.refine, L.reduced_pair

    # (a) wrong sign in the residual of step 4
    monkeypatch.setattr(L, "residual", lambda PH, PS, E, m: orig_res(PH, -PS, E, m))
    assert not pinned()
    monkeypatch.setattr(L, "residual", orig_res)
    # (b) Rayleigh-Ritz keeps the highest instead of the lowest pairs
    def rr_high(HR, SR, k):
        g, W, fb = orig_rr(-HR, SR, k)
        return -g, W, fb
    monkeypatch.setattr(L, "rayleigh_ritz", rr_high)
    assert not pinned()
    monkeypatch.setattr(L, "rayleigh_ritz", orig_rr)
    # (c) S_R formed from H-products (a transposed / swapped operand in step 8)
    monkeypatch.setattr(L, "reduced_pair", lambda Z, ZH, ZS: orig_red(Z, ZH, ZH + ZS))
    assert not pinned()
    monkeypatch.setattr(L, "reduced_pair", orig_red)
    # (d) refinement shift with the wrong sign: (H + eps_i S) instead of (H - eps_i S)
    monkeypatch.setattr(L, "refine", lambda Hs, S, e, r, p0, eta, mx: orig_ref(Hs, S, -e - 50.0, r, p0, eta, mx))
    r = L.labpsd(p, nev, 1e-9, seed=3, opts=L.Options(max_outer=200))
    monkeypatch.setattr(L, "refine", orig_ref)
    good = L.labpsd(p, nev, 1e-9, seed=3)
    assert r.iters > good.iters


# ---- global factor with eps_bar inside the spectrum (reading R3: LDL^T with 1 x 1 pivots) ----
def _interior_shift(p, below):
    H, S = p.scipy_pair()
    lam = sla.eigh(H.toarray(), S.toarray(), eigvals_only=True)
    return 0.5 * (lam[below - 1] + lam[below]), lam


@pytest.mark.parametrize("below", [1, 5, 12])
def test_interior_shift_factor_counts_the_eigenvalues_below(below):
    # Sylvester's law of inertia: H - eps S (S positive definite) has as many negative pivots
    # as the pencil has eigenvalues below eps
    p = pi.small_case(1)
    eps, lam = _interior_shift(p, below)
    H, S = p.scipy_pair()
    K = L.GlobalPreconditioner((H - eps * S).tocsr(), p.dof_node, p.grid)
    assert K.neg_pivots == below == int(np.count_nonzero(lam < eps))
    R = pi.seed_normal_block(3, p.n, 5)
    A = (H - eps * S).toarray()
    ref = -np.linalg.solve(A, R)
    assert np.abs(K.apply(R) - ref).max() <= 1e-8 * np.abs(ref).max()


def test_labpsd_with_an_interior_global_shift_matches_dense_eigh():
    # eps_bar in the gap above the second eigenvalue (a shift within a few 1e-3 of a cluster
    # makes K nearly singular and the iteration stalls near 1e-9, as shift-and-invert would)
    p = pi.small_case(1)
    eps, lam = _interior_shift(p, 2)
    Hs, S, s0 = L.make_shifted(p)          # sigma0 stays below the spectrum (R4)
    K = L.GlobalPreconditioner((Hs.loc - (eps - s0) * S).tocsr(), p.dof_node, p.grid)
    assert K.neg_pivots == 2
    r = L.labpsd(p, 16, 1e-10, seed=2, precond=K)
    assert r.converged
    assert np.allclose(r.lam, lam[:16], rtol=0, atol=1e-8 * np.abs(lam[:16]).max())


def test_global_shift_has_little_influence(small_problem):
    """Sec. 5: the choice of the global shift eps_bar barely matters.  Lowering it by 0.5 to 4
    times its distance to zero (all below the spectrum) leaves the eigenvalues unchanged to
    rounding and the outer iteration count within one of the generator's choice."""
    import dataclasses
    p = small_problem
    X0 = pi.seed_normal_block(1, p.n, 16 + L.default_m0(16))
    base = L.labpsd(p, 16, 1e-8, X0=X0)
    assert base.converged
    for f in (0.5, 2.0, 4.0):
        q = dataclasses.replace(p, eps_bar=p.eps_bar - f * abs(p.eps_bar))
        r = L.labpsd(q, 16, 1e-8, X0=X0)
        assert r.converged and abs(r.iters - base.iters) <= 1
        assert np.abs(r.lam - base.lam).max() <= 1e-12 * np.abs(base.lam).max()


def test_minres_from_the_globally_preconditioned_start_needs_few_steps(small_problem):
    """Sec. 3/5: started from the globally preconditioned vector, the local MINRES meets eta in a
    handful of steps (the paper reports 2-5).  On the small case every refined column takes at
    most 5, and a start from zero (the local-only scheme) takes more on average."""
    p = small_problem
    r = L.labpsd(p, 16, 1e-8, seed=1)
    steps = np.concatenate([np.asarray(s) for s in r.minres_steps if len(s)])
    assert r.converged and steps.size > 0 and steps.max() <= 5
    lo = L.labpsd(p, 16, 1e-8, seed=1, opts=L.Options(use_global=False, max_outer=30))
    steps0 = np.concatenate([np.asarray(s) for s in lo.minres_steps if len(s)])
    assert steps0.mean() > steps.mean()
