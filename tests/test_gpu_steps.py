"""GPU parity of every LABPSD step against the CPU oracle (through the C ABI).

Tolerances: FP64 block products (SpMM, Gram, update, residual) are compared elementwise to
1e-12 relative to the block's magnitude -- they differ from the oracle only in summation order.
The global preconditioner and MINRES act through (H - eps S)^{-1} with kappa up to ~1e9, so their
outputs are compared at 1e-6 relative, and the GPU solve is additionally required to be
backward-stable (||A P + R|| <= 1e-12 ||A|| ||P||).
"""
import numpy as np
import pytest

from oracle import labpsd as L
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


def dev(a):
    """Device copy; a 2-D block gets an even leading dimension (16-byte rows pairs)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim == 1:
        return torch.from_numpy(a).cuda()
    t = dbuf(a.shape[0], a.shape[1])
    t.copy_(torch.from_numpy(a))
    return t


def dense(a):
    """Contiguous device copy (matrices whose leading dimension is their width)."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def dbuf(n, k, fill=0.0):
    t = torch.full((n, k + (k % 2)), fill, dtype=torch.float64, device="cuda")
    return t[:, :k]


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def small():
    p = pi.small_case(1)
    return p, hb().Session.from_problem(p)


@pytest.fixture(scope="module")
def mid():
    p = pi.generate(12, 2, 4, 0.15, 3)
    return p, hb().Session.from_problem(p)


def relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("k", [1, 2, 3, 16, 19, 35, 64, 130, 300])
def test_spmm_pair(small, k):
    p, s = small
    Hs, S, _ = L.make_shifted(p)
    X = pi.seed_normal_block(k + 7, p.n, k)
    HX, SX = dbuf(p.n, k), dbuf(p.n, k)
    s.spmm_pair(dev(X), HX, SX)
    rH, rS = L.spmm_pair(Hs, S, X)
    assert relerr(host(HX), rH) <= 1e-12
    assert relerr(host(SX), rS) <= 1e-12


def test_spmm_pair_strided_input(mid):
    p, s = mid
    Hs, S, _ = L.make_shifted(p)
    big = pi.seed_normal_block(5, p.n, 40)
    Xt = dev(big)[:, 6:6 + 21]            # a column window of a wider block (ld 40, offset 6)
    HX, SX = dbuf(p.n, 21), dbuf(p.n, 21)
    s.spmm_pair(Xt, HX, SX)
    rH, rS = L.spmm_pair(Hs, S, big[:, 6:27])
    assert relerr(host(HX), rH) <= 1e-12 and relerr(host(SX), rS) <= 1e-12


@pytest.mark.parametrize("k", [1, 5, 33])
def test_spmm_shifted(mid, k):
    p, s = mid
    Hs, S, _ = L.make_shifted(p)
    X = pi.seed_normal_block(k, p.n, k)
    e = np.linspace(0.3, 40.0, k)
    Y = dbuf(p.n, k)
    s.spmm_shifted(dev(X), dev(e), Y)
    ref = Hs @ X - (S @ X) * e[None, :]
    assert relerr(host(Y), ref) <= 1e-12


def test_residual(mid):
    p, s = mid
    Hs, S, _ = L.make_shifted(p)
    X = pi.seed_normal_block(2, p.n, 24)
    PH, PS = L.spmm_pair(Hs, S, X)
    E = np.linspace(1.0, 30.0, 24)
    R = dbuf(p.n, 20)
    res = torch.zeros(20, dtype=torch.float64, device="cuda")
    s.residual(dev(PH), dev(PS), dev(E), 20, R, res)
    Rr, rr = L.residual(PH, PS, E, 20)
    assert relerr(host(R), Rr) <= 1e-13
    assert np.allclose(host(res), rr, rtol=1e-13, atol=0)


@pytest.mark.parametrize("which", ["small", "mid"])
def test_global_preconditioner(which, small, mid):
    p, s = small if which == "small" else mid
    Hs, S, _ = L.make_shifted(p)
    R = pi.seed_normal_block(9, p.n, 13)
    P = dbuf(p.n, 13)
    s.precond_apply(dev(R), P)
    Pg = host(P)
    K = L.GlobalPreconditioner(Hs, p.dof_node, p.grid)
    Po = K.apply(R)
    # backward stability of the GPU solve, then agreement with the oracle's library solve
    A = Hs.loc
    anorm = np.abs(A).sum(axis=1).max()
    assert np.abs(A @ Pg + R).max() <= 1e-12 * anorm * np.abs(Pg).max()
    assert relerr(Pg, Po) <= 1e-6


def test_global_preconditioner_many_columns(small):
    p, s = small
    Hs, S, _ = L.make_shifted(p)
    R = pi.seed_normal_block(10, p.n, 150)   # several RHS chunks of 64 and a ragged tail
    P = dbuf(p.n, 150)
    s.precond_apply(dev(R), P)
    Po = L.GlobalPreconditioner(Hs, p.dof_node, p.grid).apply(R)
    assert relerr(host(P), Po) <= 1e-8


@pytest.mark.parametrize("q,n", [(19, 646), (35, 4000), (135, 1000), (70, 33)])
def test_gram(q, n):
    Z = pi.seed_normal_block(q, n, q)
    ZH = pi.seed_normal_block(q + 1, n, q)
    ZS = pi.seed_normal_block(q + 2, n, q)
    HR = torch.zeros(q, q, dtype=torch.float64, device="cuda")
    SR = torch.zeros(q, q, dtype=torch.float64, device="cuda")
    hb().gram(dev(Z), dev(ZH), dev(ZS), HR, SR)
    rH, rS = L.reduced_pair(Z, ZH, ZS)
    assert relerr(host(HR), rH) <= 1e-12 and relerr(host(SR), rS) <= 1e-12
    assert np.array_equal(host(HR), host(HR).T)


def _rr_case(q, seed, cond=1e4):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((q, q)))
    SR = (Q * np.logspace(0, np.log10(cond), q)) @ Q.T
    SR = 0.5 * (SR + SR.T)
    B = rng.standard_normal((q, q))
    HR = 0.5 * (B + B.T)
    return HR, SR


@pytest.mark.parametrize("q,k", [(1, 1), (5, 3), (35, 19), (135, 71), (200, 120), (300, 200), (538, 282)])
def test_rayleigh_ritz(q, k):   # q >= ~190 runs the cluster kernel with its row blocks in global memory
    HR, SR = _rr_case(q, q)
    th = torch.zeros(k, dtype=torch.float64, device="cuda")
    W = torch.zeros(q, k, dtype=torch.float64, device="cuda")
    info = torch.zeros(2, dtype=torch.int32, device="cuda")
    hb().rayleigh_ritz(dense(HR), dense(SR), k, th, W, info)
    g, Wo, fb = L.rayleigh_ritz(HR, SR, k)
    thg, Wg = host(th), host(W)
    assert host(info)[0] == 0 and not fb
    scale = np.abs(g).max()
    assert np.abs(thg - g).max() <= 1e-11 * scale
    assert np.abs(Wg.T @ SR @ Wg - np.eye(k)).max() <= 1e-10
    assert np.abs(Wg.T @ HR @ Wg - np.diag(thg)).max() <= 1e-10 * scale


def test_rayleigh_ritz_degenerate_cluster():
    # a 12-fold cluster (as in the free-electron shells) must come out S_R-orthonormal
    q, k = 40, 19
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((q, q)))
    ev = np.concatenate([[0.1], np.full(6, 2.0), np.full(12, 4.0), np.linspace(6, 9, q - 19)])
    HR = (Q * ev) @ Q.T
    HR = 0.5 * (HR + HR.T)
    SR = np.eye(q)
    th = torch.zeros(k, dtype=torch.float64, device="cuda")
    W = torch.zeros(q, k, dtype=torch.float64, device="cuda")
    info = torch.zeros(2, dtype=torch.int32, device="cuda")
    hb().rayleigh_ritz(dense(HR), dense(SR), k, th, W, info)
    assert np.abs(host(th) - ev[:k]).max() <= 1e-13 * 9
    Wg = host(W)
    assert np.abs(Wg.T @ Wg - np.eye(k)).max() <= 1e-12


def test_rayleigh_ritz_fallback():
    rng = np.random.default_rng(12)
    n, q = 30, 8
    Bm = rng.standard_normal((n, n))
    Sf = Bm @ Bm.T + n * np.eye(n)
    Hf = rng.standard_normal((n, n))
    Hf = Hf + Hf.T
    Z = rng.standard_normal((n, q))
    Z[:, -1] = Z[:, 0] * 2.0 - Z[:, 1]
    HR, SR = Z.T @ Hf @ Z, Z.T @ Sf @ Z
    HR, SR = 0.5 * (HR + HR.T), 0.5 * (SR + SR.T)
    k = 4
    th = torch.zeros(k, dtype=torch.float64, device="cuda")
    W = torch.zeros(q, k, dtype=torch.float64, device="cuda")
    info = torch.zeros(2, dtype=torch.int32, device="cuda")
    hb().rayleigh_ritz(dense(HR), dense(SR), k, th, W, info)
    g, Wo, fb = L.rayleigh_ritz(HR, SR, k)
    inf = host(info)
    assert fb and inf[0] == 1 and inf[1] == q - 1
    assert np.abs(host(th) - g).max() <= 1e-9 * np.abs(g).max()


@pytest.mark.parametrize("q,k,n", [(19, 19, 646), (35, 19, 1000), (135, 71, 3001), (8, 3, 5)])
def test_update(q, k, n):
    Z = pi.seed_normal_block(q * 3, n, q)
    W = pi.seed_normal_block(q * 5, q, k)
    Zd = dbuf(n, q)
    Zd.copy_(dev(Z))
    hb().update(Zd, dense(W), k)
    out = host(Zd)
    assert relerr(out[:, :k], Z @ W) <= 1e-12
    assert np.array_equal(out[:, k:], Z[:, k:])


# ---- double-float forms (mixed precision): products of hi + lo float pairs, FP64 across
# 128-row tiles.  Bound: each entry within c * 2^-44 of |Z|^T |ZH| (the sum of the absolute
# products), a few times the FP64 summation bound at these lengths; an FP32-accurate product
# (2^-24) would miss it by ~10^6.
@pytest.mark.parametrize("q,n", [(19, 646), (35, 4000), (135, 1000), (70, 33), (135, 47620)])
def test_gram_df64(q, n):
    Z = pi.seed_normal_block(q, n, q)
    ZH = pi.seed_normal_block(q + 1, n, q)
    ZS = pi.seed_normal_block(q + 2, n, q)
    # columns of very different magnitudes, and a near-cancelling part, as in the search blocks
    sc = np.logspace(-6, 6, q)
    Z = Z * sc
    ZH = ZH / sc + 1e3 * Z
    HR = torch.zeros(q, q, dtype=torch.float64, device="cuda")
    SR = torch.zeros(q, q, dtype=torch.float64, device="cuda")
    hb().gram_df64(dev(Z), dev(ZH), dev(ZS), HR, SR)
    h, sr = host(HR), host(SR)
    exH, exS = Z.T @ ZH, Z.T @ ZS
    bH, bS = np.abs(Z).T @ np.abs(ZH), np.abs(Z).T @ np.abs(ZS)
    iu = np.triu_indices(q)
    assert np.all(np.abs(h - exH)[iu] <= 2.0 ** -44 * bH[iu] + 1e-300)
    assert np.all(np.abs(sr - exS)[iu] <= 2.0 ** -44 * bS[iu] + 1e-300)
    assert np.array_equal(h, h.T) and np.array_equal(sr, sr.T)


@pytest.mark.parametrize("q,k,n", [(19, 19, 646), (35, 19, 1000), (135, 71, 3001), (8, 3, 5), (282, 30, 700),
                                   (300, 282, 1001), (538, 282, 777), (600, 520, 301)])
# the last three read W per thread (q too large to stage it with the rows); the last in two passes
def test_update_df64(q, k, n):
    Z = pi.seed_normal_block(q * 3, n, q) * np.logspace(-4, 4, q)
    W = pi.seed_normal_block(q * 5, q, k)
    Zd = dbuf(n, q)
    Zd.copy_(dev(Z))
    hb().update_df64(Zd, dense(W), k)
    out = host(Zd)
    bound = np.abs(Z) @ np.abs(W)
    assert np.all(np.abs(out[:, :k] - Z @ W) <= 2.0 ** -44 * bound + 1e-300)
    assert np.array_equal(out[:, k:], Z[:, k:])


def test_df64_split_edge_values():
    # zeros, signs, magnitudes from 1e-28 to 1e30 and exact powers of two go through to ~2^-47;
    # magnitudes below 2^-126 enter as zero; in between (subnormal lo) at least FP32 precision
    v = np.array([0.0, -0.0, 1.0, -1.0, 2.0 ** 100, -(2.0 ** -100), 1e30, -1e-28, 3.141592653589793,
                  1.0 + 2.0 ** -40, 1e-39, -1e-300, 2.0 ** -80 * 3.141592653589793, -1e-35])
    q = v.size
    Z = np.zeros((1, q))
    Z[0] = v
    W = np.eye(q)
    Zd = dbuf(1, q)
    Zd.copy_(dev(Z))
    hb().update_df64(Zd, dense(W), q)
    out = host(Zd)[0]
    full = np.abs(v) >= 2.0 ** -96
    mid = (np.abs(v) >= 2.0 ** -126) & ~full
    assert np.all(np.abs(out[full] - v[full]) <= 2.0 ** -46 * np.abs(v[full]))
    assert np.all(np.abs(out[mid] - v[mid]) <= 2.0 ** -23 * np.abs(v[mid]))
    assert np.all(out[np.abs(v) < 2.0 ** -126] == 0.0)


def test_minres_against_oracle(mid):
    p, s = mid
    Hs, S, _ = L.make_shifted(p)
    # a realistic state: a few BPSD iterations of the oracle, then refine its localized columns
    r = L.labpsd(p, 10, 1e-8, seed=3, opts=L.Options(max_outer=6))
    K = L.GlobalPreconditioner(Hs, p.dof_node, p.grid)
    X0 = pi.seed_normal_block(3, p.n, 13)
    E = r.E_all - r.sigma0
    Psi = r.X
    PH, PS = L.spmm_pair(Hs, S, Psi)
    R, res = L.residual(PH, PS, E, 10)
    P0 = K.apply(R)
    e = E[:10]
    steps = torch.zeros(10, dtype=torch.int32, device="cuda")
    Pd = dbuf(p.n, 10)
    Pd.copy_(dev(P0))
    s.minres(dev(R), dev(e), Pd, 0.25, 20, steps)
    Pg, sg = host(Pd), host(steps)
    for j in range(10):
        xo, ko, _ = L.refine(Hs, S, e[j], R[:, j], P0[:, j], 0.25, 20)
        assert abs(int(sg[j]) - ko) <= 1, (j, sg[j], ko)
        if int(sg[j]) == ko:
            assert np.abs(Pg[:, j] - xo).max() <= 1e-6 * np.abs(xo).max()
        # the GPU iterate meets (or the cap ends) the inexact-solve criterion, Eq. approxp
        rr = np.linalg.norm(Hs @ Pg[:, j] - e[j] * (S @ Pg[:, j]) + R[:, j])
        if int(sg[j]) < 20:
            assert rr <= 0.25 * np.linalg.norm(R[:, j]) * (1 + 1e-6)


# ------------------------------------------------------------------ FP32 forms (mixed precision)
def fbuf(n, k):
    t = torch.zeros(n, (k + 3) // 4 * 4, dtype=torch.float32, device="cuda")
    return t[:, :k]


def fdev(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    t = fbuf(a.shape[0], a.shape[1])
    t.copy_(torch.from_numpy(a))
    return t


@pytest.mark.parametrize("k", [1, 5, 16, 64, 71])
def test_spmm_pair_f32_scaled(mid, k):
    p, s = mid
    Hs, S, _ = L.make_shifted(p)
    d = s.dscale()
    Hh = (Hs.loc.multiply(d[:, None]).multiply(d[None, :])).tocsr()
    Sh = (S.multiply(d[:, None]).multiply(d[None, :])).tocsr()
    X = pi.seed_normal_block(40 + k, p.n, k)
    HX, SX = fbuf(p.n, k), fbuf(p.n, k)
    s.spmm_pair_f32(fdev(X), HX, SX)
    rH, rS = Hh @ X, Sh @ X
    assert relerr(host(HX), rH) <= 2e-5 and relerr(host(SX), rS) <= 2e-5
    assert np.allclose(1.0 / d ** 2, S.diagonal(), rtol=1e-12)


@pytest.mark.parametrize("k", [1, 13, 64, 90, 100, 150, 180, 200, 300])
def test_precond_f32_scaled(mid, k):
    """FP32 preconditioner on the scaled pencil: P = -(D A D)^{-1} R, A = H - eps_bar S.
    Compared with the FP64 library solve in the energy norm of D A D (errors along its
    near-null directions, which FP32 cannot resolve, weigh little there): about u32 sqrt(kappa)."""
    p, s = mid
    Hs, S, _ = L.make_shifted(p)
    d = s.dscale()
    K = L.GlobalPreconditioner(Hs, p.dof_node, p.grid)
    R = pi.seed_normal_block(50 + k, p.n, k)
    P = fbuf(p.n, k)
    s.precond_apply_f32(fdev(R), P)
    Pg = host(P).astype(np.float64)
    ref = -K.solve(R / d[:, None]) / d[:, None]
    Ah = (Hs.loc.multiply(d[:, None]).multiply(d[None, :])).tocsr()
    err = Pg - ref
    num = np.sqrt(np.einsum("ij,ij->j", err, Ah @ err))
    den = np.sqrt(np.einsum("ij,ij->j", ref, Ah @ ref))
    assert np.isfinite(Pg).all()
    assert (num / den).max() <= 1e-2, (num / den).max()


@pytest.mark.parametrize("q,k,ndep", [(40, 19, 3), (135, 71, 10)])
def test_rayleigh_ritz_fallback_large(q, k, ndep):
    rng = np.random.default_rng(q)
    n = 3 * q
    Bm = rng.standard_normal((n, n))
    Sf = Bm @ Bm.T + n * np.eye(n)
    Hf = rng.standard_normal((n, n))
    Hf = Hf + Hf.T
    Z = rng.standard_normal((n, q))
    for t in range(ndep):
        Z[:, q - 1 - t] = Z[:, t] - 0.5 * Z[:, t + 1]
    HR, SR = Z.T @ Hf @ Z, Z.T @ Sf @ Z
    HR, SR = 0.5 * (HR + HR.T), 0.5 * (SR + SR.T)
    th = torch.zeros(k, dtype=torch.float64, device="cuda")
    W = torch.zeros(q, k, dtype=torch.float64, device="cuda")
    info = torch.zeros(2, dtype=torch.int32, device="cuda")
    hb().rayleigh_ritz(dense(HR), dense(SR), k, th, W, info)
    g, Wo, fb = L.rayleigh_ritz(HR, SR, k)
    inf = host(info)
    assert fb and inf[0] == 1 and inf[1] == q - ndep
    assert np.abs(host(th) - g).max() <= 1e-8 * np.abs(g).max()


def test_precond_f32_columns_independent_of_the_block_width(mid):
    """Each column of the FP32 sweeps is reduced in the same order whatever the block width (the
    CTA column tiles of 32, 64, 128 and 256 columns differ only in which columns share a tile), so a
    column solved in a block of 300, 130, 37 or alone must come out bit for bit the same."""
    p, s = mid
    R = pi.seed_normal_block(77, p.n, 300)
    P = fbuf(p.n, 300)
    s.precond_apply_f32(fdev(R), P)
    full = host(P)
    for cols in ([5], [299], list(range(0, 37)), list(range(100, 230))):
        Pk = fbuf(p.n, len(cols))
        s.precond_apply_f32(fdev(R[:, cols]), Pk)
        assert np.array_equal(host(Pk), full[:, cols]), cols[:3]


@pytest.mark.parametrize("k", [1, 7, 64, 130, 300])
def test_spmm_pair_df64_against_fp64(mid, k):
    """Steps 3/7 of the mixed form in double-float on the scaled pencil: within 2^-42 of |Hs||X|
    (resp. |S||X|) of the FP64 product, entry by entry, including the columns of a second pass
    (k = 300 > 256) and a ragged last column pair."""
    p, s = mid
    Hs, S, _ = L.make_shifted(p)
    X = pi.seed_normal_block(60 + k, p.n, k) * np.logspace(-3, 3, k)
    Xd = dev(X)
    HX, SX, HX2, SX2 = [dbuf(p.n, k) for _ in range(4)]
    s.spmm_pair(Xd, HX, SX)
    s.spmm_pair_df64(Xd, HX2, SX2)
    bH = np.abs(Hs.loc) @ np.abs(X)
    bS = np.abs(S) @ np.abs(X)
    assert np.all(np.abs(host(HX2) - host(HX)) <= 2.0 ** -42 * bH + 1e-300)
    assert np.all(np.abs(host(SX2) - host(SX)) <= 2.0 ** -42 * bS + 1e-300)
