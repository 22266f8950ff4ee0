"""Complex Hermitian (Bloch) input on the GPU (Sec. 2: at a Bloch vector k != 0, H is Hermitian
and S Hermitian positive definite), through hbsd_create with is_complex = 1, against the CPU
oracle's complex LABPSD on the same complex start block.

Bar: |lambda_gpu - lambda_oracle| <= 1e-9 max|lambda|; S-principal angle between the complex
spans X(:, :j) <= 1e-6 at every gap > 1e-2 max|lambda|; outer iterations within +-1 (FP64 form);
X^H S X = I to 1e-10; Res_max <= tol recomputed on the host in complex arithmetic.  The closed
form of the unenriched periodic mesh pins the Bloch eigenvalues themselves."""
import numpy as np
import pytest

from oracle import labpsd as L
from paper_1308_2445_gb300 import pufe_inputs as pi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K_BLOCH = (0.5 * np.pi, -0.5 * np.pi, 0.5 * np.pi)    # one point of the 2 x 2 x 2 k-grid


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import os
    from paper_1308_2445_gb300 import build_lib
    if not os.path.exists(build_lib.LIB):
        build_lib.build()


def hb():
    from paper_1308_2445_gb300 import hbsd
    return hbsd


def host_res(p, lam, X, sigma0):
    H, S = p.scipy_pair()
    Hs = H - sigma0 * S
    HX = Hs @ X
    R = HX - (S @ X) * (lam - sigma0)[None, :]
    return np.linalg.norm(R, axis=0) / np.linalg.norm(HX, axis=0)


def test_bloch_closed_form():
    """Unenriched 5^3 periodic mesh, V = 0.3, k = 2 pi (1/4, -1/4, 1/4): the lowest eigenvalues
    are the closed-form Q1 Bloch values (exact with 3-point Gauss)."""
    q = pi.generate(5, 0, 0, 0.1, 1, v0=0.3, kpt=K_BLOCH)
    assert np.iscomplexobj(q.h_val)
    nev = 5
    X0 = pi.seed_normal_block_complex(4, q.n, nev + L.default_m0(nev))
    s = hb().Session.from_problem(q)
    assert hb().lib().hbsd_is_complex(s.h) == 1 and hb().lib().hbsd_n(s.h) == q.n
    lam, X, it, rc, st = s.solve(nev, 1e-10, X0=X0)
    ref = pi.closed_form_eigenvalues(5, 0.3, K_BLOCH)[:nev]
    assert rc == 0 and np.iscomplexobj(X)
    assert np.abs(lam - ref).max() <= 1e-10 * np.abs(ref).max()
    s.close()


@pytest.fixture(scope="module")
def bloch_small():
    q = pi.generate(8, 2, 2, 0.25, 1, kpt=K_BLOCH)
    nev = 16
    X0 = pi.seed_normal_block_complex(1, q.n, nev + L.default_m0(nev))
    ro = L.labpsd(q, nev, 1e-8, X0=X0)
    assert ro.converged and np.iscomplexobj(ro.X)
    return q, nev, X0, ro


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_bloch_8cubed_against_the_oracle(bloch_small, form):
    import scipy.sparse as sp
    from subspace import gap_indices, s_angle
    q, nev, X0, ro = bloch_small
    prec = hb().PRECISION_MIXED if form == "mixed" else hb().PRECISION_FP64
    s = hb().Session.from_problem(q, precision=prec)
    lam, X, it, rc, st = s.solve(nev, 1e-8, X0=X0)
    assert rc == 0 and np.iscomplexobj(X) and X.shape == (q.n, nev)
    scale = np.abs(ro.lam).max()
    assert np.abs(lam - ro.lam).max() <= 1e-9 * scale
    if form == "fp64":
        assert abs(it - ro.iters) <= 1, (it, ro.iters)
    H, S = q.scipy_pair()
    S = sp.csr_matrix(S)
    assert np.abs(X.conj().T @ (S @ X) - np.eye(nev)).max() <= 1e-10
    assert host_res(q, lam, X, s.sigma0).max() <= 1e-8 * 1.001
    js = gap_indices(ro.lam, nev)
    assert js
    worst = max(s_angle(X[:, :j], ro.X[:, :j], S) for j in js)
    assert worst <= 1e-6, (form, worst)
    s.close()


def test_bloch_seeded_start_block_is_the_documented_one(bloch_small):
    """X0 = NULL draws the real parts from stream 2 and the imaginary parts from stream 6 of the
    session's seed: the same solve as the explicit block built by the generator module."""
    q, nev, _, _ = bloch_small
    s = hb().Session.from_problem(q, seed=3)
    lam_a, Xa, it_a, rc_a, _ = s.solve(nev, 1e-8)
    lam_b, Xb, it_b, rc_b, _ = s.solve(nev, 1e-8, X0=pi.seed_normal_block_complex(3, q.n, nev + L.default_m0(nev)))
    assert rc_a == rc_b == 0 and it_a == it_b
    assert np.array_equal(lam_a, lam_b) and np.array_equal(Xa, Xb)
    s.close()


def test_bloch_scf_follow_up_warm_start(bloch_small):
    """An SCF-style follow-up (V perturbed by 1%, new H values on the same pattern) warm-started
    from the previous block: the eigenpairs of the new problem, in fewer iterations than cold."""
    q, nev, X0, _ = bloch_small
    q2 = pi.generate(8, 2, 2, 0.25, 1, kpt=K_BLOCH, v_noise=0.01, noise_seed=9)
    assert np.array_equal(q2.col_idx, q.col_idx)
    s = hb().Session.from_problem(q)
    _, _, it_cold, rc, _ = s.solve(nev, 1e-8, X0=X0)
    assert rc == 0
    s.update_H(q2.h_val)
    lam, X, it_warm, rc, _ = s.solve(nev, 1e-8, warm=True)
    assert rc == 0 and it_warm < it_cold
    # the global factor keeps the first H (Sec. 4): compare with the oracle of the new problem
    ro = L.labpsd(q2, nev, 1e-8, X0=X0)
    assert np.abs(lam - ro.lam).max() <= 1e-9 * np.abs(ro.lam).max()
    assert host_res(q2, lam, X, s.sigma0).max() <= 1e-8 * 1.001
    s.close()


def test_complex_step_entry_points_act_on_the_real_equivalent_pencil(bloch_small):
    """On a complex session hbsd_spmm_pair multiplies the realified block (2n rows, real and
    imaginary part of each dof next to each other) by the real-equivalent pencil."""
    q, _, _, _ = bloch_small
    s = hb().Session.from_problem(q)
    n = q.n
    Xc = pi.seed_normal_block_complex(8, n, 6)
    Xr = np.empty((2 * n, 6))
    Xr[0::2], Xr[1::2] = Xc.real, Xc.imag
    Xd = torch.from_numpy(Xr).cuda()
    HX = torch.zeros_like(Xd)
    SX = torch.zeros_like(Xd)
    s.spmm_pair(Xd, HX, SX)
    torch.cuda.synchronize()
    H, S = q.scipy_pair()
    Hs = H - s.sigma0 * S
    for got, ref in ((HX.cpu().numpy(), Hs @ Xc), (SX.cpu().numpy(), S @ Xc)):
        assert np.abs(got[0::2] - ref.real).max() <= 1e-12 * np.abs(ref).max()
        assert np.abs(got[1::2] - ref.imag).max() <= 1e-12 * np.abs(ref).max()
    s.close()


def test_complex_and_real_inputs_do_not_mix():
    q = pi.small_case(1)
    hbsd = hb()
    rp = np.ascontiguousarray(q.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(q.col_idx, dtype=np.int32)
    hv = np.ascontiguousarray(q.h_val, dtype=np.complex128).view(np.float64)
    sv = np.ascontiguousarray(q.s_val, dtype=np.float64)
    import ctypes as C
    H = hbsd.hbsd_csr(q.n, ci.size, rp.ctypes.data_as(C.POINTER(C.c_int64)), ci.ctypes.data_as(C.POINTER(C.c_int32)),
                      hv.ctypes.data_as(C.POINTER(C.c_double)), 1)
    S = hbsd.hbsd_csr(q.n, ci.size, rp.ctypes.data_as(C.POINTER(C.c_int64)), ci.ctypes.data_as(C.POINTER(C.c_int32)),
                      sv.ctypes.data_as(C.POINTER(C.c_double)), 0)
    dn = np.ascontiguousarray(q.dof_node, dtype=np.int32)
    lb = hbsd.hbsd_local_blocks(dn.ctypes.data_as(C.POINTER(C.c_int32)), None, (C.c_int32 * 3)(*q.grid))
    o = hbsd.options_default(sigma_bar=q.eps_bar)
    h = C.c_void_p()
    rc = hbsd.lib().hbsd_create(C.byref(H), C.byref(S), C.byref(lb), C.byref(o), None, C.byref(h))
    assert rc == hbsd.HBSD_ERR_ARG and h.value is None


@pytest.mark.parametrize("mesh,atoms,enr,seed,kpt,nev", [
    (24, 4, 3, 764689141, (-0.5 * np.pi, 0.5 * np.pi, 0.5 * np.pi), 32),
    (16, 10, 2, 855858841, (0.5 * np.pi, 0.5 * np.pi, -0.5 * np.pi), 64)])
def test_bloch_solves_where_the_cluster_rayleigh_ritz_broke_down(mesh, atoms, enr, seed, kpt, nev):
    """Two Bloch problems of the served request mix on which the 16-CTA Rayleigh-Ritz once returned
    non-finite eigenvectors in the mixed form (the J-paired search block has every eigenvalue
    twice, and CholeskyQR of the inverse-iteration vectors broke down); such a call now falls
    back to the single-CTA kernel and its implicit QL iteration.  Both forms converge, to the same
    eigenvalues, with S-orthonormal complex eigenvectors."""
    p = pi.generate(mesh, atoms, enr, 0.15, seed, kpt=kpt)
    out = {}
    for prec in (hb().PRECISION_MIXED, hb().PRECISION_FP64):
        s = hb().Session.from_problem(p, precision=prec)
        lam, X, it, rc, st = s.solve(nev, 1e-8)
        s.close()
        assert rc == 0 and np.all(np.isfinite(lam))
        out[prec] = (lam, X)
    lam_m, X = out[hb().PRECISION_MIXED]
    lam_d, _ = out[hb().PRECISION_FP64]
    assert np.abs(lam_m - lam_d).max() <= 1e-9 * np.abs(lam_d).max()
    H, S = p.scipy_pair()
    assert np.abs(X.conj().T @ (S @ X) - np.eye(nev)).max() <= 1e-9
