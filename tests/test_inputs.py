"""Generator checks: symmetry, shared pattern, definiteness, Bloch conjugation, closed form."""
import numpy as np
import pytest
import scipy.linalg as sla

from paper_1308_2445_gb300 import pufe_inputs as pi


def test_splitmix64_published_sequence():
    # SplitMix64 from state 0: the first two outputs are the published 0xe220a8397b1dcdaf,
    # 0x6e789e6aa1b965f4 (Steele, Lea & Flood 2014 reference generator).
    with np.errstate(over="ignore"):
        z = pi._mix(np.array([pi._GOLDEN, pi._GOLDEN * np.uint64(2)], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4


def test_normals_moments():
    z = pi.normal(3, pi.STREAM_X0, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_small_case_structure(small_problem):
    p = small_problem
    assert 600 <= p.n <= 700
    H, S = p.scipy_pair()
    Hd, Sd = H.toarray(), S.toarray()
    assert np.array_equal(Hd, Hd.T) and np.array_equal(Sd, Sd.T)
    # same pattern by construction; no row empty; every diagonal stored
    assert np.all(np.diff(p.row_ptr) >= 27)
    np.linalg.cholesky(Sd)
    # eps_bar is below the spectrum: H - eps_bar S is positive definite
    np.linalg.cholesky(Hd - p.eps_bar * Sd)
    # enrichment dofs belong to one atom cluster and point at an enriched node
    assert np.all(p.dof_cluster[: p.grid[0] ** 3] == -1)
    assert np.all(p.dof_cluster[p.grid[0] ** 3:] >= 0)


def test_atom_separation():
    a = pi.place_atoms(5, 8, 0.15)
    for i in range(8):
        for j in range(i):
            d = a[i] - a[j]
            d -= np.round(d)
            assert np.linalg.norm(d) >= 0.3


@pytest.mark.parametrize("kpt", [None, (0.5 * np.pi, -0.5 * np.pi, 0.5 * np.pi)])
def test_closed_form_q1(kpt):
    # unenriched periodic Q1 with constant V: eigenvalues are the tensor-product symbols
    q = pi.generate(5, 0, 0, 0.1, 1, v0=0.7, kpt=kpt)
    H, S = q.scipy_pair()
    w = sla.eigh(H.toarray(), S.toarray(), eigvals_only=True)
    ref = pi.closed_form_eigenvalues(5, 0.7, kpt)
    assert np.abs(w - ref).max() <= 1e-11 * np.abs(ref).max()


def test_bloch_conjugate_pair():
    k = np.array([0.5, -0.5, 0.5]) * np.pi
    a = pi.generate(4, 1, 2, 0.3, 2, kpt=k)
    b = pi.generate(4, 1, 2, 0.3, 2, kpt=-k)
    assert np.array_equal(a.col_idx, b.col_idx)
    assert np.allclose(a.h_val, np.conj(b.h_val), atol=0, rtol=1e-15)
    H, _ = a.scipy_pair()
    Hd = H.toarray()
    assert np.array_equal(Hd, Hd.conj().T)
    assert np.abs(Hd.imag).max() > 1e-3


def test_gamma_equals_zero_k():
    a = pi.generate(4, 1, 2, 0.3, 2)
    b = pi.generate(4, 1, 2, 0.3, 2, kpt=(0.0, 0.0, 0.0))
    assert np.allclose(a.h_val, b.h_val.real, rtol=0, atol=1e-15)
    assert np.allclose(a.s_val, b.s_val.real, rtol=0, atol=1e-15)


def test_scf_noise_changes_h_only():
    a = pi.generate(4, 1, 2, 0.3, 2)
    b = pi.generate(4, 1, 2, 0.3, 2, v_noise=0.01, noise_seed=9)
    assert np.array_equal(a.s_val, b.s_val)
    assert not np.array_equal(a.h_val, b.h_val)
    assert np.abs(a.h_val - b.h_val).max() < 0.05 * np.abs(a.h_val).max()


def test_batch_spec_is_seeded_and_within_the_recipe():
    a = pi.batch_spec(1, 64)
    assert a == pi.batch_spec(1, 64) and a != pi.batch_spec(2, 64)
    assert pi.batch_spec(1, 8) == a[:8]   # a prefix of the same draws
    for mesh, atoms, enr, seed, nev in a:
        assert mesh in pi.BATCH_MESHES and nev in pi.BATCH_NEVS
        assert 4 <= atoms <= 16 and 2 <= enr <= 4 and seed >= 1
    # every mesh size and nev of the recipe occurs in 64 draws
    assert {x[0] for x in a} == set(pi.BATCH_MESHES) and {x[4] for x in a} == set(pi.BATCH_NEVS)


def test_batch_instance_places_fewer_atoms_when_they_do_not_fit():
    p, nev, atoms = pi.batch_instance((8, 4, 2, 3, 16))
    assert nev == 16 and 1 <= atoms <= 4 and p.n > 8 ** 3
