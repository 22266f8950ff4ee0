"""Pins of the oracle's first-order one-step refinement (Sec. 6, future work; reading R18):
x <- x - alpha d, d = A x - b, alpha = (A d . d) / (A d . A d), against values computed by hand,
the identity case, the residual-minimising property, a dense solve and a dense eigensolver.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import labpsd as L
from paper_1308_2445_gb300 import pufe_inputs as pi


def test_first_step_by_hand():
    # A = diag(1, 3), b = (1, 1), x0 = 0: d = (-1, -1), A d = (-1, -3), alpha = 4 / 10,
    # x1 = (0.4, 0.4), d1 = A x1 - b = (-0.6, 0.2), ||d1|| = sqrt(0.4)
    A = np.diag([1.0, 3.0])
    x, steps, hist = L.one_step(lambda y: A @ y, np.ones(2), np.zeros(2), 0.0, 1)
    assert steps == 1
    assert np.allclose(x, [0.4, 0.4], rtol=0, atol=1e-15)
    assert hist == pytest.approx([np.sqrt(2.0), np.sqrt(0.4)], rel=1e-15)


def test_multiple_of_identity_is_solved_in_one_step():
    b = pi.seed_normal_block(2, 50, 1)[:, 0]
    x, steps, hist = L.one_step(lambda y: 2.5 * y, b, np.zeros(50), 1e-13 * np.linalg.norm(b), 10)
    assert steps == 1
    assert np.abs(x - b / 2.5).max() <= 1e-15 * np.abs(b).max()


def test_residual_never_grows_even_for_an_indefinite_operator():
    p = pi.small_case(1)
    Hs, S, _ = L.make_shifted(p)
    lam = sla.eigh(Hs.toarray(), S.toarray(), eigvals_only=True)
    e = 0.5 * (lam[3] + lam[4])                           # inside the spectrum
    r = pi.seed_normal_block(5, p.n, 1)[:, 0]
    _, steps, hist = L.refine_one_step(Hs, S, e, r, np.zeros(p.n), 1e-12, 40)
    assert steps == 40
    assert all(b <= a * (1 + 1e-12) for a, b in zip(hist, hist[1:]))
    assert hist[-1] < hist[0]


def test_converges_to_the_solution_of_a_well_conditioned_system():
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    A = (Q * np.linspace(1.0, 4.0, 40)) @ Q.T
    b = rng.standard_normal(40)
    x, steps, _ = L.one_step(lambda y: A @ y, b, np.zeros(40), 1e-12 * np.linalg.norm(b), 500)
    assert steps < 500
    assert np.abs(x - np.linalg.solve(A, b)).max() <= 1e-11 * np.abs(b).max()


def test_labpsd_with_one_step_refinement_matches_dense_eigh():
    p = pi.small_case(2)
    nev = 16
    r = L.labpsd(p, nev, 1e-10, seed=3, opts=L.Options(local_solver="one_step"))
    assert r.converged and sum(r.n_local) > 0 and sum(int(s.sum()) for s in r.minres_steps) > 0
    H, S = p.scipy_pair()
    lam = sla.eigh(H.toarray(), S.toarray(), eigvals_only=True)[:nev]
    assert np.allclose(r.lam, lam, rtol=0, atol=1e-8 * np.abs(lam).max())
