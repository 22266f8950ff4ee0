"""Pins of the principal-angle helper the parity tests use (tests/subspace.py): against SciPy's
subspace_angles for S = I, against a constructed pair of subspaces at a known angle in an
ill-conditioned S inner product, and for complex bases (a complex phase per column changes no
subspace, so the angle must be zero)."""
import numpy as np
import scipy.linalg as sla

from subspace import gap_indices, s_angle, s_orthonormal


def _spd(n, cond, rng):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Q * np.geomspace(1.0, 1.0 / cond, n)[None, :]) @ Q.T


def test_euclidean_angles_match_scipy():
    rng = np.random.default_rng(1)
    for _ in range(5):
        A = rng.standard_normal((40, 6))
        B = A + 0.1 * rng.standard_normal((40, 6))
        ref = sla.subspace_angles(A, B).max()
        assert abs(s_angle(A, B, np.eye(40)) - ref) <= 1e-12


def test_known_angle_in_an_ill_conditioned_inner_product():
    rng = np.random.default_rng(2)
    n, j = 60, 5
    S = _spd(n, 1e10, rng)
    Q = s_orthonormal(rng.standard_normal((n, 2 * j)), S)       # S-orthonormal, 2j columns
    Qa, Qp = Q[:, :j], Q[:, j:]
    for theta in (1e-7, 1e-3, 0.4):
        B = np.cos(theta) * Qa + np.sin(theta) * Qp
        # any basis of the same subspaces gives the same angle
        A2 = Qa @ rng.standard_normal((j, j))
        B2 = B @ rng.standard_normal((j, j))
        got = s_angle(A2, B2, S)
        assert abs(got - theta) <= 1e-6 * theta + 1e-12, (theta, got)


def test_complex_phases_leave_the_subspace():
    rng = np.random.default_rng(3)
    n, j = 30, 4
    S = _spd(n, 1e4, rng).astype(complex)
    A = rng.standard_normal((n, j)) + 1j * rng.standard_normal((n, j))
    B = A * np.exp(1j * rng.uniform(0, 2 * np.pi, j))[None, :]
    assert s_angle(A, B, S) <= 1e-7
    C = A.copy()
    C[:, 0] = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert s_angle(A, C, S) > 1e-2


def test_gap_indices():
    lam = np.array([1.0, 1.0005, 2.0, 2.0, 3.0])
    assert gap_indices(lam, 5) == [2, 4]
