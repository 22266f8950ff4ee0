"""Principal angles between subspaces in the S inner product <x, y>_S = x^H S y, S sparse
Hermitian positive definite: the measure the parity tests compare eigenvector subspaces with.

For bases A, B (n x j, real or complex) both are first made S-orthonormal (Cholesky of their
S-Gram), then sin(theta_max) = ||(I - Qa Qa^H S) Qb||_S, the S-norm of the part of span(B)
outside span(A).  Computing the sine (not arccos of the cosines) keeps small angles accurate."""
import numpy as np


def s_orthonormal(X, S):
    G = X.conj().T @ (S @ X)
    G = 0.5 * (G + G.conj().T)
    L = np.linalg.cholesky(G)
    return np.linalg.solve(L, X.conj().T).conj().T          # X L^{-H}


def s_angle(A, B, S):
    """Largest principal angle (radians) between span(A) and span(B) in the S inner product."""
    Qa, Qb = s_orthonormal(A, S), s_orthonormal(B, S)
    M = Qb - Qa @ (Qa.conj().T @ (S @ Qb))
    G = M.conj().T @ (S @ M)
    G = 0.5 * (G + G.conj().T)
    s2 = float(np.linalg.eigvalsh(G).max())
    return float(np.arcsin(min(1.0, np.sqrt(max(s2, 0.0)))))


def gap_indices(lam, nev, rel_gap=1e-2):
    """Indices j (1 <= j < nev) where lam[j] - lam[j-1] > rel_gap * max|lam|: the subspaces
    span X(:, :j) the comparison is made on (a cluster is compared only as a whole)."""
    lam = np.asarray(lam)
    scale = np.abs(lam).max()
    return [j for j in range(1, nev) if lam[j] - lam[j - 1] > rel_gap * scale]
