"""CPU oracle: plain FP64 LABPSD (block preconditioned steepest descent with the hybrid
preconditioner) of Cai, Bai, Pask and Sukumar, Sec. 3 (outline "LABPSD", remarks 1-6)
and Sec. 4 (global factor, MINRES refinement).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import or call this module:
only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm use it.
It shares no code with the CUDA path; the only common input is the seeded generator
(paper_1308_2445_gb300.pufe_inputs), which holds none of the method's arithmetic.

Every step is written in the order and notation of the paper, with numpy / scipy
primitives (sparse matvec, dense Cholesky, dense symmetric eigensolver, sparse direct
solve) as the only library steps.  Readings of points the paper leaves open:
  R1  refinement residual: step 6(b) prints delta r_i = (H - eps_bar S) p_i + r_i; read as
      (H - eps_i S) p_i + r_i, i.e. MINRES on (H - eps_i S) p = -r_i started from the
      globally preconditioned p_i (Eq. indls / approxp).
  R3  the global factor is LDL^T with 1 x 1 pivots in a nested-dissection order (Eq. ldl without
      the 2 x 2 Bunch-Kaufman blocks): for eps_bar below the spectrum every pivot is positive
      and it is a Cholesky factorisation; for eps_bar inside it the negative pivots count the
      eigenvalues below eps_bar (Sylvester).  The oracle uses a library sparse LU without
      pivoting under that ordering (the same factorisation up to rounding); a zero pivot fails.
  R4  sigma0 = eps_bar (Sec. 5 shift making H positive definite); E is held shifted.
  R5  eps_bar = V_min - 0.1 for the synthetic matrices (a rigorous lower bound).
  R6  m0 = max(3, ceil(m/10)) (remark 1).
  R7  a cold start does one Rayleigh-Ritz on X0 (iteration 0); iters counts steps 6-11.
  R8  Res uses Euclidean norms of coefficient vectors and the shifted H (Eq. res1).
  R9  soft locking: only unconverged columns among the first m get a P column (remark 3).
  R10 at l = 1 nothing is localized (no previous Ritz value).
  R11 MINRES stops on its recurrence residual estimate <= eta ||r_i|| or after max_minres
      steps; a start already meeting eta takes 0 steps.
  R12 max_outer default 1000.
  R13 Rayleigh-Ritz on the diagonally scaled pair; if the Cholesky of the scaled S_R breaks
      down or a pivot is below 1e-14, drop S_R eigen-directions below 1e-14 * max.
  R18 the first-order one-step refinement of Sec. 6 (future work) iterates
      p <- p - alpha d with d = (H - eps_i S) p + r_i, the residual of Eq. idealp (the printed
      bracket carries -r_i, at odds with Eq. idealp's sign), alpha = (A d . d) / (A d . A d)
      minimising ||d - alpha A d||, from the globally preconditioned p, with the stopping rule
      of MINRES (||d|| <= eta ||r_i|| or max_minres steps); ||d|| is recomputed, not updated.
  R17 with a nonlocal term H = H_loc + F G F^H (Eq. fgf) the global factor is that of the
      local part H_loc^(1) - eps_bar S (Eq. ldl) and the nonlocal part enters through the
      Sherman-Morrison-Woodbury steps 1-6 of Sec. 4; every product with H (steps 3, 7 and the
      MINRES operator of 6(b)) applies the full H.

Parity unpinned: the outer iteration count and the per-column MINRES step counts of labpsd are
properties of the trajectory, pinned only in special cases (0 iterations from an exact invariant
subspace, the textbook block steepest descent reduction); its eigenpairs are pinned.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

RR_PIVOT_MIN = 1e-14


@dataclasses.dataclass
class Options:
    tau1: float = 0.1          # localisation: Res <= tau1 (remark 4)
    tau2: float = 0.1          # localisation: |eps - eps_prev| <= tau2 |eps_prev| (remark 4)
    eta: float = 0.25          # inexact-solve tolerance, Eq. approxp / Sec. 5
    max_minres: int = 20       # Sec. 5
    max_outer: int = 1000      # R12
    m0: int | None = None      # R6
    local: bool = True         # False: global preconditioner only (step 6(a) alone)
    use_global: bool = True    # False: local only, Sec. 5 (6(b) without 6(a)), reading R16
    local_solver: str = "minres"   # "one_step": the first-order one-step refinement, reading R18


def default_m0(m: int) -> int:
    return max(3, int(math.ceil(m / 10.0)))


def _ctr(A):
    return A.conj().T


# ---------------------------------------------------------------------------------------
# The shifted Hamiltonian: sparse local part plus the low-rank nonlocal part (Eq. fgf)
# ---------------------------------------------------------------------------------------
class ShiftedHamiltonian:
    """Hs = (H_loc - sigma0 S) + F G F^H, held as the sparse local part `loc` and the factors
    F (n x k) and G (k x k Hermitian) of the nonlocal term (none when F is None)."""

    def __init__(self, loc, F=None, G=None):
        self.loc = loc
        self.F = None if F is None or F.shape[1] == 0 else np.asarray(F)
        self.G = None if self.F is None else np.asarray(G)
        self.shape = loc.shape

    def toarray(self):
        """Dense Hs (small cases only)."""
        D = self.loc.toarray()
        if self.F is not None:
            D = D + self.F @ self.G @ _ctr(self.F)
        return D

    def __matmul__(self, X):
        Y = self.loc @ X
        if self.F is not None:
            Y = Y + self.F @ (self.G @ (_ctr(self.F) @ X))
        return Y


# ---------------------------------------------------------------------------------------
# Step 3 / step 7: block matrix-vector products with the shifted H and with S
# ---------------------------------------------------------------------------------------
def spmm_pair(Hs, S, X):
    """(Hs X, S X) -- LABPSD steps 3 and 7."""
    return Hs @ X, S @ X


# ---------------------------------------------------------------------------------------
# Steps 4-5: residuals and relative residual norms (Eq. res1)
# ---------------------------------------------------------------------------------------
def residual(PsiH, PsiS, E, m):
    """R = PsiH(:,1:m) - PsiS(:,1:m) E(1:m,1:m) and Res_i = ||r_i|| / ||H psi_i||."""
    R = PsiH[:, :m] - PsiS[:, :m] * E[None, :m]
    res = np.linalg.norm(R, axis=0) / np.linalg.norm(PsiH[:, :m], axis=0)
    return R, res


def localized(res, E, E_prev, tau1, tau2):
    """Remark 4: Res_i <= tau1 and |eps_i - eps_i^{l-1}| <= tau2 |eps_i^{l-1}|."""
    if E_prev is None:
        return np.zeros(res.shape[0], dtype=bool)
    m = res.shape[0]
    return (res <= tau1) & (np.abs(E[:m] - E_prev[:m]) <= tau2 * np.abs(E_prev[:m]))


# ---------------------------------------------------------------------------------------
# Step 6(a): global preconditioner K = (H - eps_bar S)^{-1}  (Eq. globalprecond, Eq. k1p)
# ---------------------------------------------------------------------------------------
def nested_dissection_nodes(N: int, leaf: int = 64) -> np.ndarray:
    """Fill-reducing node order for the periodic N^3 grid (used only to make the library
    sparse factorisation affordable; the order does not change the result beyond rounding).
    A periodic direction is cut by two planes, an open one by its middle plane; separators
    come after the two halves they split."""
    out = []

    def block(lo, hi):
        g = np.meshgrid(*[np.arange(lo[d], hi[d]) for d in range(3)], indexing="ij")
        return ((g[0] % N) + N * ((g[1] % N) + N * (g[2] % N))).ravel(order="F")

    def rec(lo, hi, per):
        size = [hi[d] - lo[d] for d in range(3)]
        if size[0] * size[1] * size[2] <= leaf:
            out.append(block(lo, hi))
            return
        d = int(np.argmax(size))
        mid = lo[d] + size[d] // 2
        if per[d]:
            a_lo, a_hi = list(lo), list(hi)
            a_lo[d], a_hi[d] = lo[d] + 1, mid
            b_lo, b_hi = list(lo), list(hi)
            b_lo[d] = mid + 1
            per2 = list(per)
            per2[d] = False
            rec(a_lo, a_hi, per2)
            rec(b_lo, b_hi, per2)
            planes = (lo[d], mid)
        else:
            a_hi = list(hi)
            a_hi[d] = mid
            b_lo = list(lo)
            b_lo[d] = mid + 1
            rec(lo, a_hi, per)
            rec(b_lo, hi, per)
            planes = (mid,)
        for pl in planes:
            s_lo, s_hi = list(lo), list(hi)
            s_lo[d], s_hi[d] = pl, pl + 1
            out.append(block(s_lo, s_hi))

    rec([0, 0, 0], [N, N, N], [True, True, True])
    return np.concatenate(out)


class GlobalPreconditioner:
    """P = -K R with K = (H^(1) - eps_bar S)^{-1}, factorised once (Sec. 4, Eq. ldl).

    A is the sparse H^(1) - eps_bar S, or a ShiftedHamiltonian whose local part is that matrix
    and whose F, G give the nonlocal term (R17): then the factor is that of the local part and
    SMW steps 1-4 run here, once."""

    def __init__(self, A, dof_node=None, grid=None, F=None, G=None):
        if isinstance(A, ShiftedHamiltonian):
            A, F, G = A.loc, A.F, A.G
        n = A.shape[0]
        if dof_node is not None and grid is not None:
            N = grid[0]
            order = nested_dissection_nodes(N)
            rank = np.empty(N ** 3, dtype=np.int64)
            rank[order] = np.arange(order.size)
            self.perm = np.lexsort((np.arange(n), rank[np.asarray(dof_node)]))
        else:
            self.perm = np.arange(n)
        Ap = sp.csr_matrix(A)[self.perm][:, self.perm].tocsc()
        self.lu = spla.splu(Ap, permc_spec="NATURAL", diag_pivot_thresh=0.0,
                            options=dict(SymmetricMode=True))
        d = self.lu.U.diagonal()
        if np.any(d == 0) or not np.all(np.isfinite(d)):
            raise np.linalg.LinAlgError("H - eps_bar S met a zero or non-finite pivot")
        self.neg_pivots = int(np.count_nonzero(d.real < 0))     # inertia (R3)
        # SMW steps 1-4 (Sec. 4), only with a nonlocal term
        self.Fhat = self.Fsmw = None
        if F is not None and F.shape[1] > 0:
            F = np.asarray(F)
            k = F.shape[1]
            Fhat = self.solve(F)                               # step 1: Fhat = (H_loc - eps_bar S)^{-1} F
            F = F @ np.asarray(G)                              # step 2: F := F G
            T = np.eye(k) + _ctr(F) @ Fhat                     # step 3: T = I + F^H Fhat
            F = _ctr(np.linalg.solve(T, _ctr(F)))              # step 4: F := F T^{-H}
            self.Fhat, self.Fsmw = Fhat, F

    def solve(self, R):
        R = np.asarray(R)
        out = np.empty_like(R, dtype=np.result_type(R.dtype, self.lu.U.dtype))
        out[self.perm] = self.lu.solve(R[self.perm])
        return out

    def apply(self, R):
        """Step 6(a): P = -K R (SMW steps 5-6 with a nonlocal term)."""
        P = -self.solve(R)                                     # step 5
        if self.Fhat is not None:
            P = P - self.Fhat @ (_ctr(self.Fsmw) @ P)          # step 6
        return P


# ---------------------------------------------------------------------------------------
# Step 6(b): locally accelerated refinement by MINRES (Sec. 4, Eq. indls; Paige-Saunders)
# ---------------------------------------------------------------------------------------
def minres(apply_A, b, x0, tol_abs, maxit):
    """Unpreconditioned MINRES (Paige & Saunders 1975) for a Hermitian A, started at x0.

    Lanczos on r0 = b - A x0 builds the tridiagonal T_k; a QR factorisation of T_k by
    Givens rotations is updated one column per step, and the solution is advanced along
    the direction vectors w_k.  phibar_k = ||b - A x_k|| in exact arithmetic; the loop
    stops as soon as phibar <= tol_abs (R11).  Returns (x, steps, phibar history)."""
    x = np.array(x0, dtype=np.result_type(x0.dtype, b.dtype), copy=True)
    r = b - apply_A(x)
    beta = float(np.linalg.norm(r))
    hist = [beta]
    if beta <= tol_abs or maxit <= 0:
        return x, 0, hist
    v_prev = np.zeros_like(r)
    v = r / beta
    beta_k = beta            # beta_k: norm that produced v_k
    # QR of T_k: rotation (c, s) of the previous step and its predecessor
    c_prev, s_prev = 1.0, 0.0
    c_pp, s_pp = 1.0, 0.0
    w_prev = np.zeros_like(r)
    w_pp = np.zeros_like(r)
    phibar = beta
    steps = 0
    beta_old = 0.0
    for k in range(1, maxit + 1):
        # Lanczos step: A v_k = beta_k v_{k-1} + alpha_k v_k + beta_{k+1} v_{k+1}
        u = apply_A(v)
        alpha = float(np.real(np.vdot(v, u)))
        u = u - alpha * v - beta_old * v_prev
        beta_next = float(np.linalg.norm(u))
        # column k of T_k is (.., beta_old, alpha, beta_next); apply the two previous rotations
        eps_k = s_pp * beta_old
        dbar = c_pp * beta_old
        delta = c_prev * dbar + s_prev * alpha
        gbar = -s_prev * dbar + c_prev * alpha
        # new rotation annihilating beta_next
        gamma = math.hypot(gbar, beta_next)
        c_k = gbar / gamma
        s_k = beta_next / gamma
        phi = c_k * phibar
        phibar = -s_k * phibar
        w = (v - delta * w_prev - eps_k * w_pp) / gamma
        x = x + phi * w
        steps = k
        hist.append(abs(phibar))
        if abs(phibar) <= tol_abs or beta_next == 0.0:
            break
        v_prev, v = v, u / beta_next
        beta_old = beta_next
        c_pp, s_pp, c_prev, s_prev = c_prev, s_prev, c_k, s_k
        w_pp, w_prev = w_prev, w
    return x, steps, hist


def refine(Hs, S, eps_i, r_i, p0, eta, maxit):
    """Step 6(b): solve (H - eps_i S) p = -r_i inexactly from p0 (R1, Eq. approxp)."""
    def apply_A(y):
        return Hs @ y - eps_i * (S @ y)
    tol_abs = eta * float(np.linalg.norm(r_i))
    return minres(apply_A, -r_i, p0, tol_abs, maxit)


def one_step(apply_A, b, x0, tol_abs, maxit):
    """First-order one-step iteration with the residual-minimising step (R18): for A x = b,
    d = A x - b, x <- x - alpha d with alpha = (A d . d) / (A d . A d).  Stops when
    ||A x - b|| <= tol_abs or after maxit steps.  Returns (x, steps, ||d|| history)."""
    x = np.array(x0, dtype=np.result_type(x0.dtype, b.dtype), copy=True)
    d = apply_A(x) - b
    dn = float(np.linalg.norm(d))
    hist = [dn]
    steps = 0
    while dn > tol_abs and steps < maxit:
        u = apply_A(d)
        uu = float(np.real(np.vdot(u, u)))
        if uu == 0.0:
            break
        alpha = float(np.real(np.vdot(u, d))) / uu
        x = x - alpha * d
        d = d - alpha * u
        dn = float(np.linalg.norm(d))
        steps += 1
        hist.append(dn)
    return x, steps, hist


def refine_one_step(Hs, S, eps_i, r_i, p0, eta, maxit):
    """Step 6(b) by the first-order one-step refinement of Sec. 6 (R18)."""
    def apply_A(y):
        return Hs @ y - eps_i * (S @ y)
    tol_abs = eta * float(np.linalg.norm(r_i))
    return one_step(apply_A, -r_i, p0, tol_abs, maxit)


# ---------------------------------------------------------------------------------------
# Steps 8-9: reduced GHEP and Rayleigh-Ritz (remark 6; R13)
# ---------------------------------------------------------------------------------------
def reduced_pair(Z, ZH, ZS):
    """Step 8: H_R = Z^H [H Z], S_R = Z^H [S Z], made exactly Hermitian as (A + A^H)/2."""
    HR = _ctr(Z) @ ZH
    SR = _ctr(Z) @ ZS
    return 0.5 * (HR + _ctr(HR)), 0.5 * (SR + _ctr(SR))


def rayleigh_ritz(HR, SR, k):
    """Step 9: lowest k eigenpairs (Gamma, W) of H_R W = S_R W Gamma, Gamma ascending.

    S_R is scaled by D = diag(S_R)^{-1/2}; with the scaled pair (D H_R D, D S_R D) = (Hd, Sd):
    Cholesky Sd = L L^H, C = L^{-1} Hd L^{-H}, C = V Theta V^H, W = D L^{-H} V.  Rank-revealing
    fallback (R13) if the Cholesky breaks down or a pivot is below RR_PIVOT_MIN.
    Returns (Gamma, W, used_fallback)."""
    d = 1.0 / np.sqrt(np.real(np.diag(SR)))
    Hd = HR * d[:, None] * d[None, :]
    Sd = SR * d[:, None] * d[None, :]
    fallback = False
    try:
        L = np.linalg.cholesky(Sd)
        if np.min(np.real(np.diag(L))) ** 2 < RR_PIVOT_MIN:
            fallback = True
    except np.linalg.LinAlgError:
        fallback = True
    if not fallback:
        Y = sla.solve_triangular(L, Hd, lower=True)
        C = _ctr(sla.solve_triangular(L, _ctr(Y), lower=True))
        C = 0.5 * (C + _ctr(C))
        theta, V = np.linalg.eigh(C)
        Wd = sla.solve_triangular(_ctr(L), V[:, :k], lower=False)
    else:
        mu, Q = np.linalg.eigh(Sd)
        keep = mu > RR_PIVOT_MIN * mu[-1]
        B = Q[:, keep] / np.sqrt(mu[keep])[None, :]
        C = _ctr(B) @ Hd @ B
        C = 0.5 * (C + _ctr(C))
        theta, V = np.linalg.eigh(C)
        if V.shape[1] < k:
            raise np.linalg.LinAlgError("search space rank below the number of wanted pairs")
        Wd = B @ V[:, :k]
    return theta[:k], Wd * d[:, None], fallback


# ---------------------------------------------------------------------------------------
# The LABPSD outline, steps 1-12
# ---------------------------------------------------------------------------------------
@dataclasses.dataclass
class Result:
    lam: np.ndarray            # nev eigenvalues (unshifted), ascending
    X: np.ndarray              # n x nev eigenvectors, S-orthonormal
    iters: int                 # outer BPSD iterations (R7)
    converged: bool
    res: np.ndarray            # final Res_i, i < nev
    E_all: np.ndarray          # final m + m0 Ritz values (unshifted)
    res_history: list          # Res_max per iteration (before the test of step 5)
    ritz_history: list         # shifted Ritz values after each Rayleigh-Ritz
    minres_steps: list         # per iteration: array of MINRES steps per refined column
    n_precond: list            # per iteration: number of preconditioned columns p
    n_local: list              # per iteration: number of localized columns a
    rr_fallbacks: int
    sigma0: float


def make_shifted(problem):
    """R4: Hs = H - sigma0 S with sigma0 = eps_bar; returns (Hs, S, sigma0), Hs a
    ShiftedHamiltonian (carrying the nonlocal term of the problem, if any)."""
    H, S = problem.scipy_pair()
    sigma0 = problem.eps_bar
    F = getattr(problem, "F", None)
    return ShiftedHamiltonian((H - sigma0 * S).tocsr(), F, getattr(problem, "G", None)), S.tocsr(), sigma0


def labpsd(problem, nev, tol, X0=None, opts: Options | None = None, seed=1,
           precond: GlobalPreconditioner | None = None, on_iteration=None) -> Result:
    """Lowest nev eigenpairs of H x = lambda S x to Res_max <= tol (remark 2)."""
    opts = opts or Options()
    m = int(nev)
    m0 = default_m0(m) if opts.m0 is None else int(opts.m0)
    w = m + m0
    Hs, S, sigma0 = make_shifted(problem)
    n = problem.n
    if precond is None and opts.use_global:
        precond = GlobalPreconditioner((Hs.loc - (problem.eps_bar - sigma0) * S).tocsr(),
                                       problem.dof_node, problem.grid, F=Hs.F, G=Hs.G)
    if X0 is None:
        from paper_1308_2445_gb300.pufe_inputs import seed_normal_block
        X0 = seed_normal_block(seed, n, w)
    X0 = np.asarray(X0)
    if X0.shape != (n, w):
        raise ValueError(f"X0 must be n x (m + m0) = {n} x {w}")

    # steps 1-3 on a cold start (R7): Rayleigh-Ritz on span(X0), then Psi_H, Psi_S
    XH, XS = spmm_pair(Hs, S, X0)
    HR, SR = reduced_pair(X0, XH, XS)
    E, W, fb = rayleigh_ritz(HR, SR, w)
    Psi, PsiH, PsiS = X0 @ W, XH @ W, XS @ W
    rr_fallbacks = int(fb)
    E_prev = None
    ritz_history = [E.copy()]
    res_history, minres_steps, n_precond, n_local = [], [], [], []
    iters = 0
    converged = False
    while True:
        # step 4: residuals of the first m columns
        R, res = residual(PsiH, PsiS, E, m)
        res_history.append(float(res.max()))
        # step 5: convergence test (remark 2)
        if res.max() <= tol:
            converged = True
            break
        if iters >= opts.max_outer:
            break
        # step 6: search directions for unconverged columns only (remark 3)
        U = np.nonzero(res > tol)[0]
        if opts.use_global:
            P = precond.apply(R[:, U])                                # 6(a)
        else:
            # local only (Sec. 5, reading R16): no global step; an unlocalized column keeps the
            # unpreconditioned direction -r_i, a localized one is refined by MINRES from zero
            P = -R[:, U]
        loc = localized(res, E, E_prev, opts.tau1, opts.tau2) if opts.local else np.zeros(m, bool)
        steps = []
        solver = refine_one_step if opts.local_solver == "one_step" else refine
        for j, i in enumerate(U):
            if loc[i]:                                                  # 6(b)
                p0 = P[:, j] if opts.use_global else np.zeros(n)
                P[:, j], k, _ = solver(Hs, S, E[i], R[:, i], p0, opts.eta, opts.max_minres)
                steps.append(k)
        minres_steps.append(np.array(steps, dtype=np.int64))
        n_precond.append(int(U.size))
        n_local.append(int(np.count_nonzero(loc[U])))
        # step 7
        PH, PS = spmm_pair(Hs, S, P)
        # step 8
        Z = np.hstack([Psi, P])
        ZH = np.hstack([PsiH, PH])
        ZS = np.hstack([PsiS, PS])
        HR, SR = reduced_pair(Z, ZH, ZS)
        # step 9
        E_new, W, fb = rayleigh_ritz(HR, SR, w)
        rr_fallbacks += int(fb)
        # steps 10-11
        Psi, PsiH, PsiS = Z @ W, ZH @ W, ZS @ W
        E_prev, E = E, E_new
        iters += 1
        ritz_history.append(E.copy())
        if on_iteration is not None:
            on_iteration(iters, res)
    return Result(lam=E[:m] + sigma0, X=Psi[:, :m], iters=iters, converged=converged,
                  res=res, E_all=E + sigma0, res_history=res_history, ritz_history=ritz_history,
                  minres_steps=minres_steps, n_precond=n_precond, n_local=n_local,
                  rr_fallbacks=rr_fallbacks, sigma0=sigma0)
