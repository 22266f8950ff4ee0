"""Seeded synthetic inputs: PUFE-like generalized eigenproblems H x = lambda S x.

This module is the one input source shared by the CPU oracle and the CUDA path.
It assembles matrices and draws random numbers; it holds none of the
eigensolver's arithmetic (no residuals, preconditioners, Rayleigh-Ritz ...).

The paper's own matrices (CuAl / CeAl partition-of-unity FE discretisations,
Sec. 2 and Sec. 5) are not available, so this generator builds a stand-in with
the same structural features (Sec. 2, Table 1): a periodic Q1 hexahedral FE
basis on the unit cube enriched, near each "atom", by products of the nodal
hat function with Gaussians (a partition-of-unity enrichment).  The result is
a sparse real-symmetric (Gamma point) or complex-Hermitian (Bloch k) pair with
H and S sharing one sparsity pattern, S positive definite and badly
conditioned, and H, S sharing a near-null space.

Definitions (all integrals by 3x3x3 Gauss-Legendre quadrature per element):
  * S_ij = int psi_i psi_j ,  H_ij = 1/2 int grad psi_i . grad psi_j + int V psi_i psi_j
  * V(r) = v0 - sum_a Z exp(-|r - R_a|^2 / width), |.| the minimum-image
    distance on the periodic unit cube.
  * enrichment: every node within r_c (minimum image) of atom a carries n_enr
    extra functions  phi_node(r) * exp(-alpha_j |r - R_a*|^2), R_a* the image
    of R_a nearest the node, alpha_j the first n_enr of (8, 20, 50, 120) * (N/8)^2
    (values stated for the 8^3 mesh, scaled with h^-2).
  * atoms: uniform in [0,1)^3 by rejection so that all pairwise minimum-image
    distances are >= 2 r_c (each enriched node then belongs to one atom).
  * Bloch k: a basis function wrapped by the lattice translation T picks up the
    phase exp(i k.T); H and S become complex Hermitian.
  * nonlocal term (optional, Sec. 4, Eq. fgf): H_nl = F G F^T with
    F_ij = int psi_i beta_j for n_proj projectors per atom -- an s channel
    beta = c exp(-d^2 / w_p) f(d) and, for n_proj = 4, three p channels
    c' d_x exp(-d^2 / w_p) f(d) (likewise y, z) -- with d the minimum-image offset
    from the atom, the smooth cutoff f(d) = (1 - d^2 / r_p^2)^2 for d < r_p (0
    beyond, so F is sparse), and c, c' normalising int beta^2 = 1 on the
    quadrature.  G is diagonal: E_s on the s channel, E_p on the p channels
    (positive, so eps_bar = V_min - 0.1 still bounds the spectrum from below).

Random numbers: SplitMix64 (Steele, Lea, Flood 2014), used as a counter-based
generator: draw t of stream s is mix(key(seed, s) + (t+1) * 0x9E3779B97F4A7C15).
Uniform doubles take the top 53 bits; normals use Box-Muller on consecutive
uniform pairs.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

ALPHAS = (8.0, 20.0, 50.0, 120.0)

# stream tags for independent draws
STREAM_ATOMS = 1
STREAM_X0 = 2
STREAM_NOISE = 3
STREAM_BATCH = 4
STREAM_REQUESTS = 5
STREAM_X0_IM = 6      # imaginary part of a complex start block


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream) * _GOLDEN)], dtype=np.uint64)
        return _mix(s + _GOLDEN)[0]


def uniform(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """count uniform doubles in [0, 1) from (seed, stream), draws offset..offset+count-1."""
    key = stream_key(seed, stream)
    with np.errstate(over="ignore"):
        t = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = _mix(key + t * _GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """count standard normals by Box-Muller from consecutive uniform pairs."""
    pairs = (count + 1) // 2
    u = uniform(seed, stream, 2 * pairs)
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-2.0 * np.log1p(-u1))
    z = np.empty(2 * pairs)
    z[0::2] = rad * np.cos(2.0 * math.pi * u2)
    z[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return z[:count]


def seed_normal_block(seed: int, n: int, w: int, stream: int = STREAM_X0) -> np.ndarray:
    """Seed-normal n x w starting block X0 (row-major, entry (i, j) = draw i*w + j)."""
    return normal(seed, stream, n * w).reshape(n, w)


def seed_normal_block_complex(seed: int, n: int, w: int) -> np.ndarray:
    """Complex start block for Hermitian (Bloch) problems: real part from the X0 stream, imaginary
    part from its own stream, both seed-normal (what the library draws for X0 = NULL)."""
    return seed_normal_block(seed, n, w) + 1j * seed_normal_block(seed, n, w, stream=STREAM_X0_IM)


@dataclasses.dataclass
class Problem:
    """A generated pair (H, S) in CSR form with one shared pattern."""
    n: int
    row_ptr: np.ndarray      # int64[n+1]
    col_idx: np.ndarray      # int32[nnz]
    h_val: np.ndarray        # float64[nnz] or complex128[nnz]
    s_val: np.ndarray        # float64[nnz] or complex128[nnz]
    dof_node: np.ndarray     # int32[n]  node carrying each dof
    dof_cluster: np.ndarray  # int32[n]  atom of an enrichment dof, -1 for nodal dofs
    grid: tuple              # (N, N, N) nodes per direction (periodic)
    atoms: np.ndarray        # float64[n_atoms, 3]
    v_min: float             # min of V over all quadrature points
    eps_bar: float           # global shift below the spectrum: v_min - 0.1
    kpt: tuple | None = None
    params: dict = dataclasses.field(default_factory=dict)
    F: np.ndarray | None = None  # n x k nonlocal projector matrix (None: no nonlocal term)
    G: np.ndarray | None = None  # k x k symmetric coupling of the projectors

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def is_complex(self) -> bool:
        return np.iscomplexobj(self.h_val)

    def scipy_pair(self):
        import scipy.sparse as sp
        shape = (self.n, self.n)
        H = sp.csr_matrix((self.h_val, self.col_idx, self.row_ptr), shape=shape)
        S = sp.csr_matrix((self.s_val, self.col_idx, self.row_ptr), shape=shape)
        return H, S


def _gauss3():
    a = 0.5 * math.sqrt(0.6)
    pts = np.array([0.5 - a, 0.5, 0.5 + a])
    wts = np.array([5.0, 8.0, 5.0]) / 18.0
    return pts, wts


def _q1_reference():
    """Shape values N[a, q] and reference gradients dN[a, q, d] at the 27 Gauss points."""
    pts, wts = _gauss3()
    qx, qy, qz = np.meshgrid(pts, pts, pts, indexing="ij")
    xi = np.stack([qx.ravel(), qy.ravel(), qz.ravel()], axis=1)  # (27, 3), q = iz + 3(iy + 3 ix)
    wx, wy, wz = np.meshgrid(wts, wts, wts, indexing="ij")
    w = (wx * wy * wz).ravel()
    corners = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)])  # (8, 3)
    f = np.where(corners[:, None, :] == 1, xi[None, :, :], 1.0 - xi[None, :, :])  # (8, 27, 3)
    df = np.where(corners[:, None, :] == 1, 1.0, -1.0) * np.ones_like(f)
    N = f.prod(axis=2)
    dN = np.empty((8, 27, 3))
    for d in range(3):
        others = [e for e in range(3) if e != d]
        dN[:, :, d] = df[:, :, d] * f[:, :, others[0]] * f[:, :, others[1]]
    return xi, w, corners, N, dN


def place_atoms(seed: int, n_atoms: int, r_c: float, max_draws: int = 100000) -> np.ndarray:
    """Uniform atoms in [0,1)^3, rejecting any closer than 2 r_c (minimum image) to an accepted one."""
    u = uniform(seed, STREAM_ATOMS, 3 * max_draws).reshape(max_draws, 3)
    atoms = []
    for cand in u:
        ok = True
        for a in atoms:
            d = cand - a
            d -= np.round(d)
            if float(np.dot(d, d)) < (2.0 * r_c) ** 2:
                ok = False
                break
        if ok:
            atoms.append(cand)
            if len(atoms) == n_atoms:
                return np.array(atoms)
    raise ValueError("could not place atoms with the requested separation")


def generate(n_el: int, n_atoms: int, n_enr: int, r_c: float, seed: int, *, Z: float = 4.0,
             width: float = 0.05, v0: float = 0.0, kpt=None, v_noise: float = 0.0,
             noise_seed: int | None = None, atoms: np.ndarray | None = None, n_proj: int = 0,
             proj_width: float = 0.01, proj_rc: float = 0.2, proj_energies=(1.0, 0.5)) -> Problem:
    """Assemble (H, S) on an n_el^3 periodic Q1 mesh of the unit cube.

    kpt: Bloch wave vector (3 floats) or None for the Gamma point (real matrices).
    v_noise: if > 0, V at every quadrature point is multiplied by (1 + v_noise * N(0,1))
             with normals from (noise_seed, STREAM_NOISE) -- an SCF-style follow-up that
             changes H but not S.
    n_proj: nonlocal projectors per atom (0: none, 1: s, 4: s and p); proj_width = w_p,
            proj_rc = r_p, proj_energies = (E_s, E_p).  Real (Gamma point) problems only.
    """
    if n_proj not in (0, 1, 4):
        raise ValueError("n_proj must be 0, 1 or 4")
    if n_proj and kpt is not None:
        raise ValueError("the nonlocal term is generated for real (Gamma point) problems only")
    N = int(n_el)
    h = 1.0 / N
    nn = N ** 3
    xi, wq, corners, Nref, dNref = _q1_reference()
    if atoms is None:
        atoms = place_atoms(seed, n_atoms, r_c) if n_atoms > 0 else np.zeros((0, 3))
    atoms = np.asarray(atoms, dtype=np.float64).reshape(-1, 3)
    # alpha_j are stated for the 8^3 reference mesh; they scale with h^-2 so that every
    # mesh resolves its Gaussians alike (alpha h^2 fixed).  Taken literally on finer
    # meshes the low-alpha enrichments fall inside the Q1 space and S is singular in FP64.
    alphas = np.array(ALPHAS[:n_enr], dtype=np.float64) * (N / 8.0) ** 2
    cplx = kpt is not None
    kvec = np.asarray(kpt, dtype=np.float64) if cplx else np.zeros(3)

    # ---- element geometry ---------------------------------------------------------------
    e_idx = np.arange(nn)
    ex, ey, ez = e_idx % N, (e_idx // N) % N, e_idx // (N * N)
    e_org = np.stack([ex, ey, ez], axis=1)                                   # (E, 3) element origin (ints)
    loc = e_org[:, None, :] + corners[None, :, :]                            # (E, 8, 3) unwrapped node ints
    wrap = loc // N                                                          # lattice translation T (0/1)
    locw = loc % N
    gnode = locw[:, :, 0] + N * (locw[:, :, 1] + N * locw[:, :, 2])          # (E, 8) global node
    rq = (e_org[:, None, :] + xi[None, :, :]) * h                            # (E, 27, 3) quadrature points

    # ---- potential at quadrature points ---------------------------------------------
    V = np.full((nn, 27), v0, dtype=np.float64)
    for a in atoms:
        d = rq - a
        d -= np.round(d)
        V -= Z * np.exp(-np.einsum("eqd,eqd->eq", d, d) / width)
    if v_noise > 0.0:
        ns = seed if noise_seed is None else noise_seed
        V *= 1.0 + v_noise * normal(ns, STREAM_NOISE, V.size).reshape(V.shape)
    v_min = float(V.min())

    # ---- enrichment bookkeeping -----------------------------------------------------
    node_ijk = np.stack([np.arange(nn) % N, (np.arange(nn) // N) % N, np.arange(nn) // (N * N)], axis=1)
    node_pos = node_ijk * h
    node_atom = np.full(nn, -1, dtype=np.int64)
    node_center = np.zeros((nn, 3))
    for ia, a in enumerate(atoms):
        d = node_pos - a
        d -= np.round(d)
        inside = np.einsum("nd,nd->n", d, d) <= r_c * r_c
        if np.any(node_atom[inside] >= 0):
            raise ValueError("enrichment spheres overlap")
        node_atom[inside] = ia
        node_center[inside] = node_pos[inside] - d[inside]                # nearest image of the atom
    enr_nodes = np.nonzero(node_atom >= 0)[0] if n_enr > 0 else np.zeros(0, dtype=np.int64)
    enr_slot = np.full(nn, -1, dtype=np.int64)
    enr_slot[enr_nodes] = np.arange(enr_nodes.size)
    n = nn + enr_nodes.size * n_enr
    dof_node = np.concatenate([np.arange(nn), np.repeat(enr_nodes, n_enr)]).astype(np.int32)
    dof_cluster = np.concatenate([np.full(nn, -1), np.repeat(node_atom[enr_nodes], n_enr)]).astype(np.int32)

    def phase_of(wrapv):
        if not cplx:
            return None
        return np.exp(1j * (wrapv @ kvec))

    rows, cols, hv, sv = [], [], [], []

    # ---- nodal (Q1-Q1) block, all elements -----------------------------------------
    G = dNref / h                                                             # (8, 27, 3)
    wJ = wq * h ** 3
    Kqq = np.einsum("aqd,bqd,q->ab", G, G, wJ)
    Mqq = np.einsum("aq,bq,q->ab", Nref, Nref, wJ)
    NN = np.einsum("aq,bq->qab", Nref, Nref).reshape(27, 64) * wJ[:, None]
    Vqq = V @ NN                                                              # (E, 64)
    Hqq = 0.5 * Kqq.reshape(1, 64) + Vqq
    Sqq = np.broadcast_to(Mqq.reshape(1, 64), Hqq.shape)
    ra = np.repeat(gnode, 8, axis=1)                                          # (E, 64) row node a
    cb = np.tile(gnode, (1, 8))                                               # (E, 64) col node b
    if cplx:
        ph = phase_of(wrap.reshape(-1, 3)).reshape(nn, 8)
        pab = np.conj(np.repeat(ph, 8, axis=1)) * np.tile(ph, (1, 8))
        Hqq = Hqq * pab
        Sqq = Sqq * pab
    rows.append(ra.ravel()); cols.append(cb.ravel())
    hv.append(np.asarray(Hqq).ravel()); sv.append(np.asarray(Sqq).ravel())

    # ---- enrichment blocks, elements that touch an enriched node ------------------
    if enr_nodes.size > 0:
        touched = np.nonzero((node_atom[gnode] >= 0).any(axis=1))[0]
        gn = gnode[touched]                                                   # (Ee, 8)
        msk = node_atom[gn] >= 0                                              # (Ee, 8)
        # centre of each local node's Gaussian, translated with the node's wrap
        cen = node_center[gn] + wrap[touched]                                 # (Ee, 8, 3)
        r = rq[touched]                                                       # (Ee, 27, 3)
        dr = r[:, None, :, :] - cen[:, :, None, :]                            # (Ee, 8, 27, 3)
        r2 = np.einsum("eaqd,eaqd->eaq", dr, dr)
        g = np.exp(-alphas[None, None, :, None] * r2[:, :, None, :])          # (Ee, 8, J, 27)
        g *= msk[:, :, None, None]
        dg = -2.0 * alphas[None, None, :, None, None] * dr[:, :, None, :, :] * g[..., None]  # (Ee,8,J,27,3)
        J = n_enr
        psi = Nref[None, :, None, :] * g                                      # (Ee, 8, J, 27)
        dpsi = G[None, :, None, :, :] * g[..., None] + Nref[None, :, None, :, None] * dg
        Ee = touched.size
        nf = 8 + 8 * J
        B = np.concatenate([np.broadcast_to(Nref, (Ee, 8, 27)), psi.reshape(Ee, 8 * J, 27)], axis=1)
        D = np.concatenate([np.broadcast_to(G, (Ee, 8, 27, 3)), dpsi.reshape(Ee, 8 * J, 27, 3)], axis=1)
        Vw = V[touched] * wJ[None, :]                                         # (Ee, 27)
        Bw = B * wJ[None, None, :]
        Me = np.einsum("eaq,ebq->eab", Bw, B)
        Ke = np.einsum("eaqd,ebqd->eab", D * wJ[None, None, :, None], D)
        Ve = np.einsum("eaq,ebq->eab", B * Vw[:, None, :], B)
        He = 0.5 * Ke + Ve
        # global dof of each local function
        gdof = np.empty((Ee, nf), dtype=np.int64)
        gdof[:, :8] = gn
        slot = enr_slot[gn]                                                   # (Ee, 8)
        edof = nn + slot[:, :, None] * J + np.arange(J)[None, None, :]
        gdof[:, 8:] = edof.reshape(Ee, 8 * J)
        valid = np.concatenate([np.ones((Ee, 8), bool), np.repeat(msk, J, axis=1)], axis=1)
        is_enr = np.concatenate([np.zeros(8, bool), np.ones(8 * J, bool)])
        keep = valid[:, :, None] & valid[:, None, :] & (is_enr[None, :, None] | is_enr[None, None, :])
        if cplx:
            phl = phase_of(wrap[touched].reshape(-1, 3)).reshape(Ee, 8)
            phf = np.concatenate([phl, np.repeat(phl, J, axis=1)], axis=1)      # (Ee, nf)
            pab = np.conj(phf[:, :, None]) * phf[:, None, :]
            He = He * pab
            Me = Me * pab
        ee, aa, bb = np.nonzero(keep)
        rows.append(gdof[ee, aa]); cols.append(gdof[ee, bb])
        hv.append(He[ee, aa, bb]); sv.append(Me[ee, aa, bb])

    # ---- nonlocal projectors F_ij = int psi_i beta_j (optional) --------------------------
    Fnl = Gnl = None
    if n_proj > 0 and atoms.shape[0] > 0:
        kp = atoms.shape[0] * n_proj
        Fnl = np.zeros((n, kp))
        if enr_nodes.size > 0:
            tpos = np.full(nn, -1, dtype=np.int64)
            tpos[touched] = np.arange(touched.size)
        for ia, a in enumerate(atoms):
            d = rq - a
            d -= np.round(d)
            r2 = np.einsum("eqd,eqd->eq", d, d)
            sup = np.nonzero((r2 < proj_rc * proj_rc).any(axis=1))[0]           # elements meeting the support
            dd, rr = d[sup], r2[sup]
            cut = np.where(rr < proj_rc * proj_rc, (1.0 - rr / (proj_rc * proj_rc)) ** 2, 0.0)
            g = np.exp(-rr / proj_width) * cut                                     # (Es, 27)
            chans = [g, dd[..., 0] * g, dd[..., 1] * g, dd[..., 2] * g][:n_proj]
            beta = np.stack(chans, axis=-1)                                        # (Es, 27, n_proj)
            norm2 = np.einsum("eqc,eqc,q->c", beta, beta, wJ)
            bw = beta * (wJ[None, :, None] / np.sqrt(norm2)[None, None, :])        # weighted, normalised
            col0 = ia * n_proj
            nodal = np.einsum("aq,eqc->eac", Nref, bw)                             # (Es, 8, n_proj)
            for c in range(n_proj):
                np.add.at(Fnl[:, col0 + c], gnode[sup].ravel(), nodal[:, :, c].ravel())
            if enr_nodes.size > 0:
                tp = tpos[sup]
                sel = np.nonzero(tp >= 0)[0]
                if sel.size:
                    te = tp[sel]
                    enr = np.einsum("efq,eqc->efc", B[te, 8:], bw[sel])              # (Et, 8J, n_proj)
                    ok = valid[te, 8:]
                    rws = gdof[te, 8:][ok]
                    for c in range(n_proj):
                        np.add.at(Fnl[:, col0 + c], rws, enr[:, :, c][ok])
        ene = np.array([proj_energies[0]] + [proj_energies[1]] * 3)[:n_proj]
        Gnl = np.diag(np.tile(ene, atoms.shape[0]))

    rows = np.concatenate(rows).astype(np.int64)
    cols = np.concatenate(cols).astype(np.int64)
    hv = np.concatenate(hv)
    sv = np.concatenate(sv)
    key = rows * n + cols
    ukey, inv = np.unique(key, return_inverse=True)
    if cplx:
        hsum = np.bincount(inv, weights=hv.real) + 1j * np.bincount(inv, weights=hv.imag)
        ssum = np.bincount(inv, weights=sv.real) + 1j * np.bincount(inv, weights=sv.imag)
    else:
        hsum = np.bincount(inv, weights=hv)
        ssum = np.bincount(inv, weights=sv)
    urow = ukey // n
    ucol = (ukey % n).astype(np.int32)
    # the pattern is symmetric; average each entry with its mirror so that H and S are
    # exactly Hermitian whatever order the element sums above were taken in
    mirror = np.searchsorted(ukey, ucol.astype(np.int64) * n + urow)
    hsum = 0.5 * (hsum + np.conj(hsum[mirror]))
    ssum = 0.5 * (ssum + np.conj(ssum[mirror]))
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(urow, minlength=n), out=row_ptr[1:])
    params = dict(n_el=N, n_atoms=int(atoms.shape[0]), n_enr=n_enr, r_c=r_c, seed=seed, Z=Z,
                  width=width, v0=v0, v_noise=v_noise, n_proj=n_proj, proj_width=proj_width,
                  proj_rc=proj_rc, proj_energies=tuple(proj_energies))
    return Problem(n=n, row_ptr=row_ptr, col_idx=ucol, h_val=hsum, s_val=ssum,
                   dof_node=dof_node, dof_cluster=dof_cluster, grid=(N, N, N), atoms=atoms,
                   v_min=v_min, eps_bar=v_min - 0.1, kpt=None if kpt is None else tuple(kvec),
                   params=params, F=Fnl, G=Gnl)


# ---- named workloads -------------------------------------------------------------------

def small_case(seed: int = 1) -> Problem:
    """8^3 Q1 elements, 2 atoms (Z=4), 2 enrichment dofs per node within r_c=0.25 (~650 dofs)."""
    return generate(8, 2, 2, 0.25, seed)


SMALL_NEV = 16


def medium_case(seed: int = 1) -> Problem:
    """32^3 Q1 elements, 8 atoms (Z=4), 4 enrichment dofs per node within r_c=0.15 (~47k dofs)."""
    return generate(32, 8, 4, 0.15, seed)


MEDIUM_NEV = 64


def medium_nonlocal_case(seed: int = 1) -> Problem:
    """The 32^3 medium case with a nonlocal term: s and p projectors on each of the 8 atoms (k = 32)."""
    return generate(32, 8, 4, 0.15, seed, n_proj=4)


def large_case(seed: int = 1) -> Problem:
    """64^3 Q1 elements, 32 atoms (Z=4), 4 enrichment dofs per node within r_c=0.08 (~320k dofs)."""
    return generate(64, 32, 4, 0.08, seed)


LARGE_NEV = 256


# ---- the batched workload: uneven independent instances ---------------------------------

BATCH_MESHES = (16, 24, 32, 40)
BATCH_NEVS = (32, 64, 128)
BATCH_RC = 0.15


def batch_spec(seed: int, count: int = 64, meshes=BATCH_MESHES, nevs=BATCH_NEVS):
    """Instance list of the batched workload, drawn from (seed, STREAM_BATCH): per instance
    (mesh, atoms, enrichment dofs per node, instance seed, nev) with the mesh from `meshes`,
    4-16 atoms, 2-4 enrichment dofs within r_c = 0.15 and nev from `nevs`, all uniform."""
    u = uniform(seed, STREAM_BATCH, 5 * count).reshape(count, 5)
    out = []
    for i in range(count):
        out.append((int(meshes[min(len(meshes) - 1, int(u[i, 0] * len(meshes)))]),
                    4 + min(12, int(u[i, 1] * 13)),
                    2 + min(2, int(u[i, 2] * 3)),
                    1 + int(u[i, 3] * (1 << 30)),
                    int(nevs[min(len(nevs) - 1, int(u[i, 4] * len(nevs)))])))
    return out


def batch_instance(spec) -> tuple:
    """(Problem, nev, atoms placed) of one batch_spec entry, real (Gamma point).  Where the drawn
    number of atoms does not fit with non-overlapping r_c spheres, one fewer is tried."""
    mesh, atoms, enr, s, nev = spec
    while True:
        try:
            return generate(mesh, atoms, enr, BATCH_RC, s), nev, atoms
        except (ValueError, RuntimeError):
            if atoms <= 1:
                raise
            atoms -= 1


def closed_form_eigenvalues(n_el: int, v0: float, kpt=None) -> np.ndarray:
    """All eigenvalues of the unenriched periodic Q1 pair with constant V = v0, ascending.

    The 1-D periodic linear element has stiffness symbol (2 - 2cos t)/h and mass symbol
    h(2 + cos t)/3 for the Fourier mode t; the Q1 pair is their tensor product and 3-point
    Gauss is exact for these integrands, so lambda = v0 + sum_d 3(1 - cos t_d)/(h^2 (2 + cos t_d))
    with t_d = (2 pi j_d + k_d) / N, j_d = 0..N-1.
    """
    N = n_el
    h = 1.0 / N
    k = np.zeros(3) if kpt is None else np.asarray(kpt, dtype=np.float64)
    lam1 = []
    for d in range(3):
        t = (2.0 * math.pi * np.arange(N) + k[d]) / N
        lam1.append(3.0 * (1.0 - np.cos(t)) / (h * h * (2.0 + np.cos(t))))
    tot = lam1[0][:, None, None] + lam1[1][None, :, None] + lam1[2][None, None, :]
    return np.sort(v0 + tot.ravel())
