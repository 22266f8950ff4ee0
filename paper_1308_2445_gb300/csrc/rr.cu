// Rayleigh-Ritz (LABPSD step 9, remark 6) on one thread-block cluster.
//
// GB300 runs FP64 at about two FMAs per clock per SM, so the O(q^3) work of the reduced
// eigenproblem is spread over the SMs of one cluster: every CTA owns a slice of rows of the
// working matrix in shared memory, broadcasts go through distributed shared memory, and the
// steps are separated by cluster barriers.
//
//   1. D = diag(S_R)^{-1/2}; Cholesky D S_R D = L L^T (row-distributed, symmetric storage, one
//      barrier per column).  A pivot below RR_PIVOT_MIN (or NaN) sets info[3] and the host
//      reruns the single-CTA kernel, whose rank-revealing branch is the reading of the paper's
//      silent breakdown case.
//   2. C = L^{-1} (D H_R D) L^{-T}, column-parallel substitutions, then C = (C + C^T)/2.
//   3. Householder tridiagonalisation of C (three barriers per column).
//   4. The k lowest eigenvalues of the tridiagonal by Sturm-count multisection (32 points per
//      warp step), one warp per eigenvalue: ascending by construction.
//   5. Eigenvectors by inverse iteration with a pivoted tridiagonal LU, eigenvalues closer than
//      1e-5 ||T|| treated as a cluster and re-orthogonalised (modified Gram-Schmidt).
//   6. Back-transforms: V <- H_0 ... H_{q-3} V, then W = D L^{-T} V.
#include <cooperative_groups.h>

#include <cfloat>
#include <cmath>

#include "common.h"

namespace cg = cooperative_groups;

namespace hbsd {

namespace {

constexpr double PIVOT_MIN = 1e-14;
constexpr int RR_THREADS_C = 256;

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sturm count: number of eigenvalues of the symmetric tridiagonal (d, e) below x.
__device__ int sturm_count(const double* d, const double* e2, int n, double x, double pivmin) {
    int cnt = 0;
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
    for (int i = 1; i < n; ++i) {
        q = d[i] - x - e2[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        if (q < 0) ++cnt;
    }
    return cnt;
}

struct RRWork {
    double *Lg, *Tg, *Cg, *Vh, *tau, *d, *e, *V, *V2, *lam;
    double *fd, *fu, *fu2, *fl, *fp;   // pivoted LU of T - lambda I per eigenvector (q x k each)
};

__device__ RRWork rr_work(double* ws, int q, int k) {
    RRWork w;
    const int64_t qq = (int64_t)q * q;
    w.Lg = ws;
    w.Tg = w.Lg + qq;
    w.Cg = w.Tg + qq;
    w.Vh = w.Cg + qq;
    w.tau = w.Vh + qq;
    w.d = w.tau + q;
    w.e = w.d + q;
    w.V = w.e + q;
    w.V2 = w.V + (int64_t)q * k;
    w.lam = w.V2 + (int64_t)q * k;
    w.fd = w.lam + k;
    w.fu = w.fd + (int64_t)q * k;
    w.fu2 = w.fu + (int64_t)q * k;
    w.fl = w.fu2 + (int64_t)q * k;
    w.fp = w.fl + (int64_t)q * k;
    return w;
}

}  // namespace

int64_t rr_cluster_ws_doubles(int q, int k) { return (int64_t)4 * q * q + 3 * q + 7 * (int64_t)q * k + k + 64; }

// shared layout: A[rb][q] | vb[q] | wb[q] | cb[q] | dv[q] | dr[q] | part[32] | flag
// drop_tol = 0: a pivot below PIVOT_MIN stops the kernel (info[3]) for the caller's fallback.
// drop_tol > 0: a pivot below drop_tol removes that column from the reduced problem (pivoted
// Cholesky rank reveal): its row of L becomes e_k and its row/column of H_R is decoupled onto an
// eigenvalue above every other one, so it never enters the lowest k.
__global__ void __launch_bounds__(RR_THREADS_C) k_rr_cluster(const double* __restrict__ HR, const double* __restrict__ SR,
                                                             int q, int k, double* __restrict__ theta,
                                                             double* __restrict__ Wout, double* __restrict__ ws,
                                                             int* __restrict__ info, double drop_tol) {
    cg::cluster_group cluster = cg::this_cluster();
    const int NC = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int rb = (q + NC - 1) / NC;
    const int r0 = rank * rb, r1 = min(q, r0 + rb);
    extern __shared__ __align__(16) double sm[];
    double* A = sm;                        // rb x q, row i at (i - r0) * q
    double* vb = A + (int64_t)rb * q;
    double* wb = vb + q;
    double* cb = wb + q;
    double* dv = cb + q;
    double* dr = dv + q;                   // 1.0 where a column was dropped
    double* part = dr + q;                 // 32
    int* flag = reinterpret_cast<int*>(part + 32);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    RRWork W = rr_work(ws, q, k);

    for (int i = tid; i < q; i += nt) {
        const double sii = SR[(int64_t)i * q + i];
        const bool usable = sii > 0.0 && isfinite(sii) && isfinite(HR[(int64_t)i * q + i]);
        // drop mode: a column with a zero or non-finite S_R diagonal is dropped up front
        dv[i] = (usable || drop_tol == 0.0) ? 1.0 / sqrt(sii) : 0.0;
        dr[i] = 0.0;
    }
    if (tid == 0) *flag = 0;
    __syncthreads();
    for (int idx = tid; idx < (r1 - r0) * q; idx += nt) {
        const int i = r0 + idx / q, j = idx % q;
        const double v = SR[(int64_t)i * q + j] * dv[i] * dv[j];
        A[idx] = (dv[i] == 0.0 || dv[j] == 0.0) ? 0.0 : v;   // 0 * inf guard for dropped columns
    }
    cluster.sync();

    // ---- 1. Cholesky, symmetric row storage: row kk (owner) holds column kk ----
    for (int kk = 0; kk < q; ++kk) {
        const int owner = kk / rb;
        if (rank == owner) {
            double* row = A + (int64_t)(kk - r0) * q;
            const double piv = row[kk];
            const bool drop = drop_tol > 0.0 && !(piv >= drop_tol);
            const bool bad = !drop && !(piv >= PIVOT_MIN);
            const double lkk = (bad || drop) ? 1.0 : sqrt(piv);
            __syncthreads();
            for (int j = kk + 1 + tid; j < q; j += nt) {
                const double l = drop ? 0.0 : row[j] / lkk;
                for (int c = 0; c < NC; ++c) cluster.map_shared_rank(cb, c)[j] = l;
            }
            if (tid == 0) {
                row[kk] = lkk;
                if (bad)
                    for (int c = 0; c < NC; ++c) *cluster.map_shared_rank(flag, c) = 1;
                if (drop)
                    for (int c = 0; c < NC; ++c) cluster.map_shared_rank(dr, c)[kk] = 1.0;
            }
        }
        cluster.sync();
        if (*flag) break;
        // own rows i > kk: A[i][kk] <- L[i][kk];  A[i][j] -= L[i][kk] L[j][kk]  for j > kk
        const int ib = max(r0, kk + 1);
        for (int idx = tid; idx < (r1 - ib) * (q - kk - 1); idx += nt) {
            const int i = ib + idx / (q - kk - 1), j = kk + 1 + idx % (q - kk - 1);
            A[(int64_t)(i - r0) * q + j] -= cb[i] * cb[j];
        }
        __syncthreads();
        for (int i = ib + tid; i < r1; i += nt) A[(int64_t)(i - r0) * q + kk] = cb[i];
        cluster.sync();
    }
    if (*flag) {
        if (rank == 0 && tid == 0) { info[0] = 0; info[3] = 1; }
        return;
    }
    // L (lower) to global; a dropped column's row is e_k
    for (int idx = tid; idx < (r1 - r0) * q; idx += nt) {
        const int i = r0 + idx / q, j = idx % q;
        double v = (j <= i) ? A[idx] : 0.0;
        if (dr[i] != 0.0) v = (j == i) ? 1.0 : 0.0;
        W.Lg[(int64_t)i * q + j] = v;
    }
    cluster.sync();

    // ---- 2. C = L^{-1} Hd L^{-T}: one warp per column, forward substitution ----
    // T(:, j) = L^{-1} Hd(:, j); stored transposed: Tg[j][i] = T(i, j)
    for (int j = r0 + warp; j < r1; j += nwarps) {
        double* x = W.Tg + (int64_t)j * q;
        for (int i = 0; i < q; ++i) {
            double acc = 0.0;
            for (int l = lane; l < i; l += 32) acc += W.Lg[(int64_t)i * q + l] * x[l];
            acc = wsum(acc);
            const double hij = (dr[i] != 0.0 || dr[j] != 0.0 || dv[i] == 0.0 || dv[j] == 0.0)
                                   ? 0.0 : HR[(int64_t)i * q + j] * dv[i] * dv[j];
            if (lane == 0) x[i] = (hij - acc) / W.Lg[(int64_t)i * q + i];
            __syncwarp();
        }
    }
    cluster.sync();
    // C(:, j) = L^{-1} T(j, :)^T ; T(j, i) = Tg[i][j];  stored Cg[j][i] = C(i, j)
    for (int j = r0 + warp; j < r1; j += nwarps) {
        double* x = W.Cg + (int64_t)j * q;
        for (int i = 0; i < q; ++i) {
            double acc = 0.0;
            for (int l = lane; l < i; l += 32) acc += W.Lg[(int64_t)i * q + l] * x[l];
            acc = wsum(acc);
            if (lane == 0) x[i] = (W.Tg[(int64_t)i * q + j] - acc) / W.Lg[(int64_t)i * q + i];
            __syncwarp();
        }
    }
    cluster.sync();
    for (int idx = tid; idx < (r1 - r0) * q; idx += nt) {
        const int i = r0 + idx / q, j = idx % q;
        A[idx] = 0.5 * (W.Cg[(int64_t)i * q + j] + W.Cg[(int64_t)j * q + i]);
    }
    if (drop_tol > 0.0) {
        // eigenvalue of the dropped (decoupled) coordinates: above the Gershgorin bound of C
        double gmax = 0.0;
        for (int i = r0 + warp; i < r1; i += nwarps) {
            double rs = 0.0;
            for (int j = lane; j < q; j += 32) rs += fabs(A[(int64_t)(i - r0) * q + j]);
            rs = wsum(rs);
            gmax = fmax(gmax, rs);
        }
        if (lane == 0) part[warp] = gmax;
        __syncthreads();
        if (tid == 0) {
            double g = 0.0;
            for (int w2 = 0; w2 < nwarps; ++w2) g = fmax(g, part[w2]);
            for (int c = 0; c < NC; ++c) cluster.map_shared_rank(cb, c)[rank] = g;
        }
        cluster.sync();
        double big = 0.0;
        for (int c = 0; c < NC; ++c) big = fmax(big, cb[c]);
        big = 2.0 * big + 1.0;
        for (int i = r0 + tid; i < r1; i += nt)
            if (dr[i] != 0.0) A[(int64_t)(i - r0) * q + i] = big;
    }
    cluster.sync();

    // ---- 3. Householder tridiagonalisation ----
    for (int kk = 0; kk + 2 < q; ++kk) {
        const int owner = kk / rb;
        if (rank == owner) {
            const double* row = A + (int64_t)(kk - r0) * q;
            double s2 = 0.0;
            for (int j = kk + 1 + tid; j < q; j += nt) s2 += row[j] * row[j];
            s2 = wsum(s2);
            if (lane == 0) part[warp] = s2;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int w = 0; w < nwarps; ++w) t += part[w];
                part[31] = t;
            }
            __syncthreads();
            s2 = part[31];
            const double x0 = row[kk + 1];
            const double tail = s2 - x0 * x0;
            double alpha, t;
            if (tail <= 0.0 || s2 == 0.0) { alpha = x0; t = 0.0; }
            else { alpha = -copysign(sqrt(s2), x0); t = 2.0 / (tail + (x0 - alpha) * (x0 - alpha)); }
            for (int j = kk + 1 + tid; j < q; j += nt) {
                const double v = (t == 0.0) ? 0.0 : (j == kk + 1 ? x0 - alpha : row[j]);
                W.Vh[(int64_t)kk * q + j] = v;
                for (int c = 0; c < NC; ++c) cluster.map_shared_rank(vb, c)[j] = v;
            }
            if (tid == 0) {
                W.tau[kk] = t;
                W.d[kk] = row[kk];
                W.e[kk] = alpha;
                for (int c = 0; c < NC; ++c) cluster.map_shared_rank(part, c)[30] = t;
            }
        }
        cluster.sync();
        const double t = part[30];
        if (t == 0.0) {           // column already reduced: uniform decision after the barrier
            cluster.sync();       // nobody may overwrite part[30] before everyone has read it
            continue;
        }
        // p_i = t * sum_j A[i][j] v_j for own rows i > kk (one warp per row)
        const int ib = max(r0, kk + 1);
        double mypart = 0.0;
        for (int i = ib + warp; i < r1; i += nwarps) {
            const double* ai = A + (int64_t)(i - r0) * q;
            double acc = 0.0;
            for (int j = kk + 1 + lane; j < q; j += 32) acc += ai[j] * vb[j];
            acc = wsum(acc) * t;
            if (lane == 0) { wb[i] = acc; mypart += acc * vb[i]; }
        }
        if (lane == 0) part[warp] = mypart;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < nwarps; ++w) s += part[w];
            for (int c = 0; c < NC; ++c) cluster.map_shared_rank(cb, c)[rank] = s;   // cb[0..NC) as partials
        }
        cluster.sync();
        double pv = 0.0;
        for (int c = 0; c < NC; ++c) pv += cb[c];
        const double K = 0.5 * t * pv;
        for (int i = ib + tid; i < r1; i += nt) {
            const double w = wb[i] - K * vb[i];
            for (int c = 0; c < NC; ++c) cluster.map_shared_rank(wb, c)[i] = w;
        }
        cluster.sync();
        for (int idx = tid; idx < (r1 - ib) * (q - kk - 1); idx += nt) {
            const int i = ib + idx / (q - kk - 1), j = kk + 1 + idx % (q - kk - 1);
            A[(int64_t)(i - r0) * q + j] -= vb[i] * wb[j] + wb[i] * vb[j];
        }
        cluster.sync();
    }
    // trailing 2 x 2 (or 1 x 1) block
    for (int i = r0 + tid; i < r1; i += nt) {
        if (i >= q - 2) {
            W.d[i] = A[(int64_t)(i - r0) * q + i];
            W.e[i] = (i + 1 < q) ? A[(int64_t)(i - r0) * q + i + 1] : 0.0;
            W.tau[i] = 0.0;
        }
    }
    cluster.sync();

    // ---- 4. lowest k eigenvalues: Sturm multisection, one warp per eigenvalue ----
    // (d, e^2 copied to shared: reuse vb / wb)
    for (int i = tid; i < q; i += nt) {
        vb[i] = W.d[i];
        wb[i] = (i < q - 1) ? W.e[i] * W.e[i] : 0.0;
    }
    __syncthreads();
    double gl = DBL_MAX, gu = -DBL_MAX, tnorm = 0.0;
    for (int i = 0; i < q; ++i) {
        const double r = (i > 0 ? fabs(W.e[i - 1]) : 0.0) + (i < q - 1 ? fabs(W.e[i]) : 0.0);
        gl = fmin(gl, vb[i] - r);
        gu = fmax(gu, vb[i] + r);
        tnorm = fmax(tnorm, fabs(vb[i]) + r);
    }
    const double pivmin = DBL_MIN * fmax(1.0, tnorm * tnorm);
    const double span = fmax(gu - gl, DBL_MIN);
    gl -= 2.0 * DBL_EPSILON * span + pivmin;
    gu += 2.0 * DBL_EPSILON * span + pivmin;
    const int gw = rank * nwarps + warp, ngw = NC * nwarps;
    for (int j = gw; j < k; j += ngw) {
        double lo = gl, hi = gu;   // invariant: count(lo) <= j < count(hi)
        for (int it = 0; it < 24; ++it) {
            const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
            const int c = sturm_count(vb, wb, q, x, pivmin);
            const unsigned below = __ballot_sync(0xffffffffu, c <= j);   // points still left of eigenvalue j
            const int nb = __popc(below);                                  // monotone in lane
            const double nlo = nb > 0 ? lo + (hi - lo) * (double)nb / 33.0 : lo;
            const double nhi = nb < 32 ? lo + (hi - lo) * (double)(nb + 1) / 33.0 : hi;
            lo = nlo;
            hi = nhi;
            if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + pivmin) break;
        }
        if (lane == 0) W.lam[j] = 0.5 * (lo + hi);
    }
    cluster.sync();

    // ---- 5. eigenvectors of the tridiagonal by inverse iteration (clusters re-orthogonalised) ----
    // A cluster is a maximal run of eigenvalues with consecutive gaps <= 1e-5 ||T|| (outside a
    // cluster inverse iteration leaves the vectors orthogonal to about eps ||T|| / gap <= 1e-11,
    // the accuracy the S-orthonormality of the Ritz block needs); one warp per
    // cluster processes its members in order (lane 0 runs the O(q) tridiagonal factor and solves,
    // the lanes share the Gram-Schmidt and normalisation), so the result does not depend on timing.
    const double ortol = 1e-5 * tnorm;
    for (int j = gw; j < k; j += ngw) {
        if (j > 0 && W.lam[j] - W.lam[j - 1] <= ortol) continue;   // not the first member of its cluster
        int jend = j + 1;
        while (jend < k && W.lam[jend] - W.lam[jend - 1] <= ortol) ++jend;
        double prev = -DBL_MAX;
        for (int m = j; m < jend; ++m) {
            double lm = W.lam[m];
            const double sep = 10.0 * DBL_EPSILON * fmax(fabs(lm), tnorm);
            if (lm <= prev + sep) lm = prev + sep;   // distinct shifts inside a cluster
            prev = lm;
            double* x = W.V + m;                      // column m, stride k
            double* fd = W.fd + m; double* fu = W.fu + m; double* fu2 = W.fu2 + m;
            double* fl = W.fl + m; double* fp = W.fp + m;
            if (lane == 0) {
                // T - lm I = P L U, Gaussian elimination with partial pivoting (U has two
                // super-diagonals; fp[i] = 1 when rows i and i+1 were exchanged)
                for (int i = 0; i < q; ++i) {
                    fd[(int64_t)i * k] = vb[i] - lm;
                    fu[(int64_t)i * k] = (i + 1 < q) ? W.e[i] : 0.0;
                    fu2[(int64_t)i * k] = 0.0;
                }
                for (int i = 0; i + 1 < q; ++i) {
                    const double sub = W.e[i];
                    double di = fd[(int64_t)i * k];
                    if (fabs(di) >= fabs(sub)) {
                        if (di == 0.0) { di = pivmin; fd[(int64_t)i * k] = di; }
                        const double f = sub / di;
                        fl[(int64_t)i * k] = f;
                        fp[(int64_t)i * k] = 0.0;
                        fd[(int64_t)(i + 1) * k] -= f * fu[(int64_t)i * k];
                    } else {
                        const double f = di / sub;
                        fl[(int64_t)i * k] = f;
                        fp[(int64_t)i * k] = 1.0;
                        fd[(int64_t)i * k] = sub;
                        const double tmp = fu[(int64_t)i * k];
                        fu[(int64_t)i * k] = fd[(int64_t)(i + 1) * k];
                        fd[(int64_t)(i + 1) * k] = tmp - f * fd[(int64_t)(i + 1) * k];
                        if (i + 2 < q) {
                            fu2[(int64_t)i * k] = fu[(int64_t)(i + 1) * k];
                            fu[(int64_t)(i + 1) * k] = -f * fu[(int64_t)(i + 1) * k];
                        }
                    }
                }
                if (fd[(int64_t)(q - 1) * k] == 0.0) fd[(int64_t)(q - 1) * k] = pivmin;
            }
            // deterministic dense start vector
            for (int i = lane; i < q; i += 32) {
                uint64_t h = 0x9E3779B97F4A7C15ull * (uint64_t)(m + 1) + 0xBF58476D1CE4E5B9ull * (uint64_t)(i + 1);
                h ^= h >> 31; h *= 0x94D049BB133111EBull; h ^= h >> 29;
                x[(int64_t)i * k] = 0.5 + (double)(h >> 11) * (1.0 / 9007199254740992.0);
            }
            __syncwarp();
            for (int iter = 0; iter < 3; ++iter) {
                if (lane == 0) {
                    for (int i = 0; i + 1 < q; ++i) {   // apply P and L^{-1}
                        double bi = x[(int64_t)i * k], bn = x[(int64_t)(i + 1) * k];
                        if (fp[(int64_t)i * k] != 0.0) { const double t2 = bi; bi = bn; bn = t2; }
                        x[(int64_t)i * k] = bi;
                        x[(int64_t)(i + 1) * k] = bn - fl[(int64_t)i * k] * bi;
                    }
                    for (int i = q - 1; i >= 0; --i) {   // U^{-1}
                        double sacc = x[(int64_t)i * k];
                        if (i + 1 < q) sacc -= fu[(int64_t)i * k] * x[(int64_t)(i + 1) * k];
                        if (i + 2 < q) sacc -= fu2[(int64_t)i * k] * x[(int64_t)(i + 2) * k];
                        x[(int64_t)i * k] = sacc / fd[(int64_t)i * k];
                    }
                }
                __syncwarp();
                // scale first (the solve can be huge), then Gram-Schmidt against earlier members
                double nrm = 0.0;
                for (int i = lane; i < q; i += 32) nrm = fmax(nrm, fabs(x[(int64_t)i * k]));
                for (int o = 16; o > 0; o >>= 1) nrm = fmax(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
                for (int i = lane; i < q; i += 32) x[(int64_t)i * k] /= nrm;
                __syncwarp();
                for (int pm = j; pm < m; ++pm) {
                    double dot = 0.0;
                    for (int i = lane; i < q; i += 32) dot += W.V[(int64_t)i * k + pm] * x[(int64_t)i * k];
                    dot = wsum(dot);
                    for (int i = lane; i < q; i += 32) x[(int64_t)i * k] -= dot * W.V[(int64_t)i * k + pm];
                    __syncwarp();
                }
                double n2 = 0.0;
                for (int i = lane; i < q; i += 32) n2 += x[(int64_t)i * k] * x[(int64_t)i * k];
                n2 = wsum(n2);
                const double inv = 1.0 / sqrt(n2);
                for (int i = lane; i < q; i += 32) x[(int64_t)i * k] *= inv;
                __syncwarp();
            }
        }
    }
    cluster.sync();

    // ---- 6. back-transforms, one warp per eigenvector ----
    for (int j = gw; j < k; j += ngw) {
        // V(:, j) <- H_0 ... H_{q-3} V(:, j): apply the reflectors from the last to the first
        for (int kk = q - 3; kk >= 0; --kk) {
            const double t = W.tau[kk];
            if (t == 0.0) continue;
            double dot = 0.0;
            for (int i = kk + 1 + lane; i < q; i += 32) dot += W.Vh[(int64_t)kk * q + i] * W.V[(int64_t)i * k + j];
            dot = wsum(dot) * t;
            for (int i = kk + 1 + lane; i < q; i += 32) W.V[(int64_t)i * k + j] -= dot * W.Vh[(int64_t)kk * q + i];
            __syncwarp();
        }
        // W(:, j) = D L^{-T} V(:, j): back substitution
        for (int i = q - 1; i >= 0; --i) {
            double acc = 0.0;
            for (int l = i + 1 + lane; l < q; l += 32) acc += W.Lg[(int64_t)l * q + i] * W.V2[(int64_t)l * k + j];
            acc = wsum(acc);
            if (lane == 0) W.V2[(int64_t)i * k + j] = (W.V[(int64_t)i * k + j] - acc) / W.Lg[(int64_t)i * q + i];
            __syncwarp();
        }
        for (int i = lane; i < q; i += 32) Wout[(int64_t)i * k + j] = dv[i] * W.V2[(int64_t)i * k + j];
        if (lane == 0) theta[j] = W.lam[j];
    }
    if (rank == 0 && tid == 0) {
        int nd = 0;
        for (int i = 0; i < q; ++i) nd += dr[i] != 0.0;
        info[0] = nd > 0 ? 1 : 0;
        info[1] = q - nd;
        info[3] = 0;
    }
}

}  // namespace hbsd

namespace hbsd {

static int cluster_size_for(int q) {
    if (q >= 96) return 16;
    if (q >= 32) return 8;
    if (q >= 8) return 4;
    return 1;
}

int rayleigh_ritz_cluster(Session* s, const double* HR, const double* SR, int q, int k, double* theta, double* W,
                          int* info_host, cudaStream_t st, double drop_tol) {
    if (q <= 0 || k <= 0 || k > q) return fail(HBSD_ERR_ARG, "rayleigh_ritz: need 0 < k <= q");
    HBSD_TRY(s->rr_ws.alloc((size_t)std::max<int64_t>(rr_cluster_ws_doubles(q, k), (int64_t)4 * q * q + 3 * q + 64)));
    HBSD_TRY(s->rr_info.alloc(4));
    HBSD_CUDA(cudaMemsetAsync(s->rr_info.p, 0, 4 * sizeof(int), st));
    // candidate cluster sizes, preferred first; a size whose row slice does not fit in shared
    // memory or that the device cannot co-schedule is skipped
    const int pref = cluster_size_for(q);
    const int cands[5] = {16, 8, 4, 2, 1};
    bool launched = false;
    for (int ci = 0; ci < 5 && !launched; ++ci) {
        const int NC = cands[ci];
        if (NC > pref && (((size_t)((q + pref - 1) / pref) * q + 5 * (size_t)q + 32) * 8 + 16) <= 220 * 1024) continue;
        if (NC > q) continue;
        const int rb = (q + NC - 1) / NC;
        const size_t smem = ((size_t)rb * q + 5 * (size_t)q + 32) * sizeof(double) + 16;
        if (smem > 220 * 1024) continue;
        HBSD_CUDA(cudaFuncSetAttribute(k_rr_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (NC > 8) HBSD_CUDA(cudaFuncSetAttribute(k_rr_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(NC, 1, 1);
        cfg.blockDim = dim3(RR_THREADS_C, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = NC;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        cudaError_t oe = cudaOccupancyMaxActiveClusters(&nclusters, k_rr_cluster, &cfg);
        if (oe != cudaSuccess || nclusters < 1) {
            (void)cudaGetLastError();
            continue;
        }
        cudaError_t le = cudaLaunchKernelEx(&cfg, k_rr_cluster, HR, SR, q, k, theta, W, s->rr_ws.p, s->rr_info.p, drop_tol);
        if (le != cudaSuccess) return fail(HBSD_ERR_CUDA, std::string("rayleigh_ritz launch: ") + cudaGetErrorString(le));
        count_launch(s);
        launched = true;
    }
    if (!launched) return rayleigh_ritz(s, HR, SR, q, k, theta, W, info_host, st);
    int info[4] = {0, 0, 0, 0};
    HBSD_CUDA(cudaMemcpyAsync(info, s->rr_info.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    HBSD_CUDA(cudaStreamSynchronize(st));
    if (info[3]) return rayleigh_ritz(s, HR, SR, q, k, theta, W, info_host, st);   // Cholesky breakdown
    if (info_host) { info_host[0] = info[0]; info_host[1] = info[1]; }
    if (info[1] < k) return fail(HBSD_ERR_RR_RANK, "rayleigh_ritz: search space rank below k");
    return 0;
}

}  // namespace hbsd
