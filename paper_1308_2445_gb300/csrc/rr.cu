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
//   4. The k lowest eigenvalues of the tridiagonal, coarse: FP32 Sturm-count multisection (32
//      points per warp step), one warp per eigenvalue.
//   5. Eigenvectors by Rayleigh-quotient inverse iteration (pivoted tridiagonal LU), one warp per
//      eigenvalue, then CholeskyQR2 of the block and the Rayleigh quotients as eigenvalues.
//   6. Back-transforms: V <- H_0 ... H_{q-3} V, then W = D L^{-T} V.
#include <cooperative_groups.h>

#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "common.h"

namespace cg = cooperative_groups;

namespace hbsd {

namespace {

constexpr double PIVOT_MIN = 1e-14;
constexpr int RR_THREADS_C = 256;

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct RRWork {
    double *Lg, *LgT, *Tg, *Cg, *Vh, *tau, *d, *e, *V, *lam, *lamr;   // lam: coarse (step 4), lamr: refined
    uint64_t* stamps;                  // phase timestamps (CTA 0, thread 0)
    double* scratch;                   // per-warp scratch when it does not fit in shared memory
};

__device__ RRWork rr_work(double* ws, int q, int k) {
    RRWork w;
    const int64_t qq = (int64_t)q * q;
    w.Lg = ws;
    w.LgT = w.Lg + qq;
    w.Tg = w.LgT + qq;
    w.Cg = w.Tg + qq;
    w.Vh = w.Cg + qq;
    w.tau = w.Vh + qq;
    w.d = w.tau + q;
    w.e = w.d + q;
    w.V = w.e + q;
    w.lam = w.V + (int64_t)q * k;
    w.lamr = w.lam + k;
    w.stamps = reinterpret_cast<uint64_t*>(w.lamr + k);
    w.scratch = w.lamr + k + 16;
    return w;
}

}  // namespace

int64_t rr_cluster_ws_doubles(int q, int k) {
    return (int64_t)5 * q * q + 3 * q + (int64_t)q * k + 2 * k + 16 + (int64_t)16 * (RR_THREADS_C / 32) * 6 * q + 64;
}

// shared layout (doubles): A[rb][q] | vb2[2][q+1] | pb[q] | cb2[2][q+1] | dv[q] | dr[q] | part[32] |
// wpart[32] | stg[LB][q] | per-warp scratch (nwarps x 6q, or in global memory when it does not fit)
// drop_tol = 0: a pivot below PIVOT_MIN stops the kernel (info[3]) for the caller's fallback.
// drop_tol > 0: a pivot below drop_tol removes that column from the reduced problem (pivoted
// Cholesky rank reveal): its row of L becomes e_k and its row/column of H_R is decoupled onto an
// eigenvalue above every other one, so it never enters the lowest k.
__global__ void __launch_bounds__(RR_THREADS_C) k_rr_cluster(const double* __restrict__ HR, const double* __restrict__ SR,
                                                             int q, int k, double* __restrict__ theta,
                                                             double* __restrict__ Wout, double* __restrict__ ws,
                                                             int* __restrict__ info, double drop_tol, int scratch_in_smem,
                                                             int LB) {
    cg::cluster_group cluster = cg::this_cluster();
    const int NC = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int rb = (q + NC - 1) / NC;
    const int r0 = rank * rb, r1 = min(q, r0 + rb);
    extern __shared__ __align__(16) double sm[];
    double* A = sm;                        // rb x q, row i at (i - r0) * q
    double* vb2 = A + (int64_t)rb * q;     // [2][q+1]: Householder vector, tau at [q]
    double* pb = vb2 + 2 * (q + 1);        // [q]: p of the current Householder step
    double* cb2 = pb + q;                  // [2][q+1]: Cholesky column, status at [q]
    double* dv = cb2 + 2 * (q + 1);
    double* dr = dv + q;                   // 1.0 where a column was dropped
    double* part = dr + q;                 // [32] per-CTA partials of the cluster
    double* wpart = part + 32;             // [32] per-warp partials inside a CTA
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    RRWork W = rr_work(ws, q, k);
    double* stg = wpart + 32;              // [LB][q]: rows staged for the warps of the CTA
    double* scr = scratch_in_smem ? (stg + (int64_t)LB * q + (int64_t)warp * 6 * q)
                                  : (W.scratch + ((int64_t)rank * nwarps + warp) * 6 * q);

    for (int i = tid; i < q; i += nt) {
        const double sii = SR[(int64_t)i * q + i];
        const bool usable = sii > 0.0 && isfinite(sii) && isfinite(HR[(int64_t)i * q + i]);
        // drop mode: a column with a zero or non-finite S_R diagonal is dropped up front
        dv[i] = (usable || drop_tol == 0.0) ? 1.0 / sqrt(sii) : 0.0;
        dr[i] = 0.0;
    }
    __syncthreads();
    for (int idx = tid; idx < (r1 - r0) * q; idx += nt) {
        const int i = r0 + idx / q, j = idx % q;
        const double v = SR[(int64_t)i * q + j] * dv[i] * dv[j];
        A[idx] = (dv[i] == 0.0 || dv[j] == 0.0) ? 0.0 : v;   // 0 * inf guard for dropped columns
    }
    if (rank == 0 && tid == 0) W.stamps[0] = gtimer();
    __syncthreads();

    // ---- 1. Cholesky, symmetric row storage (row kk of the owner holds column kk); one cluster
    //         barrier per column, the broadcast column double-buffered ----
    bool broke = false;
    for (int kk = 0; kk < q; ++kk) {
        double* cbk = cb2 + (kk & 1) * (q + 1);
        if (kk / rb == rank) {
            double* row = A + (int64_t)(kk - r0) * q;
            const double piv = row[kk];
            const bool drop = drop_tol > 0.0 && !(piv >= drop_tol);
            const bool bad = !drop && !(piv >= PIVOT_MIN);
            const double lkk = (bad || drop) ? 1.0 : sqrt(piv);
            for (int j = kk + 1 + tid; j < q; j += nt) {
                const double l = drop ? 0.0 : row[j] / lkk;
                for (int c = 0; c < NC; ++c) cluster.map_shared_rank(cbk, c)[j] = l;
            }
            if (tid == 0) {
                const double code = (bad ? 1.0 : 0.0) + (drop ? 2.0 : 0.0);
                for (int c = 0; c < NC; ++c) cluster.map_shared_rank(cbk, c)[q] = code;
            }
            __syncthreads();
            if (tid == 0) row[kk] = lkk;
        }
        cluster.sync();
        const int code = (int)cbk[q];
        if (code & 1) { broke = true; break; }
        if ((code & 2) && tid == 0) dr[kk] = 1.0;
        const int ib = max(r0, kk + 1);
        const int m = q - kk - 1;
        for (int idx = tid; idx < (r1 - ib) * m; idx += nt) {
            const int i = ib + idx / m, j = kk + 1 + idx % m;
            A[(int64_t)(i - r0) * q + j] -= cbk[i] * cbk[j];
        }
        __syncthreads();
        for (int i = ib + tid; i < r1; i += nt) A[(int64_t)(i - r0) * q + kk] = cbk[i];
        __syncthreads();
    }
    if (broke) {
        if (rank == 0 && tid == 0) { info[0] = 0; info[3] = 1; }
        return;
    }
    if (rank == 0 && tid == 0) W.stamps[1] = gtimer();
    // L (lower, a dropped column's row is e_k) to global, row-major and transposed
    for (int idx = tid; idx < (r1 - r0) * q; idx += nt) {
        const int i = r0 + idx / q, j = idx % q;
        double v = (j <= i) ? A[idx] : 0.0;
        if (dr[i] != 0.0) v = (j == i) ? 1.0 : 0.0;
        W.Lg[(int64_t)i * q + j] = v;
        W.LgT[(int64_t)j * q + i] = v;
    }
    cluster.sync();

    // ---- 2. C = L^{-1} Hd L^{-T}: one warp per column (columns in rounds of nwarps), the
    //         column in shared memory and the rows of L staged LB at a time for the whole CTA ----
    double* xv = scr;          // q
    double* bv = scr + q;      // q
    auto lower_solve_cols = [&](auto load_b, auto store_x) {
        for (int c0 = r0; c0 < r1; c0 += nwarps) {
            const int j = c0 + warp;
            const bool act = j < r1;
            if (act) load_b(j);
            __syncwarp();
            for (int i0 = 0; i0 < q; i0 += LB) {
                const int ibn = min(LB, q - i0);
                __syncthreads();
                for (int t = tid; t < ibn * q; t += nt) {
                    const int r = t / q, l = t % q;
                    stg[t] = (l <= i0 + r) ? W.Lg[(int64_t)(i0 + r) * q + l] : 0.0;
                }
                __syncthreads();
                if (act) {
                    for (int r = 0; r < ibn; ++r) {
                        const int i = i0 + r;
                        const double* li = stg + (int64_t)r * q;
                        double acc = 0.0;
                        for (int l = lane; l < i; l += 32) acc += li[l] * xv[l];
                        acc = wsum(acc);
                        if (lane == 0) xv[i] = (bv[i] - acc) / li[i];
                        __syncwarp();
                    }
                }
            }
            if (act) store_x(j);
            __syncwarp();
        }
    };
    // T(:, j) = L^{-1} Hd(:, j), Hd(:, j) = Hd(j, :) (H_R symmetric); stored Tg[j][i] = T(i, j)
    lower_solve_cols(
        [&](int j) {
            for (int i = lane; i < q; i += 32)
                bv[i] = (dr[i] != 0.0 || dr[j] != 0.0 || dv[i] == 0.0 || dv[j] == 0.0)
                            ? 0.0 : HR[(int64_t)j * q + i] * dv[i] * dv[j];
        },
        [&](int j) { for (int i = lane; i < q; i += 32) W.Tg[(int64_t)j * q + i] = xv[i]; });
    cluster.sync();
    // C(:, j) = L^{-1} T(j, :)^T, T(j, i) = Tg[i][j]; stored Cg[j][i] = C(i, j)
    lower_solve_cols(
        [&](int j) { for (int i = lane; i < q; i += 32) bv[i] = W.Tg[(int64_t)i * q + j]; },
        [&](int j) { for (int i = lane; i < q; i += 32) W.Cg[(int64_t)j * q + i] = xv[i]; });
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
            gmax = fmax(gmax, wsum(rs));
        }
        if (lane == 0) wpart[warp] = gmax;
        __syncthreads();
        if (tid == 0) {
            double g = 0.0;
            for (int w2 = 0; w2 < nwarps; ++w2) g = fmax(g, wpart[w2]);
            for (int c = 0; c < NC; ++c) cluster.map_shared_rank(part, c)[rank] = g;
        }
        cluster.sync();
        double big = 0.0;
        for (int c = 0; c < NC; ++c) big = fmax(big, part[c]);
        big = 2.0 * big + 1.0;
        for (int i = r0 + tid; i < r1; i += nt)
            if (dr[i] != 0.0) A[(int64_t)(i - r0) * q + i] = big;
    }
    __syncthreads();
    if (rank == 0 && tid == 0) W.stamps[2] = gtimer();

    // ---- 3. Householder tridiagonalisation: two cluster barriers per column ----
    // The owner of row kk (symmetric storage: row kk = column kk) forms v_kk and broadcasts it
    // (double-buffered); every CTA computes p for its rows and broadcasts them with its partial
    // p.v; after the second barrier every CTA forms w = p - K v for all indices and updates its rows.
    auto make_v = [&](int kk) {
        double* vbk = vb2 + (kk & 1) * (q + 1);
        const double* row = A + (int64_t)(kk - r0) * q;
        double s2 = 0.0;
        for (int j = kk + 1 + tid; j < q; j += nt) s2 += row[j] * row[j];
        s2 = wsum(s2);
        if (lane == 0) wpart[warp] = s2;
        __syncthreads();
        s2 = 0.0;
        for (int w2 = 0; w2 < nwarps; ++w2) s2 += wpart[w2];
        const double x0 = row[kk + 1];
        const double tail = s2 - x0 * x0;
        double alpha, t;
        if (tail <= 0.0 || s2 == 0.0) { alpha = x0; t = 0.0; }
        else { alpha = -copysign(sqrt(s2), x0); t = 2.0 / (tail + (x0 - alpha) * (x0 - alpha)); }
        for (int j = kk + 1 + tid; j < q; j += nt) {
            const double v = (t == 0.0) ? 0.0 : (j == kk + 1 ? x0 - alpha : row[j]);
            W.Vh[(int64_t)kk * q + j] = v;
            for (int c = 0; c < NC; ++c) cluster.map_shared_rank(vbk, c)[j] = v;
        }
        if (tid == 0) {
            W.tau[kk] = t;
            W.d[kk] = row[kk];
            W.e[kk] = alpha;
            for (int c = 0; c < NC; ++c) cluster.map_shared_rank(vbk, c)[q] = t;
        }
        __syncthreads();
    };
    if (q >= 3 && rank == 0) make_v(0);
    for (int kk = 0; kk + 2 < q; ++kk) {
        cluster.sync();                                           // v_kk visible everywhere
        const double* vbk = vb2 + (kk & 1) * (q + 1);
        const double t = vbk[q];
        const int ib = max(r0, kk + 1);
        if (t != 0.0) {
            double mypart = 0.0;
            for (int i = ib + warp; i < r1; i += nwarps) {
                const double* ai = A + (int64_t)(i - r0) * q;
                double acc = 0.0;
                for (int j = kk + 1 + lane; j < q; j += 32) acc += ai[j] * vbk[j];
                acc = wsum(acc) * t;
                if (lane == 0) {
                    mypart += acc * vbk[i];
                    for (int c = 0; c < NC; ++c) cluster.map_shared_rank(pb, c)[i] = acc;
                }
            }
            if (lane == 0) wpart[warp] = mypart;
            __syncthreads();
            if (tid == 0) {
                double sp = 0.0;
                for (int w2 = 0; w2 < nwarps; ++w2) sp += wpart[w2];
                for (int c = 0; c < NC; ++c) cluster.map_shared_rank(part, c)[rank] = sp;
            }
            cluster.sync();                                       // p and partials visible
            double pv = 0.0;
            for (int c = 0; c < NC; ++c) pv += part[c];
            const double K = 0.5 * t * pv;
            const int m = q - kk - 1;
            for (int idx = tid; idx < (r1 - ib) * m; idx += nt) {
                const int i = ib + idx / m, j = kk + 1 + idx % m;
                const double wi = pb[i] - K * vbk[i], wj = pb[j] - K * vbk[j];
                A[(int64_t)(i - r0) * q + j] -= vbk[i] * wj + wi * vbk[j];
            }
        }
        __syncthreads();
        if (kk + 3 < q && (kk + 1) / rb == rank) make_v(kk + 1);
    }
    cluster.sync();
    for (int i = r0 + tid; i < r1; i += nt) {   // trailing 2 x 2 (or 1 x 1) block
        if (i >= q - 2) {
            W.d[i] = A[(int64_t)(i - r0) * q + i];
            W.e[i] = (i + 1 < q) ? A[(int64_t)(i - r0) * q + i + 1] : 0.0;
            W.tau[i] = 0.0;
        }
    }
    if (rank == 0 && tid == 0) W.stamps[3] = gtimer();
    cluster.sync();

    // ---- 4. the k lowest eigenvalues, coarse: FP32 Sturm multisection (one warp each) ----
    double* dd = vb2;               // q doubles (free after step 3)
    double* ee = pb;                // q doubles
    float* df = reinterpret_cast<float*>(cb2);
    float* e2f = df + q;
    for (int i = tid; i < q; i += nt) {
        dd[i] = W.d[i];
        ee[i] = (i < q - 1) ? W.e[i] : 0.0;
        df[i] = (float)W.d[i];
        e2f[i] = (float)(ee[i] * ee[i]);
    }
    __syncthreads();
    double gl = DBL_MAX, gu = -DBL_MAX, tnorm = 0.0;
    for (int i = 0; i < q; ++i) {
        const double r = (i > 0 ? fabs(ee[i - 1]) : 0.0) + fabs(ee[i]);
        gl = fmin(gl, dd[i] - r);
        gu = fmax(gu, dd[i] + r);
        tnorm = fmax(tnorm, fabs(dd[i]) + r);
    }
    const double pivmin = DBL_MIN * fmax(1.0, tnorm * tnorm);
    const float pivf = FLT_MIN * (float)fmax(1.0, fmin(tnorm * tnorm, 1e30));
    const double span = fmax(gu - gl, DBL_MIN);
    gl -= 1e-5 * span + pivmin;
    gu += 1e-5 * span + pivmin;
    const int gw = rank * nwarps + warp, ngw = NC * nwarps;
    for (int j = gw; j < k; j += ngw) {
        double lo = gl, hi = gu;   // invariant: count(lo) <= j < count(hi)
        for (int it = 0; it < 6; ++it) {
            const float x = (float)(lo + (hi - lo) * (double)(lane + 1) / 33.0);
            int c = 0;
            float qq = df[0] - x;
            if (fabsf(qq) < pivf) qq = -pivf;
            c += qq < 0.f;
            for (int i = 1; i < q; ++i) {
                qq = df[i] - x - e2f[i - 1] / qq;
                if (fabsf(qq) < pivf) qq = -pivf;
                c += qq < 0.f;
            }
            const unsigned below = __ballot_sync(0xffffffffu, c <= j);
            const int nb = __popc(below);
            const double nlo = nb > 0 ? lo + (hi - lo) * (double)nb / 33.0 : lo;
            const double nhi = nb < 32 ? lo + (hi - lo) * (double)(nb + 1) / 33.0 : hi;
            lo = nlo;
            hi = nhi;
        }
        if (lane == 0) W.lam[j] = 0.5 * (lo + hi);
    }
    if (rank == 0 && tid == 0) W.stamps[4] = gtimer();
    cluster.sync();

    // ---- 5. eigenvectors and FP64 eigenvalues ----
    // 5a. Rayleigh-quotient inverse iteration for every wanted eigenvalue in parallel (one warp
    //     each): a solve at the coarse shift, then two at the Rayleigh quotient theta = x^T T x.
    // 5b. CholeskyQR2 of the k vectors (G = V^T V = R^T R, V <- V R^{-1}, twice): inverse
    //     iteration alone leaves vectors of close eigenvalues about eps ||T|| / gap apart from
    //     orthogonal, and ||T|| is large when S_R is ill-conditioned.
    // 5c. theta_j = x_j^T T x_j of the orthonormal vectors, ordered ascending.
    double* fdv = scr;            // q each: U diagonal, first and second super-diagonals,
    double* fuv = scr + q;        // multipliers, pivot flags, iterate
    double* fu2v = scr + 2 * q;
    double* flv = scr + 3 * q;
    double* fpv = scr + 4 * q;
    double* x = scr + 5 * q;
    auto factor = [&](double sh) {
        if (lane == 0) {
            for (int i = 0; i < q; ++i) {
                fdv[i] = dd[i] - sh;
                fuv[i] = ee[i];
                fu2v[i] = 0.0;
            }
            for (int i = 0; i + 1 < q; ++i) {
                const double sub = ee[i];
                double di = fdv[i];
                if (fabs(di) >= fabs(sub)) {
                    if (di == 0.0) { di = pivmin; fdv[i] = di; }
                    const double f = sub / di;
                    flv[i] = f;
                    fpv[i] = 0.0;
                    fdv[i + 1] -= f * fuv[i];
                } else {
                    const double f = di / sub;
                    flv[i] = f;
                    fpv[i] = 1.0;
                    fdv[i] = sub;
                    const double tmp = fuv[i];
                    fuv[i] = fdv[i + 1];
                    fdv[i + 1] = tmp - f * fdv[i + 1];
                    if (i + 2 < q) {
                        fu2v[i] = fuv[i + 1];
                        fuv[i + 1] = -f * fuv[i + 1];
                    }
                }
            }
            if (fdv[q - 1] == 0.0) fdv[q - 1] = pivmin;
        }
        __syncwarp();
    };
    auto solve = [&]() {
        if (lane == 0) {
            for (int i = 0; i + 1 < q; ++i) {
                double bi = x[i], bn = x[i + 1];
                if (fpv[i] != 0.0) { const double t2 = bi; bi = bn; bn = t2; }
                x[i] = bi;
                x[i + 1] = bn - flv[i] * bi;
            }
            for (int i = q - 1; i >= 0; --i) {
                double sacc = x[i];
                if (i + 1 < q) sacc -= fuv[i] * x[i + 1];
                if (i + 2 < q) sacc -= fu2v[i] * x[i + 2];
                x[i] = sacc / fdv[i];
            }
        }
        __syncwarp();
    };
    auto normalise = [&]() {
        double nrm = 0.0;
        for (int i = lane; i < q; i += 32) nrm = fmax(nrm, fabs(x[i]));
        for (int o = 16; o > 0; o >>= 1) nrm = fmax(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
        for (int i = lane; i < q; i += 32) x[i] /= nrm;
        __syncwarp();
        double n2 = 0.0;
        for (int i = lane; i < q; i += 32) n2 += x[i] * x[i];
        n2 = wsum(n2);
        const double inv = 1.0 / sqrt(n2);
        for (int i = lane; i < q; i += 32) x[i] *= inv;
        __syncwarp();
    };
    auto rayleigh_of = [&](const double* y, int64_t stride) {
        double acc = 0.0;
        for (int i = lane; i < q; i += 32) {
            const double yi = y[i * stride];
            acc += dd[i] * yi * yi;
            if (i + 1 < q) acc += 2.0 * ee[i] * yi * y[(i + 1) * stride];
        }
        return wsum(acc);
    };
    for (int j = gw; j < k; j += ngw) {
        for (int i = lane; i < q; i += 32) {
            uint64_t h = 0x9E3779B97F4A7C15ull * (uint64_t)(j + 1) + 0xBF58476D1CE4E5B9ull * (uint64_t)(i + 1);
            h ^= h >> 31; h *= 0x94D049BB133111EBull; h ^= h >> 29;
            x[i] = 0.5 + (double)(h >> 11) * (1.0 / 9007199254740992.0);
        }
        __syncwarp();
        factor(W.lam[j]);
        solve();
        normalise();
        double th = rayleigh_of(x, 1);
        for (int it = 0; it < 2; ++it) {
            factor(th);
            solve();
            normalise();
            th = rayleigh_of(x, 1);
        }
        for (int i = lane; i < q; i += 32) W.V[(int64_t)i * k + j] = x[i];
        __syncwarp();
    }
    cluster.sync();
    double* G = W.Cg;   // k x k (C is no longer needed)
    const int npairs = k * (k + 1) / 2;
    for (int pass = 0; pass < 2; ++pass) {
        for (int pidx = gw; pidx < npairs; pidx += ngw) {
            int a = (int)((sqrt(8.0 * pidx + 1.0) - 1.0) * 0.5);
            while ((a + 1) * (a + 2) / 2 <= pidx) ++a;
            while (a * (a + 1) / 2 > pidx) --a;
            const int b2 = pidx - a * (a + 1) / 2;   // b2 <= a
            double dot = 0.0;
            for (int i = lane; i < q; i += 32) dot += W.V[(int64_t)i * k + a] * W.V[(int64_t)i * k + b2];
            dot = wsum(dot);
            if (lane == 0) { G[(int64_t)a * k + b2] = dot; G[(int64_t)b2 * k + a] = dot; }
        }
        cluster.sync();
        if (rank == 0) {   // G = R^T R, R upper triangular in the upper triangle of G
            for (int c = 0; c < k; ++c) {
                if (tid == 0) G[(int64_t)c * k + c] = sqrt(fmax(G[(int64_t)c * k + c], DBL_MIN));
                __syncthreads();
                const double rc = G[(int64_t)c * k + c];
                for (int jj = c + 1 + tid; jj < k; jj += nt) G[(int64_t)c * k + jj] /= rc;
                __syncthreads();
                const int m = k - c - 1;
                for (int t = tid; t < m * m; t += nt) {
                    const int i2 = c + 1 + t / m, j2 = c + 1 + t % m;
                    if (j2 >= i2) G[(int64_t)i2 * k + j2] -= G[(int64_t)c * k + i2] * G[(int64_t)c * k + j2];
                }
                __syncthreads();
            }
        }
        cluster.sync();
        // V <- V R^{-1}, one warp per row of V: y_c = (v_c - sum_{l<c} y_l R[l][c]) / R[c][c]
        for (int i = r0 + warp; i < r1; i += nwarps) {
            double* yr = x;   // k <= q entries of per-warp scratch
            for (int c = lane; c < k; c += 32) yr[c] = W.V[(int64_t)i * k + c];
            __syncwarp();
            for (int c = 0; c < k; ++c) {
                double acc = 0.0;
                for (int l = lane; l < c; l += 32) acc += yr[l] * G[(int64_t)l * k + c];
                acc = wsum(acc);
                if (lane == 0) yr[c] = (yr[c] - acc) / G[(int64_t)c * k + c];
                __syncwarp();
            }
            for (int c = lane; c < k; c += 32) W.V[(int64_t)i * k + c] = yr[c];
            __syncwarp();
        }
        cluster.sync();
    }
    for (int j = gw; j < k; j += ngw) {
        const double th = rayleigh_of(W.V + j, k);
        if (lane == 0) W.lamr[j] = th;
    }
    cluster.sync();
    int* order = reinterpret_cast<int*>(W.e);   // k ints (the off-diagonal is no longer needed)
    if (rank == 0 && tid == 0) {
        for (int j = 0; j < k; ++j) order[j] = j;
        for (int j = 1; j < k; ++j) {
            const int v = order[j];
            int t = j - 1;
            while (t >= 0 && W.lamr[order[t]] > W.lamr[v]) { order[t + 1] = order[t]; --t; }
            order[t + 1] = v;
        }
    }
    if (rank == 0 && tid == 0) W.stamps[5] = gtimer();
    cluster.sync();

    // ---- 6. back-transforms, one warp per eigenvector (rounds of the cluster's warps), the
    //         vector in shared memory, reflectors and rows of L^T staged LB at a time ----
    const int rounds = (k + ngw - 1) / ngw;
    for (int rd = 0; rd < rounds; ++rd) {
        const int j = rd * ngw + gw;
        const bool act = j < k;
        const int src = act ? order[j] : 0;
        if (act)
            for (int i = lane; i < q; i += 32) xv[i] = W.V[(int64_t)i * k + src];
        __syncwarp();
        // V(:, j) <- H_0 ... H_{q-3} V(:, j): reflectors from the last to the first
        for (int kk1 = q - 3; kk1 >= 0; kk1 -= LB) {
            const int kk0 = max(0, kk1 - LB + 1);
            __syncthreads();
            for (int t = tid; t < (kk1 - kk0 + 1) * q; t += nt) stg[t] = W.Vh[(int64_t)kk0 * q + t];
            __syncthreads();
            if (act) {
                for (int kk = kk1; kk >= kk0; --kk) {
                    const double tt = W.tau[kk];
                    if (tt == 0.0) continue;
                    const double* vh = stg + (int64_t)(kk - kk0) * q;
                    double dot = 0.0;
                    for (int i = kk + 1 + lane; i < q; i += 32) dot += vh[i] * xv[i];
                    dot = wsum(dot) * tt;
                    for (int i = kk + 1 + lane; i < q; i += 32) xv[i] -= dot * vh[i];
                    __syncwarp();
                }
            }
        }
        // x <- L^{-T} x (row i of L^T = column i of L), rows from the last to the first
        for (int i1 = q - 1; i1 >= 0; i1 -= LB) {
            const int i0 = max(0, i1 - LB + 1);
            __syncthreads();
            for (int t = tid; t < (i1 - i0 + 1) * q; t += nt) stg[t] = W.LgT[(int64_t)i0 * q + t];
            __syncthreads();
            if (act) {
                for (int i = i1; i >= i0; --i) {
                    const double* lt = stg + (int64_t)(i - i0) * q;
                    double acc = 0.0;
                    for (int l = i + 1 + lane; l < q; l += 32) acc += lt[l] * xv[l];
                    acc = wsum(acc);
                    if (lane == 0) xv[i] = (xv[i] - acc) / lt[i];
                    __syncwarp();
                }
            }
        }
        if (act) {
            for (int i = lane; i < q; i += 32) Wout[(int64_t)i * k + j] = dv[i] * xv[i];
            if (lane == 0) theta[j] = W.lamr[src];
        }
        __syncwarp();
    }
    if (rank == 0 && tid == 0) {
        W.stamps[6] = gtimer();
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
    const int nwarps = RR_THREADS_C / 32;
    bool launched = false;
    for (int ci = 0; ci < 5 && !launched; ++ci) {
        const int NC = cands[ci];
        if (NC > q) continue;
        const int rb = (q + NC - 1) / NC;
        const size_t base = ((size_t)rb * q + 2 * (size_t)(q + 1) + q + 2 * (size_t)(q + 1) + 2 * (size_t)q + 64) *
                            sizeof(double);
        if (base > 220 * 1024) continue;
        if (NC > pref) {
            const int rbp = (q + pref - 1) / pref;
            const size_t basep = ((size_t)rbp * q + 6 * (size_t)q + 68) * sizeof(double);
            if (basep <= 220 * 1024) continue;   // the preferred size fits: do not go larger
        }
        int LB = 32;
        while (LB > 4 && base + (size_t)LB * q * sizeof(double) > 200 * 1024) LB /= 2;
        const size_t stgb = (size_t)LB * q * sizeof(double);
        if (base + stgb > 220 * 1024) continue;
        const size_t scr = (size_t)nwarps * 6 * q * sizeof(double);
        const int in_smem = (base + stgb + scr <= 220 * 1024) ? 1 : 0;
        const size_t smem = base + stgb + (in_smem ? scr : 0);
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
        cudaError_t le = cudaLaunchKernelEx(&cfg, k_rr_cluster, HR, SR, q, k, theta, W, s->rr_ws.p, s->rr_info.p,
                                            drop_tol, in_smem, LB);
        if (le != cudaSuccess) return fail(HBSD_ERR_CUDA, std::string("rayleigh_ritz launch: ") + cudaGetErrorString(le));
        count_launch(s);
        launched = true;
    }
    if (!launched) return rayleigh_ritz(s, HR, SR, q, k, theta, W, info_host, st);
    int info[4] = {0, 0, 0, 0};
    HBSD_CUDA(cudaMemcpyAsync(info, s->rr_info.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    HBSD_CUDA(cudaStreamSynchronize(st));
    if (std::getenv("HBSD_TRACE") && !info[3]) {
        uint64_t t[7];
        const int64_t off = (int64_t)5 * q * q + 3 * q + (int64_t)q * k + 2 * k;
        HBSD_CUDA(cudaMemcpy(t, s->rr_ws.p + off, sizeof(t), cudaMemcpyDeviceToHost));
        std::fprintf(stderr, "[hbsd]   RR phases us: chol %.0f C %.0f tridiag %.0f eig %.0f invit %.0f back %.0f\n",
                     (t[1] - t[0]) * 1e-3, (t[2] - t[1]) * 1e-3, (t[3] - t[2]) * 1e-3, (t[4] - t[3]) * 1e-3,
                     (t[5] - t[4]) * 1e-3, (t[6] - t[5]) * 1e-3);
    }
    if (info[3]) return rayleigh_ritz(s, HR, SR, q, k, theta, W, info_host, st);   // Cholesky breakdown
    if (info_host) { info_host[0] = info[0]; info_host[1] = info[1]; }
    if (info[1] < k) return fail(HBSD_ERR_RR_RANK, "rayleigh_ritz: search space rank below k");
    return 0;
}

}  // namespace hbsd
