// Rayleigh-Ritz (LABPSD step 9, remark 6) on one thread-block cluster.
//
// GB300 executes FP64 at two lanes per clock per SM: a dependent FP64 FMA takes about 64
// clocks, a division or square root about 640, while a cluster barrier costs about 0.2 us
// (0.8 us with a broadcast).  The reduced eigenproblem (q up to a few hundred) is therefore
// organised around short dependent chains: every CTA of the cluster owns a slice of rows in
// shared memory, pivots use one reciprocal square root and broadcast reciprocals, triangular
// solves are right-looking with the triangle staged in shared memory, and the Cholesky runs by
// row panels with one barrier per CTA.
//
//   1. D = diag(S_R)^{-1/2}; Cholesky D S_R D = L L^T by row panels (one barrier per CTA).
//      A pivot below RR_PIVOT_MIN (or NaN) sets info[3] and the host reruns the single-CTA
//      kernel, whose rank-revealing branch is the reading of the paper's silent breakdown case.
//   2. C = L^{-1} (D H_R D) L^{-T} by column-parallel forward substitutions, C = (C + C^T)/2.
//   3. Householder tridiagonalisation T = Q^T C Q (two barriers per column); the owners of the
//      rows of Q accumulate Q = H_0 H_1 ... on the fly.
//   4. The k lowest eigenvalues of T, coarse: FP32 Sturm-count multisection, one warp each.
//   5. Eigenvectors of T: an inverse-iteration solve at the coarse shift, then one solve at the
//      Rayleigh quotient; CholeskyQR of the block (a second pass when the vectors were far from
//      orthogonal); eigenvalues as Rayleigh quotients, sorted.
//   6. W = D L^{-T} Q Z: Y = Q Z by rows, then column-parallel back substitutions.
#include <cooperative_groups.h>

#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "common.h"

namespace cg = cooperative_groups;

namespace hbsd {

namespace {

constexpr double PIVOT_MIN = 1e-14;
constexpr int RR_THREADS_C = 512;
constexpr int RR_NW = RR_THREADS_C / 32;
constexpr double CHOLQR_SECOND_PASS = 1e-2;   // max |V^T V - I| above which CholeskyQR runs twice
constexpr size_t RR_SMEM_MAX = 225 * 1024;

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

// 1/d: an FP32 estimate refined by two Newton steps r <- r + r (1 - d r) (each roughly doubles
// the correct bits, 24 -> 48 -> full precision); operands outside the FP32 normal range use the
// IEEE division.
__device__ __forceinline__ double rcp64(double d) {
    const double ad = fabs(d);
    if (!(ad > 1e-30 && ad < 1e30)) return 1.0 / d;
    double r = (double)(1.0f / (float)d);
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    return fma(r, e, r);
}

// cluster barrier in two halves: work placed between them overlaps the barrier's latency
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// order-preserving integer key of a double (sorting on the integer pipe)
__device__ __forceinline__ unsigned long long dkey(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// (a, b), b <= a, of the p-th entry of a packed lower triangle
__device__ __forceinline__ void tri_index(int p, int& a, int& b) {
    a = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
    while ((a + 1) * (a + 2) / 2 <= p) ++a;
    while (a * (a + 1) / 2 > p) --a;
    b = p - a * (a + 1) / 2;
}

struct RRWork {
    double *Lg, *LgT, *Tg, *Cg, *V, *Y, *Gpart, *d, *e, *lam, *lamr, *scratch;
    uint64_t* stamps;
};

__host__ __device__ inline int64_t rr_stamp_offset(int q, int k, int nc) {
    return (int64_t)4 * q * q + (int64_t)2 * q * k + (int64_t)nc * k * (k + 1) / 2 + 2 * q + 2 * k;
}

__device__ RRWork rr_work(double* ws, int q, int k, int nc) {
    RRWork w;
    const int64_t qq = (int64_t)q * q;
    w.Lg = ws;
    w.LgT = w.Lg + qq;
    w.Tg = w.LgT + qq;
    w.Cg = w.Tg + qq;
    w.V = w.Cg + qq;
    w.Y = w.V + (int64_t)q * k;
    w.Gpart = w.Y + (int64_t)q * k;
    w.d = w.Gpart + (int64_t)nc * k * (k + 1) / 2;
    w.e = w.d + q;
    w.lam = w.e + q;
    w.lamr = w.lam + k;
    w.stamps = reinterpret_cast<uint64_t*>(ws + rr_stamp_offset(q, k, nc));
    w.scratch = ws + rr_stamp_offset(q, k, nc) + 16;
    return w;
}

// Shared-memory layout (doubles), fixed part:
//   A[rb q] | Qr[rb q] | vb2[2 (q+1)] | pb[q] | cb2[2 rb (q+2)] | dv[q] | dr[q] | rinv[q] | dd[q] |
//   ee[q] | fl[2 q] (floats: d, e^2, e) | red[64] | rinvG[k] | ord[k]
// then one region reused by the phases:
//   phases 2 and 6: Ls[q q] (when stage_l) | xw[NW q]
//   phase 5:        G[k k] | Vr[rb k] | yw[NW k] | scr[nwr 6q] (when scr_sm)
struct RRLayout {
    int64_t fixed, p26, p5, total;
};
// grows: the row blocks A, Qr, cb2 and the phase-5 G, Vr live in a per-CTA region of the global
// workspace instead (large q); shared memory keeps the q-vectors and the per-warp buffers.
inline RRLayout rr_layout(int q, int k, int rb, int nwr, int stage_l, int scr_sm, int grows = 0) {
    RRLayout L;
    L.fixed = (grows ? 0 : (int64_t)2 * rb * q + (int64_t)2 * rb * (q + 2)) + 2 * (q + 1) + q + 5 * q + 2 * q + 64 +
              2 * k;
    L.p26 = (stage_l ? (int64_t)q * q : 0) + (int64_t)RR_NW * q;
    L.p5 = (grows ? 0 : (int64_t)k * k + (int64_t)rb * k) + (int64_t)RR_NW * k + (scr_sm ? (int64_t)nwr * 6 * q : 0);
    L.total = L.fixed + (L.p26 > L.p5 ? L.p26 : L.p5);
    return L;
}
// doubles of one CTA's global row region (grows): A | Qr | cb2 | G | Vr
__host__ __device__ inline int64_t rr_grows_per(int q, int k, int rb) {
    return (int64_t)2 * rb * q + (int64_t)2 * rb * (q + 2) + (int64_t)k * k + (int64_t)rb * k;
}

}  // namespace

__host__ __device__ int64_t rr_cluster_ws_doubles(int q, int k, int nc, int grows) {
    const int rb = (q + nc - 1) / nc;
    return rr_stamp_offset(q, k, nc) + 16 + (int64_t)nc * RR_NW * 6 * q + 64 +
           (grows ? (int64_t)nc * rr_grows_per(q, k, rb) : 0) + 3 * k;   // + per-vector diagnostics
}

// drop_tol = 0: a pivot below PIVOT_MIN stops the kernel (info[3]) for the caller's fallback.
// drop_tol > 0: a pivot below drop_tol removes that column from the reduced problem (pivoted
// Cholesky rank reveal): its row of L becomes e_k and its row/column of H_R is decoupled onto an
// eigenvalue above every other one, so it never enters the lowest k.
__global__ void __launch_bounds__(RR_THREADS_C, 1)
    k_rr_cluster(const double* __restrict__ HR, const double* __restrict__ SR, int q, int k,
                 double* __restrict__ theta, double* __restrict__ Wout, double* __restrict__ ws,
                 int* __restrict__ info, double drop_tol, int stage_l, int scr_sm, int grows) {
    cg::cluster_group cluster = cg::this_cluster();
    const int NC = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int rb = (q + NC - 1) / NC;
    const int r0 = min(q, rank * rb), r1 = min(q, r0 + rb);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwr = min((k + NC - 1) / NC, RR_NW);   // inverse-iteration warps per CTA
    extern __shared__ __align__(16) double sm[];
    RRWork W = rr_work(ws, q, k, NC);
    // global row regions of the CTAs (grows): A | Qr | cb2 | G | Vr, one region per rank
    double* const Rg = W.scratch + (int64_t)NC * RR_NW * 6 * q;
    const int64_t rper = rr_grows_per(q, k, rb);
    // per-vector diagnostics of the eigenvector phase (read by the host under HBSD_RRDBG=2)
    double* const vdiag = ws + rr_cluster_ws_doubles(q, k, 16, 1) - 3 * k;
    double* A;                                    // rb x q: row i at (i - r0) * q
    double* Qr;                                   // rb x q: rows of Q
    double* vb2;                                  // [2][q+1]: Householder vector, tau at [q]
    double* pb;                                   // [q]
    double* cb2;                                  // [2][rb][q+2]: Cholesky panels, code at [q], 1/l_cc at [q+1]
    double* dv;
    if (grows) {
        A = Rg + (int64_t)rank * rper;
        Qr = A + (int64_t)rb * q;
        cb2 = Qr + (int64_t)rb * q;
        vb2 = sm;
        pb = vb2 + 2 * (q + 1);
        dv = pb + q;
    } else {
        A = sm;
        Qr = A + (int64_t)rb * q;
        vb2 = Qr + (int64_t)rb * q;
        pb = vb2 + 2 * (q + 1);
        cb2 = pb + q;
        dv = cb2 + (int64_t)2 * rb * (q + 2);
    }
    double* dr = dv + q;                          // 1.0 where a column was dropped
    double* rinv = dr + q;                        // 1 / L_ii
    double* dd = rinv + q;                        // tridiagonal
    double* ee = dd + q;
    float* df = reinterpret_cast<float*>(ee + q); // floats: d[q], e^2[q], e[q] (in 2q doubles)
    float* e2f = df + q;
    float* ef = e2f + q;
    double* red = ee + 3 * q;                     // [0..31] per-warp partials, [32..63] cluster values
    double* rinvG = red + 64;                     // [k]
    int* ord = reinterpret_cast<int*>(rinvG + k); // [k]
    double* big = rinvG + 2 * k;
    const bool stamp = rank == 0 && tid == 0;

    for (int i = tid; i < q; i += nt) {
        const double sii = SR[(int64_t)i * q + i];
        const bool usable = sii > 0.0 && isfinite(sii) && isfinite(HR[(int64_t)i * q + i]);
        // drop mode: a column with a zero or non-finite S_R diagonal is dropped up front
        dv[i] = (usable || drop_tol == 0.0) ? rsqrt(sii) : 0.0;
        dr[i] = 0.0;
    }
    __syncthreads();
    for (int idx = tid; idx < (r1 - r0) * q; idx += nt) {
        const int i = r0 + idx / q, j = idx % q;
        const double v = SR[(int64_t)i * q + j] * dv[i] * dv[j];
        A[idx] = (dv[i] == 0.0 || dv[j] == 0.0) ? 0.0 : v;   // 0 * inf guard for dropped columns
    }
    if (stamp) W.stamps[0] = gtimer();
    __syncthreads();

    // ---- 1. Cholesky by row panels: panel b = the rows of CTA b (symmetric storage, row c holds
    //         column c).  CTA b factors its rows (sequential pivots inside the CTA), broadcasts
    //         them, and the later CTAs apply the rank-rb update to their rows: one cluster
    //         barrier per panel. ----
    bool broke = false;
    for (int b = 0; b < NC; ++b) {
        const int p0 = min(q, b * rb), p1 = min(q, p0 + rb);
        if (p0 >= q) break;
        double* pbk = cb2 + (int64_t)(b & 1) * rb * (q + 2);   // row c at (c - p0) (q + 2); code, 1/l_cc after
        if (rank == b) {
            for (int c = p0; c < p1; ++c) {
                double* row = A + (int64_t)(c - r0) * q;
                const double piv = row[c];
                const bool drop = drop_tol > 0.0 && !(piv >= drop_tol);
                const bool bad = !drop && !(piv >= PIVOT_MIN);
                const double inv = (bad || drop) ? 1.0 : rsqrt(piv);
                __syncthreads();
                for (int j = c + 1 + tid; j < q; j += nt) row[j] = drop ? 0.0 : row[j] * inv;   // L(j, c)
                if (tid == 0) {
                    row[c] = (bad || drop) ? 1.0 : piv * inv;
                    double* pr = pbk + (int64_t)(c - p0) * (q + 2);
                    pr[q] = (bad ? 1.0 : 0.0) + (drop ? 2.0 : 0.0);
                    pr[q + 1] = inv;
                }
                __syncthreads();
                const int m = q - c - 1;
                for (int idx = tid; idx < (p1 - c - 1) * m; idx += nt) {   // the panel's later rows
                    const int i = c + 1 + idx / m, j = c + 1 + idx % m;
                    double* a = A + (int64_t)(i - r0) * q + j;
                    *a = fma(-row[i], row[j], *a);
                }
                __syncthreads();   // the next pivot is read only after this update
            }
        }
        cluster.sync();
        if (rank != b) {
            // pull L(j, c), j >= p1, and the codes and 1/l_cc of the panel rows from CTA b
            const double* srcA = grows ? Rg + (int64_t)b * rper : cluster.map_shared_rank(A, b);
            const double* srcP = grows ? Rg + (int64_t)b * rper + (int64_t)2 * rb * q + (int64_t)(b & 1) * rb * (q + 2)
                                       : cluster.map_shared_rank(pbk, b);
            const int w = (rank > b ? q - p1 : 0) + 2;
            for (int idx = tid; idx < (p1 - p0) * w; idx += nt) {
                const int c = p0 + idx / w, jj = idx % w;
                const int j = jj < w - 2 ? p1 + jj : q + (jj - (w - 2));
                pbk[(int64_t)(c - p0) * (q + 2) + j] =
                    j < q ? srcA[(int64_t)(c - p0) * q + j] : srcP[(int64_t)(c - p0) * (q + 2) + j];
            }
            __syncthreads();
        }
        int codes = 0;
        for (int c = p0; c < p1; ++c) codes |= (int)pbk[(int64_t)(c - p0) * (q + 2) + q];
        if (codes & 1) { broke = true; break; }
        for (int c = p0 + tid; c < p1; c += nt) {
            const double* pr = pbk + (int64_t)(c - p0) * (q + 2);
            if ((int)pr[q] & 2) dr[c] = 1.0;
            rinv[c] = pr[q + 1];
        }
        if (rank > b && r0 < r1) {
            const int m = q - p1;
            const int np = p1 - p0;
            for (int idx = tid; idx < (r1 - r0) * m; idx += nt) {
                const int i = r0 + idx / m, j = p1 + idx % m;
                if (j < i) continue;   // lower part of the owned rows is rewritten below
                double acc = A[(int64_t)(i - r0) * q + j];
                for (int c = 0; c < np; ++c) {
                    const double* pr = pbk + (int64_t)c * (q + 2);
                    acc = fma(-pr[i], pr[j], acc);
                }
                A[(int64_t)(i - r0) * q + j] = acc;
            }
            for (int idx = tid; idx < (r1 - r0) * np; idx += nt) {   // L(i, c) of the owned rows
                const int i = r0 + idx / np, c = idx % np;
                A[(int64_t)(i - r0) * q + p0 + c] = pbk[(int64_t)c * (q + 2) + i];
            }
        }
        __syncthreads();
    }
    if (broke) {
        if (rank == 0 && tid == 0) { info[0] = 0; info[3] = 1; }
        return;
    }
    if (stamp) W.stamps[1] = gtimer();
    // L (lower; a dropped column's row is e_k) to global, row-major and transposed.  Owned row i
    // holds L(i, j) for j < r0 in column j; inside its own panel L(i, j) sits in row j, column i.
    for (int idx = tid; idx < (r1 - r0) * q; idx += nt) {
        const int i = r0 + idx / q, j = idx % q;
        double v = 0.0;
        if (j < r0) v = A[idx];
        else if (j <= i) v = A[(int64_t)(j - r0) * q + i];
        if (dr[i] != 0.0) v = (j == i) ? 1.0 : 0.0;
        W.Lg[(int64_t)i * q + j] = v;
        W.LgT[(int64_t)j * q + i] = v;
    }
    cluster.sync();

    // ---- 2. C = L^{-1} Hd L^{-T}: right-looking forward substitutions, one warp per column ----
    const double* Lt = stage_l ? big : W.LgT;     // row i of L^T = column i of L
    double* xw = big + (stage_l ? (int64_t)q * q : 0);
    double* xv = xw + (int64_t)warp * q;
    if (stage_l) {
        for (int t = tid; t < q * q; t += nt) big[t] = W.LgT[t];
        __syncthreads();
    }
    auto fwd_solve = [&]() {   // L x = b in place (xv), rows top-down
        for (int i = 0; i < q; ++i) {
            const double xi = xv[i] * rinv[i];
            __syncwarp();
            if (lane == 0) xv[i] = xi;
            const double* li = Lt + (int64_t)i * q;
            for (int l = i + 1 + lane; l < q; l += 32) xv[l] = fma(-li[l], xi, xv[l]);
            __syncwarp();
        }
    };
    // T(:, j) = L^{-1} Hd(:, j) (H_R symmetric); stored Tg[j][i] = T(i, j)
    for (int j = r0 + warp; j < r1; j += RR_NW) {
        for (int i = lane; i < q; i += 32)
            xv[i] = (dr[i] != 0.0 || dr[j] != 0.0 || dv[i] == 0.0 || dv[j] == 0.0)
                        ? 0.0 : HR[(int64_t)j * q + i] * dv[i] * dv[j];
        __syncwarp();
        fwd_solve();
        for (int i = lane; i < q; i += 32) W.Tg[(int64_t)j * q + i] = xv[i];
        __syncwarp();
    }
    cluster.sync();
    // C(:, j) = L^{-1} T(j, :)^T, T(j, i) = Tg[i][j]; stored Cg[j][i] = C(i, j)
    for (int j = r0 + warp; j < r1; j += RR_NW) {
        for (int i = lane; i < q; i += 32) xv[i] = W.Tg[(int64_t)i * q + j];
        __syncwarp();
        fwd_solve();
        for (int i = lane; i < q; i += 32) W.Cg[(int64_t)j * q + i] = xv[i];
        __syncwarp();
    }
    cluster.sync();
    for (int idx = tid; idx < (r1 - r0) * q; idx += nt) {
        const int i = r0 + idx / q, j = idx % q;
        A[idx] = 0.5 * (W.Cg[(int64_t)i * q + j] + W.Cg[(int64_t)j * q + i]);
        Qr[idx] = (i == j) ? 1.0 : 0.0;
    }
    if (drop_tol > 0.0) {
        // eigenvalue of the dropped (decoupled) coordinates: above the Gershgorin bound of C
        __syncthreads();
        double gmax = 0.0;
        for (int i = r0 + warp; i < r1; i += RR_NW) {
            double rs = 0.0;
            for (int j = lane; j < q; j += 32) rs += fabs(A[(int64_t)(i - r0) * q + j]);
            gmax = fmax(gmax, wsum(rs));
        }
        if (lane == 0) red[warp] = gmax;
        __syncthreads();
        if (tid == 0) {
            double g = 0.0;
            for (int w2 = 0; w2 < RR_NW; ++w2) g = fmax(g, red[w2]);
            for (int c = 0; c < NC; ++c) cluster.map_shared_rank(red, c)[32 + rank] = g;
        }
        cluster.sync();
        double bigv = 0.0;
        for (int c = 0; c < NC; ++c) bigv = fmax(bigv, red[32 + c]);
        bigv = 2.0 * bigv + 1.0;
        for (int i = r0 + tid; i < r1; i += nt)
            if (dr[i] != 0.0) A[(int64_t)(i - r0) * q + i] = bigv;
    }
    __syncthreads();
    if (stamp) W.stamps[2] = gtimer();

    // ---- 3. Householder tridiagonalisation, Q accumulated: two cluster barriers per column ----
    // One warp of the owner of row kk forms v_kk and broadcasts it (double-buffered); every CTA
    // computes p = tau A v for its rows and broadcasts it; after the second barrier every warp
    // forms p.v from the broadcast vectors, w = p - K v replaces p, and the owned rows of C take
    // the rank-2 update.  H_kk is applied to the owned rows of Q while the owner of the next row
    // forms the next reflector.
    // v_kk into the owner's own buffer: one warp computes it, then all threads push it on
    auto make_v = [&](int kk) {   // called by the whole owner CTA
        double* vbk = vb2 + (kk & 1) * (q + 1);
        const double* row = A + (int64_t)(kk - r0) * q;
        if (warp == 0) {
            double s2 = 0.0;
            for (int j = kk + 1 + lane; j < q; j += 32) s2 = fma(row[j], row[j], s2);
            s2 = wsum(s2);
            const double x0 = row[kk + 1];
            const double tail = s2 - x0 * x0;
            double alpha, t;
            if (tail <= 0.0 || s2 == 0.0) {
                alpha = x0;
                t = 0.0;
            } else {
                alpha = -copysign(s2 * rsqrt(s2), x0);
                t = rcp64(s2 - alpha * x0);   // 2 / v^T v with v^T v = 2 (s2 - alpha x0)
            }
            for (int j = kk + 1 + lane; j < q; j += 32)
                vbk[j] = (t == 0.0) ? 0.0 : (j == kk + 1 ? x0 - alpha : row[j]);
            if (lane == 0) {
                vbk[q] = t;
                W.d[kk] = row[kk];
                W.e[kk] = alpha;
            }
        }
        __syncthreads();
        const int m = q - kk;   // entries kk+1 .. q-1 and tau
        for (int idx = tid; idx < m * NC; idx += nt) {
            const int c = idx / m, j = kk + 1 + idx % m;
            if (c != rank) cluster.map_shared_rank(vbk, c)[j] = vbk[j];
        }
    };
    auto q_update = [&](int kk) {   // Q <- Q H_kk on the owned rows
        const double* vbk = vb2 + (kk & 1) * (q + 1);
        const double t = vbk[q];
        if (t == 0.0) return;
        for (int i = r0 + warp; i < r1; i += RR_NW) {
            double* qi = Qr + (int64_t)(i - r0) * q;
            double sq = 0.0;
            for (int j = kk + 1 + lane; j < q; j += 32) sq = fma(qi[j], vbk[j], sq);
            sq = wsum(sq) * t;
            for (int j = kk + 1 + lane; j < q; j += 32) qi[j] = fma(-sq, vbk[j], qi[j]);
        }
    };
    long long tp[6] = {0, 0, 0, 0, 0, 0};   // per-CTA step-part clocks (thread 0), for tracing
    long long tc = clock64();
    auto tick = [&](int s) {
        if (tid == 0) {
            const long long t2 = clock64();
            tp[s] += t2 - tc;
            tc = t2;
        }
    };
    if (q >= 3 && r0 == 0 && r1 > 0) make_v(0);
    for (int kk = 0; kk + 2 < q; ++kk) {
        tick(5);
        cluster_arrive();                                         // v_kk on its way
        if (kk > 0) q_update(kk - 1);                             // H_{kk-1} on Q meanwhile
        tick(4);
        cluster_wait();                                           // v_kk visible everywhere
        tick(0);
        const double* vbk = vb2 + (kk & 1) * (q + 1);
        const double t = vbk[q];
        const int ib = max(r0, kk + 1);
        if (t != 0.0) {
            for (int i = ib + warp; i < r1; i += RR_NW) {
                const double* ai = A + (int64_t)(i - r0) * q;
                double acc = 0.0;
                for (int j = kk + 1 + lane; j < q; j += 32) acc = fma(ai[j], vbk[j], acc);
                acc = wsum(acc) * t;
                if (lane < NC) cluster.map_shared_rank(pb, lane)[i] = acc;
            }
            tick(1);
            cluster.sync();                                       // p visible everywhere
            tick(2);
            double pv = 0.0;
            for (int i = kk + 1 + lane; i < q; i += 32) pv = fma(pb[i], vbk[i], pv);
            const double K = 0.5 * t * wsum(pv);
            __syncthreads();                                      // every warp has read p
            for (int j = kk + 1 + tid; j < q; j += nt) pb[j] = fma(-K, vbk[j], pb[j]);   // w
            __syncthreads();
            const int m = q - kk - 1;
            for (int idx = tid; idx < (r1 - ib) * m; idx += nt) {
                const int i = ib + idx / m, j = kk + 1 + idx % m;
                double* a = A + (int64_t)(i - r0) * q + j;
                *a = fma(-vbk[i], pb[j], fma(-pb[i], vbk[j], *a));
            }
        } else {
            cluster.sync();                                       // keeps the barrier count uniform
        }
        __syncthreads();
        tick(3);
        if (kk + 3 < q && kk + 1 >= r0 && kk + 1 < r1) make_v(kk + 1);
    }
    if (q >= 3) {
        cluster_arrive();
        q_update(q - 3);
        cluster_wait();
    }
    tick(5);
    if (tid == 0)
        for (int x2 = 0; x2 < 6; ++x2) W.Cg[rank * 8 + x2] = (double)tp[x2];
    cluster.sync();
    for (int i = r0 + tid; i < r1; i += nt) {   // trailing 2 x 2 (or 1 x 1) block
        if (i >= q - 2) {
            W.d[i] = A[(int64_t)(i - r0) * q + i];
            W.e[i] = (i + 1 < q) ? A[(int64_t)(i - r0) * q + i + 1] : 0.0;
        }
    }
    if (stamp) W.stamps[3] = gtimer();
    cluster.sync();

    // ---- 4. the k lowest eigenvalues, coarse: FP32 Sturm multisection (one warp each) ----
    for (int i = tid; i < q; i += nt) {
        dd[i] = W.d[i];
        ee[i] = (i < q - 1) ? W.e[i] : 0.0;
        df[i] = (float)dd[i];
        ef[i] = (float)ee[i];
        e2f[i] = (float)(ee[i] * ee[i]);
    }
    __syncthreads();
    if (warp == 0) {   // Gershgorin interval and ||T||, lanes over the rows
        double gl = DBL_MAX, gu = -DBL_MAX, tn = 0.0;
        for (int i = lane; i < q; i += 32) {
            const double r = (i > 0 ? fabs(ee[i - 1]) : 0.0) + fabs(ee[i]);
            gl = fmin(gl, dd[i] - r);
            gu = fmax(gu, dd[i] + r);
            tn = fmax(tn, fabs(dd[i]) + r);
        }
        for (int o = 16; o > 0; o >>= 1) {
            gl = fmin(gl, __shfl_xor_sync(0xffffffffu, gl, o));
            gu = fmax(gu, __shfl_xor_sync(0xffffffffu, gu, o));
            tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
        }
        if (lane == 0) { red[32] = gl; red[33] = gu; red[34] = tn; }
    }
    __syncthreads();
    const double tnorm = red[34];
    const double pivmin = DBL_MIN * fmax(1.0, tnorm * tnorm);
    const float pivf = FLT_MIN * (float)fmax(1.0, fmin(tnorm * tnorm, 1e30));
    double gl = red[32], gu = red[33];
    const double span = fmax(gu - gl, DBL_MIN);
    gl -= 1e-5 * span + pivmin;
    gu += 1e-5 * span + pivmin;
    const int gw = rank * RR_NW + warp, ngw = NC * RR_NW;
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
    if (stamp) W.stamps[4] = gtimer();
    cluster.sync();

    // ---- 5a. eigenvectors of T; eigenvector j on CTA j % NC, warp j / NC ----
    // Inverse iteration at the coarse shift from a fixed pseudo-random start, then one solve at
    // the Rayleigh quotient theta = x^T T x.  Pivoted tridiagonal LU with reciprocal pivots,
    // sequential on lane 0; pivots below eps ||T|| are raised to it, so that a shift on an
    // eigenvalue amplifies the wanted direction by about 1/eps instead of overflowing.
    const int64_t goff = (int64_t)2 * rb * q + (int64_t)2 * rb * (q + 2);   // G in a global row region
    double* G = grows ? Rg + (int64_t)rank * rper + goff : big;   // phase-5 region
    double* Vr = G + (int64_t)k * k;
    double* yw = grows ? big : Vr + (int64_t)rb * k;
    double* scr_base = yw + (int64_t)RR_NW * k;
    {
        double* scr = scr_sm ? scr_base + (int64_t)warp * 6 * q : W.scratch + ((int64_t)rank * RR_NW + warp) * 6 * q;
        double* fdv = scr;             // reciprocals of the U diagonal
        double* fuv = scr + q;         // first super-diagonal
        double* fu2v = scr + 2 * q;    // second super-diagonal
        double* flv = scr + 3 * q;     // multipliers
        double* fpv = scr + 4 * q;     // pivot flags
        double* x = scr + 5 * q;       // iterate
        const double ptd = fmax(DBL_EPSILON * tnorm, pivmin);
        auto floor_piv = [&](double d) { return fabs(d) < ptd ? (d < 0.0 ? -ptd : ptd) : d; };
        auto solve64 = [&](double sh) {   // x <- (T - sh I)^{-1} x
            if (lane == 0) {
                for (int i = 0; i < q; ++i) { fdv[i] = dd[i] - sh; fuv[i] = ee[i]; fu2v[i] = 0.0; }
                for (int i = 0; i + 1 < q; ++i) {
                    const double sub = ee[i];
                    const double di = fdv[i];
                    if (fabs(di) >= fabs(sub)) {
                        const double ri = rcp64(floor_piv(di));
                        const double f = sub * ri;
                        fdv[i] = ri;
                        flv[i] = f;
                        fpv[i] = 0.0;
                        fdv[i + 1] = fma(-f, fuv[i], fdv[i + 1]);
                    } else {
                        const double ri = rcp64(floor_piv(sub));
                        const double f = di * ri;
                        flv[i] = f;
                        fpv[i] = 1.0;
                        const double tmp = fuv[i];
                        fuv[i] = fdv[i + 1];
                        fdv[i] = ri;
                        fdv[i + 1] = fma(-f, fdv[i + 1], tmp);
                        if (i + 2 < q) { fu2v[i] = fuv[i + 1]; fuv[i + 1] = -f * fuv[i + 1]; }
                    }
                }
                fdv[q - 1] = rcp64(floor_piv(fdv[q - 1]));
                for (int i = 0; i + 1 < q; ++i) {
                    double bi = x[i], bn = x[i + 1];
                    if (fpv[i] != 0.0) { const double t2 = bi; bi = bn; bn = t2; }
                    x[i] = bi;
                    x[i + 1] = fma(-flv[i], bi, bn);
                }
                for (int i = q - 1; i >= 0; --i) {
                    double sacc = x[i];
                    if (i + 1 < q) sacc = fma(-fuv[i], x[i + 1], sacc);
                    if (i + 2 < q) sacc = fma(-fu2v[i], x[i + 2], sacc);
                    x[i] = sacc * fdv[i];
                }
            }
            __syncwarp();
        };
        // x / ||x||; false (x untouched) when an entry of x is not finite or x is zero
        // (fmax drops NaN, so the entries are tested one by one)
        auto normalise = [&]() {
            double mx = 0.0;
            bool bad = false;
            for (int i = lane; i < q; i += 32) {
                bad |= !isfinite(x[i]);
                mx = fmax(mx, fabs(x[i]));
            }
            if (__any_sync(0xffffffffu, bad)) return false;
            for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (!(mx > 0.0 && isfinite(mx))) return false;
            const double sc = 1.0 / mx;
            double n2 = 0.0;
            for (int i = lane; i < q; i += 32) { x[i] *= sc; n2 = fma(x[i], x[i], n2); }
            const double inr = rsqrt(wsum(n2));
            for (int i = lane; i < q; i += 32) x[i] *= inr;
            __syncwarp();
            return true;
        };
        for (int j = rank + NC * warp; j < k && warp < nwr; j += NC * nwr) {
            for (int i = lane; i < q; i += 32) {
                uint64_t h = 0x9E3779B97F4A7C15ull * (uint64_t)(j + 1) + 0xBF58476D1CE4E5B9ull * (uint64_t)(i + 1);
                h ^= h >> 31;
                h *= 0x94D049BB133111EBull;
                h ^= h >> 29;
                x[i] = 0.5 + (double)(h >> 11) * (1.0 / 9007199254740992.0);
            }
            __syncwarp();
            solve64(W.lam[j]);
            normalise();
            for (int i = lane; i < q; i += 32) W.V[(int64_t)i * k + j] = x[i];   // kept if the next solve fails
            double th = 0.0;
            for (int i = lane; i < q; i += 32) {
                th = fma(dd[i] * x[i], x[i], th);
                if (i + 1 < q) th = fma(2.0 * ee[i] * x[i], x[i + 1], th);
            }
            th = wsum(th);
            __syncwarp();
            solve64(th);
            bool ok2 = normalise();
            if (ok2)
                for (int i = lane; i < q; i += 32) W.V[(int64_t)i * k + j] = x[i];
            // Rayleigh-quotient iteration until the residual ||T x - theta x|| is below
            // 1e-12 ||T|| (a start vector nearly orthogonal to the wanted eigenvector leaves a
            // neighbour's component after the first solve): at most three more solves
            // only for a separated eigenvalue: inside a cluster narrower than 1e-6 ||T|| further
            // solves would pull several vectors onto one eigenvector, while the mixing they
            // remove there costs almost nothing (it is weighted by the cluster width).  A vector
            // is accepted only while its quotient stays in eigenvalue j's interval (midpoints to
            // the neighbouring coarse eigenvalues): unguarded, the iteration can settle on a
            // neighbour and duplicate its vector.
            double gapj = DBL_MAX;
            if (j > 0) gapj = fmin(gapj, fabs(W.lam[j] - W.lam[j - 1]));
            if (j + 1 < k) gapj = fmin(gapj, fabs(W.lam[j + 1] - W.lam[j]));
            const bool separated = gapj > 1e-6 * tnorm;
            const double lo_j = j > 0 ? 0.5 * (W.lam[j - 1] + W.lam[j]) : -DBL_MAX;
            const double hi_j = j + 1 < k ? 0.5 * (W.lam[j] + W.lam[j + 1]) : DBL_MAX;
            auto rayleigh = [&]() {
                double t2 = 0.0;
                for (int i = lane; i < q; i += 32) {
                    t2 = fma(dd[i] * x[i], x[i], t2);
                    if (i + 1 < q) t2 = fma(2.0 * ee[i] * x[i], x[i + 1], t2);
                }
                return wsum(t2);
            };
            int extra = 0;
            if (ok2 && separated) {
                double th2 = rayleigh();
                while (extra < 3 && th2 >= lo_j && th2 <= hi_j) {
                    double r2 = 0.0;
                    for (int i = lane; i < q; i += 32) {
                        double ti = fma(dd[i] - th2, x[i], 0.0);
                        if (i > 0) ti = fma(ee[i - 1], x[i - 1], ti);
                        if (i + 1 < q) ti = fma(ee[i], x[i + 1], ti);
                        r2 = fma(ti, ti, r2);
                    }
                    r2 = wsum(r2);
                    __syncwarp();
                    th = th2;
                    if (r2 <= (1e-12 * tnorm) * (1e-12 * tnorm)) break;   // far below what the caller resolves
                    solve64(th);
                    ++extra;
                    if (!normalise()) break;               // W.V keeps the last accepted vector
                    th2 = rayleigh();
                    __syncwarp();
                    if (th2 < lo_j || th2 > hi_j) break;   // left the interval: rejected
                    for (int i = lane; i < q; i += 32) W.V[(int64_t)i * k + j] = x[i];
                    __syncwarp();
                }
            }
            if (lane == 0) {
                vdiag[j] = ok2 ? 1.0 + extra : 0.0;
                vdiag[k + j] = th;
                vdiag[2 * k + j] = W.lam[j];
            }
            __syncwarp();
        }
    }
    cluster.sync();
    if (stamp) W.stamps[7] = gtimer();

    // ---- 5b. CholeskyQR of V (q x k): G = V^T V over the cluster, R = chol(G) redundantly in
    //          every CTA, V <- V R^{-1} on the owned rows; a second pass when G was far from I ----
    const int npairs = k * (k + 1) / 2;
    for (int pass = 0; pass < 2; ++pass) {
        for (int t = tid; t < (r1 - r0) * k; t += nt) Vr[t] = W.V[(int64_t)r0 * k + t];
        __syncthreads();
        for (int p = tid; p < npairs; p += nt) {   // partial G over the owned rows
            int a, b;
            tri_index(p, a, b);
            double s = 0.0;
            for (int i = 0; i < r1 - r0; ++i) s = fma(Vr[(int64_t)i * k + a], Vr[(int64_t)i * k + b], s);
            W.Gpart[(int64_t)rank * npairs + p] = s;
        }
        cluster.sync();
        {   // each CTA sums a slice of the pairs and sends both triangles to every CTA
            const int per = (npairs + NC - 1) / NC;
            const int p0 = rank * per, p1 = min(npairs, p0 + per);
            for (int p = p0 + tid; p < p1; p += nt) {
                int a, b;
                tri_index(p, a, b);
                double s = 0.0;
                for (int c = 0; c < NC; ++c) s += W.Gpart[(int64_t)c * npairs + p];
                for (int c = 0; c < NC; ++c) {
                    double* Gc = grows ? Rg + (int64_t)c * rper + goff : cluster.map_shared_rank(G, c);
                    Gc[(int64_t)a * k + b] = s;
                    Gc[(int64_t)b * k + a] = s;
                }
            }
        }
        cluster.sync();
        // distance from orthonormality (the same in every CTA)
        double off = 0.0;
        for (int t = tid; t < k * k; t += nt) off = fmax(off, fabs(G[t] - ((t / k == t % k) ? 1.0 : 0.0)));
        for (int o = 16; o > 0; o >>= 1) off = fmax(off, __shfl_xor_sync(0xffffffffu, off, o));
        if (lane == 0) red[warp] = off;
        // G = R^T R, R upper triangular: row c of R in row c of G (columns > c), 1/R_cc in rinvG
        for (int c = 0; c < k; ++c) {
            __syncthreads();
            const double inv = rsqrt(fmax(G[(int64_t)c * k + c], DBL_MIN));
            for (int jj = c + 1 + tid; jj < k; jj += nt) G[(int64_t)c * k + jj] *= inv;
            if (tid == 0) rinvG[c] = inv;
            __syncthreads();
            const int m = k - c - 1;
            const int tri = m * (m + 1) / 2;
            for (int t = tid; t < tri; t += nt) {   // upper triangle of the trailing block
                int a, b;
                tri_index(t, a, b);                  // entry (row c+1+b, column c+1+a), b <= a
                const int i2 = c + 1 + b, j2 = c + 1 + a;
                double* g = G + (int64_t)i2 * k + j2;
                *g = fma(-G[(int64_t)c * k + i2], G[(int64_t)c * k + j2], *g);
            }
        }
        __syncthreads();
        // V <- V R^{-1} on the owned rows: y R = v, one warp per row, right-looking
        for (int i = r0 + warp; i < r1; i += RR_NW) {
            double* y = yw + (int64_t)warp * k;
            for (int c = lane; c < k; c += 32) y[c] = Vr[(int64_t)(i - r0) * k + c];
            __syncwarp();
            for (int c = 0; c < k; ++c) {
                const double yc = y[c] * rinvG[c];
                __syncwarp();
                if (lane == 0) y[c] = yc;
                const double* rc = G + (int64_t)c * k;
                for (int l = c + 1 + lane; l < k; l += 32) y[l] = fma(-rc[l], yc, y[l]);
                __syncwarp();
            }
            for (int c = lane; c < k; c += 32) W.V[(int64_t)i * k + c] = y[c];
            __syncwarp();
        }
        double offmax = 0.0;
        for (int w2 = 0; w2 < RR_NW; ++w2) offmax = fmax(offmax, red[w2]);
        cluster.sync();
        if (stamp) W.stamps[8 + pass] = gtimer();
        if (!(offmax > CHOLQR_SECOND_PASS)) break;
    }
    // eigenvalues: Rayleigh quotients of the orthonormal vectors
    for (int j = gw; j < k; j += ngw) {
        double acc = 0.0;
        for (int i = lane; i < q; i += 32) {
            const double yi = W.V[(int64_t)i * k + j];
            acc = fma(dd[i] * yi, yi, acc);
            if (i + 1 < q) acc = fma(2.0 * ee[i] * yi, W.V[(int64_t)(i + 1) * k + j], acc);
        }
        acc = wsum(acc);
        if (lane == 0) W.lamr[j] = acc;
    }
    cluster.sync();
    // ascending order (ties by index), computed identically in every CTA
    for (int j = tid; j < k; j += nt) {
        const unsigned long long kj = dkey(W.lamr[j]);
        int r = 0;
        for (int i = 0; i < k; ++i) {
            const unsigned long long ki = dkey(W.lamr[i]);
            r += (ki < kj) || (ki == kj && i < j);
        }
        ord[r] = j;
    }
    __syncthreads();
    if (stamp) W.stamps[5] = gtimer();

    // ---- 6. back-transforms: Y = Q Z (owned rows), then x = L^{-T} y (one warp per column) ----
    for (int idx = tid; idx < (r1 - r0) * k; idx += nt) {
        const int i = r0 + idx / k, j = idx % k;
        const double* qi = Qr + (int64_t)(i - r0) * q;
        const int src = ord[j];
        double s0 = 0.0, s1 = 0.0;
        int l = 0;
        for (; l + 1 < q; l += 2) {
            s0 = fma(qi[l], W.V[(int64_t)l * k + src], s0);
            s1 = fma(qi[l + 1], W.V[(int64_t)(l + 1) * k + src], s1);
        }
        if (l < q) s0 = fma(qi[l], W.V[(int64_t)l * k + src], s0);
        W.Y[(int64_t)i * k + j] = s0 + s1;
    }
    cluster.sync();
    const double* Lr = stage_l ? big : W.Lg;   // row i of L
    if (stage_l) {
        for (int t = tid; t < q * q; t += nt) big[t] = W.Lg[t];
        __syncthreads();
    }
    for (int j = rank + NC * warp; j < k; j += NC * RR_NW) {
        for (int i = lane; i < q; i += 32) xv[i] = W.Y[(int64_t)i * k + j];
        __syncwarp();
        for (int i = q - 1; i >= 0; --i) {   // L^T x = y, rows bottom-up
            const double xi = xv[i] * rinv[i];
            __syncwarp();
            if (lane == 0) xv[i] = xi;
            const double* li = Lr + (int64_t)i * q;
            for (int l = lane; l < i; l += 32) xv[l] = fma(-li[l], xi, xv[l]);
            __syncwarp();
        }
        bool bad = false;   // a non-finite output (an eigenvector block that CholeskyQR could not
                            // orthonormalise) sends the call to the single-CTA QL solver
        for (int i = lane; i < q; i += 32) {
            const double v = dv[i] * xv[i];
            bad |= !isfinite(v);
            Wout[(int64_t)i * k + j] = v;
        }
        if (lane == 0) {
            theta[j] = W.lamr[ord[j]];
            bad |= !isfinite(theta[j]);
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&info[2], 1);
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
    // 16 CTAs halve each CTA's rows in the tridiagonal reduction; measured faster from q ~ 48
    if (q >= 48) return 16;
    if (q >= 32) return 8;
    if (q >= 8) return 4;
    return 1;
}

int rayleigh_ritz_cluster(Session* s, const double* HR, const double* SR, int q, int k, double* theta, double* W,
                          int* info_host, cudaStream_t st, double drop_tol) {
    if (q <= 0 || k <= 0 || k > q) return fail(HBSD_ERR_ARG, "rayleigh_ritz: need 0 < k <= q");
    HBSD_TRY(s->rr_ws.alloc((size_t)std::max<int64_t>(rr_cluster_ws_doubles(q, k, 16, 1), (int64_t)4 * q * q + 3 * q + 64)));
    HBSD_TRY(s->rr_info.alloc(4));
    static const bool trace = std::getenv("HBSD_TRACE") != nullptr || std::getenv("HBSD_RRDBG") != nullptr;
    static thread_local cudaEvent_t tev[4];
    static thread_local bool tev_made = false;
    if (trace && !tev_made) {
        for (auto& e : tev) cudaEventCreate(&e);
        tev_made = true;
    }
    if (trace) cudaEventRecord(tev[0], st);
    HBSD_CUDA(cudaMemsetAsync(s->rr_info.p, 0, 4 * sizeof(int), st));
    // candidate cluster sizes, preferred first; a size whose shared-memory layout does not fit
    // or that the device cannot co-schedule is skipped
    const int pref = cluster_size_for(q);
    // candidates: shared-memory rows on 16, 8, 4, 2, 1 CTAs, then global rows on 16 CTAs (large q)
    const int cands[6] = {16, 8, 4, 2, 1, 16};
    bool launched = false;
    int used_nc = 0, used_stage = 0;
    for (int ci = 0; ci < 6 && !launched; ++ci) {
        const int NC = cands[ci];
        const int grows = ci == 5 ? 1 : 0;
        if ((!grows && NC > pref) || NC > q) continue;
        const int rb = (q + NC - 1) / NC;
        const int nwr = std::min((k + NC - 1) / NC, RR_NW);
        int stage_l = grows ? 0 : 1, scr_sm = 1;
        RRLayout L = rr_layout(q, k, rb, nwr, stage_l, scr_sm, grows);
        if ((size_t)L.total * sizeof(double) > RR_SMEM_MAX) { scr_sm = 0; L = rr_layout(q, k, rb, nwr, stage_l, scr_sm, grows); }
        if ((size_t)L.total * sizeof(double) > RR_SMEM_MAX) { stage_l = 0; L = rr_layout(q, k, rb, nwr, stage_l, scr_sm, grows); }
        if ((size_t)L.total * sizeof(double) > RR_SMEM_MAX) continue;
        const size_t smem = (size_t)L.total * sizeof(double);
        // attribute and co-scheduling checks are host calls of tens of microseconds: once per
        // (cluster size, shared-memory size)
        static std::mutex cache_mu;   // sessions of a server call this from several threads
        std::lock_guard<std::mutex> cache_lk(cache_mu);
        static size_t attr_smem = 0;
        static bool nonportable = false;
        static int ok_cache[17] = {0};
        static size_t ok_smem[17] = {0};
        if (smem > attr_smem) {
            HBSD_CUDA(cudaFuncSetAttribute(k_rr_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr_smem = smem;
        }
        if (NC > 8 && !nonportable) {
            HBSD_CUDA(cudaFuncSetAttribute(k_rr_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
            nonportable = true;
        }
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
        if (ok_smem[NC] == 0 || smem > ok_smem[NC]) {   // co-scheduling check for this size
            int nclusters = 0;
            cudaError_t oe = cudaOccupancyMaxActiveClusters(&nclusters, k_rr_cluster, &cfg);
            if (oe != cudaSuccess) (void)cudaGetLastError();
            ok_cache[NC] = (oe == cudaSuccess && nclusters >= 1) ? 1 : -1;
            ok_smem[NC] = smem;
        }
        if (ok_cache[NC] < 0) continue;
        cudaError_t le = cudaLaunchKernelEx(&cfg, k_rr_cluster, HR, SR, q, k, theta, W, s->rr_ws.p, s->rr_info.p,
                                            drop_tol, stage_l, scr_sm, grows);
        if (le != cudaSuccess) return fail(HBSD_ERR_CUDA, std::string("rayleigh_ritz launch: ") + cudaGetErrorString(le));
        count_launch(s);
        if (trace) cudaEventRecord(tev[1], st);
        launched = true;
        used_nc = NC;
        used_stage = stage_l;
    }
    if (!launched) return rayleigh_ritz(s, HR, SR, q, k, theta, W, info_host, st);
    int info[4] = {0, 0, 0, 0};
    HBSD_CUDA(cudaMemcpyAsync(info, s->rr_info.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    {
        static const char* dbg = std::getenv("HBSD_RRDBG");
        if (dbg && dbg[0] == '2') {
            std::vector<double> vd(3 * (size_t)k);
            HBSD_CUDA(cudaMemcpyAsync(vd.data(), s->rr_ws.p + rr_cluster_ws_doubles(q, k, 16, 1) - 3 * k,
                                      3 * k * sizeof(double), cudaMemcpyDeviceToHost, st));
            HBSD_CUDA(cudaStreamSynchronize(st));
            for (int j = 0; j < k; ++j)
                std::fprintf(stderr, "[hbsd]   RR vec %d solves-after-first %d theta %.12e coarse %.12e\n", j, (int)vd[j],
                             vd[k + j], vd[2 * k + j]);
        }
    }
    if (trace) cudaEventRecord(tev[2], st);
    HBSD_CUDA(cudaStreamSynchronize(st));
    if (trace) {
        cudaEventRecord(tev[3], st);
        cudaEventSynchronize(tev[3]);
        float a = 0.f, b = 0.f, c = 0.f;
        cudaEventElapsedTime(&a, tev[0], tev[1]);
        cudaEventElapsedTime(&b, tev[1], tev[2]);
        cudaEventElapsedTime(&c, tev[2], tev[3]);
        s->dbg_rr_kernel_ms += a + b;
        s->dbg_rr_wake_ms += c;
        if (std::getenv("HBSD_TRACE"))
            std::fprintf(stderr, "[hbsd]   RR events: memset+launch %.3f ms, after launch %.3f ms\n", a, b);
    }
    if (std::getenv("HBSD_TRACE") && !info[3]) {
        uint64_t t[10];
        HBSD_CUDA(cudaMemcpy(t, s->rr_ws.p + rr_stamp_offset(q, k, used_nc), sizeof(t), cudaMemcpyDeviceToHost));
        double tpv[16 * 8];
        const int64_t gp = (int64_t)3 * q * q;
        HBSD_CUDA(cudaMemcpy(tpv, s->rr_ws.p + gp, sizeof(double) * 8 * used_nc, cudaMemcpyDeviceToHost));
        for (int c = 0; c < used_nc; c += std::max(1, used_nc - 1))
            std::fprintf(stderr, "[hbsd]   RR tridiag CTA %d us: wait1 %.0f p %.0f sync2 %.0f upd %.0f qupd %.0f makev %.0f\n", c,
                         tpv[c * 8 + 0] / 2070.0, tpv[c * 8 + 1] / 2070.0, tpv[c * 8 + 2] / 2070.0, tpv[c * 8 + 3] / 2070.0,
                         tpv[c * 8 + 4] / 2070.0, tpv[c * 8 + 5] / 2070.0);
        std::fprintf(stderr,
                     "[hbsd]   RR q %d k %d NC %d stage %d us: chol %.0f C %.0f tridiag %.0f eig %.0f rqi %.0f "
                     "cholqr %.0f back %.0f\n",
                     q, k, used_nc, used_stage, (t[1] - t[0]) * 1e-3, (t[2] - t[1]) * 1e-3, (t[3] - t[2]) * 1e-3,
                     (t[4] - t[3]) * 1e-3, (t[7] - t[4]) * 1e-3, (t[5] - t[7]) * 1e-3, (t[6] - t[5]) * 1e-3);
    }
    // Cholesky breakdown (info[3]) or a non-finite output (info[2]): the single-CTA kernel, whose
    // implicit QL iteration gives orthonormal eigenvectors of T whatever the multiplicities (the
    // J-paired blocks of a complex session have every eigenvalue twice)
    if (info[3] || info[2]) return rayleigh_ritz(s, HR, SR, q, k, theta, W, info_host, st);
    if (info_host) { info_host[0] = info[0]; info_host[1] = info[1]; }
    if (info[1] < k) return fail(HBSD_ERR_RR_RANK, "rayleigh_ritz: search space rank below k");
    return 0;
}

}  // namespace hbsd
