// Double-float ("df64") block products for the mixed form: steps 8 (Gram) and 10-11 (update).
//
// GB300 issues FP32 FMAs at 128 lanes per clock per SM and FP64 FMAs at 2, so a product whose
// FP64 rate is the bound runs faster as pairs of floats (hi + lo, Dekker 1971; Knuth's
// TwoSum): a product of two pairs is hi*hi exactly (TwoProd by FMA) plus the two cross terms,
// and the running sum is a pair kept by TwoSum and renormalised every few terms.  About 48
// significant bits per term; the Gram sums keep FP64 across 128-row tiles, so their long sums
// carry FP64 accuracy.
//
// The pair arithmetic (split, TwoProd + TwoSum, renormalisation) is in df64.h.
#include <mutex>

#include "common.h"
#include "df64.h"

namespace hbsd {

namespace {

using df::split_d;
using df::dfma;
using df::renorm;
using df::to_d;

struct Seg2d {
    const double* p0;
    int64_t ld0;
    int q0;
    const double* p1;
    int64_t ld1;
    __device__ __forceinline__ double at(int64_t i, int c) const {
        return c < q0 ? p0[i * ld0 + c] : p1[i * ld1 + (c - q0)];
    }
};

constexpr int GT = 32;          // output tile edge
constexpr int GR = 32;          // rows per shared-memory stage
constexpr int GFLUSH = 4;       // stages per FP64 flush (128 rows)

// One CTA: a 32 x 32 tile (a-block <= b-block) of Z^T H Z and Z^T S Z over a chunk of rows.
__global__ void __launch_bounds__(256) k_gram_df64(Seg2d Z, Seg2d ZH, Seg2d ZS, int q,
                                                   int64_t n, int64_t rows_per_chunk, double* __restrict__ partial) {
    __shared__ float2 sz[GR][GT + 1], sh[GR][GT + 1], ss[GR][GT + 1];
    // tile pair (ta <= tb) from the packed-triangle index of the block
    const int pidx = blockIdx.x;
    int tb = (int)((sqrtf(8.0f * (float)pidx + 1.0f) - 1.0f) * 0.5f);
    while ((tb + 1) * (tb + 2) / 2 <= pidx) ++tb;
    while (tb * (tb + 1) / 2 > pidx) --tb;
    const int ta = pidx - tb * (tb + 1) / 2;
    const int a0 = ta * GT, b0 = tb * GT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads, 2 x 2 outputs each
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
    const int64_t r1 = min(n, r0 + rows_per_chunk);
    double aH[2][2] = {{0, 0}, {0, 0}}, aS[2][2] = {{0, 0}, {0, 0}};
    float hH[2][2], lH[2][2], hS[2][2], lS[2][2];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) { hH[u][v] = lH[u][v] = hS[u][v] = lS[u][v] = 0.f; }
    int stage = 0;
    for (int64_t i0 = r0; i0 < r1; i0 += GR, ++stage) {
        for (int t = threadIdx.x; t < GR * GT; t += 256) {
            const int rr = t / GT, cc = t % GT;
            const int64_t i = i0 + rr;
            const bool ok = i < r1;
            sz[rr][cc] = split_d((ok && a0 + cc < q) ? Z.at(i, a0 + cc) : 0.0);
            sh[rr][cc] = split_d((ok && b0 + cc < q) ? ZH.at(i, b0 + cc) : 0.0);
            ss[rr][cc] = split_d((ok && b0 + cc < q) ? ZS.at(i, b0 + cc) : 0.0);
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < GR; ++rr) {
            const float2 z0 = sz[rr][ty * 2], z1 = sz[rr][ty * 2 + 1];
            const float2 h0 = sh[rr][tx * 2], h1 = sh[rr][tx * 2 + 1];
            const float2 s0 = ss[rr][tx * 2], s1 = ss[rr][tx * 2 + 1];
            dfma(z0, h0, hH[0][0], lH[0][0]); dfma(z0, h1, hH[0][1], lH[0][1]);
            dfma(z1, h0, hH[1][0], lH[1][0]); dfma(z1, h1, hH[1][1], lH[1][1]);
            dfma(z0, s0, hS[0][0], lS[0][0]); dfma(z0, s1, hS[0][1], lS[0][1]);
            dfma(z1, s0, hS[1][0], lS[1][0]); dfma(z1, s1, hS[1][1], lS[1][1]);
            if ((rr & 7) == 7) {
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int v = 0; v < 2; ++v) { renorm(hH[u][v], lH[u][v]); renorm(hS[u][v], lS[u][v]); }
            }
        }
        __syncthreads();
        if ((stage % GFLUSH) == GFLUSH - 1 || i0 + GR >= r1) {
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    aH[u][v] += to_d(hH[u][v], lH[u][v]);
                    aS[u][v] += to_d(hS[u][v], lS[u][v]);
                    hH[u][v] = lH[u][v] = hS[u][v] = lS[u][v] = 0.f;
                }
        }
    }
    const int64_t qq = (int64_t)q * q;
    double* ph = partial + (int64_t)blockIdx.y * 2 * qq;
    double* ps = ph + qq;
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) {
            const int a = a0 + ty * 2 + u, b = b0 + tx * 2 + v;
            if (a < q && b < q) {
                ph[(int64_t)a * q + b] = aH[u][v];
                ps[(int64_t)a * q + b] = aS[u][v];
            }
        }
}

// Sum the chunks in order; entry (a, b), a <= b, of Z^T X Z is used for both (a, b) and (b, a).
__global__ void __launch_bounds__(256) k_gram_final_upper(const double* __restrict__ partial, int nchunks, int q,
                                                          double* __restrict__ HR, double* __restrict__ SR) {
    // 32 entries per block (lanes), the chunks split over the 8 warps, then summed in warp order:
    // the order is fixed, so the result is deterministic.  Entries a <= b are summed and mirrored.
    __shared__ double rh[8][33], rs[8][33];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int64_t qq = (int64_t)q * q;
    const int64_t idx = (int64_t)blockIdx.x * 32 + lane;
    const int a = (int)(idx / q), b = (int)(idx - (int64_t)(idx / q) * q);
    const bool on = idx < qq && a <= b;
    double h = 0.0, sv = 0.0;
    if (on)
        for (int c = g; c < nchunks; c += 8) {
            const double* ph = partial + (int64_t)c * 2 * qq;
            h += ph[idx];
            sv += ph[qq + idx];
        }
    rh[g][lane] = h;
    rs[g][lane] = sv;
    __syncthreads();
    if (g == 0 && on) {
        double H = 0.0, S = 0.0;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            H += rh[t][lane];
            S += rs[t][lane];
        }
        HR[idx] = H;
        SR[idx] = S;
        HR[(int64_t)b * q + a] = H;
        SR[(int64_t)b * q + a] = S;
    }
}

// W (q x k, FP64) -> pairs
__global__ void k_split_w(const double* __restrict__ W, int64_t cnt, float2* __restrict__ W2) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
        W2[t] = split_d(W[t]);
}

// Z0(:, 0:k) <- [Z0 Z1] W.  Threads are flattened over (row group, column): kc = min(k, 256)
// columns per pass, ng = min(256 / kc, 8) row groups of UR rows, so a CTA covers ng * UR rows;
// the rows (split) and W (q x k pairs) are staged in shared memory, W shared by the row groups.
// Every output sums its q terms in column order, the running pair renormalised after each
// term whose index is 7 mod 8 (the loops run in blocks of RN = 8 terms and a short tail).
constexpr int UR = 8;
constexpr int RN = 8;

__global__ void __launch_bounds__(256) k_update_df64(double* __restrict__ Z0, int64_t ld0, int q0,
                                                     const double* __restrict__ Z1, int64_t ld1, int q1, int64_t n,
                                                     const float2* __restrict__ W2, int k, int ng) {
    extern __shared__ __align__(16) float2 smu[];
    const int q = q0 + q1;
    const int rows = ng * UR;
    float2* zrow = smu;                      // [rows][q]
    float2* wsm = smu + (int64_t)rows * q;   // [q][k]
    const int64_t i0 = (int64_t)blockIdx.x * rows;
    for (int t = threadIdx.x; t < rows * q; t += 256) {
        const int rr = t / q, c = t % q;
        const int64_t i = i0 + rr;
        double v = 0.0;
        if (i < n) v = c < q0 ? Z0[i * ld0 + c] : Z1[i * ld1 + (c - q0)];
        zrow[t] = split_d(v);
    }
    for (int t = threadIdx.x; t < q * k; t += 256) wsm[t] = W2[t];
    __syncthreads();
    const int kc = min(k, 256);
    const int g = threadIdx.x / kc, cl = threadIdx.x % kc;
    if (g >= ng) return;
    const float2* zr = zrow + (int64_t)g * UR * q;
    for (int jb = 0; jb < k; jb += kc) {
        const int j = jb + cl;
        if (j >= k) continue;
        float ah[UR], al[UR];
#pragma unroll
        for (int u = 0; u < UR; ++u) { ah[u] = 0.f; al[u] = 0.f; }
        const float2* wc = wsm + j;
        int c = 0;
        for (; c + RN <= q; c += RN) {
#pragma unroll
            for (int cc = 0; cc < RN; ++cc) {
                const float2 wv = wc[(c + cc) * k];
#pragma unroll
                for (int u = 0; u < UR; ++u) dfma(zr[u * q + c + cc], wv, ah[u], al[u]);
            }
#pragma unroll
            for (int u = 0; u < UR; ++u) renorm(ah[u], al[u]);
        }
        for (; c < q; ++c) {
            const float2 wv = wc[c * k];
#pragma unroll
            for (int u = 0; u < UR; ++u) dfma(zr[u * q + c], wv, ah[u], al[u]);
        }
#pragma unroll
        for (int u = 0; u < UR; ++u) {
            const int64_t i = i0 + g * UR + u;
            if (i < n) Z0[i * ld0 + j] = to_d(ah[u], al[u]);
        }
    }
}

// The same product for q too large to stage W with the rows: UR rows per CTA staged once
// (split), one output column per thread (blockDim.x columns per pass, a multiple of 32 chosen so
// the passes are even), each thread reading its own column of W straight from L2, RN terms at a
// time (no other thread of the CTA reads it, so staging it would buy nothing).  Same term order
// and renormalisation as above.  In place: the outputs are written only after every row of the
// CTA was staged, and only the staged copy is read.
__global__ void __launch_bounds__(512) k_update_df64_kt(double* __restrict__ Z0, int64_t ld0, int q0,
                                                        const double* __restrict__ Z1, int64_t ld1, int q1, int64_t n,
                                                        const float2* __restrict__ W2, int k) {
    extern __shared__ __align__(16) float2 smu[];
    const int q = q0 + q1;
    const int nt = blockDim.x;
    float2* zrow = smu;                     // [UR][q]
    const int64_t i0 = (int64_t)blockIdx.x * UR;
    for (int t = threadIdx.x; t < UR * q; t += nt) {
        const int rr = t / q, c = t % q;
        const int64_t i = i0 + rr;
        double v = 0.0;
        if (i < n) v = c < q0 ? Z0[i * ld0 + c] : Z1[i * ld1 + (c - q0)];
        zrow[t] = split_d(v);
    }
    __syncthreads();
    for (int jb = 0; jb < k; jb += nt) {
        const int j = jb + threadIdx.x;
        if (j >= k) break;   // no barrier follows
        float ah[UR], al[UR];
#pragma unroll
        for (int u = 0; u < UR; ++u) { ah[u] = 0.f; al[u] = 0.f; }
        const float2* wc = W2 + j;
        int c = 0;
        for (; c + RN <= q; c += RN) {
            float2 wv[RN];
#pragma unroll
            for (int cc = 0; cc < RN; ++cc) wv[cc] = __ldg(wc + (int64_t)(c + cc) * k);
#pragma unroll
            for (int cc = 0; cc < RN; ++cc) {
#pragma unroll
                for (int u = 0; u < UR; ++u) dfma(zrow[u * q + c + cc], wv[cc], ah[u], al[u]);
            }
#pragma unroll
            for (int u = 0; u < UR; ++u) renorm(ah[u], al[u]);
        }
        for (; c < q; ++c) {
            const float2 wv = __ldg(wc + (int64_t)c * k);
#pragma unroll
            for (int u = 0; u < UR; ++u) dfma(zrow[u * q + c], wv, ah[u], al[u]);
        }
#pragma unroll
        for (int u = 0; u < UR; ++u) {
            const int64_t i = i0 + u;
            if (i < n) Z0[i * ld0 + j] = to_d(ah[u], al[u]);
        }
    }
}

}  // namespace

int gram2_df64(Session* s, const double* Z0, int64_t ld0, int q0, const double* Z1, int64_t ld1, int q1,
               const double* H0, int64_t ldh0, const double* H1, int64_t ldh1, const double* S0, int64_t lds0,
               const double* S1, int64_t lds1, int64_t n, double* HR, double* SR, cudaStream_t st) {
    const int q = q0 + q1;
    if (q <= 0) return 0;
    const int tb = ceil_div(q, GT);
    const int ntile = tb * (tb + 1) / 2;
    // chunks of rows: enough CTAs for every SM several times over, a multiple of the stage height
    int nch = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, ceil_div(152 * 8, ntile)));
    int64_t rpc = round_up((n + nch - 1) / nch, GR);
    nch = (int)((n + rpc - 1) / rpc);
    HBSD_TRY(s->ws.alloc((size_t)nch * 2 * q * q + 64));
    Seg2d Z{Z0, ld0, q0, Z1, ld1}, ZH{H0, ldh0, q0, H1, ldh1}, ZS{S0, lds0, q0, S1, lds1};
    k_gram_df64<<<dim3(ntile, nch), 256, 0, st>>>(Z, ZH, ZS, q, n, rpc, s->ws.p);
    HBSD_LAUNCHED(s);
    const int64_t qq = (int64_t)q * q;
    k_gram_final_upper<<<ceil_div(qq, 32), 256, 0, st>>>(s->ws.p, nch, q, HR, SR);
    HBSD_LAUNCHED(s);
    return 0;
}

int update2_df64(Session* s, double* Z0, int64_t ld0, int q0, const double* Z1, int64_t ld1, int q1, int64_t n,
                 const double* W, int k, cudaStream_t st, bool split_w) {
    const int q = q0 + q1;
    if (k > q0) return fail(HBSD_ERR_ARG, "update: k must not exceed the first segment width");
    // W staged whole when it fits with the rows (kernel k_update_df64), else read by each
    // thread from L2 (k_update_df64_kt: passes of nt <= 512 columns, as even as multiples of 32
    // allow, one pass for k <= 512)
    const int kc0 = std::min(k, 256);
    const int ng = std::max(1, std::min(256 / kc0, 8));
    const int rows = ng * UR;
    const size_t smem_whole = ((size_t)rows * q + (size_t)q * k) * sizeof(float2);
    const bool whole = smem_whole <= 220 * 1024;
    const int npass = ceil_div(k, 512);
    const int nt = (int)round_up(ceil_div(k, npass), 32);
    const size_t smem = whole ? smem_whole : (size_t)UR * q * sizeof(float2);
    if (smem > 220 * 1024) return fail(HBSD_ERR_ARG, "update: q too large for the double-float kernel");
    {
        static std::mutex attr_mu;
        static size_t attr = 0;
        std::lock_guard<std::mutex> lk(attr_mu);
        if (smem > 48 * 1024 && smem > attr) {
            HBSD_CUDA(cudaFuncSetAttribute(k_update_df64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            HBSD_CUDA(cudaFuncSetAttribute(k_update_df64_kt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr = smem;
        }
    }
    HBSD_TRY(s->df_w.alloc((size_t)q * k));
    if (split_w) {
        const int64_t cnt = (int64_t)q * k;
        k_split_w<<<ceil_div(cnt, 256), 256, 0, st>>>(W, cnt, s->df_w.p);
        HBSD_LAUNCHED(s);
    }
    if (whole) k_update_df64<<<ceil_div(n, rows), 256, smem, st>>>(Z0, ld0, q0, Z1, ld1, q1, n, s->df_w.p, k, ng);
    else k_update_df64_kt<<<ceil_div(n, UR), nt, smem, st>>>(Z0, ld0, q0, Z1, ld1, q1, n, s->df_w.p, k);
    HBSD_LAUNCHED(s);
    return 0;
}

}  // namespace hbsd
