// SELL-C-sigma storage of the shared (H, S) pattern and the fused block SpMM that produces
// H X and S X in one pass over the pattern (LABPSD steps 3 and 7; Sec. 4 footnote: H and S
// share one sparsity pattern, so one column index serves two values).
//
// Layout: rows are sorted by length (descending) inside windows of sigma rows, grouped into
// slices of C rows and padded to the slice's longest row.  Entry j of slot t of slice s is at
// slice_ptr[s] + j*C + t, so the C rows of a slice read their j-th entries from one contiguous
// segment.  Values are interleaved as (h - sigma0 s, s): one 16-byte (FP64) or 8-byte (FP32)
// load yields both.
//
// Block vectors are row-major, so the X-row that a nonzero needs is one contiguous vector.
// A row is handled by lpr lanes; each lane owns VW consecutive columns per chunk (one 16-byte
// vector load), so the gather of an X row is coalesced and vectorised.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "common.h"
#include "df64.h"

namespace hbsd {

int sell_build(Sell& m, int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
               const double* hval, const double* sval, double sigma0) {
    const int C = m.C;
    const int sigma = m.sigma;
    m.n = n;
    m.nnz = row_ptr[n];
    std::vector<int32_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    for (int64_t w0 = 0; w0 < n; w0 += sigma) {
        int64_t w1 = std::min<int64_t>(n, w0 + sigma);
        std::stable_sort(order.begin() + w0, order.begin() + w1, [&](int32_t a, int32_t b) {
            return (row_ptr[a + 1] - row_ptr[a]) > (row_ptr[b + 1] - row_ptr[b]);
        });
    }
    m.n_slots = round_up(n, C);
    m.n_slices = m.n_slots / C;
    std::vector<int32_t> slot_row(m.n_slots, -1);
    for (int64_t i = 0; i < n; ++i) slot_row[i] = order[i];
    std::vector<int64_t> sptr(m.n_slices + 1, 0);
    std::vector<int32_t> slen(m.n_slices, 0);
    for (int64_t s = 0; s < m.n_slices; ++s) {
        int64_t mx = 0;
        for (int t = 0; t < C; ++t) {
            int32_t r = slot_row[s * C + t];
            if (r >= 0) mx = std::max<int64_t>(mx, row_ptr[r + 1] - row_ptr[r]);
        }
        slen[s] = (int32_t)mx;
        sptr[s + 1] = sptr[s] + mx * C;
    }
    m.stored = sptr[m.n_slices];
    m.h_slice_ptr = sptr;
    m.h_slot_row = slot_row;
    // D = diag(S)^{-1/2} (the diagonal entry of each row of S)
    m.h_dscale.assign(n, 1.0);
    for (int64_t r = 0; r < n; ++r)
        for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e)
            if (col_idx[e] == r && sval[e] > 0.0) m.h_dscale[r] = 1.0 / std::sqrt(sval[e]);
    std::vector<int32_t> cols(m.stored, 0);
    std::vector<double2> hs(m.stored, make_double2(0.0, 0.0));
    m.h_entry_of_csr.assign(m.nnz, -1);
    for (int64_t s = 0; s < m.n_slices; ++s) {
        for (int t = 0; t < C; ++t) {
            int32_t r = slot_row[s * C + t];
            int64_t len = r >= 0 ? row_ptr[r + 1] - row_ptr[r] : 0;
            int32_t pad_col = (r >= 0 && len > 0) ? col_idx[row_ptr[r + 1] - 1] : 0;
            for (int64_t j = 0; j < slen[s]; ++j) {
                int64_t pos = sptr[s] + j * C + t;
                if (j < len) {
                    int64_t e = row_ptr[r] + j;
                    cols[pos] = col_idx[e];
                    double hv = hval[e];
                    double sv = sval[e];
                    double shifted = hv - sigma0 * sv;
                    hs[pos] = make_double2(shifted, sv);
                    m.h_entry_of_csr[e] = pos;
                } else {
                    cols[pos] = pad_col;
                }
            }
        }
    }
    HBSD_TRY(m.slice_ptr.alloc(m.n_slices + 1));
    HBSD_TRY(m.slice_len.alloc(m.n_slices));
    HBSD_TRY(m.cols.alloc(m.stored));
    HBSD_TRY(m.hs.alloc(m.stored));
    HBSD_TRY(m.slot_row.alloc(m.n_slots));
    HBSD_CUDA(cudaMemcpy(m.slice_ptr.p, sptr.data(), sptr.size() * 8, cudaMemcpyHostToDevice));
    HBSD_CUDA(cudaMemcpy(m.slice_len.p, slen.data(), slen.size() * 4, cudaMemcpyHostToDevice));
    HBSD_CUDA(cudaMemcpy(m.cols.p, cols.data(), cols.size() * 4, cudaMemcpyHostToDevice));
    HBSD_CUDA(cudaMemcpy(m.hs.p, hs.data(), hs.size() * sizeof(double2), cudaMemcpyHostToDevice));
    HBSD_CUDA(cudaMemcpy(m.slot_row.p, slot_row.data(), slot_row.size() * 4, cudaMemcpyHostToDevice));
    m.h_cols = cols;
    HBSD_TRY(m.dscale.alloc(n));
    HBSD_CUDA(cudaMemcpy(m.dscale.p, m.h_dscale.data(), n * 8, cudaMemcpyHostToDevice));
    {
        std::vector<double> dinv(n);
        for (int64_t i = 0; i < n; ++i) dinv[i] = 1.0 / m.h_dscale[i];
        HBSD_TRY(m.dinv.alloc(n));
        HBSD_CUDA(cudaMemcpy(m.dinv.p, dinv.data(), n * 8, cudaMemcpyHostToDevice));
    }
    HBSD_TRY(m.hs32.alloc(m.stored));
    return sell_fill_fp32(m, hs.data(), cols.data(), slot_row.data());
}

// FP32 values of the diagonally scaled pencil (D Hs D, D S D), D = diag(S)^{-1/2}, for the FP32
// step entry points: FP32 works only on this pencil, because the unscaled basis spans ~30 orders
// of magnitude.
int sell_fill_fp32(Sell& m, const double2* hs, const int32_t* cols, const int32_t* slot_row) {
    std::vector<float2> hs32(m.stored, make_float2(0.f, 0.f));
    std::vector<float4> hsdf(m.stored, make_float4(0.f, 0.f, 0.f, 0.f));
    // double-float pair of a double: the nearest float, then the nearest float to the remainder
    auto pair = [](double v, float& hi, float& lo) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    };
    for (int64_t sl = 0; sl < m.n_slices; ++sl) {
        const int64_t len = (m.h_slice_ptr[sl + 1] - m.h_slice_ptr[sl]) / m.C;
        for (int t = 0; t < m.C; ++t) {
            const int32_t r = slot_row[sl * m.C + t];
            if (r < 0) continue;
            for (int64_t j = 0; j < len; ++j) {
                const int64_t pos = m.h_slice_ptr[sl] + j * m.C + t;
                const double f = m.h_dscale[r] * m.h_dscale[cols[pos]];
                hs32[pos] = make_float2((float)(f * hs[pos].x), (float)(f * hs[pos].y));
                float a, b, c, d;
                pair(f * hs[pos].x, a, b);
                pair(f * hs[pos].y, c, d);
                hsdf[pos] = make_float4(a, b, c, d);
            }
        }
    }
    HBSD_CUDA(cudaMemcpy(m.hs32.p, hs32.data(), hs32.size() * sizeof(float2), cudaMemcpyHostToDevice));
    HBSD_TRY(m.hsdf.alloc(m.stored));
    HBSD_CUDA(cudaMemcpy(m.hsdf.p, hsdf.data(), hsdf.size() * sizeof(float4), cudaMemcpyHostToDevice));
    return 0;
}

int sell_update_h(Sell& m, const double* hval, const double* sval, double sigma0) {
    std::vector<double2> hs(m.stored, make_double2(0.0, 0.0));
    for (int64_t e = 0; e < m.nnz; ++e) {
        int64_t pos = m.h_entry_of_csr[e];
        double shifted = hval[e] - sigma0 * sval[e];
        hs[pos] = make_double2(shifted, sval[e]);
    }
    HBSD_CUDA(cudaMemcpy(m.hs.p, hs.data(), hs.size() * sizeof(double2), cudaMemcpyHostToDevice));
    return sell_fill_fp32(m, hs.data(), m.h_cols.data(), m.h_slot_row.data());
}

// ---- kernels ------------------------------------------------------------------------
template <class T> struct VecOf;
template <> struct VecOf<double> { using V = double2; using P = double2; static constexpr int W = 2; };
template <> struct VecOf<float> { using V = float4; using P = float2; static constexpr int W = 4; };

template <class T>
__device__ __forceinline__ void vload(const T* p, T (&v)[VecOf<T>::W]);
template <>
__device__ __forceinline__ void vload<double>(const double* p, double (&v)[2]) {
    double2 t = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = t.x; v[1] = t.y;
}
template <>
__device__ __forceinline__ void vload<float>(const float* p, float (&v)[4]) {
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

template <class T>
__device__ __forceinline__ void vstore(T* p, const T (&v)[VecOf<T>::W], int valid);
template <>
__device__ __forceinline__ void vstore<double>(double* p, const double (&v)[2], int valid) {
    if (valid >= 2) *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    else if (valid == 1) p[0] = v[0];
}
template <>
__device__ __forceinline__ void vstore<float>(float* p, const float (&v)[4], int valid) {
    if (valid >= 4) *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else for (int i = 0; i < valid; ++i) p[i] = v[i];
}

__device__ __forceinline__ void ldhs(const double2* hs, int64_t e, double& h, double& s) {
    double2 t = __ldg(hs + e);
    h = t.x; s = t.y;
}
__device__ __forceinline__ void ldhs(const float2* hs, int64_t e, float& h, float& s) {
    float2 t = __ldg(hs + e);
    h = t.x; s = t.y;
}

// MODE 0: pair (HX, SX).  MODE 1: shifted, Y = HX - e_j SX.
template <class T, int CH, int MODE>
__global__ void __launch_bounds__(256) k_spmm(
    const int64_t* __restrict__ slice_ptr, const int32_t* __restrict__ slice_len,
    const int32_t* __restrict__ cols, const typename VecOf<T>::P* __restrict__ hs,
    const int32_t* __restrict__ slot_row, int64_t n_slots, int C, const T* __restrict__ X,
    int64_t ldx, int k, int lpr_log2, T* __restrict__ Y0, int64_t ld0, T* __restrict__ Y1,
    int64_t ld1, const T* __restrict__ shifts) {
    constexpr int VW = VecOf<T>::W;
    const int lpr = 1 << lpr_log2;
    const int lane = threadIdx.x & (lpr - 1);
    const int64_t slot = (int64_t)blockIdx.x * (blockDim.x >> lpr_log2) + (threadIdx.x >> lpr_log2);
    if (slot >= n_slots) return;
    const int64_t sl = slot / C;
    const int t = (int)(slot - sl * C);
    const int64_t base = slice_ptr[sl] + t;
    const int len = slice_len[sl];
    T ah[CH][VW], as[CH][VW];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int v = 0; v < VW; ++v) { ah[c][v] = T(0); as[c][v] = T(0); }
    int col0[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) col0[c] = VW * (lane + c * lpr);
#pragma unroll 4
    for (int j = 0; j < len; ++j) {
        const int64_t e = base + (int64_t)j * C;
        const int cj = __ldg(cols + e);
        T hv, sv;
        ldhs(hs, e, hv, sv);
        const T* xr = X + (int64_t)cj * ldx;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            if (col0[c] < k) {
                T x[VW];
                vload<T>(xr + col0[c], x);
#pragma unroll
                for (int v = 0; v < VW; ++v) {
                    ah[c][v] = fma(hv, x[v], ah[c][v]);
                    as[c][v] = fma(sv, x[v], as[c][v]);
                }
            }
        }
    }
    const int row = slot_row[slot];
    if (row < 0) return;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const int cc = col0[c];
        if (cc >= k) continue;
        const int valid = min(VW, k - cc);
        if (MODE == 0) {
            vstore<T>(Y0 + (int64_t)row * ld0 + cc, ah[c], valid);
            vstore<T>(Y1 + (int64_t)row * ld1 + cc, as[c], valid);
        } else {
            T y[VW];
#pragma unroll
            for (int v = 0; v < VW; ++v) {
                T ev = (cc + v < k) ? shifts[cc + v] : T(0);
                y[v] = ah[c][v] - ev * as[c][v];
            }
            vstore<T>(Y0 + (int64_t)row * ld0 + cc, y, valid);
        }
    }
}

template <class T>
static const typename VecOf<T>::P* values_of(const Sell& m);
template <>
const double2* values_of<double>(const Sell& m) { return m.hs.p; }
template <>
const float2* values_of<float>(const Sell& m) { return m.hs32.p; }

// most lanes per row: the autotuner's choice for the session, else 32
static int spmm_lanes(const Session* s) {
    const int v = s ? s->tune_spmm_lpr : 0;
    return (v == 4 || v == 8 || v == 16) ? v : 32;
}

template <class T, int MODE>
static int spmm_launch(Session* s, const Sell& m, const T* X, int64_t ldx, int k, T* Y0, int64_t ld0,
                       T* Y1, int64_t ld1, const T* e, cudaStream_t st) {
    constexpr int VW = VecOf<T>::W;
    if (k <= 0) return 0;
    if ((ldx % VW) || (ld0 % VW) || (MODE == 0 && (ld1 % VW)))
        return fail(HBSD_ERR_ARG, "spmm: leading dimensions must be multiples of the vector width");
    // columns are processed in passes of at most lpr_max lanes * VW * 4 chunks; each row gets the
    // smallest power-of-two number of lanes (up to lpr_max, the autotuner's choice) that covers
    // its vectors in at most 4 chunks
    const int lpr_max = spmm_lanes(s);
    const int pass_cols = lpr_max * VW * 4;
    for (int c0 = 0; c0 < k; c0 += pass_cols) {
        const int kk = std::min(pass_cols, k - c0);
        int vecs = ceil_div(kk, VW);
        int lpr = 1, lg = 0;
        while (lpr < vecs && lpr < lpr_max) { lpr <<= 1; ++lg; }
        const int ch = ceil_div(vecs, lpr);
        const int rows_per_cta = 256 / lpr;
        const int grid = ceil_div(m.n_slots, rows_per_cta);
        const T* Xc = X + c0;
        T* Y0c = Y0 + c0;
        T* Y1c = Y1 ? Y1 + c0 : nullptr;
        const T* ec = e ? e + c0 : nullptr;
#define HBSD_SPMM_CASE(CHV)                                                                    \
    case CHV:                                                                                  \
        k_spmm<T, CHV, MODE><<<grid, 256, 0, st>>>(m.slice_ptr.p, m.slice_len.p, m.cols.p,      \
                                                   values_of<T>(m), m.slot_row.p, m.n_slots,   \
                                                   m.C, Xc, ldx, kk, lg, Y0c, ld0, Y1c, ld1, ec); \
        break;
        switch (ch) {
            HBSD_SPMM_CASE(1)
            HBSD_SPMM_CASE(2)
            HBSD_SPMM_CASE(3)
            HBSD_SPMM_CASE(4)
            default:
                return fail(HBSD_ERR_ARG, "spmm: internal chunking error");
        }
#undef HBSD_SPMM_CASE
        HBSD_LAUNCHED(s);
    }
    return 0;
}

// ---- double-float SpMM on the scaled pencil (mixed form) ------------------------------------------
// X2 = D^-1 X as double-float pairs (the FP64 scaling, then split_d's exact bit split)
__global__ void k_split_scaled(const double* __restrict__ X, int64_t ldx, int k, int64_t n,
                               const double* __restrict__ dinv, float2* __restrict__ X2, int64_t ld2) {
    const int64_t total = n * k;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k;
        const int j = (int)(t - i * k);
        X2[i * ld2 + j] = df::split_d(X[i * ldx + j] * dinv[i]);
    }
}

// Pair mode of k_spmm in double-float: per stored entry the (hi, lo) of D Hs D and of D S D, per
// column pair one float4 of X2; sums by df::dfma, renormalised every 8 entries; the row result is
// scaled back by D^-1 in FP64.
template <int CH>
__global__ void __launch_bounds__(256) k_spmm_df64(
    const int64_t* __restrict__ slice_ptr, const int32_t* __restrict__ slice_len, const int32_t* __restrict__ cols,
    const float4* __restrict__ hsdf, const int32_t* __restrict__ slot_row, int64_t n_slots, int C,
    const float2* __restrict__ X2, int64_t ld2, int k, int lpr_log2, const double* __restrict__ dinv,
    double* __restrict__ Y0, int64_t ld0, double* __restrict__ Y1, int64_t ld1) {
    const int lpr = 1 << lpr_log2;
    const int lane = threadIdx.x & (lpr - 1);
    const int64_t slot = (int64_t)blockIdx.x * (blockDim.x >> lpr_log2) + (threadIdx.x >> lpr_log2);
    if (slot >= n_slots) return;
    const int64_t sl = slot / C;
    const int t = (int)(slot - sl * C);
    const int64_t base = slice_ptr[sl] + t;
    const int len = slice_len[sl];
    float ah[CH][2][2], as[CH][2][2];   // [chunk][column of the pair][hi, lo]
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int v = 0; v < 2; ++v) { ah[c][v][0] = ah[c][v][1] = as[c][v][0] = as[c][v][1] = 0.f; }
    int col0[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) col0[c] = 2 * (lane + c * lpr);
    for (int j = 0; j < len; ++j) {
        const int64_t e = base + (int64_t)j * C;
        const int cj = __ldg(cols + e);
        const float4 hv = __ldg(hsdf + e);
        const float2 h2 = make_float2(hv.x, hv.y), s2 = make_float2(hv.z, hv.w);
        const float2* xr = X2 + (int64_t)cj * ld2;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            if (col0[c] < k) {
                const float4 x = __ldg(reinterpret_cast<const float4*>(xr + col0[c]));
                const float2 x0 = make_float2(x.x, x.y), x1 = make_float2(x.z, x.w);
                df::dfma(h2, x0, ah[c][0][0], ah[c][0][1]);
                df::dfma(s2, x0, as[c][0][0], as[c][0][1]);
                df::dfma(h2, x1, ah[c][1][0], ah[c][1][1]);
                df::dfma(s2, x1, as[c][1][0], as[c][1][1]);
            }
        }
        if ((j & 7) == 7) {
#pragma unroll
            for (int c = 0; c < CH; ++c)
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    df::renorm(ah[c][v][0], ah[c][v][1]);
                    df::renorm(as[c][v][0], as[c][v][1]);
                }
        }
    }
    const int row = slot_row[slot];
    if (row < 0) return;
    const double di = dinv[row];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const int cc = col0[c];
        if (cc >= k) continue;
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            if (cc + v >= k) break;
            Y0[(int64_t)row * ld0 + cc + v] = df::to_d(ah[c][v][0], ah[c][v][1]) * di;
            Y1[(int64_t)row * ld1 + cc + v] = df::to_d(as[c][v][0], as[c][v][1]) * di;
        }
    }
}

int spmm_pair_df64(Session* s, const Sell& m, const double* X, int64_t ldx, int k, double* HX, int64_t ldhx,
                   double* SX, int64_t ldsx, cudaStream_t st) {
    if (k <= 0) return 0;
    const int64_t ld2 = round_up(k, 2);
    HBSD_TRY(s->x2.alloc((size_t)m.n * ld2));
    {
        const int64_t total = m.n * k;
        const int g = (int)std::min<int64_t>(std::max<int64_t>(1, (total + 255) / 256), 8192);
        k_split_scaled<<<g, 256, 0, st>>>(X, ldx, k, m.n, m.dinv.p, s->x2.p, ld2);
        HBSD_LAUNCHED(s);
    }
    const int lpr_max = spmm_lanes(s);
    const int pass_cols = lpr_max * 2 * 4;
    for (int c0 = 0; c0 < k; c0 += pass_cols) {
        const int kk = std::min(pass_cols, k - c0);
        const int vecs = ceil_div(kk, 2);
        int lpr = 1, lg = 0;
        while (lpr < vecs && lpr < lpr_max) { lpr <<= 1; ++lg; }
        const int ch = ceil_div(vecs, lpr);
        const int rows_per_cta = 256 / lpr;
        const int grid = ceil_div(m.n_slots, rows_per_cta);
#define HBSD_SPMM_DF_CASE(CHV)                                                                                 case CHV:                                                                                                      k_spmm_df64<CHV><<<grid, 256, 0, st>>>(m.slice_ptr.p, m.slice_len.p, m.cols.p, m.hsdf.p, m.slot_row.p,                                                  m.n_slots, m.C, s->x2.p + c0, ld2, kk, lg, m.dinv.p, HX + c0, ldhx,                                                SX + c0, ldsx);                                                     break;
        switch (ch) {
            HBSD_SPMM_DF_CASE(1)
            HBSD_SPMM_DF_CASE(2)
            HBSD_SPMM_DF_CASE(3)
            HBSD_SPMM_DF_CASE(4)
            default:
                return fail(HBSD_ERR_ARG, "spmm_df64: internal chunking error");
        }
#undef HBSD_SPMM_DF_CASE
        HBSD_LAUNCHED(s);
    }
    return nl_apply_add<double>(s, X, ldx, k, HX, ldhx, st);
}

// Both add the nonlocal term F G F^T X of the session (Eq. fgf) to the H product.
template <class T>
int spmm_pair(Session* s, const Sell& m, const T* X, int64_t ldx, int k, T* HX, int64_t ldhx,
              T* SX, int64_t ldsx, cudaStream_t st) {
    HBSD_TRY((spmm_launch<T, 0>(s, m, X, ldx, k, HX, ldhx, SX, ldsx, nullptr, st)));
    return nl_apply_add<T>(s, X, ldx, k, HX, ldhx, st);
}

template <class T>
int spmm_shifted(Session* s, const Sell& m, const T* X, int64_t ldx, int k, const T* e, T* Y,
                 int64_t ldy, cudaStream_t st) {
    HBSD_TRY((spmm_launch<T, 1>(s, m, X, ldx, k, Y, ldy, nullptr, 0, e, st)));
    return nl_apply_add<T>(s, X, ldx, k, Y, ldy, st);
}

template int spmm_pair<double>(Session*, const Sell&, const double*, int64_t, int, double*, int64_t,
                               double*, int64_t, cudaStream_t);
template int spmm_pair<float>(Session*, const Sell&, const float*, int64_t, int, float*, int64_t,
                              float*, int64_t, cudaStream_t);
template int spmm_shifted<double>(Session*, const Sell&, const double*, int64_t, int, const double*,
                                  double*, int64_t, cudaStream_t);
template int spmm_shifted<float>(Session*, const Sell&, const float*, int64_t, int, const float*,
                                 float*, int64_t, cudaStream_t);

}  // namespace hbsd
