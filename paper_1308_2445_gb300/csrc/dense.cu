// Dense block kernels of the LABPSD iteration:
//   col_dots / residual  -- steps 4-5 (Eq. res1), deterministic two-pass reductions
//   gram2                -- step 8: H_R = Z^T [H Z], S_R = Z^T [S Z] over Z = [Psi P]
//   update2              -- steps 10-11: Z(:, 0:k) := [Psi P] W, row-local and in place
//   rayleigh_ritz        -- step 9: scaled Cholesky + symmetric eigensolver in FP64
// Z = [Psi P] is passed as two row-major segments so that Psi and P keep their own
// (16-byte aligned) buffers.
#include <cfloat>
#include <cmath>
#include <mutex>

#include "common.h"

namespace hbsd {

// ---- block reductions ------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// partial[b * k + j] = sum over rows of chunk b of A(i,j) * B(i,j); 32 columns x 8 row lanes
template <class T>
__global__ void __launch_bounds__(256) k_coldot_partial(const T* __restrict__ A, int64_t lda,
                                                         const T* __restrict__ B, int64_t ldb,
                                                         int64_t n, int k, int64_t rows_per_chunk,
                                                         double* __restrict__ partial) {
    __shared__ double red[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_chunk;
    const int64_t r1 = min(n, r0 + rows_per_chunk);
    for (int j0 = 0; j0 < k; j0 += 32) {
        const int j = j0 + tx;
        double acc = 0.0;
        if (j < k)
            for (int64_t i = r0 + ty; i < r1; i += 8) acc += (double)A[i * lda + j] * (double)B[i * ldb + j];
        red[ty][tx] = acc;
        __syncthreads();
        if (ty == 0 && j < k) {
            double s = 0.0;
            for (int t = 0; t < 8; ++t) s += red[t][tx];
            partial[(int64_t)blockIdx.x * k + j] = s;
        }
        __syncthreads();
    }
}

__global__ void k_sum_partials(const double* __restrict__ partial, int nchunks, int k,
                               double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    double s = 0.0;
    for (int b = 0; b < nchunks; ++b) s += partial[(int64_t)b * k + j];
    out[j] = s;
}

static int reduction_chunks(int64_t n, int64_t* rows_per_chunk) {
    int nch = (int)std::min<int64_t>(304, std::max<int64_t>(1, (n + 255) / 256));
    *rows_per_chunk = (n + nch - 1) / nch;
    return nch;
}

template <class T>
int col_dots(Session* s, const T* A, int64_t lda, const T* B, int64_t ldb, int64_t n, int k,
             double* out, cudaStream_t st) {
    if (k <= 0) return 0;
    int64_t rpc;
    int nch = reduction_chunks(n, &rpc);
    HBSD_TRY(s->ws.alloc((size_t)nch * k + 64));
    k_coldot_partial<T><<<nch, 256, 0, st>>>(A, lda, B, ldb, n, k, rpc, s->ws.p);
    HBSD_LAUNCHED(s);
    k_sum_partials<<<ceil_div(k, 128), 128, 0, st>>>(s->ws.p, nch, k, out);
    HBSD_LAUNCHED(s);
    return 0;
}
template int col_dots<double>(Session*, const double*, int64_t, const double*, int64_t, int64_t, int,
                              double*, cudaStream_t);
template int col_dots<float>(Session*, const float*, int64_t, const float*, int64_t, int64_t, int,
                             double*, cudaStream_t);

// ---- residual (steps 4-5) ------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_residual_partial(const T* __restrict__ PH, int64_t ldh,
                                                           const T* __restrict__ PS, int64_t lds,
                                                           const double* __restrict__ E, int m,
                                                           T* __restrict__ R, int64_t ldr, int64_t n,
                                                           int64_t rows_per_chunk,
                                                           double* __restrict__ partial) {
    __shared__ double red_r[8][33], red_h[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_chunk;
    const int64_t r1 = min(n, r0 + rows_per_chunk);
    for (int j0 = 0; j0 < m; j0 += 32) {
        const int j = j0 + tx;
        double ar = 0.0, ah = 0.0;
        if (j < m) {
            const T ej = (T)E[j];
            for (int64_t i = r0 + ty; i < r1; i += 8) {
                const T h = PH[i * ldh + j];
                const T r = h - PS[i * lds + j] * ej;
                if (R) R[i * ldr + j] = r;
                ar += (double)r * (double)r;
                ah += (double)h * (double)h;
            }
        }
        red_r[ty][tx] = ar;
        red_h[ty][tx] = ah;
        __syncthreads();
        if (ty == 0 && j < m) {
            double sr = 0.0, sh = 0.0;
            for (int t = 0; t < 8; ++t) { sr += red_r[t][tx]; sh += red_h[t][tx]; }
            partial[((int64_t)blockIdx.x * m + j) * 2 + 0] = sr;
            partial[((int64_t)blockIdx.x * m + j) * 2 + 1] = sh;
        }
        __syncthreads();
    }
}

__global__ void k_residual_final(const double* __restrict__ partial, int nchunks, int m,
                                 double* __restrict__ res, double* __restrict__ rnorm) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double sr = 0.0, sh = 0.0;
    for (int b = 0; b < nchunks; ++b) {
        sr += partial[((int64_t)b * m + j) * 2 + 0];
        sh += partial[((int64_t)b * m + j) * 2 + 1];
    }
    res[j] = sqrt(sr) / sqrt(sh);
    if (rnorm) rnorm[j] = sqrt(sr);
}

template <class T>
int residual(Session* s, const T* PH, int64_t ldh, const T* PS, int64_t lds, const double* E, int m,
             T* R, int64_t ldr, int64_t n, double* res, double* rnorm, cudaStream_t st) {
    int64_t rpc;
    int nch = reduction_chunks(n, &rpc);
    HBSD_TRY(s->ws.alloc((size_t)nch * m * 2 + 64));
    k_residual_partial<T><<<nch, 256, 0, st>>>(PH, ldh, PS, lds, E, m, R, ldr, n, rpc, s->ws.p);
    HBSD_LAUNCHED(s);
    k_residual_final<<<ceil_div(m, 128), 128, 0, st>>>(s->ws.p, nch, m, res, rnorm);
    HBSD_LAUNCHED(s);
    return 0;
}
template int residual<double>(Session*, const double*, int64_t, const double*, int64_t, const double*,
                              int, double*, int64_t, int64_t, double*, double*, cudaStream_t);
template int residual<float>(Session*, const float*, int64_t, const float*, int64_t, const double*,
                             int, float*, int64_t, int64_t, double*, double*, cudaStream_t);

// ---- Gram (step 8) ---------------------------------------------------------------------
template <class T>
struct Seg2 {
    const T* p0; int64_t ld0; int q0;
    const T* p1; int64_t ld1;
    __device__ __forceinline__ T at(int64_t i, int c) const {
        return c < q0 ? p0[i * ld0 + c] : p1[i * ld1 + (c - q0)];
    }
};

// One CTA: 32 x 32 output tile (a-block, b-block) over a chunk of rows.  Each 32-row tile is
// accumulated in T, the tiles in FP64 (for T = float this keeps the long sums in FP64).
template <class T>
__global__ void __launch_bounds__(256) k_gram_partial(Seg2<T> Z, Seg2<T> ZH, Seg2<T> ZS, int q, int64_t n,
                                                      int64_t rows_per_chunk, int tiles,
                                                      double* __restrict__ partial) {
    __shared__ T sz[32][33], sh[32][33], ss[32][33];
    const int tile = blockIdx.x;
    const int ta = tile / tiles, tb = tile % tiles;
    const int a0 = ta * 32, b0 = tb * 32;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 2 x 2 outputs
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
    const int64_t r1 = min(n, r0 + rows_per_chunk);
    double accH[2][2] = {{0, 0}, {0, 0}}, accS[2][2] = {{0, 0}, {0, 0}};
    for (int64_t i0 = r0; i0 < r1; i0 += 32) {
        for (int t = threadIdx.x; t < 32 * 32; t += 256) {
            const int rr = t >> 5, cc = t & 31;
            const int64_t i = i0 + rr;
            const bool ok = i < r1;
            sz[rr][cc] = (ok && a0 + cc < q) ? Z.at(i, a0 + cc) : T(0);
            sh[rr][cc] = (ok && b0 + cc < q) ? ZH.at(i, b0 + cc) : T(0);
            ss[rr][cc] = (ok && b0 + cc < q) ? ZS.at(i, b0 + cc) : T(0);
        }
        __syncthreads();
        T tH[2][2] = {{0, 0}, {0, 0}}, tS[2][2] = {{0, 0}, {0, 0}};
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr) {
            const T z0 = sz[rr][ty * 2], z1 = sz[rr][ty * 2 + 1];
            const T h0 = sh[rr][tx * 2], h1 = sh[rr][tx * 2 + 1];
            const T s0 = ss[rr][tx * 2], s1 = ss[rr][tx * 2 + 1];
            tH[0][0] = fma(z0, h0, tH[0][0]); tH[0][1] = fma(z0, h1, tH[0][1]);
            tH[1][0] = fma(z1, h0, tH[1][0]); tH[1][1] = fma(z1, h1, tH[1][1]);
            tS[0][0] = fma(z0, s0, tS[0][0]); tS[0][1] = fma(z0, s1, tS[0][1]);
            tS[1][0] = fma(z1, s0, tS[1][0]); tS[1][1] = fma(z1, s1, tS[1][1]);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 2; ++v) { accH[u][v] += (double)tH[u][v]; accS[u][v] += (double)tS[u][v]; }
        __syncthreads();
    }
    const int64_t qq = (int64_t)q * q;
    double* ph = partial + (int64_t)blockIdx.y * 2 * qq;
    double* ps = ph + qq;
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) {
            const int a = a0 + ty * 2 + u, b = b0 + tx * 2 + v;
            if (a < q && b < q) {
                ph[(int64_t)a * q + b] = accH[u][v];
                ps[(int64_t)a * q + b] = accS[u][v];
            }
        }
}

// Sum the chunks in order and symmetrise: X_R = (A + A^T) / 2.
__global__ void k_gram_final(const double* __restrict__ partial, int nchunks, int q,
                             double* __restrict__ HR, double* __restrict__ SR) {
    const int64_t qq = (int64_t)q * q;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= qq) return;
    const int a = (int)(idx / q), b = (int)(idx % q);
    double h_ab = 0, h_ba = 0, s_ab = 0, s_ba = 0;
    for (int c = 0; c < nchunks; ++c) {
        const double* ph = partial + (int64_t)c * 2 * qq;
        h_ab += ph[(int64_t)a * q + b];
        h_ba += ph[(int64_t)b * q + a];
        s_ab += ph[qq + (int64_t)a * q + b];
        s_ba += ph[qq + (int64_t)b * q + a];
    }
    HR[idx] = 0.5 * (h_ab + h_ba);
    SR[idx] = 0.5 * (s_ab + s_ba);
}

template <class T>
int gram2(Session* s, const T* Z0, int64_t ld0, int q0, const T* Z1, int64_t ld1, int q1,
          const T* H0, int64_t ldh0, const T* H1, int64_t ldh1, const T* S0,
          int64_t lds0, const T* S1, int64_t lds1, int64_t n, double* HR, double* SR,
          cudaStream_t st) {
    const int q = q0 + q1;
    if (q <= 0) return 0;
    const int tiles = ceil_div(q, 32);
    int nch = (int)std::max<int64_t>(1, std::min<int64_t>((n + 127) / 128, ceil_div(1216, tiles * tiles)));
    const int64_t rpc = (n + nch - 1) / nch;
    nch = (int)((n + rpc - 1) / rpc);
    const size_t need = (size_t)nch * 2 * q * q;
    HBSD_TRY(s->ws.alloc(need + 64));
    Seg2<T> Z{Z0, ld0, q0, Z1, ld1}, ZH{H0, ldh0, q0, H1, ldh1}, ZS{S0, lds0, q0, S1, lds1};
    dim3 grid(tiles * tiles, nch);
    k_gram_partial<T><<<grid, 256, 0, st>>>(Z, ZH, ZS, q, n, rpc, tiles, s->ws.p);
    HBSD_LAUNCHED(s);
    const int64_t qq = (int64_t)q * q;
    k_gram_final<<<ceil_div(qq, 256), 256, 0, st>>>(s->ws.p, nch, q, HR, SR);
    HBSD_LAUNCHED(s);
    return 0;
}
template int gram2<double>(Session*, const double*, int64_t, int, const double*, int64_t, int, const double*, int64_t,
                           const double*, int64_t, const double*, int64_t, const double*, int64_t, int64_t, double*,
                           double*, cudaStream_t);
template int gram2<float>(Session*, const float*, int64_t, int, const float*, int64_t, int, const float*, int64_t,
                          const float*, int64_t, const float*, int64_t, const float*, int64_t, int64_t, double*,
                          double*, cudaStream_t);

// ---- cross Gram of the complex recovery ----------------------------------------------------
// Sum the chunks in order; A1 = (X - X^T) / 2 (the antisymmetric part of Z^T V1), A2 = (Y + Y^T) / 2.
__global__ void k_gram_final_skew(const double* __restrict__ partial, int nchunks, int q,
                                  double* __restrict__ A1, double* __restrict__ A2) {
    const int64_t qq = (int64_t)q * q;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= qq) return;
    const int a = (int)(idx / q), b = (int)(idx % q);
    double x_ab = 0, x_ba = 0, y_ab = 0, y_ba = 0;
    for (int c = 0; c < nchunks; ++c) {
        const double* px = partial + (int64_t)c * 2 * qq;
        x_ab += px[(int64_t)a * q + b];
        x_ba += px[(int64_t)b * q + a];
        y_ab += px[qq + (int64_t)a * q + b];
        y_ba += px[qq + (int64_t)b * q + a];
    }
    A1[idx] = 0.5 * (x_ab - x_ba);
    A2[idx] = 0.5 * (y_ab + y_ba);
}

int gram_skew(Session* s, const double* Z, int64_t ldz, const double* V1, int64_t ldv1, const double* V2,
              int64_t ldv2, int64_t n, int q, double* A1, double* A2, cudaStream_t st) {
    if (q <= 0) return 0;
    const int tiles = ceil_div(q, 32);
    int nch = (int)std::max<int64_t>(1, std::min<int64_t>((n + 127) / 128, ceil_div(1216, tiles * tiles)));
    const int64_t rpc = (n + nch - 1) / nch;
    nch = (int)((n + rpc - 1) / rpc);
    HBSD_TRY(s->ws.alloc((size_t)nch * 2 * q * q + 64));
    Seg2<double> A{Z, ldz, q, nullptr, 0}, B1{V1, ldv1, q, nullptr, 0}, B2{V2, ldv2, q, nullptr, 0};
    dim3 grid(tiles * tiles, nch);
    k_gram_partial<double><<<grid, 256, 0, st>>>(A, B1, B2, q, n, rpc, tiles, s->ws.p);
    HBSD_LAUNCHED(s);
    const int64_t qq = (int64_t)q * q;
    k_gram_final_skew<<<ceil_div(qq, 256), 256, 0, st>>>(s->ws.p, nch, q, A1, A2);
    HBSD_LAUNCHED(s);
    return 0;
}

// ---- allocation-free Gram ---------------------------------------------------------------
// Scratch for hbsd_gram_noalloc: a file-scope device array, so the call needs no cudaMalloc.
// Every device that loads the library holds it (16 MiB) until the process exits.
constexpr size_t GRAM_STATIC_DOUBLES = size_t(1) << 21;
static __device__ __align__(256) double g_gram_static[GRAM_STATIC_DOUBLES];

// Device address of g_gram_static on the current device, looked up once per device.  In host
// code the symbol names a host-side stand-in, not device memory, so kernels must be given this
// address instead.  The cached address belongs to the device's primary context: after a
// cudaDeviceReset the module may load elsewhere, so the library must not be used across a reset.
static int gram_static_address(double** out) {
    static std::mutex mu;
    static double* addr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HBSD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return fail(HBSD_ERR_ARG, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_gram_static);
        if (e != cudaSuccess)
            return fail(HBSD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        addr[dev] = static_cast<double*>(p);
    }
    *out = addr[dev];
    return 0;
}

int gram_noalloc(const double* Z, int64_t ldz, const double* ZH, int64_t ldzh, const double* ZS, int64_t ldzs,
                 int64_t n, int q, double* HR, double* SR, cudaStream_t st) {
    if (q <= 0 || n <= 0) return fail(HBSD_ERR_ARG, "gram_noalloc: need n > 0 and q > 0");
    const size_t per_chunk = (size_t)2 * q * q;
    if (q > GRAM_NOALLOC_MAX_Q || per_chunk > GRAM_STATIC_DOUBLES)
        return fail(HBSD_ERR_ARG, "gram_noalloc: q = " + std::to_string(q) +
                                      " exceeds the static scratch (2 q^2 <= 2^21 doubles, q <= 1024)");
    double* scratch = nullptr;
    HBSD_TRY(gram_static_address(&scratch));
    const int tiles = ceil_div(q, 32);
    int nch = (int)std::max<int64_t>(1, std::min<int64_t>((n + 127) / 128, ceil_div(1216, tiles * tiles)));
    nch = (int)std::min<size_t>((size_t)nch, GRAM_STATIC_DOUBLES / per_chunk);
    const int64_t rpc = (n + nch - 1) / nch;
    nch = (int)((n + rpc - 1) / rpc);
    // every partial element read by k_gram_final is written by k_gram_partial: nothing to clear
    Seg2<double> A{Z, ldz, q, nullptr, 0}, AH{ZH, ldzh, q, nullptr, 0}, AS{ZS, ldzs, q, nullptr, 0};
    dim3 grid(tiles * tiles, nch);
    k_gram_partial<double><<<grid, 256, 0, st>>>(A, AH, AS, q, n, rpc, tiles, scratch);
    HBSD_LAUNCHED(nullptr);
    const int64_t qq = (int64_t)q * q;
    k_gram_final<<<ceil_div(qq, 256), 256, 0, st>>>(scratch, nch, q, HR, SR);
    HBSD_LAUNCHED(nullptr);
    return 0;
}

// ---- update (steps 10-11) ------------------------------------------------------------------
// 16 rows per CTA staged in shared memory; thread (jc, rg): column j = jc + 64*jb, rows 4*rg..4*rg+3
template <class T>
__global__ void __launch_bounds__(256) k_update(T* __restrict__ Z0, int64_t ld0, int q0,
                                                const T* __restrict__ Z1, int64_t ld1, int q1,
                                                int64_t n, const double* __restrict__ W, int k) {
    extern __shared__ __align__(16) unsigned char zraw[];
    T* zrow = reinterpret_cast<T*>(zraw);  // [16][q]
    const int q = q0 + q1;
    const int64_t i0 = (int64_t)blockIdx.x * 16;
    for (int t = threadIdx.x; t < 16 * q; t += 256) {
        const int rr = t / q, c = t % q;
        const int64_t i = i0 + rr;
        T v = T(0);
        if (i < n) v = c < q0 ? Z0[i * ld0 + c] : Z1[i * ld1 + (c - q0)];
        zrow[rr * q + c] = v;
    }
    __syncthreads();
    const int jc = threadIdx.x & 63, rg = threadIdx.x >> 6;
    for (int jb = 0; jb * 64 < k; ++jb) {
        const int j = jb * 64 + jc;
        if (j >= k) continue;
        T acc[4] = {0, 0, 0, 0};
        for (int c = 0; c < q; ++c) {
            const T wv = (T)__ldg(W + (int64_t)c * k + j);
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fma(zrow[(rg * 4 + u) * q + c], wv, acc[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t i = i0 + rg * 4 + u;
            if (i < n) Z0[i * ld0 + j] = acc[u];
        }
    }
}

template <class T>
int update2(Session* s, T* Z0, int64_t ld0, int q0, const T* Z1, int64_t ld1, int q1,
            int64_t n, const double* W, int k, cudaStream_t st) {
    const int q = q0 + q1;
    if (k > q0) return fail(HBSD_ERR_ARG, "update: k must not exceed the first segment width");
    const size_t smem = (size_t)16 * q * sizeof(T);
    if (smem > 200 * 1024) return fail(HBSD_ERR_ARG, "update: q too large");
    if (smem > 48 * 1024) {   // the cap, once: concurrent sessions never lower it under each other
        static std::once_flag once;
        static cudaError_t e = cudaSuccess;
        std::call_once(once, [] {
            e = cudaFuncSetAttribute(k_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        });
        HBSD_CUDA(e);
    }
    k_update<T><<<ceil_div(n, 16), 256, smem, st>>>(Z0, ld0, q0, Z1, ld1, q1, n, W, k);
    HBSD_LAUNCHED(s);
    return 0;
}
template int update2<double>(Session*, double*, int64_t, int, const double*, int64_t, int, int64_t, const double*, int,
                             cudaStream_t);
template int update2<float>(Session*, float*, int64_t, int, const float*, int64_t, int, int64_t, const double*, int,
                            cudaStream_t);

// ---- Rayleigh-Ritz (step 9), one CTA, FP64 ------------------------------------------------
constexpr int RR_THREADS = 512;
constexpr double RR_PIVOT_MIN = 1e-14;

__device__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        red[32] = s;
    }
    __syncthreads();
    return red[32];
}

// Householder reduction of the symmetric nn x nn matrix A (row-major, ld lda) to tridiagonal
// (d, e), followed by accumulation of Q = H_0 H_1 ... H_{nn-3} into Q (ld lda).
__device__ void tridiagonalize(double* A, int nn, int lda, double* Q, double* d, double* e,
                               double* tau, double* pv, double* red) {
    for (int kk = 0; kk + 2 < nn; ++kk) {
        double s2 = 0.0;
        for (int i = kk + 1 + threadIdx.x; i < nn; i += blockDim.x) s2 += A[(int64_t)i * lda + kk] * A[(int64_t)i * lda + kk];
        s2 = block_sum(s2, red);
        const double x0 = A[(int64_t)(kk + 1) * lda + kk];
        const double tail = s2 - x0 * x0;
        if (threadIdx.x == 0) d[kk] = A[(int64_t)kk * lda + kk];
        if (tail <= 0.0 || s2 == 0.0) {
            if (threadIdx.x == 0) { e[kk] = x0; tau[kk] = 0.0; }
            for (int i = kk + 1 + threadIdx.x; i < nn; i += blockDim.x) A[(int64_t)i * lda + kk] = 0.0;
            __syncthreads();
            continue;
        }
        const double alpha = -copysign(sqrt(s2), x0);
        const double v0 = x0 - alpha;
        const double vtv = tail + v0 * v0;
        const double t = 2.0 / vtv;
        __syncthreads();
        if (threadIdx.x == 0) { e[kk] = alpha; tau[kk] = t; A[(int64_t)(kk + 1) * lda + kk] = v0; }
        __syncthreads();
        // p = t * A22 v
        for (int i = kk + 1 + threadIdx.x; i < nn; i += blockDim.x) {
            double acc = 0.0;
            for (int j = kk + 1; j < nn; ++j) acc += A[(int64_t)i * lda + j] * A[(int64_t)j * lda + kk];
            pv[i] = t * acc;
        }
        __syncthreads();
        double pvv = 0.0;
        for (int i = kk + 1 + threadIdx.x; i < nn; i += blockDim.x) pvv += pv[i] * A[(int64_t)i * lda + kk];
        pvv = block_sum(pvv, red);
        const double K = 0.5 * t * pvv;
        for (int i = kk + 1 + threadIdx.x; i < nn; i += blockDim.x) pv[i] -= K * A[(int64_t)i * lda + kk];
        __syncthreads();
        // A22 -= v w^T + w v^T
        const int m = nn - kk - 1;
        for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
            const int i = kk + 1 + idx / m, j = kk + 1 + idx % m;
            A[(int64_t)i * lda + j] -= A[(int64_t)i * lda + kk] * pv[j] + pv[i] * A[(int64_t)j * lda + kk];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (nn >= 2) {
            d[nn - 2] = A[(int64_t)(nn - 2) * lda + nn - 2];
            e[nn - 2] = A[(int64_t)(nn - 1) * lda + nn - 2];
        }
        d[nn - 1] = A[(int64_t)(nn - 1) * lda + nn - 1];
        e[nn - 1] = 0.0;
    }
    // Q = I, then Q <- H_kk Q for kk = nn-3 .. 0 (each H_kk acts on rows/cols > kk)
    for (int idx = threadIdx.x; idx < nn * nn; idx += blockDim.x)
        Q[(int64_t)(idx / nn) * lda + idx % nn] = (idx / nn == idx % nn) ? 1.0 : 0.0;
    __syncthreads();
    for (int kk = nn - 3; kk >= 0; --kk) {
        const double t = tau[kk];
        if (t == 0.0) continue;
        // u_j = sum_i v_i Q_ij  (i, j > kk)
        for (int j = kk + 1 + threadIdx.x; j < nn; j += blockDim.x) {
            double acc = 0.0;
            for (int i = kk + 1; i < nn; ++i) acc += A[(int64_t)i * lda + kk] * Q[(int64_t)i * lda + j];
            pv[j] = acc;
        }
        __syncthreads();
        const int m = nn - kk - 1;
        for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
            const int i = kk + 1 + idx / m, j = kk + 1 + idx % m;
            Q[(int64_t)i * lda + j] -= t * A[(int64_t)i * lda + kk] * pv[j];
        }
        __syncthreads();
    }
}

// Implicit QL with a Wilkinson-type shift on the tridiagonal (d, e) (e[i] couples i and i+1);
// the rotations of each sweep are generated by thread 0 and applied by all threads, one row of
// Q each, in generation order.  Returns false if an eigenvalue needed more than 60 sweeps.
__device__ bool tridiagonal_ql(double* d, double* e, int nn, double* Q, int lda, double* rc,
                               double* rs, int* ri, int* ctl) {
    constexpr int DONE = -2, FAILED = -1;
    for (int l = 0; l < nn; ++l) {
        for (int iter = 0;; ++iter) {
            if (threadIdx.x == 0) {
                int m = l;
                while (m < nn - 1) {
                    const double dd = fabs(d[m]) + fabs(d[m + 1]);
                    if (fabs(e[m]) <= DBL_EPSILON * dd) break;
                    ++m;
                }
                if (m == l) {
                    ctl[0] = DONE;
                } else if (iter >= 60) {
                    ctl[0] = FAILED;
                } else {
                    double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
                    double r = hypot(g, 1.0);
                    g = d[m] - d[l] + e[l] / (g + copysign(r, g));
                    double s = 1.0, c = 1.0, p = 0.0;
                    bool early = false;
                    int nrot = 0;
                    for (int i = m - 1; i >= l; --i) {
                        const double f = s * e[i];
                        const double b = c * e[i];
                        r = hypot(f, g);
                        e[i + 1] = r;
                        if (r == 0.0) {  // deflation inside the sweep
                            d[i + 1] -= p;
                            e[m] = 0.0;
                            early = true;
                            break;
                        }
                        s = f / r;
                        c = g / r;
                        g = d[i + 1] - p;
                        r = (d[i] - g) * s + 2.0 * c * b;
                        p = s * r;
                        d[i + 1] = g + p;
                        g = c * r - b;
                        rc[nrot] = c;
                        rs[nrot] = s;
                        ri[nrot] = i;
                        ++nrot;
                    }
                    if (!early) {
                        d[l] -= p;
                        e[l] = g;
                        e[m] = 0.0;
                    }
                    ctl[0] = nrot;
                }
            }
            __syncthreads();
            const int nrot = ctl[0];
            __syncthreads();
            if (nrot == DONE) break;
            if (nrot == FAILED) return false;
            for (int row = threadIdx.x; row < nn; row += blockDim.x) {
                double* qr = Q + (int64_t)row * lda;
                for (int t = 0; t < nrot; ++t) {
                    const int i = ri[t];
                    const double f = qr[i + 1];
                    qr[i + 1] = rs[t] * qr[i] + rc[t] * f;
                    qr[i] = rc[t] * qr[i] - rs[t] * f;
                }
            }
            __syncthreads();
        }
    }
    return true;
}

// order[0..nn) = indices of d ascending (stable)
__device__ void sort_ascending(const double* d, int nn, int* order) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < nn; ++i) order[i] = i;
        for (int i = 1; i < nn; ++i) {
            const int v = order[i];
            int j = i - 1;
            while (j >= 0 && d[order[j]] > d[v]) { order[j + 1] = order[j]; --j; }
            order[j + 1] = v;
        }
    }
    __syncthreads();
}

// Full symmetric eigendecomposition of the nn x nn matrix A (destroyed): eigenvalues in d,
// eigenvectors in the columns of Q (unsorted).
__device__ bool sym_eig(double* A, int nn, int lda, double* Q, double* d, double* e, double* tau,
                        double* pv, double* red, double* rc, double* rs, int* ri, int* ctl) {
    if (nn == 1) {
        if (threadIdx.x == 0) { d[0] = A[0]; Q[0] = 1.0; }
        __syncthreads();
        return true;
    }
    tridiagonalize(A, nn, lda, Q, d, e, tau, pv, red);
    __syncthreads();
    return tridiagonal_ql(d, e, nn, Q, lda, rc, rs, ri, ctl);
}

// workspace: 4*q*q + 4*q doubles; shared: 4 q-vectors + ints
__global__ void __launch_bounds__(RR_THREADS) k_rayleigh_ritz(const double* __restrict__ HR,
                                                              const double* __restrict__ SR, int q,
                                                              int k, double* __restrict__ theta,
                                                              double* __restrict__ W,
                                                              double* __restrict__ ws,
                                                              int* __restrict__ info) {
    extern __shared__ double sh[];
    double* d = sh;                 // q
    double* e = d + q;              // q
    double* tau = e + q;            // q
    double* rc = tau + q;           // q
    double* rs = rc + q;            // q
    double* red = rs + q;           // 40
    int* ri = (int*)(red + 40);     // q
    int* order = ri + q;            // q
    int* ctl = order + q;           // 4
    const int64_t qq = (int64_t)q * q;
    double* A = ws;                 // scaled H_R, then C
    double* B = A + qq;             // scaled S_R, then L
    double* Q = B + qq;             // eigenvectors
    double* T = Q + qq;             // scratch
    double* dvec = T + qq;          // q
    double* pv = dvec + q;          // q
    for (int i = threadIdx.x; i < q; i += blockDim.x) dvec[i] = 1.0 / sqrt(SR[(int64_t)i * q + i]);
    __syncthreads();
    for (int64_t idx = threadIdx.x; idx < qq; idx += blockDim.x) {
        const int i = (int)(idx / q), j = (int)(idx % q);
        A[idx] = HR[idx] * dvec[i] * dvec[j];
        B[idx] = SR[idx] * dvec[i] * dvec[j];
    }
    if (threadIdx.x == 0) { ctl[3] = 0; info[0] = 0; info[1] = q; info[2] = 0; }
    __syncthreads();
    // Cholesky D S_R D = L L^T (lower, in B); a pivot below RR_PIVOT_MIN (or NaN) -> fallback
    for (int kk = 0; kk < q; ++kk) {
        if (threadIdx.x == 0) {
            const double piv = B[(int64_t)kk * q + kk];
            if (!(piv >= RR_PIVOT_MIN)) ctl[3] = 1;
            else B[(int64_t)kk * q + kk] = sqrt(piv);
        }
        __syncthreads();
        if (ctl[3]) break;
        const double lkk = B[(int64_t)kk * q + kk];
        for (int i = kk + 1 + threadIdx.x; i < q; i += blockDim.x) B[(int64_t)i * q + kk] /= lkk;
        __syncthreads();
        const int m = q - kk - 1;
        for (int64_t idx = threadIdx.x; idx < (int64_t)m * m; idx += blockDim.x) {
            const int i = kk + 1 + (int)(idx / m), j = kk + 1 + (int)(idx % m);
            if (j <= i) B[(int64_t)i * q + j] -= B[(int64_t)i * q + kk] * B[(int64_t)j * q + kk];
        }
        __syncthreads();
    }
    const bool fallback = ctl[3] != 0;
    if (!fallback) {
        // T = L^{-1} A (column-parallel forward substitution)
        for (int j = threadIdx.x; j < q; j += blockDim.x) {
            for (int i = 0; i < q; ++i) {
                double acc = A[(int64_t)i * q + j];
                for (int l = 0; l < i; ++l) acc -= B[(int64_t)i * q + l] * T[(int64_t)l * q + j];
                T[(int64_t)i * q + j] = acc / B[(int64_t)i * q + i];
            }
        }
        __syncthreads();
        // C = L^{-1} T^T  -> into A
        for (int j = threadIdx.x; j < q; j += blockDim.x) {
            for (int i = 0; i < q; ++i) {
                double acc = T[(int64_t)j * q + i];
                for (int l = 0; l < i; ++l) acc -= B[(int64_t)i * q + l] * A[(int64_t)l * q + j];
                A[(int64_t)i * q + j] = acc / B[(int64_t)i * q + i];
            }
        }
        __syncthreads();
        for (int64_t idx = threadIdx.x; idx < qq; idx += blockDim.x) {
            const int i = (int)(idx / q), j = (int)(idx % q);
            if (j > i) {
                const double v = 0.5 * (A[(int64_t)i * q + j] + A[(int64_t)j * q + i]);
                A[(int64_t)i * q + j] = v;
                A[(int64_t)j * q + i] = v;
            }
        }
        __syncthreads();
        if (!sym_eig(A, q, q, Q, d, e, tau, pv, red, rc, rs, ri, ctl)) {
            if (threadIdx.x == 0) info[2] = 1;
            return;
        }
        sort_ascending(d, q, order);
        for (int j = threadIdx.x; j < k; j += blockDim.x) theta[j] = d[order[j]];
        // W(:, j) = D L^{-T} V(:, order[j])
        for (int j = threadIdx.x; j < k; j += blockDim.x) {
            const int src = order[j];
            for (int i = q - 1; i >= 0; --i) {
                double acc = Q[(int64_t)i * q + src];
                for (int l = i + 1; l < q; ++l) acc -= B[(int64_t)l * q + i] * T[(int64_t)l * q + j];
                T[(int64_t)i * q + j] = acc / B[(int64_t)i * q + i];
            }
        }
        __syncthreads();
        for (int64_t idx = threadIdx.x; idx < (int64_t)q * k; idx += blockDim.x) {
            const int i = (int)(idx / k), j = (int)(idx % k);
            W[idx] = dvec[i] * T[(int64_t)i * q + j];
        }
        return;
    }
    // ---- rank-revealing fallback: eigen-directions of D S_R D above RR_PIVOT_MIN * max ----
    if (threadIdx.x == 0) info[0] = 1;
    for (int64_t idx = threadIdx.x; idx < qq; idx += blockDim.x) {
        const int i = (int)(idx / q), j = (int)(idx % q);
        B[idx] = SR[idx] * dvec[i] * dvec[j];
    }
    __syncthreads();
    if (!sym_eig(B, q, q, Q, d, e, tau, pv, red, rc, rs, ri, ctl)) {
        if (threadIdx.x == 0) info[2] = 1;
        return;
    }
    sort_ascending(d, q, order);
    // kept directions: mu > RR_PIVOT_MIN * mu_max, in ascending order of mu
    if (threadIdx.x == 0) {
        const double mu_max = d[order[q - 1]];
        int r = 0;
        for (int t = 0; t < q; ++t)
            if (d[order[t]] > RR_PIVOT_MIN * mu_max) order[r++] = order[t];
        ctl[0] = r;
        info[1] = r;
    }
    __syncthreads();
    const int r = ctl[0];
    if (r < k) return;
    // Bm(:, t) = Q(:, order[t]) / sqrt(mu) -> stored in B (q x r, ld q)
    for (int64_t idx = threadIdx.x; idx < (int64_t)q * r; idx += blockDim.x) {
        const int i = (int)(idx / r), t = (int)(idx % r);
        B[(int64_t)i * q + t] = Q[(int64_t)i * q + order[t]] / sqrt(d[order[t]]);
    }
    __syncthreads();
    // T = Hd Bm (q x r), Hd = A (scaled H_R)
    for (int64_t idx = threadIdx.x; idx < (int64_t)q * r; idx += blockDim.x) {
        const int i = (int)(idx / r), t = (int)(idx % r);
        double acc = 0.0;
        for (int l = 0; l < q; ++l) acc += A[(int64_t)i * q + l] * B[(int64_t)l * q + t];
        T[(int64_t)i * q + t] = acc;
    }
    __syncthreads();
    // C = Bm^T T (r x r) -> A (ld q), symmetrised
    for (int64_t idx = threadIdx.x; idx < (int64_t)r * r; idx += blockDim.x) {
        const int a = (int)(idx / r), b = (int)(idx % r);
        double acc = 0.0;
        for (int l = 0; l < q; ++l) acc += B[(int64_t)l * q + a] * T[(int64_t)l * q + b];
        Q[(int64_t)a * q + b] = acc;
    }
    __syncthreads();
    for (int64_t idx = threadIdx.x; idx < (int64_t)r * r; idx += blockDim.x) {
        const int a = (int)(idx / r), b = (int)(idx % r);
        A[(int64_t)a * q + b] = 0.5 * (Q[(int64_t)a * q + b] + Q[(int64_t)b * q + a]);
    }
    __syncthreads();
    if (!sym_eig(A, r, q, Q, d, e, tau, pv, red, rc, rs, ri, ctl)) {
        if (threadIdx.x == 0) info[2] = 1;
        return;
    }
    sort_ascending(d, r, order);
    for (int j = threadIdx.x; j < k; j += blockDim.x) theta[j] = d[order[j]];
    __syncthreads();
    // W = D Bm V(:, order[:k])
    for (int64_t idx = threadIdx.x; idx < (int64_t)q * k; idx += blockDim.x) {
        const int i = (int)(idx / k), j = (int)(idx % k);
        double acc = 0.0;
        for (int t = 0; t < r; ++t) acc += B[(int64_t)i * q + t] * Q[(int64_t)t * q + order[j]];
        W[idx] = dvec[i] * acc;
    }
}

int rayleigh_ritz(Session* s, const double* HR, const double* SR, int q, int k, double* theta,
                  double* W, int* info_host, cudaStream_t st) {
    if (q <= 0 || k <= 0 || k > q) return fail(HBSD_ERR_ARG, "rayleigh_ritz: need 0 < k <= q");
    HBSD_TRY(s->rr_ws.alloc((size_t)4 * q * q + 3 * q + 64));
    HBSD_TRY(s->rr_info.alloc(4));
    const size_t smem = (size_t)(5 * q + 40) * sizeof(double) + (size_t)(2 * q + 4) * sizeof(int);
    if (smem > 200 * 1024) return fail(HBSD_ERR_ARG, "rayleigh_ritz: q too large");
    if (smem > 48 * 1024) {   // the cap, once (see update2)
        static std::once_flag once;
        static cudaError_t e = cudaSuccess;
        std::call_once(once, [] {
            e = cudaFuncSetAttribute(k_rayleigh_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        });
        HBSD_CUDA(e);
    }
    k_rayleigh_ritz<<<1, RR_THREADS, smem, st>>>(HR, SR, q, k, theta, W, s->rr_ws.p, s->rr_info.p);
    HBSD_LAUNCHED(s);
    int info[4] = {0, 0, 0, 0};
    HBSD_CUDA(cudaMemcpyAsync(info, s->rr_info.p, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
    HBSD_CUDA(cudaStreamSynchronize(st));
    if (info_host) { info_host[0] = info[0]; info_host[1] = info[1]; }
    if (info[2]) return fail(HBSD_ERR_RR_RANK, "rayleigh_ritz: QL iteration did not converge");
    if (info[1] < k) return fail(HBSD_ERR_RR_RANK, "rayleigh_ritz: search space rank below k");
    return 0;
}

}  // namespace hbsd
