// FP64-accurate block update Y = [Z0 Z1] W (steps 10-11) on the bf16 tensor cores, by exact
// slices (the splitting idea of Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication", Numer. Algorithms 59, 2012).
//
// Every row of a segment Z_g (g = 0: Psi, q0 columns; g = 1: P, q1 columns) is written in fixed
// point against its largest entry, |z| < 2^E: z / 2^E = 2^-6 sum_s A_s with A_s = +-d_s 2^(-6 s),
// d_s in [0, 63] the s-th 6-bit digit of the truncated 48-bit magnitude (s = 0..7).  Every column of
// W_g likewise against its own largest entry.  Each A_s and B_t is exact in bf16, each product
// d_s d_t < 2^12 is exact, and the L + 1 products of one level L = s + t summed over q <= 640 terms
// stay below 2^24 in units of 2^(-6 L) for L <= 5, so a tensor-core FP32 accumulator that holds one
// such level only is exact.  Levels 0-5 get one accumulator each; levels 6-8 share one (2^-36 below
// the leading level, so its FP32 rounding stays near 2^-55 of it); levels >= 9 are dropped (each of
// their terms is below 2^-49 times the product of the row and column scales, under the 2^-47 of the
// operands' truncation).  The segments run one after the other on the same accumulators with
// their own row scales, so a row whose P entries are far larger than its Psi entries (directions
// K r carry large components along the near-null space of S) loses nothing on its Psi part.  After
// each segment the epilogue adds its levels 0-5 in integer arithmetic (exact multiples of 2^-30
// of the leading unit), then the shared accumulator of levels 6-8 and the scales in FP64.
#include <algorithm>
#include <mutex>
#include <string>

#include "common.h"
#include "tc.h"

namespace hbsd {
namespace {

constexpr int OZ_N = 64;                        // output columns per CTA (N of every MMA)
constexpr int OZ_DIG = 8;                       // 6-bit digits per operand
constexpr int OZ_ACC = 7;                       // accumulators: levels 0..5 exact, 6..8 shared
constexpr int OZ_LMAX = 8;                      // highest level kept (pairs of digits a + b <= 8)
constexpr int OZ_SLICERS = 256;                 // warps 0-7: slicing and epilogue
constexpr int OZ_THREADS = OZ_SLICERS + 32;     // warp 8: MMA issue
constexpr int OZ_NS = 3;                        // stage buffers
constexpr int OZ_A_SLICE = 128 * 16 * 2;        // bytes of one 128 x 16 bf16 slice tile
constexpr int OZ_B_SLICE = OZ_N * 16 * 2;       // bytes of one OZ_N x 16 bf16 slice tile
constexpr int OZ_STAGE = OZ_DIG * (OZ_A_SLICE + OZ_B_SLICE);
constexpr uint32_t OZ_TMEM_COLS = 512;          // 7 accumulators, one per 64 columns
constexpr int OZ_ACC_STRIDE = 64;               // TMEM column stride between accumulators
constexpr uint64_t OZ_WAIT_NS = 2000000000ull;
constexpr int OZ_MAX_Q = OZ_MAX_Q_SEG;          // per segment: keeps the level-5 sums below 2^24

struct OzSeg {
    const double* Z;        // n x q, ld
    int64_t ld;
    int q;
    int qpad;               // q rounded up to 16
    const uint16_t* B;      // bf16 slices of W_g: [OZ_DIG][kpad][qpad], row j = output column j
    const int* rowexp;      // exponent field of the largest |Z_g(i, :)| (0: the row is zero)
    const int* colexp;      // exponent field of the largest |W_g(:, j)|
};

__device__ __forceinline__ int exp_field(double x) {
    return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF);
}

// 48-bit truncated magnitude of |x| / 2^(E) in units of 2^-48, E from the exponent field emax of the
// largest entry (|x| < 2^(emax - 1022)); sign in *neg
__device__ __forceinline__ unsigned long long fixed48(double x, int emax, bool* neg) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    *neg = (b >> 63) != 0;
    const int ex = (int)((b >> 52) & 0x7FF);
    if (ex == 0 && (b & 0xFFFFFFFFFFFFFull) == 0) return 0ull;
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (ex ? (1ull << 52) : 0ull);
    const int sh = 5 + emax - (ex ? ex : 1);
    return sh >= 64 ? 0ull : (m >> sh);
}

// bf16 bits of +-d 2^(-6 s) (exact: d < 64)
__device__ __forceinline__ uint32_t digit_bf16(unsigned long long F, int s, bool neg) {
    const uint32_t d = (uint32_t)(F >> (42 - 6 * s)) & 63u;
    const float v = (float)d * __uint_as_float((uint32_t)(127 - 6 * s) << 23);
    return (__float_as_uint(v) >> 16) | (neg && d ? 0x8000u : 0u);
}

// bf16 bits of the 8 digits of x (without integer-to-float conversions: d | 0x4B000000 read as a
// float is 2^23 + d exactly)
__device__ __forceinline__ void digits8(double x, int emax, uint32_t (&bits)[OZ_DIG]) {
    bool neg;
    const unsigned long long F = fixed48(x, emax, &neg);
    const uint32_t hi = (uint32_t)(F >> 24), lo = (uint32_t)F & 0xFFFFFFu;
    const uint32_t sgn = neg ? 0x8000u : 0u;
#pragma unroll
    for (int s = 0; s < OZ_DIG; ++s) {
        const uint32_t d = (s < 4 ? (hi >> (18 - 6 * s)) : (lo >> (18 - 6 * (s - 4)))) & 63u;
        const float f = (__uint_as_float(0x4B000000u | d) - 8388608.0f) * __uint_as_float((uint32_t)(127 - 6 * s) << 23);
        bits[s] = (__float_as_uint(f) >> 16) | (d ? sgn : 0u);
    }
}

// rowexp[i] = exponent field of max_k |Z(i, k)|
__global__ void k_oz_rowexp(const double* __restrict__ Z, int64_t ld, int q, int64_t n, int* __restrict__ rowexp) {
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (i >= n) return;
    int e = 0;
    for (int k = threadIdx.x & 31; k < q; k += 32) e = max(e, exp_field(Z[i * ld + k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if ((threadIdx.x & 31) == 0) rowexp[i] = e;
}

// colexp[j] over rows [r0, r0 + q) of W (q x k, row-major, ld k); B slices of those rows
__global__ void k_oz_wslices(const double* __restrict__ W, int k, int r0, int q, int qpad, int kpad,
                             int* __restrict__ colexp, uint16_t* __restrict__ B) {
    const int j = blockIdx.x;
    __shared__ int se[32];
    int e = 0;
    if (j < k)
        for (int r = threadIdx.x; r < q; r += blockDim.x) e = max(e, exp_field(W[(int64_t)(r0 + r) * k + j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if ((threadIdx.x & 31) == 0) se[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        int m = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, se[w]);
        se[0] = m;
        colexp[j] = m;
    }
    __syncthreads();
    const int emax = se[0];
    for (int r = threadIdx.x; r < qpad; r += blockDim.x) {
        bool neg = false;
        const unsigned long long F = (j < k && r < q) ? fixed48(W[(int64_t)(r0 + r) * k + j], emax, &neg) : 0ull;
#pragma unroll
        for (int s = 0; s < OZ_DIG; ++s)
            B[((int64_t)s * kpad + j) * qpad + r] = (uint16_t)digit_bf16(F, s, neg);
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(tc::smem_u32(mbar)) : "memory");
}

// Warp roles: warps 0-7 (OZ_SLICERS threads) slice Z into the stage buffers, load the W slices and
// run the epilogue; warp 8 issues the MMAs (lane 0).  Stages cycle through OZ_NS buffers: full[s]
// completes when the slicers have filled stage s, empty[s] when the MMAs that read it are done.
// segdone completes when a segment's MMAs are done; accfree when the slicers have read its
// accumulators, before the next segment overwrites them.
__global__ void __launch_bounds__(OZ_THREADS, 1) k_update_oz(OzSeg s0, OzSeg s1, int64_t n, int k, int kpad,
                                                              double* __restrict__ Y, int64_t ldy,
                                                              int* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t oz_smem[];
    __shared__ __align__(8) uint64_t full[OZ_NS], empty[OZ_NS], segdone, accfree;
    __shared__ uint32_t tslot;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t row0 = (int64_t)blockIdx.x * 128;
    const int j0 = blockIdx.y * OZ_N;
    uint8_t* base = oz_smem + ((1024 - (tc::smem_u32(oz_smem) & 1023)) & 1023);   // 1 KB aligned
    if (tid == 0) {
        for (int i = 0; i < OZ_NS; ++i) {
            tc::mbar_init(&full[i], OZ_SLICERS);
            tc::mbar_init(&empty[i], 1);
        }
        tc::mbar_init(&segdone, 1);
        tc::mbar_init(&accfree, OZ_SLICERS);
        s_fail = 0;
    }
    if (warp == 0) tc::tmem_alloc(&tslot, OZ_TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tslot;
    const int n0 = (s0.q + 15) / 16, n1 = (s1.q + 15) / 16, total = n0 + n1;

    if (warp == OZ_SLICERS / 32) {   // ---- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16_f32(128, OZ_N);
            uint32_t init_mask = 0;
            for (int t = 0; t < total; ++t) {
                const int st = t % OZ_NS;
                if (t == n0) {   // the slicers have read segment 0's accumulators
                    if (!tc::mbar_wait(&accfree, 0u, OZ_WAIT_NS)) { s_fail = 1; break; }
                    init_mask = 0;
                }
                if (!tc::mbar_wait(&full[st], (uint32_t)((t / OZ_NS) & 1), OZ_WAIT_NS)) { s_fail = 1; break; }
                tc::fence_after_sync();
                uint8_t* stA = base + st * OZ_STAGE;
                uint8_t* stB = stA + OZ_DIG * OZ_A_SLICE;
#pragma unroll 1
                for (int a = 0; a < OZ_DIG; ++a) {
                    const uint64_t ad = tc::smem_desc(tc::smem_u32(stA + a * OZ_A_SLICE), 128, 256);
#pragma unroll 1
                    for (int b = 0; b < OZ_DIG && a + b <= OZ_LMAX; ++b) {
                        const int acc = min(a + b, OZ_ACC - 1);
                        const uint64_t bd = tc::smem_desc(tc::smem_u32(stB + b * OZ_B_SLICE), 128, 256);
                        tc::mma_bf16(tbase + (uint32_t)(acc * OZ_ACC_STRIDE), ad, bd, idesc, (init_mask >> acc) & 1u);
                        init_mask |= 1u << acc;
                    }
                }
                tc::mma_commit(&empty[st]);
                if (t == n0 - 1 || t == total - 1) tc::mma_commit(&segdone);
            }
        }
    } else {   // ---- slicers and epilogue
        const int arow = tid >> 1, ahalf = tid & 1;
        const int64_t agrow = row0 + arow;
        const int er = (warp & 3) * 32 + lane, ch = warp >> 2;   // epilogue: row, column half (32 columns)
        const int64_t egrow = row0 + er;
        const uint32_t lane_addr = tbase + ((uint32_t)((warp & 3) * 32) << 16);
        double y[32];
#pragma unroll
        for (int v = 0; v < 32; ++v) y[v] = 0.0;
        int segs = 0;
        for (int t = 0; t < total; ++t) {
            const int st = t % OZ_NS;
            const int g = t < n0 ? 0 : 1;
            const OzSeg& sg = g ? s1 : s0;
            const int kk = (g ? t - n0 : t) * 16;
            uint8_t* stA = base + st * OZ_STAGE;
            uint8_t* stB = stA + OZ_DIG * OZ_A_SLICE;
            if (t >= OZ_NS && !tc::mbar_wait(&empty[st], (uint32_t)((t / OZ_NS - 1) & 1), OZ_WAIT_NS)) {
                s_fail = 1;
                break;
            }
            {   // A slices: the 8 digits of the thread's 8 entries of its row
                const int emax_a = agrow < n ? sg.rowexp[agrow] : 0;
                double x[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int col = kk + ahalf * 8 + c;
                    x[c] = (agrow < n && col < sg.q) ? sg.Z[agrow * sg.ld + col] : 0.0;
                }
                uint32_t packed[OZ_DIG][4];
#pragma unroll
                for (int c = 0; c < 8; c += 2) {
                    uint32_t b0[OZ_DIG], b1[OZ_DIG];
                    digits8(x[c], emax_a, b0);
                    digits8(x[c + 1], emax_a, b1);
#pragma unroll
                    for (int d = 0; d < OZ_DIG; ++d) packed[d][c >> 1] = b0[d] | (b1[d] << 16);
                }
                const uint32_t off = (uint32_t)(ahalf * 128 + (arow >> 3) * 256 + (arow & 7) * 16);
#pragma unroll
                for (int d = 0; d < OZ_DIG; ++d)
                    *reinterpret_cast<uint4*>(stA + d * OZ_A_SLICE + off) =
                        make_uint4(packed[d][0], packed[d][1], packed[d][2], packed[d][3]);
            }
#pragma unroll
            for (int i = 0; i < OZ_DIG * OZ_N * 2 / OZ_SLICERS; ++i) {   // B slices: 16-byte halves of rows
                const int e = tid + OZ_SLICERS * i;
                const int d = e / (OZ_N * 2), rem = e % (OZ_N * 2), jr = rem >> 1, hf = rem & 1;
                *reinterpret_cast<uint4*>(stB + d * OZ_B_SLICE + hf * 128 + (jr >> 3) * 256 + (jr & 7) * 16) =
                    *reinterpret_cast<const uint4*>(sg.B + ((int64_t)d * kpad + j0 + jr) * sg.qpad + kk + hf * 8);
            }
            tc::fence_proxy_async();
            mbar_arrive(&full[st]);
            if (t == n0 - 1 || t == total - 1) {
                // fold the segment in: levels 0-5 are exact multiples of 2^-30 (summed as integers),
                // the shared 6-8 accumulator is added in FP64; z w = 2^(E_r + E_c - 12) sum_L D_L,
                // E = exponent field - 1022
                if (!tc::mbar_wait(&segdone, (uint32_t)(segs & 1), OZ_WAIT_NS)) {
                    s_fail = 1;
                    break;
                }
                tc::fence_after_sync();
                const int e_row = egrow < n ? sg.rowexp[egrow] : 0;
#pragma unroll
                for (int c0 = 0; c0 < 32; c0 += 8) {
                    long long I[8];
                    float lowlev[8];
#pragma unroll
                    for (int v = 0; v < 8; ++v) I[v] = 0;
#pragma unroll
                    for (int a = 0; a < OZ_ACC; ++a) {
                        uint32_t rr[8];
                        const uint32_t ta = lane_addr + (uint32_t)(a * OZ_ACC_STRIDE + ch * 32 + c0);
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                                     : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]),
                                       "=r"(rr[6]), "=r"(rr[7])
                                     : "r"(ta));
                        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                        if (a < OZ_ACC - 1) {
#pragma unroll
                            for (int v = 0; v < 8; ++v)
                                I[v] += __float2ll_rn(__uint_as_float(rr[v]) * 1073741824.0f);
                        } else {
#pragma unroll
                            for (int v = 0; v < 8; ++v) lowlev[v] = __uint_as_float(rr[v]);
                        }
                    }
#pragma unroll
                    for (int v = 0; v < 8; ++v) {
                        const int j = j0 + ch * 32 + c0 + v;
                        if (j < k) {
                            const int sc = e_row + sg.colexp[j] - 2044 - 12;
                            y[c0 + v] += ldexp((double)I[v], sc - 30) + ldexp((double)lowlev[v], sc);
                        }
                    }
                }
                tc::fence_before_sync();
                mbar_arrive(&accfree);
                ++segs;
            }
        }
        if (!s_fail && egrow < n) {
#pragma unroll
            for (int v = 0; v < 32; ++v) {
                const int j = j0 + ch * 32 + v;
                if (j < k) Y[egrow * ldy + j] = y[v];
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, OZ_TMEM_COLS);
    if (tid == 0 && s_fail) atomicExch(status, 1);
}

}  // namespace

size_t oz_smem_bytes() { return (size_t)OZ_NS * OZ_STAGE + 1024; }

// Y (n x k, ld ldy; may not alias Z0, Z1) = [Z0 Z1] W, W (q0 + q1) x k row-major (ld k), device.
int update_oz(Session* s, const double* Z0, int64_t ld0, int q0, const double* Z1, int64_t ld1, int q1, int64_t n,
              const double* W, int k, double* Y, int64_t ldy, cudaStream_t st, int* status_out) {
    if (q0 < 1 || q1 < 0 || q0 > OZ_MAX_Q || q1 > OZ_MAX_Q || k < 1 || n < 1)
        return fail(HBSD_ERR_ARG, "update_oz: need 1 <= q0 <= 640, 0 <= q1 <= 640, k >= 1, n >= 1");
    const int kpad = (int)round_up(k, OZ_N);
    const int qp0 = (int)round_up(q0, 16), qp1 = (int)round_up(std::max(q1, 1), 16);
    const size_t bsl0 = (size_t)OZ_DIG * kpad * qp0, bsl1 = (size_t)OZ_DIG * kpad * qp1;
    // workspace (ints): row exponents 2 n, column exponents 2 kpad, status; then the bf16 slices
    const size_t ints = (size_t)2 * n + 2 * kpad + 4;
    const size_t bytes = ints * 4 + (bsl0 + bsl1) * 2 + 64;
    HBSD_TRY(s->oz_ws.alloc((bytes + 7) / 8));
    int* re0 = reinterpret_cast<int*>(s->oz_ws.p);
    int* re1 = re0 + n;
    int* ce0 = re1 + n;
    int* ce1 = ce0 + kpad;
    int* status = ce1 + kpad;
    uint16_t* B0 = reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(s->oz_ws.p) + ((ints * 4 + 63) / 64) * 64);
    uint16_t* B1 = B0 + bsl0;
    if (status_out) status = status_out;
    else HBSD_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
    const int rows_per_block = 8;
    k_oz_rowexp<<<ceil_div(n, rows_per_block), 32 * rows_per_block, 0, st>>>(Z0, ld0, q0, n, re0);
    HBSD_LAUNCHED(s);
    if (q1 > 0) {
        k_oz_rowexp<<<ceil_div(n, rows_per_block), 32 * rows_per_block, 0, st>>>(Z1, ld1, q1, n, re1);
        HBSD_LAUNCHED(s);
    }
    k_oz_wslices<<<kpad, 256, 0, st>>>(W, k, 0, q0, qp0, kpad, ce0, B0);
    HBSD_LAUNCHED(s);
    if (q1 > 0) {
        k_oz_wslices<<<kpad, 256, 0, st>>>(W, k, q0, q1, qp1, kpad, ce1, B1);
        HBSD_LAUNCHED(s);
    }
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(k_update_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes());
    });
    HBSD_CUDA(attr);
    OzSeg a{Z0, ld0, q0, qp0, B0, re0, ce0};
    OzSeg b{Z1, ld1, q1, qp1, B1, re1, ce1};
    dim3 grid(ceil_div(n, 128), kpad / OZ_N);
    k_update_oz<<<grid, OZ_THREADS, oz_smem_bytes(), st>>>(a, b, n, k, kpad, Y, ldy, status);
    HBSD_LAUNCHED(s);
    if (status_out) return 0;
    int h = 0;
    HBSD_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    HBSD_CUDA(cudaStreamSynchronize(st));
    if (h) return fail(HBSD_ERR_TIMEOUT, "update_oz: an MMA completion wait gave up");
    return 0;
}

}  // namespace hbsd
