// Tensor-core (tcgen05) building block: D = A B^T with bf16 A (M x K) and B (N x K), FP32
// accumulation in tensor memory.  The split-slice FP64 products of the mixed form are sums of such
// products over exact bf16 slices of FP64 operands; hbsd_tc_gemm_bf16 exposes the block on its
// own so that its operand layout and accumulation are checked against a plain product.
#include <algorithm>
#include <string>

#include "common.h"
#include "tc.h"

namespace hbsd {
namespace {

constexpr int TC_THREADS = 128;
constexpr uint64_t TC_WAIT_NS = 2000000000ull;   // 2 s per wait, then the call reports a timeout

// One CTA: rows [128 b, 128 b + 128) of D, all N columns; K in steps of 16 (one MMA each).
// variant 0: descriptor leading offset = distance of K-adjacent core matrices (128 B), stride
// offset = distance of row-adjacent ones (256 B); variant 1 gives the two fields swapped.
__global__ void __launch_bounds__(TC_THREADS) k_tc_gemm_bf16(const uint16_t* __restrict__ A,
                                                             const uint16_t* __restrict__ B, float* __restrict__ D,
                                                             int N, int K, int variant, int* __restrict__ status) {
    __shared__ __align__(1024) uint8_t sA[16384];   // 4 KB used; the rest keeps any descriptor reading in bounds
    __shared__ __align__(1024) uint8_t sB[16384];   // 8 KB used
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t row0 = (int64_t)blockIdx.x * 128;
    const uint32_t ncols = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
    if (tid == 0) {
        tc::mbar_init(&mbar, 1);
        s_fail = 0;
    }
    if (warp == 0) tc::tmem_alloc(&tslot, ncols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tslot;
    const uint32_t idesc = tc::idesc_bf16_f32(128, N);
    const uint32_t lbo = variant == 0 ? 128 : 256, sbo = variant == 0 ? 256 : 128;
    uint32_t phase = 0;
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = tid; e < 128 * 16; e += TC_THREADS) {
            const int r = e >> 4, k = e & 15;
            *reinterpret_cast<uint16_t*>(sA + tc::kmajor16_offset(r, k)) = A[(row0 + r) * K + k0 + k];
        }
        for (int e = tid; e < N * 16; e += TC_THREADS) {
            const int r = e >> 4, k = e & 15;
            *reinterpret_cast<uint16_t*>(sB + tc::kmajor16_offset(r, k)) = B[(int64_t)r * K + k0 + k];
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint64_t ad = tc::smem_desc(tc::smem_u32(sA), lbo, sbo);
            const uint64_t bd = tc::smem_desc(tc::smem_u32(sB), lbo, sbo);
            tc::mma_bf16(tbase, ad, bd, idesc, k0 > 0 ? 1u : 0u);
            tc::mma_commit(&mbar);
        }
        // the MMA has read the tiles (and written D) before they are refilled
        if (!tc::mbar_wait(&mbar, phase, TC_WAIT_NS)) s_fail = 1;
        phase ^= 1u;
        __syncthreads();
        if (s_fail) break;
    }
    tc::fence_after_sync();
    if (!s_fail) {
        // warp w reads TMEM lanes 32 w .. 32 w + 31 = rows of D
        const int r = warp * 32 + (tid & 31);
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (c0 + i < N) D[(row0 + r) * N + c0 + i] = v[i];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, ncols);
    if (tid == 0 && s_fail) atomicExch(status, 1);
}

}  // namespace

int tc_gemm_bf16(const uint16_t* A, const uint16_t* B, float* D, int M, int N, int K, int variant, cudaStream_t st) {
    if (M <= 0 || M % 128 || N < 16 || N > 256 || N % 16 || K <= 0 || K % 16 || (variant != 0 && variant != 1))
        return fail(HBSD_ERR_ARG, "tc_gemm_bf16: M multiple of 128, N multiple of 16 in [16, 256], K multiple of 16");
    DBuf<int> status;
    HBSD_TRY(status.alloc(1));
    HBSD_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int), st));
    k_tc_gemm_bf16<<<M / 128, TC_THREADS, 0, st>>>(A, B, D, N, K, variant, status.p);
    HBSD_LAUNCHED(nullptr);
    int h = 0;
    HBSD_CUDA(cudaMemcpyAsync(&h, status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HBSD_CUDA(cudaStreamSynchronize(st));
    if (h) return fail(HBSD_ERR_TIMEOUT, "tc_gemm_bf16: an MMA completion wait gave up");
    return 0;
}

}  // namespace hbsd

extern "C" int hbsd_tc_gemm_bf16(const uint16_t* A, const uint16_t* B, float* D, int M, int N, int K, int variant,
                                 void* stream) {
    return hbsd::guarded([&]() -> int {
        if (!A || !B || !D) return hbsd::fail(HBSD_ERR_ARG, "NULL argument");
        return hbsd::tc_gemm_bf16(A, B, D, M, N, K, variant, (cudaStream_t)stream);
    });
}
