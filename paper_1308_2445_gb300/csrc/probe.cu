// Peak probes: sustained FMA throughput of the SIMT pipes (FP64 and FP32), the denominators of
// the "alu" rooflines of the FP64 path.  Each thread runs 8 independent FMA chains so that the
// pipe, not the dependency latency, is the limit; the grid covers every SM several times.
#include "common.h"

namespace hbsd {
namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma_chain(T* out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == (T)-12345.0) out[0] = s;  // keeps the chains alive; never true for these inputs
}

template <class T>
int probe(cudaStream_t st, double* flops) {
    int dev = 0, sms = 0;
    HBSD_CUDA(cudaGetDevice(&dev));
    HBSD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DBuf<T> out;
    HBSD_TRY(out.alloc(1));
    const int blocks = sms * 8;
    const int iters = sizeof(T) == 8 ? 4096 : 65536;
    cudaEvent_t e0, e1;
    HBSD_CUDA(cudaEventCreate(&e0));
    HBSD_CUDA(cudaEventCreate(&e1));
    k_fma_chain<T><<<blocks, 256, 0, st>>>(out.p, iters / 8, (T)0.999, (T)1e-4);  // warm-up
    HBSD_CUDA(cudaEventRecord(e0, st));
    k_fma_chain<T><<<blocks, 256, 0, st>>>(out.p, iters, (T)0.999, (T)1e-4);
    HBSD_CUDA(cudaEventRecord(e1, st));
    HBSD_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    HBSD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *flops = 2.0 * 8.0 * (double)iters * blocks * 256 / (ms * 1e-3);
    return 0;
}

}  // namespace
}  // namespace hbsd

extern "C" int hbsd_probe_peak(int which, void* stream, double* flops_per_s) {
    if (!flops_per_s) return hbsd::fail(HBSD_ERR_ARG, "NULL output");
    cudaStream_t st = (cudaStream_t)stream;
    if (which == 0) return hbsd::probe<double>(st, flops_per_s);
    if (which == 1) return hbsd::probe<float>(st, flops_per_s);
    return hbsd::fail(HBSD_ERR_ARG, "which must be 0 (FP64) or 1 (FP32)");
}
