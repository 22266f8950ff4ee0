// Double-float arithmetic: a value as an unevaluated sum hi + lo of two floats (Dekker 1971;
// Knuth's TwoSum), for FP64-bound products on GB300's FP32 pipes (128 FP32 lanes per clock
// per SM against 2 FP64).
//
// split_d builds the pair without the FP64 pipe: hi = the FP64 value truncated to 24 bits, from
// its sign, exponent and top mantissa bits; lo = the remaining 29 mantissa bits converted by the
// integer-to-float unit and scaled by the exponent.  The pair carries ~47 bits for magnitudes
// above 2^-96; below that lo is an FP32 subnormal and the precision falls towards 24 bits, and
// magnitudes below 2^-126 enter as zero.  dfma adds the product of two pairs (TwoProd by FMA
// for hi*hi plus the two cross terms) to a running pair by TwoSum; renorm restores |lo| <= ulp(hi)/2.
// The _rn intrinsics are never contracted into FMAs, which would break the error-free steps.
#pragma once
#include <cuda_runtime.h>

namespace hbsd {
namespace df {

__device__ __forceinline__ float2 split_d(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi32 = (unsigned)(b >> 32);
    const unsigned sign = hi32 & 0x80000000u;
    const int e = (int)((hi32 >> 20) & 0x7FFu);
    float h = 0.f, l = 0.f;
    if (e >= 897) {
        if (e > 1150) {
            h = __uint_as_float(sign | 0x7F800000u);   // beyond the FP32 range: +-inf, never silent
        } else {
            const unsigned top23 = ((hi32 & 0xFFFFFu) << 3) | (unsigned)((b >> 29) & 7u);
            h = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | top23);
            const unsigned low29 = (unsigned)(b & 0x1FFFFFFFull);
            if (e >= 949) {   // lo = low29 * 2^(e - 1075), the scale a normal float
                l = __fmul_rn(__uint_as_float(sign | ((unsigned)(e - 948) << 23)), __uint2float_rn(low29));
            } else {          // the same in two normal-range factors, 2^-64 and 2^(e - 1011)
                l = __fmul_rn(__fmul_rn(__uint2float_rn(low29), __uint_as_float(sign | (63u << 23))),
                              __uint_as_float((unsigned)(e - 884) << 23));
            }
        }
    }
    return make_float2(h, l);
}

// (sh, sl) += a * b for double-float a, b
__device__ __forceinline__ void dfma(const float2 a, const float2 b, float& sh, float& sl) {
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);   // rounding error of p, exact
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float t = __fadd_rn(sh, p);   // TwoSum(sh, p)
    const float bp = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    sl = __fadd_rn(sl, __fadd_rn(err, e));
    sh = t;
}

__device__ __forceinline__ void renorm(float& sh, float& sl) {   // FastTwoSum, |sh| >= |sl|
    const float t = __fadd_rn(sh, sl);
    sl = __fsub_rn(sl, __fsub_rn(t, sh));
    sh = t;
}

__device__ __forceinline__ double to_d(float sh, float sl) { return __dadd_rn((double)sh, (double)sl); }


}  // namespace df
}  // namespace hbsd
