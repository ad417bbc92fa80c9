// Float-float arithmetic: unevaluated sums of two floats (h + l, about 48
// significant bits) from error-free transforms, for the kernels that need
// near-FP64 accuracy on GB300's FP32 pipe (FP64 runs at 1/64 of its rate).
//   two_sum: Knuth's TwoSum (exact s + e = a + b, any a, b);
//   fast_two_sum: Dekker's Fast2Sum (exact when exponent(a) >= exponent(b));
//   products: the FMA gives the exact error of a float product.
// All operations use round-to-nearest intrinsics, which the compiler never
// contracts or reassociates.
#pragma once

#include <cuda_runtime.h>

namespace bpm {
namespace ffm {

struct ffv {
    float h, l;
};

__device__ __forceinline__ ffv two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ffv{s, e};
}
// exact when a == 0 or exponent(a) >= exponent(b)
__device__ __forceinline__ ffv fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return ffv{s, __fsub_rn(b, __fsub_rn(s, a))};
}
// a*b as an unnormalised pair p + e (the product of the low parts dropped)
__device__ __forceinline__ ffv mul_u(ffv a, ffv b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return ffv{p, e};
}
__device__ __forceinline__ ffv sqr_u(ffv a) {
    const float p = __fmul_rn(a.h, a.h);
    float e = __fmaf_rn(a.h, a.h, -p);
    e = __fmaf_rn(__fadd_rn(a.h, a.h), a.l, e);
    return ffv{p, e};
}
__device__ __forceinline__ ffv neg(ffv a) { return ffv{-a.h, -a.l}; }
// a + b, TwoSum on the high parts, the low parts added (unnormalised)
__device__ __forceinline__ ffv add_ff(ffv a, ffv b) {
    const ffv s = two_sum(a.h, b.h);
    return ffv{s.h, __fadd_rn(__fadd_rn(a.l, b.l), s.l)};
}
__device__ __forceinline__ ffv norm_ff(ffv a) { return two_sum(a.h, a.l); }
// a c for a constant c that is exact in FP32
__device__ __forceinline__ ffv mulc(ffv a, float c) {
    const float p = __fmul_rn(c, a.h);
    return ffv{p, __fmaf_rn(c, a.l, __fmaf_rn(c, a.h, -p))};
}
// 1/a for a > 0 in the float normal range: the FP32 reciprocal, then one
// Newton step y + y (1 - a y) with the residual from exact products
__device__ __forceinline__ ffv rcp_ff(ffv a) {
    const float y = __frcp_rn(a.h);
    const float p = __fmul_rn(a.h, y);
    const float err = __fmaf_rn(a.h, y, -p);  // a.h y = p + err exactly
    float r = __fsub_rn(__fsub_rn(1.0f, p), err);  // 1 - p is exact near 1
    r = __fmaf_rn(-a.l, y, r);
    return fast_two_sum(y, __fmul_rn(y, r));
}

// float -> double by integer operations (exponent rebias and mantissa shift),
// so that no conversion instruction occupies the narrow FP64 pipe; zero and
// subnormal floats give zero, infinities and NaN stay non-finite
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f), a = u & 0x7fffffffu, e = u & 0x7f800000u;
    unsigned hi = (a >> 3) + (e == 0x7f800000u ? 0x70000000u : 0x38000000u);
    unsigned lo = u << 29;
    if (e == 0u) hi = lo = 0u;
    return __hiloint2double((int)(hi | (u & 0x80000000u)), (int)lo);
}
__device__ __forceinline__ double to_double(ffv a) { return widen(a.h) + widen(a.l); }

// double -> float-float by integer operations: the high float is x cut to
// its leading 24 bits, the low float the next bits (rounded to 24), so
// h + l = x within 2^-48 |x|.  For |x| between 2^-126 and 2^127; outside
// that range it returns zero (callers pass values far inside it).
__device__ __forceinline__ ffv split_d(double x) {
    const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
    const unsigned a = hw & 0x7fffffffu, sg = hw & 0x80000000u;
    if (a < 0x38100000u || a >= 0x47f00000u) return ffv{0.f, 0.f};
    const float h = __uint_as_float(sg | ((a - 0x38000000u) << 3) | (lw >> 29));
    // the 29 remaining mantissa bits m, worth m 2^(E - 1075) (E the biased
    // exponent); zero when that scale is below the float range
    const unsigned E = a >> 20;
    const float l = E >= 949u ? __fmul_rn(__uint2float_rn(lw & 0x1fffffffu), __uint_as_float((E - 948u) << 23)) : 0.f;
    return ffv{h, sg ? -l : l};
}

}  // namespace ffm
}  // namespace bpm
