// Double-float ("float-float") arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.  GB300 issues FP32
// at 64 times its FP64 rate, so a handful of FP32 operations per double-float
// operation is far cheaper than native FP64 where FP64 issue is the bound.
//
// The building blocks are the classical error-free transformations: Knuth's TwoSum
// (the exact rounding error of a + b from six additions), Dekker's FastTwoSum (three,
// when |a| >= |b|) and the exact product error a b - fl(a b) from one fused
// multiply-add.  Every operation is written with explicitly rounded intrinsics so that
// the compiler cannot contract or reorder it.
#pragma once

#include <cstdint>

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {  // |a| >= |b| (or a = 0)
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// exact double-float of a double (round to nearest twice)
__host__ __device__ __forceinline__ ff ff_from_double(double x) {
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = ff_two_sum(a.hi, b.hi);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ff_fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_sqr(ff a) {
    const float p = __fmul_rn(a.hi, a.hi);
    float e = __fmaf_rn(a.hi, a.hi, -p);
    e = __fmaf_rn(__fmul_rn(2.0f, a.hi), a.lo, e);
    return ff_fast_two_sum(p, e);
}

// sqrt(a) for a >= 0.  y = 1/sqrt(hi) from the hardware estimate refined by one FP32
// Newton step y (3 - hi y^2) / 2 (about one unit in the last place), s = hi y, then one
// Newton (Heron) step s + (a - s^2) y / 2 with a - s^2 formed exactly: the step squares
// s's relative error (~1e-7 -> ~1e-14).  No IEEE square-root or division sequence.
// a = 0 gives 0.
__device__ __forceinline__ ff ff_sqrt(ff a) {
    if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
    const float y0 = rsqrtf(a.hi);
    const float y = __fmul_rn(y0, __fmaf_rn(__fmul_rn(-0.5f * a.hi, y0), y0, 1.5f));
    const float s = __fmul_rn(a.hi, y);
    const float p = __fmul_rn(s, s);
    const float pe = __fmaf_rn(s, s, -p);                              // s^2 = p + pe exactly
    const float e = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo);  // a - s^2
    return ff_fast_two_sum(s, __fmul_rn(e, __fmul_rn(0.5f, y)));
}

// (a + b) - c for a float a and double-floats b, c where a - c.hi is formed exactly first:
// the cell offset plus a point's in-cell offset minus the reference point's.
__device__ __forceinline__ ff ff_sum3(float a, ff b, ff c) {
    const ff base = ff_two_sum(a, -c.hi);
    return ff_add({base.hi, __fsub_rn(base.lo, c.lo)}, b);
}

// A float as a double, by the IEEE 754 layouts (binary32: 1 sign, 8 exponent bits biased
// by 127, 23 fraction bits; binary64: 11 exponent bits biased by 1023, 52 fraction bits):
// for a normal float keep the sign, rebias the exponent by 1023 - 127 = 896 and widen the
// fraction by 29 bits.  Integer instructions only; zeros keep their sign, and subnormals,
// infinities and NaNs take the hardware conversion.  Exact, like any float-to-double widening.
__device__ __forceinline__ double f2d_exact(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xFFu;
    const uint64_t sign = (uint64_t)(b >> 31) << 63;
    if ((b << 1) == 0u) return __longlong_as_double((long long)sign);
    if (e == 0u || e == 0xFFu) return (double)f;
    return __longlong_as_double((long long)(sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29)));
}

// A small integer (|n| < 2^22) as a float without a conversion instruction: placed in the
// fraction of 1.5 * 2^23, whose unit in the last place is 1, then the bias subtracted.
// Exact for every n in range.
__device__ __forceinline__ float small_int_to_float(int n) {
    return __fsub_rn(__int_as_float(0x4B400000 + n), 12582912.0f);
}

// hi + lo rounded to a double: two exact widenings and one FP64 addition.
__device__ __forceinline__ double ff_to_double(ff a) { return f2d_exact(a.hi) + f2d_exact(a.lo); }
