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

// sqrt(a) for a >= 0: s = sqrtf(hi) (correctly rounded, relative error <= 2^-24), then one
// Newton (Heron) step s + (a - s^2) / (2 s) with a - s^2 formed exactly, which squares the
// relative error (below 1e-14 with the rounding of the step).  a = 0 gives 0.
__device__ __forceinline__ ff ff_sqrt(ff a) {
    if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
    const float s = __fsqrt_rn(a.hi);
    const float p = __fmul_rn(s, s);
    const float pe = __fmaf_rn(s, s, -p);                              // s^2 = p + pe exactly
    const float e = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo);  // a - s^2
    return ff_fast_two_sum(s, __fmul_rn(e, __fdiv_rn(0.5f, s)));
}

// The exact sum hi + lo as a double (two conversions and one FP64 addition).
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }
