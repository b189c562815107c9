// Float-float ("double-single") arithmetic for the compensated-float32 epilogue.
//
// A value is the unevaluated sum hi + lo of two float32 numbers with |lo| <= ulp(hi) / 2, about
// 48 significant bits. The building blocks are the error-free transformations of Knuth (TwoSum:
// a + b = s + e exactly, any order of magnitude) and Dekker (TwoProd: a * b = p + e exactly, here
// with one fused multiply-add for e), and Dekker's renormalisation (FastTwoSum, |a| >= |b|).
// Every operation is an explicitly rounded intrinsic, so no compiler contraction or
// reassociation changes a result: the same inputs give the same bits in every kernel.
#pragma once

#include <cuda_runtime.h>

namespace tvspec {

struct ff {
    float hi, lo;
};

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// s + e = a + b exactly when |a| >= |b| or a == 0 (Dekker).
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = a * b exactly (Dekker's product with a fused multiply-add for the error term).
__device__ __forceinline__ ff ff_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_from_float(float a) { return {a, 0.0f}; }

// The float-float nearest to a float64 value (hi = the float nearest to it, lo = the rest).
__device__ __forceinline__ ff ff_from_double(double a) {
    const float hi = __double2float_rn(a);
    return {hi, __double2float_rn(__dsub_rn(a, (double)hi))};
}

// hi + lo exactly (both fit in a float64 significand).
__device__ __forceinline__ double ff_to_double(ff a) { return __dadd_rn((double)a.hi, (double)a.lo); }

// Rounded to float32 (hi already is the float nearest to hi + lo after renormalisation).
__device__ __forceinline__ float ff_to_float(ff a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

// a + b: TwoSum of the high parts and of the low parts, the errors folded back (the accurate
// variant: relative error about 2^-46 even under cancellation).
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = ff_two_sum(a.hi, b.hi);
    const ff t = ff_two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = ff_fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return ff_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

// a * b: exact product of the high parts plus the first-order cross terms.
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    ff p = ff_two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return ff_fast_two_sum(p.hi, p.lo);
}

// 2 a (exact).
__device__ __forceinline__ ff ff_twice(ff a) { return {__fmul_rn(2.0f, a.hi), __fmul_rn(2.0f, a.lo)}; }

__device__ __forceinline__ bool ff_isfinite(ff a) { return isfinite(a.hi) && isfinite(a.lo); }

}  // namespace tvspec
