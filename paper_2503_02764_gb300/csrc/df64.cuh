// Double-FP32 ("df") arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi)/2, giving a 48-bit significand with the FP32 exponent
// range. Built from error-free transformations:
//   two_sum       Knuth, TAOCP vol. 2, Sect. 4.2.2 (exact a + b = s + e, any order);
//   fast_two_sum  Dekker 1971, "A floating-point technique for extending the available
//                 precision" (exact when |a| >= |b|);
//   two_prod      a*b = p + e exactly with one fused multiply-add (Ogita, Rump and
//                 Oishi 2005, "Accurate sum and dot product").
// The df add/mul below are the usual "sloppy" double-word forms (relative error a few
// units of 2^-48). FP64 issues at 1/58 of the FP32 rate on this GPU, so these FP32
// sequences are the cheap way to reach FP64-grade accuracy in the memory-bound kernels.
#pragma once

namespace fld {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ df df_add_f(df x, float y) {
    df s = two_sum(x.hi, y);
    s.lo = __fadd_rn(s.lo, x.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_mul(df x, df y) {
    df p = two_prod(x.hi, y.hi);
    p.lo = __fmaf_rn(x.hi, y.lo, p.lo);
    p.lo = __fmaf_rn(x.lo, y.hi, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_mul_f(df x, float y) {
    df p = two_prod(x.hi, y);
    p.lo = __fmaf_rn(x.lo, y, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// Unnormalised double-word forms for short sums of products: the hi words combine
// exactly (two_sum / two_prod) and the lo words accumulate without the renormalising
// fast_two_sum, each step adding O(2^-24 |lo|) to the error. A few of them in a row keep
// the result within a few units of 2^-47 of the operands' magnitude, at about half the
// instructions of the renormalised forms; only the final value is rounded.
__device__ __forceinline__ df dw_add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return s;
}

__device__ __forceinline__ df dw_sub(df x, df y) {
    df s = two_sum(x.hi, -y.hi);
    s.lo = __fadd_rn(s.lo, __fsub_rn(x.lo, y.lo));
    return s;
}

// x * y without the lo * lo term
__device__ __forceinline__ df dw_mul(df x, df y) {
    df p = two_prod(x.hi, y.hi);
    p.lo = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
    return p;
}

// x / y: quotient estimate q1 = hi/hi, its df remainder x - q1 y, one correction term
// (the long-division step of double-word arithmetic).
__device__ __forceinline__ df df_div(df x, df y) {
    const float q1 = __fdiv_rn(x.hi, y.hi);
    const df r = df_sub(x, df_mul_f(y, q1));
    const float q2 = __fdiv_rn(r.hi, y.hi);
    return fast_two_sum(q1, q2);
}

// sqrt(x), x > 0: s = sqrt(hi), corrected by the df remainder (x - s^2)/(2 s) (Karp's
// one-step refinement).
__device__ __forceinline__ df df_sqrt(df x) {
    const float s = __fsqrt_rn(x.hi);
    const df r = df_sub(x, two_prod(s, s));
    return fast_two_sum(s, __fdiv_rn(r.hi, 2.f * s));
}

// 1/sqrt(x), x > 0: FP32 seed, then two Newton-Raphson steps y + y (1 - x y^2)/2 in df
// (the first leaves O(seed error^2) ~ 1e-13, the second the df rounding).
__device__ __forceinline__ df df_rsqrt(df x) {
    const float y0 = rsqrtf(x.hi);
    const df e0 = df_sub({1.f, 0.f}, df_mul(x, two_prod(y0, y0)));
    const df y1 = df_add_f(df_mul_f(e0, 0.5f * y0), y0);
    const df e1 = df_sub({1.f, 0.f}, df_mul(x, df_mul(y1, y1)));
    return df_add(y1, df_mul(df_mul_f(e1, 0.5f), y1));
}

// |x.hi| within [2^-80, 2^80]: comfortably inside the FP32 normal range, so the lo word
// keeps its full precision through products of a few such values.
__device__ __forceinline__ bool df_safe(float v) {
    const float a = fabsf(v);
    return a > 8.3e-25f && a < 1.2e24f;
}

// split an FP64 value into the nearest df (hi = RN(v), lo = RN(v - hi))
__device__ __forceinline__ df df_from_double(double v) {
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}

__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }

}  // namespace fld
