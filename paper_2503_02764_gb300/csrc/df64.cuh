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

// The same two conversions in integer arithmetic (FP64 instructions issue at 1/58 of the
// FP32 rate here, and a conversion costs about two of them), bit-identical to the FP64
// forms above; each returns false outside its window and the caller then uses those.
//
// split: v * 2^k2 -> (RN32, RN32 of the remainder), for 2^-48 <= |v 2^k2| < 2^80. hi is
// the double's significand rounded to 24 bits (ties to even, a carry moving it to the next
// binade); the remainder v - hi is an integer number of the double's ulps below 2^29,
// rounded to 24 bits by the int -> float conversion and scaled through its exponent field.
__device__ __forceinline__ bool df_split_i(double v, int k2, df& out) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned sgn = (unsigned)(b >> 63);
    const int e = (int)((b >> 52) & 0x7FF) + k2;
    if (((b >> 52) & 0x7FF) == 0 || e < 1023 - 48 || e >= 1023 + 80) return false;
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    unsigned mf = (unsigned)(m >> 29);
    const unsigned rem = (unsigned)(m & 0x1FFFFFFFu);
    int ef = e - 1023 + 127;
    if (rem > 0x10000000u || (rem == 0x10000000u && (mf & 1u))) {
        if (++mf == 0x800000u) {
            mf = 0;
            ++ef;
        }
    }
    out.hi = __uint_as_float((sgn << 31) | ((unsigned)ef << 23) | mf);
    const unsigned long long hd =
        ((unsigned long long)(ef - 127 + 1023 - k2) << 52) | ((unsigned long long)mf << 29);
    const long long du = (long long)((b & 0x7FFFFFFFFFFFFFFFull) - hd);
    if (du == 0) {
        out.lo = 0.f;
        return true;
    }
    unsigned fb = __float_as_uint(__int2float_rn((int)du));
    fb = (fb & 0x807FFFFFu) | ((unsigned)((int)((fb >> 23) & 0xFF) + (e - 1075)) << 23);
    const float lo = __uint_as_float(fb);
    out.lo = sgn ? -lo : lo;
    return true;
}

// join: (hi, lo) -> RN64(hi + lo) * 2^k2 for a normalised pair with 2^-100 < |hi| < 2^100.
// hi's bits become the double's; lo is added as an integer number of the result's ulps
// (rounded to nearest, ties to even, when lo reaches below them). A sum leaving hi's binade
// (only an unnormalised pair does) takes the FP64 form; a subtraction from a binade start
// lands one binade down and is counted in that binade's ulp.
__device__ __forceinline__ bool df_join_i(df x, int k2, double& out) {
    const unsigned hb = __float_as_uint(x.hi);
    const int eh = (int)((hb >> 23) & 0xFF);
    if (eh < 127 - 100 || eh > 127 + 100) return false;
    const unsigned sgn = hb >> 31;
    const unsigned hm = hb & 0x7FFFFFu;
    const unsigned long long hd =
        ((unsigned long long)(eh - 127 + 1023) << 52) | ((unsigned long long)hm << 29);
    const unsigned lb = __float_as_uint(x.lo);
    const int el = (int)((lb >> 23) & 0xFF);
    unsigned long long res = hd;
    if ((lb & 0x7FFFFFFFu) != 0) {
        if (el == 0) return false;
        const bool sub = (lb >> 31) != sgn;
        const unsigned long long Ml = (unsigned long long)((lb & 0x7FFFFFu) | 0x800000u);
        int sh = (el - 150) - (eh - 179);
        if (sub && hm == 0) sh += 1;
        unsigned long long units;
        if (sh >= 0) {
            if (sh > 8) return false;
            units = Ml << sh;
        } else if (-sh >= 40) {
            units = 0;
        } else {
            const int r = -sh;
            const unsigned long long q = Ml >> r, rm = Ml & ((1ull << r) - 1), half = 1ull << (r - 1);
            units = q;
            if (rm > half) {
                units = q + 1;
            } else if (rm == half) {
                const unsigned long long t = sub ? hd - q : hd + q;
                if (t & 1ull) units = q + 1;
            }
        }
        res = sub ? hd - units : hd + units;
        const unsigned long long eres = res >> 52, ehd = hd >> 52;
        if (!(eres == ehd || (sub && hm == 0 && eres + 1 == ehd))) return false;
    }
    const int ef = (int)(res >> 52) + k2;
    if (ef <= 0 || ef >= 2047) return false;
    res = (res & 0xFFFFFFFFFFFFFull) | ((unsigned long long)ef << 52);
    out = __longlong_as_double((long long)((((unsigned long long)sgn) << 63) | res));
    return true;
}

// the conversions with the integer form first
__device__ __forceinline__ df df_from_double_i(double v, int k2 = 0) {
    df r;
    if (df_split_i(v, k2, r)) return r;
    return df_from_double(k2 ? ldexp(v, k2) : v);
}
__device__ __forceinline__ double df_to_double_i(df x, int k2 = 0) {
    double r;
    if (df_join_i(x, k2, r)) return r;
    const double v = df_to_double(x);
    return k2 ? ldexp(v, k2) : v;
}

}  // namespace fld
