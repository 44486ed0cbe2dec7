// m1_df.cuh — double-word ("double-float") arithmetic on pairs of FP32 numbers.
//
// The FP64 residual and J v of the implicit step are bound by the FP64 pipe,
// which on this GPU issues about 1/64 of the FP32 rate. A double-word number
// x = hi + lo (|lo| <= ulp(hi) / 2) carries about 48 significant bits, and its
// operations are short sequences of FP32 operations on the full-rate pipe, so
// the residual keeps ~1e-14 relative accuracy per operation at a fraction of
// the FP64 cost. The exponent range is FP32's: magnitudes must stay within
// about 2^+-100. The library selects this arithmetic for grids whose scalars
// (c, a_r, dx) are near 1, and a residual whose components leave the range
// is computed again in FP64 (the FP32 inner solver has the same range).
//
// The algorithms are the double-word building blocks analysed by M. Joldes,
// J.-M. Muller and V. Popescu, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic", ACM TOMS 44 (2017), built on
// the error-free transforms of Knuth (2Sum), Dekker (Fast2Sum) and the FMA
// product error; relative error bounds with u = 2^-24:
//   DW + DW (accurate)  3u^2 + 13u^3      DW x FP  2u^2
//   DW x DW             4u^2              DW / DW  15u^2 + 56u^3
// The square root is one Newton (Heron) correction of the FP32 root, s + (x -
// s^2) / (2 s), with s^2 formed exactly by the FMA product error.
//
// Every rounding step uses the __f*_rn intrinsics, which the compiler never
// contracts into an FMA: the error-free transforms depend on each sum and
// product being rounded exactly once.
#pragma once

#include <cuda_runtime.h>

namespace m1 {

struct DF;
__device__ __forceinline__ DF df_from_double(double x);

struct DF {
    float hi, lo;
    DF() = default;
    __host__ __device__ constexpr DF(float h, float l) : hi(h), lo(l) {}
    // a double as a double-word (df_from_double)
    __device__ __forceinline__ DF(double x);
    __device__ __forceinline__ DF(float x) : hi(x), lo(0.0f) {}
    __device__ __forceinline__ DF(int x) : hi((float)x), lo(0.0f) {}  // exact for |x| < 2^24
};

// ---------------------------------------------------------------- error-free transforms
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {  // |a| >= |b| (or a = 0)
    const float s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    return DF(s, __fsub_rn(b, z));
}
__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float ap = __fsub_rn(s, b);
    const float bp = __fsub_rn(s, ap);
    const float da = __fsub_rn(a, ap);
    const float db = __fsub_rn(b, bp);
    return DF(s, __fadd_rn(da, db));
}
__device__ __forceinline__ DF df_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return DF(p, __fmaf_rn(a, b, -p));
}

// A double as hi + lo without FP64 operations (the FP64 pipe is the scarce
// one): hi is x cut to its leading 24 significant bits, built from the bit
// fields; lo is the other 29 mantissa bits, converted to FP32 (rounded) and
// scaled by the exponent; a Fast2Sum then normalises the pair. The result is
// within 2^-53 |x| of x for 2^-74 <= |x| < 2^128. Below 2^-74 lo is dropped
// (24 bits kept), below 2^-126 (FP32's normal range, zero included) the result
// is 0; from 2^128 on it is +-inf, and NaN stays NaN.
__device__ __forceinline__ DF df_from_double(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int top = (unsigned int)(b >> 32);
    const int ed = (int)((top >> 20) & 0x7ffu);  // biased FP64 exponent
    const unsigned int sign = top & 0x80000000u;
    if (ed < 897) return DF(0.0f, 0.0f);
    if (ed > 1150) {
        const bool nan = ed == 2047 && (b << 12) != 0ull;
        return DF(__uint_as_float(nan ? 0x7fc00000u : (sign | 0x7f800000u)), 0.0f);
    }
    const unsigned int mhi = (unsigned int)(b >> 29) & 0x7fffffu;  // leading 23 stored mantissa bits
    const float hi = __uint_as_float(sign | ((unsigned int)(ed - 896) << 23) | mhi);
    const unsigned int mlo = (unsigned int)b & 0x1fffffffu;  // the remaining 29 bits, worth 2^(ed - 1075) each
    float lo = 0.0f;
    if (mlo != 0u && ed >= 949) {
        const float scale = __uint_as_float((unsigned int)(ed - 948) << 23);  // 2^(ed - 1075)
        lo = __fmul_rn(__uint2float_rn(mlo), scale);
        if (sign) lo = -lo;
    }
    return df_fast_two_sum(hi, lo);
}
__device__ __forceinline__ DF::DF(double x) : DF(df_from_double(x)) {}

// ---------------------------------------------------------------- arithmetic
__device__ __forceinline__ DF operator+(DF x, DF y) {
    const DF s = df_two_sum(x.hi, y.hi);
    const DF t = df_two_sum(x.lo, y.lo);
    const float c = __fadd_rn(s.lo, t.hi);
    const DF v = df_fast_two_sum(s.hi, c);
    const float w = __fadd_rn(t.lo, v.lo);
    return df_fast_two_sum(v.hi, w);
}
__device__ __forceinline__ DF operator-(DF x) { return DF(-x.hi, -x.lo); }
__device__ __forceinline__ DF operator-(DF x, DF y) { return x + (-y); }
__device__ __forceinline__ DF df_mul_f(DF x, float y) {
    const DF c = df_two_prod(x.hi, y);
    const float cl3 = __fmaf_rn(x.lo, y, c.lo);
    return df_fast_two_sum(c.hi, cl3);
}
__device__ __forceinline__ DF operator*(DF x, DF y) {
    const DF c = df_two_prod(x.hi, y.hi);
    const float tl0 = __fmul_rn(x.lo, y.lo);
    const float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
    const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
    const float cl3 = __fadd_rn(c.lo, cl2);
    return df_fast_two_sum(c.hi, cl3);
}
__device__ __forceinline__ DF operator/(DF x, DF y) {
    const float th = __fdiv_rn(x.hi, y.hi);
    const DF r = df_mul_f(y, th);
    const float ph = __fsub_rn(x.hi, r.hi);
    const float dl = __fsub_rn(x.lo, r.lo);
    const float d = __fadd_rn(ph, dl);
    const float tl = __fdiv_rn(d, y.hi);
    return df_fast_two_sum(th, tl);
}
__device__ __forceinline__ DF df_sqrt(DF x) {
    if (!(x.hi > 0.0f)) return DF(0.0f, 0.0f);
    const float s = __fsqrt_rn(x.hi);
    const DF p = df_two_prod(s, s);  // s^2 exactly
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), p.lo), x.lo);
    const float t = __fdiv_rn(r, __fmul_rn(2.0f, s));
    return df_fast_two_sum(s, t);
}

// mixed operands: a double (from memory or a scalar of the grid) is first
// rounded to the nearest double-word
__device__ __forceinline__ DF operator+(DF x, double y) { return x + DF(y); }
__device__ __forceinline__ DF operator+(double x, DF y) { return DF(x) + y; }
__device__ __forceinline__ DF operator-(DF x, double y) { return x - DF(y); }
__device__ __forceinline__ DF operator-(double x, DF y) { return DF(x) - y; }
__device__ __forceinline__ DF operator*(DF x, double y) { return x * DF(y); }
__device__ __forceinline__ DF operator*(double x, DF y) { return DF(x) * y; }
__device__ __forceinline__ DF operator/(DF x, double y) { return x / DF(y); }
__device__ __forceinline__ DF operator/(double x, DF y) { return DF(x) / y; }
__device__ __forceinline__ DF& operator+=(DF& x, DF y) { return x = x + y; }
__device__ __forceinline__ DF& operator-=(DF& x, DF y) { return x = x - y; }

// ---------------------------------------------------------------- comparisons
// (normalised pairs: the order of (hi, lo) lexicographically is the order of hi + lo)
__device__ __forceinline__ bool operator>(DF a, DF b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator<(DF a, DF b) { return b > a; }
__device__ __forceinline__ bool operator>=(DF a, DF b) { return !(b > a); }
__device__ __forceinline__ bool operator<=(DF a, DF b) { return !(a > b); }

// ---------------------------------------------------------------- conversions
__device__ __forceinline__ double df_to_double(DF x) { return (double)x.hi + (double)x.lo; }

}  // namespace m1
