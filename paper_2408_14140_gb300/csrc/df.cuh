// Double-float arithmetic for the FP64-field pass sums.
//
// GB300 issues two FP64 operations per clock per SM against 128 FP32 (or
// INT32) operations, so the FP64 forms of the interpolation and gather sums
// were bound by the FP64 pipe.  Here a double value is carried as an
// unevaluated pair of floats hi + lo (Dekker 1971, "A floating-point
// technique for extending the available precision"), with
//   * products from the FMA remainder: fma(a, b, -a*b) is the exact error of
//     the float product a*b (the cross terms a.hi*b.lo + a.lo*b.hi are
//     added, a.lo*b.lo is dropped);
//   * sums from Knuth's TwoSum (the exact rounding error of a float sum from
//     six additions), followed by a renormalisation of (hi, lo);
//   * conversions between double and float pairs by bit manipulation on the
//     integer pipe: a double's top 24 significant bits (truncated) form hi and
//     its next 29 bits, rounded to 24, form lo, so a split is within 2^-47 of
//     the double (|x| >= 2^-74; smaller magnitudes keep only hi, and values
//     below 2^-126 become 0).
// Every float operation is an explicit _rn intrinsic, so the compiler cannot
// contract a product into a following sum (which would break TwoSum).
// The pair carries about 48 significant bits; sums of a few dozen terms stay
// within ~1e-13 of the exact result, inside the library's 1e-12 gate for
// FP64 fields.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbib {

// double -> (hi, lo), integer pipe only.
__device__ __forceinline__ float2 df_split(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
    const unsigned sgn = h32 & 0x80000000u;
    const int e = (int)((h32 >> 20) & 0x7ffu);  // biased exponent (bias 1023)
    const unsigned mh = ((h32 & 0xfffffu) << 3) | (l32 >> 29);  // top 23 stored bits
    if (e <= 896) return make_float2(__uint_as_float(sgn), __uint_as_float(sgn));  // |x| < 2^-126
    if (e >= 1151) {  // beyond float range, Inf or NaN: keep the class
        const unsigned nan = (e == 2047 && ((h32 & 0xfffffu) | l32)) ? 0x400000u : 0u;
        return make_float2(__uint_as_float(sgn | 0x7f800000u | nan), 0.0f);
    }
    const float hi = __uint_as_float(sgn | ((unsigned)(e - 896) << 23) | mh);
    float lo = 0.0f;
    if (e >= 949) {
        // remaining 29 bits r, worth r * 2^(e - 1075)
        const unsigned r = l32 & 0x1fffffffu;
        const float scale = __uint_as_float((unsigned)(e - 948) << 23);
        lo = __uint_as_float(__float_as_uint(__fmul_rn(__uint2float_rn(r), scale)) | sgn);
    }
    return make_float2(hi, lo);
}

// float -> double, exact, integer pipe only (float subnormals become 0).
__device__ __forceinline__ double df_widen(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned sgn = b & 0x80000000u;
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned m = b & 0x7fffffu;
    unsigned h32, l32;
    if (e == 0) {
        h32 = sgn;
        l32 = 0;
    } else if (e == 255) {
        h32 = sgn | 0x7ff00000u | (m >> 3) | (m ? 0x80000u : 0u);
        l32 = 0;
    } else {
        h32 = sgn | ((e + 896u) << 20) | (m >> 3);
        l32 = m << 29;
    }
    return __hiloint2double((int)h32, (int)l32);
}

// (hi, lo) -> double: one FP64 addition.
__device__ __forceinline__ double df_to_double(float2 v) { return __dadd_rn(df_widen(v.x), df_widen(v.y)); }

// Renormalise s + e (|e| small against s) into a pair.
__device__ __forceinline__ float2 df_fast_two_sum(float s, float e) {
    const float h = __fadd_rn(s, e);
    return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}

// a * b of two pairs.
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    return df_fast_two_sum(p, e);
}

// a + b of two pairs: TwoSum of the high parts, the low parts added to its
// error, renormalised.
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    const float s = __fadd_rn(a.x, b.x);
    const float bb = __fsub_rn(s, a.x);
    const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
    return df_fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}

__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

// a * k for a power of two k: exact.
__device__ __forceinline__ float2 df_scale(float2 a, float k) { return make_float2(__fmul_rn(a.x, k), __fmul_rn(a.y, k)); }

// Square root of a pair a > 0 (a.x a normal float): one Newton (Heron) step
// q = q0 + (a - q0^2) / (2 q0) from the FP32 root q0, the residual from the
// exact FMA square (a.x - q0^2 is exact: q0^2 is within a factor 2 of a.x).
// The start's relative error below 2^-24 leaves about 2^-47.
__device__ __forceinline__ float2 df_sqrt(float2 a) {
    const float q0 = __fsqrt_rn(a.x);
    const float p = __fmul_rn(q0, q0);
    const float pe = __fmaf_rn(q0, q0, -p);
    const float res = __fadd_rn(__fsub_rn(__fsub_rn(a.x, p), pe), a.y);
    return df_fast_two_sum(q0, __fmul_rn(res, __fdiv_rn(0.5f, q0)));
}

// Running sum of pair products, renormalised after every term.
struct DFAcc {
    float hi, lo;
    __device__ __forceinline__ DFAcc() : hi(0.0f), lo(0.0f) {}
    __device__ __forceinline__ void add_prod(float2 a, float2 b) {
        const float p = __fmul_rn(a.x, b.x);
        float pe = __fmaf_rn(a.x, b.x, -p);
        pe = __fmaf_rn(a.x, b.y, pe);
        pe = __fmaf_rn(a.y, b.x, pe);
        // TwoSum(hi, p)
        const float s = __fadd_rn(hi, p);
        const float bb = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
        const float2 r = df_fast_two_sum(s, __fadd_rn(lo, __fadd_rn(err, pe)));
        hi = r.x;
        lo = r.y;
    }
    __device__ __forceinline__ float2 get() const { return make_float2(hi, lo); }
    __device__ __forceinline__ double value() const { return df_to_double(get()); }
};

}  // namespace gbib
