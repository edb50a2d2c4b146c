// Double-float ("double-word") arithmetic on the binary32 pipes.
//
// A real number is the unevaluated sum hi + lo of two binary32 values with
// |lo| <= ulp(hi)/2, giving a 48-bit significand.  The building blocks are
// the classical error-free transformations:
//   two_sum       -- Knuth, TAOCP vol. 2 (s + e = a + b exactly)
//   fast_two_sum  -- Dekker 1971 (needs |a| >= |b| or a = 0)
//   two_prod      -- via fused multiply-add (p + e = a * b exactly)
// and the double-word algorithms of Joldes, Muller and Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic",
// ACM TOMS 2017 (SloppyDWPlusDW, DWTimesDW with FMA).  The compensated
// accumulation used by the block product is the Dot2 scheme of Ogita, Rump
// and Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 2005,
// extended with the cross terms of double-word inputs.
//
// Every operation is written with explicit __fadd_rn / __fmul_rn / __fmaf_rn
// so that the compiler can neither contract nor reassociate them.
#pragma once
#include <cuda_runtime.h>

namespace bttb {

struct df { float hi, lo; };

// Complex double-float, stored as float4 {re.hi, im.hi, re.lo, im.lo}.
struct __align__(16) cdf { float rh, ih, rl, il; };

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// SloppyDWPlusDW: 11 flops.  Error bounded relative to |x| + |y|, which is
// what the normwise error of an FFT butterfly needs.
__device__ __forceinline__ df df_add(df x, df y) {
    float s, e;
    two_sum(x.hi, y.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
    df r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

// DWTimesDW (FMA variant, lo*lo term dropped): 8 flops.
__device__ __forceinline__ df df_mul(df x, df y) {
    float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    df r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

// x * 2^k for a power-of-two float k: exact.
__device__ __forceinline__ df df_scale_pow2(df x, float k) { return df{x.hi * k, x.lo * k}; }

// Re or Im of a complex product as a two-term compensated dot product:
//   a*c + sb*b*d  (sb = +1 or -1), all operands double-float.
__device__ __forceinline__ df df_dot2(df a, df c, df b, df d, float sb) {
    float p1 = __fmul_rn(a.hi, c.hi);
    float e1 = __fmaf_rn(a.hi, c.hi, -p1);
    float bh = sb * b.hi, bl = sb * b.lo;
    float p2 = __fmul_rn(bh, d.hi);
    float e2 = __fmaf_rn(bh, d.hi, -p2);
    float s, t;
    two_sum(p1, p2, s, t);
    t = __fadd_rn(t, __fadd_rn(e1, e2));
    t = __fmaf_rn(a.hi, c.lo, t);
    t = __fmaf_rn(a.lo, c.hi, t);
    t = __fmaf_rn(bh, d.lo, t);
    t = __fmaf_rn(bl, d.hi, t);
    df r;
    two_sum(s, t, r.hi, r.lo);
    return r;
}

// Reciprocal and square root: one Newton step from the binary32 estimate with
// the residual formed exactly by FMA (Karp and Markstein, "High-precision
// division and square root", ACM TOMS 1997); relative error ~2^-46.
__device__ __forceinline__ df df_recip(df b) {
    const float r0 = __frcp_rn(b.hi);
    float e = __fmaf_rn(-b.hi, r0, 1.0f);          // 1 - b.hi r0, exact
    e = __fmaf_rn(-b.lo, r0, e);
    df r;
    fast_two_sum(r0, __fmul_rn(r0, e), r.hi, r.lo);
    return r;
}

__device__ __forceinline__ df df_sqrt(df a) {
    if (!(a.hi > 0.f)) return df{0.f, 0.f};
    const float s0 = __fsqrt_rn(a.hi);
    const float p = __fmul_rn(s0, s0);
    const float pe = __fmaf_rn(s0, s0, -p);        // s0^2 = p + pe exactly
    const float e = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo);
    df r;
    fast_two_sum(s0, __fdiv_rn(e, __fmul_rn(2.0f, s0)), r.hi, r.lo);
    return r;
}

// Complex double-float helpers (value type; storage is cdf).
struct dfc { df re, im; };
__device__ __forceinline__ dfc dfc_load(cdf v) { return dfc{df{v.rh, v.rl}, df{v.ih, v.il}}; }
__device__ __forceinline__ cdf dfc_store(dfc v) { return cdf{v.re.hi, v.im.hi, v.re.lo, v.im.lo}; }
__device__ __forceinline__ dfc dfc_add(dfc a, dfc b) { return dfc{df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ dfc dfc_sub(dfc a, dfc b) { return dfc{df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
__device__ __forceinline__ dfc dfc_conj(dfc a) { return dfc{a.re, df_neg(a.im)}; }
__device__ __forceinline__ dfc dfc_neg(dfc a) { return dfc{df_neg(a.re), df_neg(a.im)}; }
__device__ __forceinline__ dfc dfc_mul(dfc a, dfc b) {
    return dfc{df_dot2(a.re, b.re, a.im, b.im, -1.f), df_dot2(a.re, b.im, a.im, b.re, 1.f)};
}
__device__ __forceinline__ dfc dfc_scale(dfc a, df k) { return dfc{df_mul(a.re, k), df_mul(a.im, k)}; }
__device__ __forceinline__ df dfc_abs2(dfc a) { return df_dot2(a.re, a.re, a.im, a.im, 1.f); }

// Conversions between binary64 and double-float (binary64 pipe, used only
// at the boundary of the library: a handful of operations per element).
__device__ __forceinline__ df df_from_double(double v) {
    float h = __double2float_rn(v);
    float l = __double2float_rn(v - (double)h);
    return df{h, l};
}
__device__ __forceinline__ double df_to_double(df v) { return (double)v.hi + (double)v.lo; }

// ---------------------------------------------------------------------------
// Compensated accumulator for sum_k a_k * c_k with double-float a_k, c_k.
// S collects the rounded binary32 products through two_sum; s collects every
// rounding error and the hi*lo cross terms in plain binary32 (Dot2).
// ---------------------------------------------------------------------------
struct dacc { float S, s; };

__device__ __forceinline__ void dacc_mac(dacc &acc, float ah, float al, float ch, float cl) {
    float p = __fmul_rn(ah, ch);
    float pe = __fmaf_rn(ah, ch, -p);
    float t, e;
    two_sum(acc.S, p, t, e);
    acc.S = t;
    float lo = __fmaf_rn(ah, cl, pe);
    lo = __fmaf_rn(al, ch, lo);
    acc.s = __fadd_rn(acc.s, __fadd_rn(e, lo));
}

// Merge two accumulators (used by tree reductions).
__device__ __forceinline__ void dacc_add(dacc &acc, dacc o) {
    float t, e;
    two_sum(acc.S, o.S, t, e);
    acc.S = t;
    acc.s = __fadd_rn(acc.s, __fadd_rn(e, o.s));
}

__device__ __forceinline__ df dacc_result(dacc acc) {
    df r;
    two_sum(acc.S, acc.s, r.hi, r.lo);
    return r;
}

}  // namespace bttb
