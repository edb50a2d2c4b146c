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
