// Number systems the kernels are instantiated for.  Each provides the complex
// operations a radix butterfly and a block product need, plus conversions from
// and to the storage types a caller's vectors may have.  Every rounding step is
// an explicit intrinsic (no compiler contraction), so the same butterfly gives
// the same bits in every kernel that runs it (the strided FFT passes and the
// fused two-level FFT).
//
//   F64N : IEEE binary64 (double2), on the binary64 pipe
//   DF64 : double-float complex (cdf = float4), on the binary32 pipes
//   F32  : IEEE binary32 (float2)
#pragma once
#include "check.cuh"
#include <cuda_runtime.h>
#include "df64.cuh"

namespace bttb {

// Real constants of the radix-3 / radix-5 butterflies, per number system.
struct RadixConsts {
    double c1, c2, s1, s2, s3;   // cos(2pi/5), cos(4pi/5), sin(2pi/5), sin(4pi/5), sin(pi/3)
};

struct F64N {
    using C = double2;           // storage and arithmetic
    using K = double;            // real constant
    static constexpr int kind = 2;
    __device__ static C zero() { return make_double2(0.0, 0.0); }
    __device__ static C add(C a, C b) { return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)); }
    __device__ static C sub(C a, C b) { return make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y)); }
    // a * (s i), s = +1 or -1
    __device__ static C mul_i(C a, int s) { return s > 0 ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x); }
    __device__ static C mul_k(C a, K k) { return make_double2(__dmul_rn(a.x, k), __dmul_rn(a.y, k)); }
    __device__ static C half(C a) { return make_double2(__dmul_rn(0.5, a.x), __dmul_rn(0.5, a.y)); }
    // a * w (conj(w) when cj)
    __device__ static C cmul(C a, C w, bool cj) {
        double wi = cj ? -w.y : w.y;
        return make_double2(__fma_rn(a.x, w.x, -__dmul_rn(a.y, wi)), __fma_rn(a.x, wi, __dmul_rn(a.y, w.x)));
    }
    __device__ static K kconst(double v) { return v; }
    __device__ static C from_c128(double2 v) { return v; }
    __device__ static C from_c64(float2 v) { return make_double2(v.x, v.y); }
    __device__ static C from_cdf(float4 v) { return make_double2((double)v.x + v.z, (double)v.y + v.w); }
    __device__ static double2 to_c128(C v) { return v; }
    __device__ static float2 to_c64(C v) { return make_float2((float)v.x, (float)v.y); }
    __device__ static float4 to_cdf(C v) {
        df r = df_from_double(v.x), i = df_from_double(v.y);
        return make_float4(r.hi, i.hi, r.lo, i.lo);
    }
};

struct DF64 {
    using C = cdf;
    using K = df;
    static constexpr int kind = 0;
    __device__ static C zero() { return cdf{0.f, 0.f, 0.f, 0.f}; }
    __device__ static df re(C a) { return df{a.rh, a.rl}; }
    __device__ static df im(C a) { return df{a.ih, a.il}; }
    __device__ static C mk(df r, df i) { return cdf{r.hi, i.hi, r.lo, i.lo}; }
    __device__ static C add(C a, C b) { return mk(df_add(re(a), re(b)), df_add(im(a), im(b))); }
    __device__ static C sub(C a, C b) { return mk(df_sub(re(a), re(b)), df_sub(im(a), im(b))); }
    __device__ static C mul_i(C a, int s) {
        return s > 0 ? mk(df_neg(im(a)), re(a)) : mk(im(a), df_neg(re(a)));
    }
    __device__ static C mul_k(C a, K k) { return mk(df_mul(re(a), k), df_mul(im(a), k)); }
    __device__ static C half(C a) { return mk(df_scale_pow2(re(a), 0.5f), df_scale_pow2(im(a), 0.5f)); }
    __device__ static C cmul(C a, C w, bool cj) {
        df wr = re(w), wi = im(w);
        if (cj) wi = df_neg(wi);
        // (ar + i ai)(wr + i wi) = (ar wr - ai wi) + i (ar wi + ai wr)
        df r = df_dot2(re(a), wr, im(a), wi, -1.f);
        df i = df_dot2(re(a), wi, im(a), wr, 1.f);
        return mk(r, i);
    }
    __device__ static K kconst(double v) { return df_from_double(v); }
    __device__ static C from_c128(double2 v) { return mk(df_from_double(v.x), df_from_double(v.y)); }
    __device__ static C from_c64(float2 v) { return cdf{v.x, v.y, 0.f, 0.f}; }
    __device__ static C from_cdf(float4 v) { return cdf{v.x, v.y, v.z, v.w}; }
    __device__ static double2 to_c128(C v) { return make_double2(df_to_double(re(v)), df_to_double(im(v))); }
    __device__ static float2 to_c64(C v) { return make_float2(v.rh + v.rl, v.ih + v.il); }
    __device__ static float4 to_cdf(C v) { return make_float4(v.rh, v.ih, v.rl, v.il); }
};

struct F32 {
    using C = float2;
    using K = float;
    static constexpr int kind = 1;
    __device__ static C zero() { return make_float2(0.f, 0.f); }
    __device__ static C add(C a, C b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
    __device__ static C sub(C a, C b) { return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y)); }
    __device__ static C mul_i(C a, int s) { return s > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x); }
    __device__ static C mul_k(C a, K k) { return make_float2(__fmul_rn(a.x, k), __fmul_rn(a.y, k)); }
    __device__ static C half(C a) { return make_float2(__fmul_rn(0.5f, a.x), __fmul_rn(0.5f, a.y)); }
    __device__ static C cmul(C a, C w, bool cj) {
        float wi = cj ? -w.y : w.y;
        return make_float2(__fmaf_rn(a.x, w.x, -__fmul_rn(a.y, wi)), __fmaf_rn(a.x, wi, __fmul_rn(a.y, w.x)));
    }
    __device__ static K kconst(double v) { return (float)v; }
    __device__ static C from_c128(double2 v) { return make_float2((float)v.x, (float)v.y); }
    __device__ static C from_c64(float2 v) { return v; }
    __device__ static C from_cdf(float4 v) { return make_float2(v.x, v.y); }
    __device__ static double2 to_c128(C v) { return make_double2(v.x, v.y); }
    __device__ static float2 to_c64(C v) { return v; }
    __device__ static float4 to_cdf(C v) { return make_float4(v.x, v.y, 0.f, 0.f); }
};

// Storage formats of a vector a kernel reads or writes.
enum VecFmt { FMT_C128 = 0, FMT_C64 = 1, FMT_CDF = 2 };

// The storage format a number system keeps its own intermediates in.
template <class A> constexpr int native_fmt = A::kind == 2 ? FMT_C128 : (A::kind == 0 ? FMT_CDF : FMT_C64);

template <class A, int FMT>
__device__ __forceinline__ typename A::C load_vec(const void *base, long idx) {
    if constexpr (FMT == FMT_C128) return A::from_c128(gld(reinterpret_cast<const double2 *>(base) + idx));
    else if constexpr (FMT == FMT_C64) return A::from_c64(gld(reinterpret_cast<const float2 *>(base) + idx));
    else return A::from_cdf(gld(reinterpret_cast<const float4 *>(base) + idx));
}

template <class A, int FMT>
__device__ __forceinline__ void store_vec(void *base, long idx, typename A::C v) {
    if constexpr (FMT == FMT_C128) gst(reinterpret_cast<double2 *>(base) + idx, A::to_c128(v));
    else if constexpr (FMT == FMT_C64) gst(reinterpret_cast<float2 *>(base) + idx, A::to_c64(v));
    else gst(reinterpret_cast<float4 *>(base) + idx, A::to_cdf(v));
}

}  // namespace bttb
