// Accumulators of the per-bin block product v_k = G_k u_k (Eq. (multL)) in each number system, shared by
// the block-product kernels: binary32 and binary64 FMA chains, double-float with compensated (Dot2)
// accumulation; and the spectrum element type a number system reads (the double-float product reads two
// binary32 planes).
#pragma once
#include "arith.cuh"

namespace bttb {

template <class A> struct Acc;

template <> struct Acc<DF64> {
    dacc re, im;
    __device__ void zero() { re = dacc{0.f, 0.f}; im = dacc{0.f, 0.f}; }
    __device__ void mac(float2 gh, float2 gl, cdf u) {
        // re += g.re u.re - g.im u.im ; im += g.re u.im + g.im u.re
        dacc_mac(re, gh.x, gl.x, u.rh, u.rl);
        dacc_mac(re, -gh.y, -gl.y, u.ih, u.il);
        dacc_mac(im, gh.x, gl.x, u.ih, u.il);
        dacc_mac(im, gh.y, gl.y, u.rh, u.rl);
    }
    __device__ cdf result() const {
        df r = dacc_result(re), i = dacc_result(im);
        return cdf{r.hi, i.hi, r.lo, i.lo};
    }
    __device__ void merge(const Acc &o) {
        dacc_add(re, o.re);
        dacc_add(im, o.im);
    }
};

template <> struct Acc<F32> {
    float2 a;
    __device__ void zero() { a = make_float2(0.f, 0.f); }
    __device__ void mac(float2 g, float2, float2 u) {
        a.x = fmaf(g.x, u.x, a.x);
        a.x = fmaf(-g.y, u.y, a.x);
        a.y = fmaf(g.x, u.y, a.y);
        a.y = fmaf(g.y, u.x, a.y);
    }
    __device__ float2 result() const { return a; }
    __device__ void merge(const Acc &o) {
        a.x = __fadd_rn(a.x, o.a.x);
        a.y = __fadd_rn(a.y, o.a.y);
    }
};

template <> struct Acc<F64N> {
    double2 a;
    __device__ void zero() { a = make_double2(0.0, 0.0); }
    __device__ void mac(double2 g, double2, double2 u) {
        a.x = fma(g.x, u.x, a.x);
        a.x = fma(-g.y, u.y, a.x);
        a.y = fma(g.x, u.y, a.y);
        a.y = fma(g.y, u.x, a.y);
    }
    __device__ double2 result() const { return a; }
    __device__ void merge(const Acc &o) {
        a.x = __dadd_rn(a.x, o.a.x);
        a.y = __dadd_rn(a.y, o.a.y);
    }
};

template <class A> struct GElem { using T = float2; static constexpr int planes = 1; };
template <> struct GElem<DF64> { using T = float2; static constexpr int planes = 2; };
template <> struct GElem<F64N> { using T = double2; static constexpr int planes = 1; };

// Two consecutive rows of one spectrum column, loaded as one vector.
template <class GT> struct Pair;
template <> struct Pair<float2> {
    using V = float4;
    __device__ static float2 lo(const V &v) { return make_float2(v.x, v.y); }
    __device__ static float2 hi(const V &v) { return make_float2(v.z, v.w); }
};
template <> struct Pair<double2> {
    struct __align__(32) V { double2 a, b; };
    __device__ static double2 lo(const V &v) { return v.a; }
    __device__ static double2 hi(const V &v) { return v.b; }
};

}  // namespace bttb
