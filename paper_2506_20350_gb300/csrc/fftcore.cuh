// Building blocks of the in-project FFTs shared by the strided passes, the fused two-level FFT and the
// fused y-level transform + block product: radix-2/3/4/5 butterflies, and Stockham stages over sequences
// held in shared memory.  Every rounding step is an explicit intrinsic (arith.cuh), so each kernel that
// runs the same stages gets the same bits.
#pragma once
#include "arith.cuh"
#include "internal.h"

namespace bttb {

// ---------------------------------------------------------------------------
// Radix butterflies.  sg = -1 for the forward transform (exp(-2 pi i kn/R)),
// +1 for the inverse (unnormalised).  The radix-3 and radix-5 forms are the
// usual symmetric splittings into sums and differences of mirrored inputs.
// ---------------------------------------------------------------------------
template <class A>
struct Butterfly {
    using C = typename A::C;
    using K = typename A::K;

    __device__ static void r2(C *v) {
        C a = A::add(v[0], v[1]), b = A::sub(v[0], v[1]);
        v[0] = a;
        v[1] = b;
    }
    __device__ static void r4(C *v, int sg) {
        C a0 = A::add(v[0], v[2]), a1 = A::sub(v[0], v[2]);
        C a2 = A::add(v[1], v[3]), a3 = A::mul_i(A::sub(v[1], v[3]), sg);
        v[0] = A::add(a0, a2);
        v[2] = A::sub(a0, a2);
        v[1] = A::add(a1, a3);
        v[3] = A::sub(a1, a3);
    }
    __device__ static void r3(C *v, int sg, K s3) {
        C s = A::add(v[1], v[2]), d = A::sub(v[1], v[2]);
        C y0 = A::add(v[0], s);
        C t = A::sub(v[0], A::half(s));
        C u = A::mul_i(A::mul_k(d, s3), sg);
        v[0] = y0;
        v[1] = A::add(t, u);
        v[2] = A::sub(t, u);
    }
    __device__ static void r5(C *v, int sg, K c1, K c2, K s1, K s2) {
        C a1 = A::add(v[1], v[4]), a2 = A::add(v[2], v[3]);
        C b1 = A::sub(v[1], v[4]), b2 = A::sub(v[2], v[3]);
        C y0 = A::add(A::add(v[0], a1), a2);
        C t1 = A::add(A::add(v[0], A::mul_k(a1, c1)), A::mul_k(a2, c2));
        C t2 = A::add(A::add(v[0], A::mul_k(a1, c2)), A::mul_k(a2, c1));
        C u1 = A::mul_i(A::add(A::mul_k(b1, s1), A::mul_k(b2, s2)), sg);
        C u2 = A::mul_i(A::sub(A::mul_k(b1, s2), A::mul_k(b2, s1)), sg);
        v[0] = y0;
        v[1] = A::add(t1, u1);
        v[4] = A::sub(t1, u1);
        v[2] = A::add(t2, u2);
        v[3] = A::sub(t2, u2);
    }
};

template <class A>
__device__ __forceinline__ typename A::K real_const(const typename A::C &c);
template <>
__device__ __forceinline__ double real_const<F64N>(const double2 &c) { return c.x; }
template <>
__device__ __forceinline__ df real_const<DF64>(const cdf &c) { return df{c.rh, c.rl}; }
template <>
__device__ __forceinline__ float real_const<F32>(const float2 &c) { return c.x; }

template <class A>
__device__ __forceinline__ typename A::C scale_by(typename A::C v, double s);
template <>
__device__ __forceinline__ double2 scale_by<F64N>(double2 v, double s) { return make_double2(v.x * s, v.y * s); }
template <>
__device__ __forceinline__ cdf scale_by<DF64>(cdf v, double s) { return DF64::mul_k(v, df_from_double(s)); }
template <>
__device__ __forceinline__ float2 scale_by<F32>(float2 v, double s) {
    float f = (float)s;
    return make_float2(v.x * f, v.y * f);
}

struct Fft2Side {
    int M, nst;
    int radix[kMaxRadixStages];
    unsigned nsmagic[kMaxRadixStages];
};

// One Stockham stage of radix R over nb sequences of length m*R with element stride es: sequence t starts
// at offset (t div g) * gs + (t mod g) (g = 1: t * gs).  The flat work index is split by multiply-high
// divisions (exact below 2^16).
template <class A, int R, bool INV>
__device__ __forceinline__ void fft2_stage(const typename A::C *__restrict__ src, typename A::C *__restrict__ dst,
                                           const typename A::C *tw, int m, int Ns, unsigned nsmagic, int tstep,
                                           int es, int nb, unsigned nbmagic, int gs, typename A::K s3,
                                           typename A::K c1, typename A::K c2, typename A::K s1, typename A::K s2) {
    using C = typename A::C;
    constexpr int sg = INV ? 1 : -1;
    const int total = m * nb;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int j = nb == 1 ? idx : (int)__umulhi((unsigned)idx, nbmagic);
        const int off = (idx - j * nb) * gs;
        const int q = Ns == 1 ? j : (int)__umulhi((unsigned)j, nsmagic);
        const int k = j - q * Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = sld(src + (j + r * m) * es + off);
        if (k != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = A::cmul(v[r], tw[r * k * tstep], INV);
        }
        if constexpr (R == 2) Butterfly<A>::r2(v);
        else if constexpr (R == 3) Butterfly<A>::r3(v, sg, s3);
        else if constexpr (R == 4) Butterfly<A>::r4(v, sg);
        else Butterfly<A>::r5(v, sg, c1, c2, s1, s2);
        const int dbase = q * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) sst(dst + (dbase + r * Ns) * es + off, v[r]);
    }
}

// All stages of one level; returns the buffer that holds the result.
template <class A, bool INV>
__device__ typename A::C *fft2_level(typename A::C *src, typename A::C *dst, const typename A::C *tw,
                                      const Fft2Side &sd, int es, int nb, int gs) {
    using C = typename A::C;
    using K = typename A::K;
    const int M = sd.M;
    const K s3 = real_const<A>(tw[M + 4]);
    const K c1 = real_const<A>(tw[M + 0]), c2 = real_const<A>(tw[M + 1]);
    const K s1 = real_const<A>(tw[M + 2]), s2 = real_const<A>(tw[M + 3]);
    const unsigned nbm = nb > 1 ? (unsigned)((0x100000000ull + nb - 1) / nb) : 0u;
    int Ns = 1;
    for (int s = 0; s < sd.nst; ++s) {
        const int R = sd.radix[s];
        const int m = M / R, tstep = M / (Ns * R);
        const unsigned mg = sd.nsmagic[s];
        switch (R) {
            case 2: fft2_stage<A, 2, INV>(src, dst, tw, m, Ns, mg, tstep, es, nb, nbm, gs, s3, c1, c2, s1, s2); break;
            case 3: fft2_stage<A, 3, INV>(src, dst, tw, m, Ns, mg, tstep, es, nb, nbm, gs, s3, c1, c2, s1, s2); break;
            case 4: fft2_stage<A, 4, INV>(src, dst, tw, m, Ns, mg, tstep, es, nb, nbm, gs, s3, c1, c2, s1, s2); break;
            default: fft2_stage<A, 5, INV>(src, dst, tw, m, Ns, mg, tstep, es, nb, nbm, gs, s3, c1, c2, s1, s2); break;
        }
        __syncthreads();
        C *t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

constexpr int kFftThreads = 256;

// One Stockham stage of radix R over the P interleaved sequences: thread (pp, j0) takes the butterflies
// j = j0, j0 + jstep, ... of batch index pp.  With Ns the product of the earlier radices, butterfly j reads
// src[j + r m] (m = M/R), twiddles inputs r >= 1 by w^(r k tstep) (k = j mod Ns) and writes
// dst[(j div Ns) Ns R + k + r Ns].  j div Ns is one high multiply by nsmagic = ceil(2^32 / Ns), exact for
// j, Ns < 2^16.
template <class A, int R, bool INV>
__device__ __forceinline__ void fft_stage(const typename A::C *__restrict__ src, typename A::C *__restrict__ dst,
                                          const typename A::C *tw, int m, int Ns, unsigned nsmagic, int tstep,
                                          int lP, int pp, int j0, int jstep, typename A::K s3, typename A::K c1,
                                          typename A::K c2, typename A::K s1, typename A::K s2) {
    using C = typename A::C;
    constexpr int sg = INV ? 1 : -1;
    for (int j = j0; j < m; j += jstep) {
        const int q = Ns == 1 ? j : (int)__umulhi((unsigned)j, nsmagic);
        const int k = j - q * Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = sld(src + ((j + r * m) << lP) + pp);
        if (k != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = A::cmul(v[r], tw[r * k * tstep], INV);
        }
        if constexpr (R == 2) Butterfly<A>::r2(v);
        else if constexpr (R == 3) Butterfly<A>::r3(v, sg, s3);
        else if constexpr (R == 4) Butterfly<A>::r4(v, sg);
        else Butterfly<A>::r5(v, sg, c1, c2, s1, s2);
        const int dbase = q * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) sst(dst + ((dbase + r * Ns) << lP) + pp, v[r]);
    }
}

// All stages of one strided pass over the P interleaved sequences of a CTA (buffers [n][P], n < M),
// called after a barrier that follows the twiddle staging; returns the buffer that holds the result.
template <class A, bool INV>
__device__ __forceinline__ typename A::C *fft_pass_stages(const FftPass &a, typename A::C *src, typename A::C *dst,
                                                          const typename A::C *tw) {
    using C = typename A::C;
    using K = typename A::K;
    const int M = a.M, lP = a.log2P;
    const int tid = threadIdx.x, nt = kFftThreads;
    const int pp = tid & (a.P - 1), j0 = tid >> lP, jstep = nt >> lP;
    const K s3 = real_const<A>(tw[M + 4]);
    const K c1 = real_const<A>(tw[M + 0]), c2 = real_const<A>(tw[M + 1]);
    const K s1 = real_const<A>(tw[M + 2]), s2 = real_const<A>(tw[M + 3]);
    int Ns = 1;
    for (int s = 0; s < a.nst; ++s) {
        const int R = a.radix[s];
        const int m = M / R;
        const int tstep = M / (Ns * R);
        const unsigned mg = a.nsmagic[s];
        switch (R) {
            case 2: fft_stage<A, 2, INV>(src, dst, tw, m, Ns, mg, tstep, lP, pp, j0, jstep, s3, c1, c2, s1, s2); break;
            case 3: fft_stage<A, 3, INV>(src, dst, tw, m, Ns, mg, tstep, lP, pp, j0, jstep, s3, c1, c2, s1, s2); break;
            case 4: fft_stage<A, 4, INV>(src, dst, tw, m, Ns, mg, tstep, lP, pp, j0, jstep, s3, c1, c2, s1, s2); break;
            default: fft_stage<A, 5, INV>(src, dst, tw, m, Ns, mg, tstep, lP, pp, j0, jstep, s3, c1, c2, s1, s2); break;
        }
        __syncthreads();
        C *t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

}  // namespace bttb
