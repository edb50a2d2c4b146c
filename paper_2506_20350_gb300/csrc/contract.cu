// Per-bin block product  v_k = G_k u_k  (Eq. (multL): the block-diagonal
// matrix diag_b(F C_1) applied to the transformed vector), for every bin k of
// the mx x my grid and up to kContractKC right-hand sides at a time.
//
// This kernel streams the whole spectrum once per product and is bound by HBM
// bandwidth.  Design:
//  - persistent CTAs (one per SM); bins are dealt out round-robin and a CTA
//    walks the column chunks of each of its bins in order;
//  - one producer warp issues bulk asynchronous copies (cp.async.bulk with an
//    evict-first L2 policy) of the spectrum chunk -- one plane for binary32 and
//    binary64, the hi and lo planes for double-float -- plus the bin's
//    transformed vectors into a ring of shared-memory stages guarded by
//    mbarrier transaction counts;
//  - eight consumer warps: thread (p, g) owns output row p and the g-th slice
//    of the chunk's columns; the spectrum is stored column-major per bin, so a
//    warp reads consecutive rows of one column (conflict-free) and the vector
//    entry is a broadcast;
//  - double-float accumulation is compensated (Dot2); the G partial sums of a
//    row are combined through shared memory at the end of each bin.
#include <cstdio>

#include "arith.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace bttb {

constexpr int kConsumerWarps = 8;
constexpr int kContractThreads = (kConsumerWarps + 1) * 32;
constexpr int kMaxStages = 8;

struct ContractArgs {
    const void *g0, *g1;          // spectrum planes (g1: double-float low plane)
    long gbs;                     // bin stride of a plane (elements)
    const void *u;                // transformed vectors, column c0 of the group
    void *v;
    long ubs;                     // bin stride of u/v (elements)
    int nbins, b, kc;             // kc = columns in this group (<= kContractKC)
    int Qc, nchunks, G, nstages;
    uint32_t st_bytes, off_g1, off_u, red_off;
    int *err;
};

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
};

template <class A> struct GElem { using T = float2; static constexpr int planes = 1; };
template <> struct GElem<DF64> { using T = float2; static constexpr int planes = 2; };
template <> struct GElem<F64N> { using T = double2; static constexpr int planes = 1; };

__host__ __device__ constexpr uint32_t round_up16(uint32_t x) { return (x + 15u) & ~15u; }
__host__ __device__ constexpr uint32_t round_up128(uint32_t x) { return (x + 127u) & ~127u; }

template <class A>
__global__ void __launch_bounds__(kContractThreads, 1) contract_kernel(const ContractArgs a) {
    using C = typename A::C;
    using GT = typename GElem<A>::T;
    constexpr int NPL = GElem<A>::planes;
    constexpr int KC = kContractKC;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + kMaxStages;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 2 * kMaxStages * sizeof(uint64_t));
    unsigned char *stages = smem + 256;
    C *red = reinterpret_cast<C *>(smem + a.red_off);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < a.nstages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    const int total = a.nbins * a.nchunks;
    const int b = a.b;

    if (warp == kConsumerWarps) {
        // ---------------- producer ----------------
        if (lane == 0) {
            const uint64_t pol_stream = l2_policy_evict_first();
            const uint64_t pol_keep = l2_policy_evict_last();
            int i = 0;
            int issued_last = -1;
            for (int w = blockIdx.x * a.nchunks; w < total; ++w, ++i) {
                if (w % a.nchunks == 0 && i > 0) w += (gridDim.x - 1) * a.nchunks;   // next bin of this CTA
                if (w >= total) break;
                const int s = i % a.nstages;
                const uint32_t ph = (uint32_t)(i / a.nstages) & 1u;
                if (!mbar_wait_bounded(&empty[s], ph ^ 1u, abort_flag)) break;
                const int bin = w / a.nchunks, ch = w % a.nchunks;
                const int q0 = ch * a.Qc;
                const int qn = min(a.Qc, b - q0);
                const uint32_t gbytes = round_up16((uint32_t)(qn * b) * (uint32_t)sizeof(GT));
                const uint32_t ubytes = round_up16((uint32_t)(a.kc * b) * (uint32_t)sizeof(C));
                unsigned char *st = stages + (size_t)s * a.st_bytes;
                mbar_arrive_expect_tx(&full[s], gbytes * NPL + ubytes);
                const long goff = (long)bin * a.gbs + (long)q0 * b;
                bulk_g2s(st, reinterpret_cast<const GT *>(a.g0) + goff, gbytes, &full[s], pol_stream);
                if (NPL == 2)
                    bulk_g2s(st + a.off_g1, reinterpret_cast<const GT *>(a.g1) + goff, gbytes, &full[s], pol_stream);
                bulk_g2s(st + a.off_u, reinterpret_cast<const C *>(a.u) + (long)bin * a.ubs, ubytes, &full[s],
                         pol_keep);
                issued_last = i;
            }
            if (*abort_flag) {
                // Drain the copies that may still be in flight before exiting.
                for (int d = issued_last; d >= 0 && d > issued_last - a.nstages; --d)
                    mbar_wait_drain(&full[d % a.nstages], (uint32_t)(d / a.nstages) & 1u);
                atomicOr(a.err, DEVERR_TIMEOUT);
            }
        }
        return;
    }

    // ---------------- consumers ----------------
    const int nact = a.G * b;
    const bool active = tid < nact;
    const int p = active ? tid % b : 0;
    const int g = active ? tid / b : 0;
    Acc<A> acc[KC];
    int i = 0;
    for (int w = blockIdx.x * a.nchunks; w < total; ++w, ++i) {
        if (w % a.nchunks == 0 && i > 0) w += (gridDim.x - 1) * a.nchunks;       // next bin of this CTA
        if (w >= total) break;
        const int s = i % a.nstages;
        const uint32_t ph = (uint32_t)(i / a.nstages) & 1u;
        const int bin = w / a.nchunks, ch = w % a.nchunks;
        const bool ok = mbar_wait_bounded(&full[s], ph, abort_flag);
        if (!ok && lane == 0) atomicOr(a.err, DEVERR_TIMEOUT);
        if (ch == 0) {
#pragma unroll
            for (int c = 0; c < KC; ++c) acc[c].zero();
        }
        if (ok && active) {
            const int q0 = ch * a.Qc;
            const int qn = min(a.Qc, b - q0);
            const int qa = (g * qn) / a.G, qb = ((g + 1) * qn) / a.G;
            const unsigned char *st = stages + (size_t)s * a.st_bytes;
            const GT *gs0 = reinterpret_cast<const GT *>(st);
            const GT *gs1 = reinterpret_cast<const GT *>(st + a.off_g1);
            const C *us = reinterpret_cast<const C *>(st + a.off_u);
#pragma unroll 4
            for (int q = qa; q < qb; ++q) {
                const GT gv0 = gs0[q * b + p];
                const GT gv1 = NPL == 2 ? gs1[q * b + p] : gv0;
#pragma unroll
                for (int c = 0; c < KC; ++c)
                    if (c < a.kc) acc[c].mac(gv0, gv1, us[c * b + q0 + q]);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (ch == a.nchunks - 1) {
            if (active) {
#pragma unroll
                for (int c = 0; c < KC; ++c)
                    if (c < a.kc) red[((long)g * KC + c) * b + p] = acc[c].result();
            }
            named_barrier_sync(1, kConsumerWarps * 32);
            for (int idx = tid; idx < a.kc * b; idx += kConsumerWarps * 32) {
                const int c = idx / b, pr = idx % b;
                C sum = red[(long)c * b + pr];
                for (int gg = 1; gg < a.G; ++gg) sum = A::add(sum, red[((long)gg * KC + c) * b + pr]);
                store_vec<A, native_fmt<A>>(a.v, (long)bin * a.ubs + (long)c * b + pr, sum);
            }
            named_barrier_sync(1, kConsumerWarps * 32);
        }
    }
}

template <class A>
constexpr int prec_of() { return A::kind == 0 ? BTTB_MV_FP64 : (A::kind == 1 ? BTTB_MV_FP32 : BTTB_MV_FP64_NATIVE); }

template <class A>
static int launch_contract(Plan *p, const void *u, void *v, int k) {
    using C = typename A::C;
    using GT = typename GElem<A>::T;
    constexpr int NPL = GElem<A>::planes;
    const int b = p->b;
    ContractArgs a{};
    a.gbs = p->gbs;
    a.ubs = p->ubs;
    a.nbins = (int)p->bins;
    a.b = b;
    a.err = p->d_err;
    a.G = (kConsumerWarps * 32) / b;
    if (a.G < 1) a.G = 1;
    if constexpr (A::kind == 0) {
        a.g0 = p->ghat_hi;
        a.g1 = p->ghat_lo;
    } else if constexpr (A::kind == 1) {
        a.g0 = p->ghat_hi;
        a.g1 = nullptr;
    } else {
        a.g0 = p->ghat_f64;
        a.g1 = nullptr;
    }
    if (!a.g0 || (NPL == 2 && !a.g1))
        return set_error(p, BTTB_ERR_INVALID_ARG, "plan does not keep the spectrum copy this precision reads");

    const size_t budget = p->smem_optin > 0 ? p->smem_optin : 200 * 1024;
    const uint32_t ubytes_max = round_up128((uint32_t)(kContractKC * b) * sizeof(C));
    const uint32_t red_bytes = round_up128((uint32_t)(a.G * kContractKC * b) * sizeof(C));
    // Largest chunk of columns such that >= 3 stages fit (>= 2 for very wide blocks).
    int Qc = b;
    int nst = 0;
    for (; Qc >= 1; --Qc) {
        if (Qc < b && (Qc * b) % 2) continue;             // keep 16-byte aligned chunk starts
        uint32_t gbytes = round_up128((uint32_t)(Qc * b) * sizeof(GT));
        uint32_t st = gbytes * NPL + ubytes_max;
        size_t avail = budget - 256 - red_bytes;
        int ns = (int)(avail / st);
        if (ns > kMaxStages) ns = kMaxStages;
        if (ns >= 3 || (ns >= 2 && Qc <= 8)) {
            nst = ns;
            break;
        }
    }
    if (Qc < 1 || nst < 2) return set_error(p, BTTB_ERR_INVALID_ARG, "block too large for the shared-memory pipeline");
    a.Qc = Qc;
    a.nchunks = (b + Qc - 1) / Qc;
    a.nstages = nst;
    const uint32_t gbytes = round_up128((uint32_t)(Qc * b) * sizeof(GT));
    a.off_g1 = gbytes;
    a.off_u = gbytes * NPL;
    a.st_bytes = gbytes * NPL + ubytes_max;
    a.red_off = 256 + a.st_bytes * nst;
    const size_t smem = a.red_off + red_bytes;

    auto kern = contract_kernel<A>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return check_cuda(p, e, "contract smem attribute");
    const int grid = a.nbins < p->nsm ? a.nbins : p->nsm;     // whole bins per CTA, chunks in order
    for (int c0 = 0; c0 < k; c0 += kContractKC) {
        a.kc = (k - c0) < kContractKC ? (k - c0) : kContractKC;
        a.u = reinterpret_cast<const C *>(u) + (long)c0 * b;
        a.v = reinterpret_cast<C *>(v) + (long)c0 * b;
        const int tok = prof_begin(p, BTTB_K_BLOCK_PRODUCT_PREC + prec_of<A>());
        kern<<<grid, kContractThreads, smem, p->stream>>>(a);
        count_launch(p);
        // algorithmic bytes: spectrum planes once, transformed vectors in and out
        prof_end(p, tok, (double)a.nbins * ((double)b * b * sizeof(GT) * NPL + 2.0 * a.kc * b * sizeof(C)));
        e = cudaGetLastError();
        if (e != cudaSuccess) return check_cuda(p, e, "contract launch");
    }
    return BTTB_OK;
}

int contract_launch(Plan *p, int prec, const void *u, void *v, int k) {
    switch (prec) {
        case PREC_F32: return launch_contract<F32>(p, u, v, k);
        case PREC_F64N: return launch_contract<F64N>(p, u, v, k);
        default: return launch_contract<DF64>(p, u, v, k);
    }
}

}  // namespace bttb
