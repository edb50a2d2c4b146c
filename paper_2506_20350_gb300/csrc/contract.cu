// Per-bin block product  v_k = G_k u_k  (Eq. (multL): the block-diagonal
// matrix diag_b(F C_1) applied to the transformed vector), for every bin k of
// the mx x my grid and up to four right-hand sides per launch.
//
// This kernel streams the whole spectrum once per product and is bound by HBM
// bandwidth.  Design:
//  - persistent CTAs (one per SM) of eight warps; bins are dealt out
//    round-robin over CTAs, then over the CTA's warps, and one warp owns one
//    bin at a time (lane l accumulates rows l*R .. l*R+R-1 over all columns),
//    so a bin needs no cross-warp reduction and no barrier;
//  - each warp streams its bins' column chunks through a private ring of
//    shared-memory stages: lane 0 issues bulk asynchronous copies
//    (cp.async.bulk, evict-first L2 policy for the spectrum) of the spectrum
//    chunk -- one plane for binary32 and binary64, the hi and lo planes for
//    double-float -- plus the bin's transformed vectors, one mbarrier per stage
//    counting the bytes in;
//  - the spectrum is stored column-major per bin, so a lane reads R
//    consecutive rows of one column (a 16-byte vector for R = 2) and the
//    vector entry is a broadcast;
//  - the spectrum does not depend on the preceding kernel, so each warp starts
//    streaming its first chunk before the programmatic-dependent-launch wait;
//    only the transformed vectors wait for the preceding FFT pass;
//  - double-float accumulation is compensated (Dot2); every mbarrier wait is
//    bounded by the global timer and reports a timeout instead of hanging.
// A second kernel (contract_multi_kernel, below) covers many right-hand sides.
#include <cstdio>

#include "arith.cuh"
#include "blockprod.cuh"
#include "fftcore.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace bttb {

constexpr int kConsumerWarps = 8;
constexpr int kMaxStages = 8;


struct ContractArgs {
    const void *g0, *g1;          // spectrum planes (g1: double-float low plane)
    long gbs;                     // bin stride of a plane (elements)
    const void *u;                // transformed vectors, column c0 of the group
    void *v;
    long ubs;                     // bin stride of u/v (elements)
    int nbins, b, kc;             // kc = columns in this group (<= the launch width KC)
    const int *active;            // optional per-column flags of this group (offset to column c0)
    int Qc, nchunks, G, nstages;
    uint32_t st_bytes, off_g1, off_u, red_off;
    int *err;
    unsigned long long wait_ns;   // bound of every pipeline wait
    int withhold;                 // test hook: warp 0 of CTA 0 withholds the arrival of its first item
};

__host__ __device__ constexpr uint32_t round_up16(uint32_t x) { return (x + 15u) & ~15u; }
__host__ __device__ constexpr uint32_t round_up128(uint32_t x) { return (x + 127u) & ~127u; }

// KC: right-hand sides per launch (compile time); R: rows per lane (b <= 32 R).
//
// One warp owns one bin at a time: lane l accumulates rows l*R .. l*R+R-1 over
// all columns, so a bin needs no cross-warp reduction and no barrier.  Each
// warp streams its bins' column chunks through a private ring of kWarpStages
// shared-memory stages (lane 0 issues the bulk copies kWarpStages-1 items
// ahead; an mbarrier per stage counts the bytes in).  Bins are dealt out
// round-robin over CTAs, then over the CTA's warps.
constexpr int kWarpStages = 2;

template <class A, int KC, int R, bool VEC>
__global__ void __launch_bounds__(kConsumerWarps * 32, 1) contract_kernel(const ContractArgs a) {
    using C = typename A::C;
    using GT = typename GElem<A>::T;
    constexpr int NPL = GElem<A>::planes;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem) + warp * kWarpStages;
    unsigned char *stages = smem + 256 + (size_t)warp * kWarpStages * a.st_bytes;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 8 * kConsumerWarps * kWarpStages);
    if (threadIdx.x == 0) *abort_flag = 0;
    if (lane == 0) {
        for (int s = 0; s < kWarpStages; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const int b = a.b;
    // bins of this warp: blockIdx.x + gridDim.x * (warp + kConsumerWarps * r)
    const int first = blockIdx.x + gridDim.x * warp;
    const int step = gridDim.x * kConsumerWarps;
    const int nbw = first < a.nbins ? (a.nbins - 1 - first) / step + 1 : 0;
    const int nitems = nbw * a.nchunks;
    const uint64_t pol_stream = l2_policy_evict_first();
    const uint64_t pol_keep = l2_policy_evict_last();

    // An item's stage fills in two parts: the spectrum chunk (expect_tx, no arrival) and the bin's
    // transformed vectors (arrive.expect_tx); the phase completes when both have landed.
    auto issue_g = [&](int it) {
        const int s = it % kWarpStages;
        const int bin = first + step * (it / a.nchunks), ch = it % a.nchunks;
        const int q0 = ch * a.Qc;
        const int qn = min(a.Qc, b - q0);
        const uint32_t gbytes = round_up16((uint32_t)(qn * b) * (uint32_t)sizeof(GT));
        unsigned char *st = stages + (size_t)s * a.st_bytes;
        mbar_expect_tx(&full[s], gbytes * NPL);
        const long goff = (long)bin * a.gbs + (long)q0 * b;
        bulk_g2s(st, reinterpret_cast<const GT *>(a.g0) + goff, gbytes, &full[s], pol_stream);
        if (NPL == 2)
            bulk_g2s(st + a.off_g1, reinterpret_cast<const GT *>(a.g1) + goff, gbytes, &full[s], pol_stream);
    };
    // test hook: the first item of warp 0 of CTA 0 gets its bytes but not its arrival, so its wait runs out
    const bool withheld0 = a.withhold && blockIdx.x == 0 && warp == 0;
    auto issue_u = [&](int it) {
        const int s = it % kWarpStages;
        const int bin = first + step * (it / a.nchunks);
        const uint32_t ubytes = round_up16((uint32_t)(a.kc * b) * (uint32_t)sizeof(C));
        unsigned char *st = stages + (size_t)s * a.st_bytes;
        if (withheld0 && it == 0) mbar_expect_tx(&full[s], ubytes);
        else mbar_arrive_expect_tx(&full[s], ubytes);
        bulk_g2s(st + a.off_u, reinterpret_cast<const C *>(a.u) + (long)bin * a.ubs, ubytes, &full[s], pol_keep);
    };
    // The spectrum does not depend on the preceding kernel: start streaming it before the
    // dependency wait, so that its first DRAM round trip overlaps that kernel's tail.
    const int npre = min(kWarpStages - 1, nitems);
    if (lane == 0)
        for (int it = 0; it < npre; ++it) issue_g(it);
    pdl_wait();
    if (a.active) {                                        // skip a group of finished columns (uniform)
        bool any = false;
        for (int c = 0; c < a.kc; ++c) any |= a.active[c] != 0;
        if (!any) {
            // let the prefetched copies land before the CTA's shared memory goes away
            if (lane == 0)
                for (int it = 0; it < npre; ++it) {
                    mbar_arrive(&full[it % kWarpStages]);
                    mbar_wait_drain(&full[it % kWarpStages], 0u);
                }
            return;
        }
    }
    if (lane == 0)
        for (int it = 0; it < npre; ++it) issue_u(it);

    Acc<A> acc[KC][R];
    const int p0 = lane * R;
    bool failed = false;
    int it = 0;
    for (; it < nitems; ++it) {
        const int s = it % kWarpStages;
        const uint32_t ph = (uint32_t)(it / kWarpStages) & 1u;
        // keep kWarpStages-1 items in flight: the stage refilled now was released last iteration
        if (lane == 0 && it + kWarpStages - 1 < nitems) {
            issue_g(it + kWarpStages - 1);
            issue_u(it + kWarpStages - 1);
        }
        const int bin = first + step * (it / a.nchunks), ch = it % a.nchunks;
        // a wait that ran out (or saw another warp's abort) ends the warp's loop; the decision is uniform
        // over the warp, so no lane goes on to issue or read a stage the others gave up on
        const bool ok = mbar_wait_bounded(&full[s], ph, abort_flag, a.wait_ns);
        if (__any_sync(0xffffffffu, !ok)) {
            failed = true;
            break;
        }
        if (ch == 0) {
#pragma unroll
            for (int c = 0; c < KC; ++c)
#pragma unroll
                for (int r = 0; r < R; ++r) acc[c][r].zero();
        }
        {
            const int q0 = ch * a.Qc;
            const int qn = min(a.Qc, b - q0);
            const unsigned char *st = stages + (size_t)s * a.st_bytes;
            const GT *gs0 = reinterpret_cast<const GT *>(st) + p0;
            const GT *gs1 = reinterpret_cast<const GT *>(st + a.off_g1) + p0;
            const C *us = reinterpret_cast<const C *>(st + a.off_u) + q0;
            if (p0 < b) {
#pragma unroll 2
                for (int q = 0; q < qn; ++q) {
                    if constexpr (R == 2 && VEC) {               // b even: row pairs are 16-byte aligned
                        using PV = typename Pair<GT>::V;
                        const PV v0 = *reinterpret_cast<const PV *>(gs0 + q * b);
                        const PV v1 = NPL == 2 ? *reinterpret_cast<const PV *>(gs1 + q * b) : v0;
#pragma unroll
                        for (int c = 0; c < KC; ++c) {
                            const C u = us[c * b + q];
                            acc[c][0].mac(Pair<GT>::lo(v0), Pair<GT>::lo(v1), u);
                            acc[c][1].mac(Pair<GT>::hi(v0), Pair<GT>::hi(v1), u);
                        }
                    } else {
                        GT v0[R], v1[R];
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            v0[r] = p0 + r < b ? gs0[q * b + r] : GT{};
                            v1[r] = NPL == 2 && p0 + r < b ? gs1[q * b + r] : v0[r];
                        }
#pragma unroll
                        for (int c = 0; c < KC; ++c) {
                            const C u = us[c * b + q];
#pragma unroll
                            for (int r = 0; r < R; ++r) acc[c][r].mac(v0[r], v1[r], u);
                        }
                    }
                }
            }
        }
        // all lanes are done reading stage s before lane 0 may refill it (next iteration)
        __syncwarp();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (ch == a.nchunks - 1) {
#pragma unroll
            for (int c = 0; c < KC; ++c)
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (c < a.kc && p0 + r < b)
                        store_vec<A, native_fmt<A>>(a.v, (long)bin * a.ubs + (long)c * b + p0 + r, acc[c][r].result());
        }
    }
    pdl_trigger();
    if (failed && lane == 0) {
        atomicOr(a.err, DEVERR_TIMEOUT);
        // Items it .. it+kWarpStages-1 were issued and not consumed, each into its own stage (every earlier
        // item completed its phase).  A withheld arrival is supplied now; then each item's copies are drained
        // (bounded) before the CTA's shared memory goes away.
        for (int d = it; d < nitems && d < it + kWarpStages; ++d) {
            if (withheld0 && d == 0) mbar_arrive(&full[d % kWarpStages]);
            mbar_wait_drain(&full[d % kWarpStages], (uint32_t)(d / kWarpStages) & 1u);
        }
    }
}

// ---------------------------------------------------------------------------
// The whole product in one persistent kernel (one CTA per SM, cooperative launch): the four strided FFT
// passes (x forward, y forward, y inverse, x inverse: App. B) and the block product above run as phases,
// separated by grid-wide barriers.  Each warp's spectrum ring is filled at kernel start, so the first
// spectrum stages land while the forward transforms run, and no launch gap separates the phases.  The
// phases run the same stages and the same per-lane accumulation as the separate kernels, so the result is
// bit for bit the one of the strided-pass route.  Every CTA arrives at every barrier (a CTA whose wait ran
// out skips its work but keeps arriving), and every wait is bounded.
// ---------------------------------------------------------------------------
struct ProdArgs {
    FftPass px, py, pyi, pxi;     // x forward (x -> U), y forward (U -> u^), y inverse (v^ -> V), x inverse (V -> y)
    int fmt_x, fmt_y;             // formats of x and y
    ContractArgs c;               // the block product (u = u^, v = v^)
    unsigned long long *gbar;     // arrival counter: monotonic, 4 * gridDim.x arrivals per launch
    uint32_t off_tw, off_b0, off_b1, off_ring;
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Barrier k (0..3) of this launch.  Thread 0 arrives and waits (bounded) until every CTA has arrived;
// the launch's first arrival value fixes the base of its four barriers.
__device__ __forceinline__ void prod_grid_barrier(unsigned long long *gbar, int k, unsigned long long *base_s,
                                                  volatile int *abort, int *err, unsigned long long limit) {
    asm volatile("fence.proxy.async.global;" ::: "memory");   // generic writes before later bulk-copy reads
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned long long old = atomicAdd(gbar, 1ull);
        const unsigned long long per = 4ull * gridDim.x;
        if (k == 0) *base_s = old - old % per;
        const unsigned long long target = *base_s + (unsigned long long)(k + 1) * gridDim.x;
        if (old + 1 < target) {
            const unsigned long long t0 = global_ns();
            while (ld_acquire_u64(gbar) < target) {
                if (global_ns() - t0 > limit) {
                    *abort = 1;
                    atomicOr(err, DEVERR_TIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

template <class A>
__device__ __forceinline__ typename A::C prod_load(const void *base, long idx, int fmt) {
    if (fmt == FMT_C128) return A::from_c128(__ldcg(reinterpret_cast<const double2 *>(base) + idx));
    if (fmt == FMT_C64) return A::from_c64(__ldcg(reinterpret_cast<const float2 *>(base) + idx));
    return A::from_cdf(__ldcg(reinterpret_cast<const float4 *>(base) + idx));
}
template <class A>
__device__ __forceinline__ void prod_store(void *base, long idx, typename A::C v, int fmt) {
    if (fmt == FMT_C128) reinterpret_cast<double2 *>(base)[idx] = A::to_c128(v);
    else if (fmt == FMT_C64) reinterpret_cast<float2 *>(base)[idx] = A::to_c64(v);
    else reinterpret_cast<float4 *>(base)[idx] = A::to_cdf(v);
}

// One strided pass as a phase: the CTAs take its (outer index, basis chunk, column) items in turn.  Inputs
// are read through L2 (other CTAs wrote them in this launch).
template <class A, bool INV>
__device__ void prod_fft_phase(const FftPass &a, int infmt, int outfmt, typename A::C *tw, typename A::C *b0,
                               typename A::C *b1, bool skip) {
    using C = typename A::C;
    const int M = a.M, P = a.P, lP = a.log2P, tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < M + 5; i += nt) tw[i] = reinterpret_cast<const C *>(a.tw)[i];
    __syncthreads();
    const int npc = (a.pdim + P - 1) / P;
    const long items = (long)a.O * npc * a.ncols;
    const long sel = a.in_sel ? (long)(*a.in_sel) * a.in_sel_stride : 0;
    for (long it = blockIdx.x; it < items && !skip; it += gridDim.x) {
        const int o = (int)(it % a.O);
        const long rest = it / a.O;
        const int pc = (int)(rest % npc), c = (int)(rest / npc);
        if (a.active && !a.active[c]) continue;              // uniform per CTA
        const int p0 = pc * P;
        const long ibase = (long)c * a.in_cs + (long)o * a.in_os + sel;
        const double scl = a.in_scale ? a.in_scale[c] : 1.0;
        for (int idx = tid; idx < M * P; idx += nt) {
            const int n = idx >> lP, q = idx & (P - 1), pi = p0 + q;
            C v = A::zero();
            if (n < a.nin && pi < a.pdim) {
                v = prod_load<A>(a.in, ibase + (long)n * a.in_ns + pi, infmt);
                if (a.in_scale) v = scale_by<A>(v, scl);
            }
            b0[idx] = v;
        }
        __syncthreads();
        const C *res = fft_pass_stages<A, INV>(a, b0, b1, tw);
        const long obase = (long)c * a.out_cs + (long)o * a.out_os;
        for (int idx = tid; idx < a.nout * P; idx += nt) {
            const int n = idx >> lP, q = idx & (P - 1), pi = p0 + q;
            if (pi < a.pdim) prod_store<A>(a.out, obase + (long)n * a.out_ns + pi, res[idx], outfmt);
        }
        __syncthreads();
    }
}

template <class A, int KC, int R, bool VEC>
__global__ void __launch_bounds__(kConsumerWarps * 32, 1) product_kernel(const ProdArgs pa) {
    using C = typename A::C;
    using GT = typename GElem<A>::T;
    constexpr int NPL = GElem<A>::planes;
    extern __shared__ __align__(128) unsigned char smem[];
    const ContractArgs &a = pa.c;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem) + warp * kWarpStages;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 8 * kConsumerWarps * kWarpStages);
    unsigned long long *base_s = reinterpret_cast<unsigned long long *>(smem + 8 * kConsumerWarps * kWarpStages + 16);
    C *tw = reinterpret_cast<C *>(smem + pa.off_tw);
    C *b0 = reinterpret_cast<C *>(smem + pa.off_b0);
    C *b1 = reinterpret_cast<C *>(smem + pa.off_b1);
    unsigned char *stages = smem + pa.off_ring + (size_t)warp * kWarpStages * a.st_bytes;
    if (threadIdx.x == 0) *abort_flag = 0;
    if (lane == 0) {
        for (int s = 0; s < kWarpStages; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const int b = a.b;
    const int first = blockIdx.x + gridDim.x * warp;
    const int step = gridDim.x * kConsumerWarps;
    const int nbw = first < a.nbins ? (a.nbins - 1 - first) / step + 1 : 0;
    const int nitems = nbw * a.nchunks;
    const uint64_t pol_stream = l2_policy_evict_first();
    const uint64_t pol_keep = l2_policy_evict_last();
    const bool withheld0 = a.withhold && blockIdx.x == 0 && warp == 0;
    auto issue_g = [&](int it) {
        const int s = it % kWarpStages;
        const int bin = first + step * (it / a.nchunks), ch = it % a.nchunks;
        const int q0 = ch * a.Qc;
        const int qn = min(a.Qc, b - q0);
        const uint32_t gbytes = round_up16((uint32_t)(qn * b) * (uint32_t)sizeof(GT));
        unsigned char *st = stages + (size_t)s * a.st_bytes;
        mbar_expect_tx(&full[s], gbytes * NPL);
        const long goff = (long)bin * a.gbs + (long)q0 * b;
        bulk_g2s(st, reinterpret_cast<const GT *>(a.g0) + goff, gbytes, &full[s], pol_stream);
        if (NPL == 2)
            bulk_g2s(st + a.off_g1, reinterpret_cast<const GT *>(a.g1) + goff, gbytes, &full[s], pol_stream);
    };
    auto issue_u = [&](int it) {
        const int s = it % kWarpStages;
        const int bin = first + step * (it / a.nchunks);
        const uint32_t ubytes = round_up16((uint32_t)(a.kc * b) * (uint32_t)sizeof(C));
        unsigned char *st = stages + (size_t)s * a.st_bytes;
        if (withheld0 && it == 0) mbar_expect_tx(&full[s], ubytes);
        else mbar_arrive_expect_tx(&full[s], ubytes);
        bulk_g2s(st + a.off_u, reinterpret_cast<const C *>(a.u) + (long)bin * a.ubs, ubytes, &full[s], pol_keep);
    };
    // the spectrum does not depend on x: fill both stages of every warp's ring now
    const int npre = min(kWarpStages, nitems);
    if (lane == 0)
        for (int it = 0; it < npre; ++it) issue_g(it);
    pdl_wait();
    bool any = true;
    if (a.active) {
        any = false;
        for (int c = 0; c < a.kc; ++c) any |= a.active[c] != 0;
    }
    if (!any) {                                           // uniform over the grid: no barrier is entered
        if (lane == 0)
            for (int it = 0; it < npre; ++it) {
                mbar_arrive(&full[it % kWarpStages]);
                mbar_wait_drain(&full[it % kWarpStages], 0u);
            }
        pdl_trigger();
        return;
    }
    // ---- forward transforms: level 1 (x -> U), level 2 (U -> u^)
    prod_fft_phase<A, false>(pa.px, pa.fmt_x, native_fmt<A>, tw, b0, b1, *abort_flag != 0);
    prod_grid_barrier(pa.gbar, 0, base_s, abort_flag, a.err, a.wait_ns);
    prod_fft_phase<A, false>(pa.py, native_fmt<A>, native_fmt<A>, tw, b0, b1, *abort_flag != 0);
    prod_grid_barrier(pa.gbar, 1, base_s, abort_flag, a.err, a.wait_ns);

    // ---- block product (as contract_kernel); the vectors' part of the pre-filled stages now
    bool failed = *abort_flag != 0;
    int issued = npre;
    if (lane == 0 && !failed)
        for (int it = 0; it < npre; ++it) issue_u(it);
    if (failed) issued = 0;                               // the spectrum parts are drained below
    Acc<A> acc[KC][R];
    const int p0 = lane * R;
    int it = 0;
    for (; it < nitems && !failed; ++it) {
        const int s = it % kWarpStages;
        const uint32_t ph = (uint32_t)(it / kWarpStages) & 1u;
        const int bin = first + step * (it / a.nchunks), ch = it % a.nchunks;
        const bool ok = mbar_wait_bounded(&full[s], ph, abort_flag, a.wait_ns);
        if (__any_sync(0xffffffffu, !ok)) {
            failed = true;
            break;
        }
        if (ch == 0) {
#pragma unroll
            for (int c = 0; c < KC; ++c)
#pragma unroll
                for (int r = 0; r < R; ++r) acc[c][r].zero();
        }
        {
            const int q0 = ch * a.Qc;
            const int qn = min(a.Qc, b - q0);
            const unsigned char *st = stages + (size_t)s * a.st_bytes;
            const GT *gs0 = reinterpret_cast<const GT *>(st) + p0;
            const GT *gs1 = reinterpret_cast<const GT *>(st + a.off_g1) + p0;
            const C *us = reinterpret_cast<const C *>(st + a.off_u) + q0;
            if (p0 < b) {
#pragma unroll 2
                for (int q = 0; q < qn; ++q) {
                    if constexpr (R == 2 && VEC) {
                        using PV = typename Pair<GT>::V;
                        const PV v0 = *reinterpret_cast<const PV *>(gs0 + q * b);
                        const PV v1 = NPL == 2 ? *reinterpret_cast<const PV *>(gs1 + q * b) : v0;
#pragma unroll
                        for (int c = 0; c < KC; ++c) {
                            const C u = us[c * b + q];
                            acc[c][0].mac(Pair<GT>::lo(v0), Pair<GT>::lo(v1), u);
                            acc[c][1].mac(Pair<GT>::hi(v0), Pair<GT>::hi(v1), u);
                        }
                    } else {
                        GT v0[R], v1[R];
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            v0[r] = p0 + r < b ? gs0[q * b + r] : GT{};
                            v1[r] = NPL == 2 && p0 + r < b ? gs1[q * b + r] : v0[r];
                        }
#pragma unroll
                        for (int c = 0; c < KC; ++c) {
                            const C u = us[c * b + q];
#pragma unroll
                            for (int r = 0; r < R; ++r) acc[c][r].mac(v0[r], v1[r], u);
                        }
                    }
                }
            }
        }
        __syncwarp();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (ch == a.nchunks - 1) {
#pragma unroll
            for (int c = 0; c < KC; ++c)
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (c < a.kc && p0 + r < b)
                        store_vec<A, native_fmt<A>>(a.v, (long)bin * a.ubs + (long)c * b + p0 + r, acc[c][r].result());
        }
        // stage s is free: refill it with the item kWarpStages ahead
        if (lane == 0 && it + kWarpStages < nitems) {
            issue_g(it + kWarpStages);
            issue_u(it + kWarpStages);
            ++issued;
        }
    }
    if (lane == 0) {
        if (failed) {
            atomicOr(a.err, DEVERR_TIMEOUT);
            *abort_flag = 1;
            // items it .. issued-1 are outstanding (each in its own stage); before the block product started
            // only the spectrum parts of the first npre were issued: supply their arrivals and drain them
            const int lo = issued == 0 ? 0 : it, hi = issued == 0 ? npre : issued;
            for (int d = lo; d < hi && d < lo + kWarpStages; ++d) {
                if (issued == 0 || (withheld0 && d == 0)) mbar_arrive(&full[d % kWarpStages]);
                mbar_wait_drain(&full[d % kWarpStages], (uint32_t)(d / kWarpStages) & 1u);
            }
        }
    }
    prod_grid_barrier(pa.gbar, 2, base_s, abort_flag, a.err, a.wait_ns);
    // ---- inverse transforms: level 2 (v^ -> V), level 1 (V -> y)
    prod_fft_phase<A, true>(pa.pyi, native_fmt<A>, native_fmt<A>, tw, b0, b1, *abort_flag != 0);
    prod_grid_barrier(pa.gbar, 3, base_s, abort_flag, a.err, a.wait_ns);
    pdl_trigger();
    prod_fft_phase<A, true>(pa.pxi, native_fmt<A>, pa.fmt_y, tw, b0, b1, *abort_flag != 0);
}

template <class A>
constexpr int prec_of() { return A::kind == 0 ? BTTB_MV_FP64 : (A::kind == 1 ? BTTB_MV_FP32 : BTTB_MV_FP64_NATIVE); }

// Largest number of right-hand sides one launch of the block product carries.
template <class A> constexpr int max_kc() { return A::kind == 1 ? 4 : 2; }

template <class A, int KC, int R, bool VEC>
static int launch_contract_impl(Plan *p, const void *u, void *v, int k, const int *active) {
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
    a.wait_ns = p->wait_ns;
    a.withhold = 0;
    if (p->withhold > 0) {                                 // test hook, never inside a captured graph
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(p->stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
            a.withhold = 1;
            --p->withhold;
        }
    }
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

    // Per-warp stages: largest column chunk whose kConsumerWarps * kWarpStages stages fit.
    const size_t budget = (p->smem_optin > 0 ? p->smem_optin : 200 * 1024) - 256;
    const uint32_t ubytes_max = round_up128((uint32_t)(KC * b) * sizeof(C));
    int Qc = b;
    for (; Qc >= 1; --Qc) {
        if (Qc < b && (Qc * b) % 2) continue;             // keep 16-byte aligned chunk starts
        const size_t st = (size_t)round_up128((uint32_t)(Qc * b) * sizeof(GT)) * NPL + ubytes_max;
        if (st * kConsumerWarps * kWarpStages <= budget) break;
    }
    if (Qc < 1) return set_error(p, BTTB_ERR_INVALID_ARG, "block too large for the shared-memory pipeline");
    {   // balance the chunks (e.g. 60 columns as 3 x 20, not 29 + 29 + 2)
        const int nch = (b + Qc - 1) / Qc;
        int q2 = (b + nch - 1) / nch;
        if (q2 < b && (q2 * b) % 2) ++q2;
        if (q2 <= Qc) Qc = q2;
    }
    const uint32_t gbytes = round_up128((uint32_t)(Qc * b) * sizeof(GT));
    a.Qc = Qc;
    a.nchunks = (b + Qc - 1) / Qc;
    a.nstages = kWarpStages;
    a.off_g1 = gbytes;
    a.off_u = gbytes * NPL;
    a.st_bytes = gbytes * NPL + ubytes_max;
    const size_t smem = 256 + (size_t)a.st_bytes * kConsumerWarps * kWarpStages;

    auto kern = contract_kernel<A, KC, R, VEC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_optin);
    if (e != cudaSuccess) return check_cuda(p, e, "contract smem attribute");
    const long warps_needed = a.nbins;
    int grid = (int)((warps_needed + kConsumerWarps - 1) / kConsumerWarps);
    if (grid > p->nsm) grid = p->nsm;
    for (int c0 = 0; c0 < k; c0 += KC) {
        a.kc = (k - c0) < KC ? (k - c0) : KC;
        a.u = reinterpret_cast<const C *>(u) + (long)c0 * b;
        a.v = reinterpret_cast<C *>(v) + (long)c0 * b;
        a.active = active ? active + c0 : nullptr;
        const int tok = prof_begin(p, BTTB_K_BLOCK_PRODUCT_PREC + prec_of<A>());
        e = launch_pdl(kern, dim3(grid), dim3(kConsumerWarps * 32), smem, p->stream, a);
        a.withhold = 0;                                    // one launch per injection
        count_launch(p);
        if (e != cudaSuccess) return check_cuda(p, e, "contract launch");
        // algorithmic bytes: spectrum planes once, transformed vectors in and out
        prof_end(p, tok, (double)a.nbins * ((double)b * b * sizeof(GT) * NPL + 2.0 * a.kc * b * sizeof(C)));
        e = cudaGetLastError();
        if (e != cudaSuccess) return check_cuda(p, e, "contract launch");
    }
    return BTTB_OK;
}

// ---------------------------------------------------------------- whole-product kernel: host side

constexpr size_t kProdFftBytes = 32 * 1024;   // shared-memory area of the transform phases

// The four strided passes of matvec_run, with one column per item (the items are dealt out over the CTAs).
static int prod_passes(Plan *p, int fprec, int P, const void *x, long ldx, void *y, long ldy, int k,
                       const int *in_sel, long in_sel_stride, const double *in_scale, const int *active,
                       ProdArgs &pa) {
    const int nx = p->nx, ny = p->ny, b = p->b, mx = p->mx, my = p->my;
    const long plane = (long)ny * mx * b;
    FftPass &a = pa.px, &c = pa.py, &d = pa.pyi, &e = pa.pxi;
    a = FftPass{};
    a.in = x; a.out = p->wsB;
    a.in_cs = ldx; a.in_os = (long)nx * b; a.in_ns = b;
    a.out_cs = plane; a.out_os = (long)mx * b; a.out_ns = b;
    a.in_sel = in_sel; a.in_sel_stride = in_sel_stride; a.in_scale = in_scale; a.active = active;
    a.O = ny; a.pdim = b; a.ncols = k; a.nin = nx; a.nout = mx; a.M = mx;
    c = FftPass{};
    c.in = p->wsB; c.out = p->wsA;
    c.in_cs = plane; c.in_os = b; c.in_ns = (long)mx * b;
    c.out_cs = b; c.out_os = p->ubs; c.out_ns = (long)mx * p->ubs;
    c.O = mx; c.pdim = b; c.ncols = k; c.active = active; c.nin = ny; c.nout = my; c.M = my;
    d = FftPass{};
    d.in = p->wsB; d.out = p->wsA;
    d.in_cs = b; d.in_os = p->ubs; d.in_ns = (long)mx * p->ubs;
    d.out_cs = plane; d.out_os = b; d.out_ns = (long)mx * b;
    d.O = mx; d.pdim = b; d.ncols = k; d.active = active; d.nin = my; d.nout = ny; d.M = my;
    e = FftPass{};
    e.in = p->wsA; e.out = y;
    e.in_cs = plane; e.in_os = (long)mx * b; e.in_ns = b;
    e.out_cs = ldy; e.out_os = (long)nx * b; e.out_ns = b;
    e.O = ny; e.pdim = b; e.ncols = k; e.active = active; e.nin = mx; e.nout = nx; e.M = mx;
    for (FftPass *q : {&a, &c, &d, &e}) {
        q->cpb = 1;
        const int rc = fft_pass_prepare(p, *q, fprec, P);
        if (rc != BTTB_OK) return rc;
        if (q->P != P) return set_error(p, BTTB_ERR_INVALID_ARG, "whole-product kernel: pass chunk mismatch");
    }
    return BTTB_OK;
}

// Shared-memory layout of the whole-product kernel; false if the ring does not fit.
template <class A, int KC>
static bool prod_layout(const Plan *p, int &P, ContractArgs &a, ProdArgs &pa, size_t &smem) {
    using C = typename A::C;
    using GT = typename GElem<A>::T;
    constexpr int NPL = GElem<A>::planes;
    const int b = p->b, Mmax = std::max(p->mx, p->my);
    P = 1;
    while (P < 16 && P < b) P <<= 1;
    while (P > 1 && ((size_t)Mmax + 8 + 2 * (size_t)Mmax * P) * sizeof(C) > kProdFftBytes) P >>= 1;
    pa.off_tw = 256;
    pa.off_b0 = round_up16(256 + (uint32_t)(Mmax + 8) * sizeof(C));
    pa.off_b1 = pa.off_b0 + (uint32_t)(Mmax * P) * sizeof(C);
    pa.off_ring = round_up128(pa.off_b1 + (uint32_t)(Mmax * P) * sizeof(C));
    const size_t optin = p->smem_optin > 0 ? p->smem_optin : 200 * 1024;
    if (pa.off_ring >= optin) return false;
    const size_t budget = optin - pa.off_ring;
    const uint32_t ubytes_max = round_up128((uint32_t)(KC * b) * sizeof(C));
    int Qc = b;
    for (; Qc >= 1; --Qc) {
        if (Qc < b && (Qc * b) % 2) continue;
        const size_t st = (size_t)round_up128((uint32_t)(Qc * b) * sizeof(GT)) * NPL + ubytes_max;
        if (st * kConsumerWarps * kWarpStages <= budget) break;
    }
    if (Qc < 1) return false;
    {
        const int nch = (b + Qc - 1) / Qc;
        int q2 = (b + nch - 1) / nch;
        if (q2 < b && (q2 * b) % 2) ++q2;
        if (q2 <= Qc) Qc = q2;
    }
    const uint32_t gbytes = round_up128((uint32_t)(Qc * b) * sizeof(GT));
    a.Qc = Qc;
    a.nchunks = (b + Qc - 1) / Qc;
    a.nstages = kWarpStages;
    a.off_g1 = gbytes;
    a.off_u = gbytes * NPL;
    a.st_bytes = gbytes * NPL + ubytes_max;
    smem = pa.off_ring + (size_t)a.st_bytes * kConsumerWarps * kWarpStages;
    return smem <= optin;
}

template <class A> constexpr int prod_kc(int k) { return k == 1 ? 1 : (A::kind == 1 ? 4 : 2); }

template <class A, int KC, int R>
static int launch_product(Plan *p, const void *x, int xfmt, long ldx, void *y, int yfmt, long ldy, int k,
                          const int *in_sel, long in_sel_stride, const double *in_scale, const int *active) {
    using GT = typename GElem<A>::T;
    constexpr int NPL = GElem<A>::planes;
    constexpr bool VEC = R == 2;
    ProdArgs pa{};
    ContractArgs &a = pa.c;
    int P = 0;
    size_t smem = 0;
    if (!prod_layout<A, KC>(p, P, a, pa, smem)) return set_error(p, BTTB_ERR_INVALID_ARG, "whole-product kernel does not fit");
    int rc = prod_passes(p, A::kind == 0 ? PREC_DF64 : PREC_F32, P, x, ldx, y, ldy, k, in_sel, in_sel_stride, in_scale,
                         active, pa);
    if (rc != BTTB_OK) return rc;
    pa.fmt_x = xfmt;
    pa.fmt_y = yfmt;
    pa.gbar = p->d_gbar;
    a.gbs = p->gbs;
    a.ubs = p->ubs;
    a.nbins = (int)p->bins;
    a.b = p->b;
    a.kc = k;
    a.err = p->d_err;
    a.wait_ns = p->wait_ns;
    a.withhold = 0;
    if (p->withhold > 0) {                                 // test hook, never inside a captured graph
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(p->stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
            a.withhold = 1;
            --p->withhold;
        }
    }
    a.g0 = p->ghat_hi;
    a.g1 = A::kind == 0 ? p->ghat_lo : nullptr;
    a.u = p->wsA;
    a.v = p->wsB;
    a.active = active;
    if (!a.g0 || (NPL == 2 && !a.g1))
        return set_error(p, BTTB_ERR_INVALID_ARG, "plan does not keep the spectrum copy this precision reads");
    auto kern = product_kernel<A, KC, R, VEC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_optin);
    if (e != cudaSuccess) return check_cuda(p, e, "whole-product smem attribute");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p->nsm);
    cfg.blockDim = dim3(kConsumerWarps * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = p->stream;
    // Cooperative launch: every CTA is resident before any reaches a grid barrier.  No programmatic early
    // launch: the kernel starts once its predecessor has finished, so co-residency needs no other guarantee.
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int tok = prof_begin(p, BTTB_K_BLOCK_PRODUCT_PREC + (A::kind == 0 ? BTTB_MV_FP64 : BTTB_MV_FP32));
    e = cudaLaunchKernelEx(&cfg, kern, pa);
    count_launch(p);
    if (e != cudaSuccess) return check_cuda(p, e, "whole-product launch");
    // algorithmic bytes of the whole product: spectrum planes once, x in, y out
    auto esz = [](int f) { return f == FMT_C64 ? 8.0 : 16.0; };
    prof_end(p, tok, (double)p->bins * p->b * p->b * sizeof(GT) * NPL + (double)k * p->n * (esz(xfmt) + esz(yfmt)));
    return check_cuda(p, cudaGetLastError(), "whole-product launch");
}

bool product_persistent_fits(Plan *p, int prec, int k) {
    if (!p->d_gbar || p->in_batch || p->b > 128 || (p->b > 32 && p->b <= 64 && p->b % 2)) return false;
    if (prec != PREC_DF64 && prec != PREC_F32) return false;
    if (k < 1 || k > (prec == PREC_DF64 ? 2 : 4)) return false;
    static thread_local int coop = -1, coop_dev = -1;
    if (coop < 0 || coop_dev != p->dev) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, p->dev) != cudaSuccess) v = 0;
        coop = v;
        coop_dev = p->dev;
    }
    if (!coop) return false;
    int P = 0;
    size_t smem = 0;
    ContractArgs a{};
    ProdArgs pa{};
    return prec == PREC_DF64 ? (k == 1 ? prod_layout<DF64, 1>(p, P, a, pa, smem) : prod_layout<DF64, 2>(p, P, a, pa, smem))
                             : (k == 1 ? prod_layout<F32, 1>(p, P, a, pa, smem) : prod_layout<F32, 4>(p, P, a, pa, smem));
}

template <class A, int KC>
static int launch_product_r(Plan *p, const void *x, int xfmt, long ldx, void *y, int yfmt, long ldy, int k,
                            const int *in_sel, long in_sel_stride, const double *in_scale, const int *active) {
    switch ((p->b + 31) / 32) {
        case 1: return launch_product<A, KC, 1>(p, x, xfmt, ldx, y, yfmt, ldy, k, in_sel, in_sel_stride, in_scale, active);
        case 2: return launch_product<A, KC, 2>(p, x, xfmt, ldx, y, yfmt, ldy, k, in_sel, in_sel_stride, in_scale, active);
        case 3: return launch_product<A, KC, 3>(p, x, xfmt, ldx, y, yfmt, ldy, k, in_sel, in_sel_stride, in_scale, active);
        default: return launch_product<A, KC, 4>(p, x, xfmt, ldx, y, yfmt, ldy, k, in_sel, in_sel_stride, in_scale, active);
    }
}

int product_persistent_launch(Plan *p, const void *x, int xfmt, long ldx, void *y, int yfmt, long ldy, int k,
                              int prec, const int *in_sel, long in_sel_stride, const double *in_scale,
                              const int *active) {
    if (!product_persistent_fits(p, prec, k)) return set_error(p, BTTB_ERR_INVALID_ARG, "whole-product kernel does not fit");
    if (prec == PREC_DF64)
        return k == 1 ? launch_product_r<DF64, 1>(p, x, xfmt, ldx, y, yfmt, ldy, k, in_sel, in_sel_stride, in_scale, active)
                      : launch_product_r<DF64, 2>(p, x, xfmt, ldx, y, yfmt, ldy, k, in_sel, in_sel_stride, in_scale, active);
    return k == 1 ? launch_product_r<F32, 1>(p, x, xfmt, ldx, y, yfmt, ldy, k, in_sel, in_sel_stride, in_scale, active)
                  : launch_product_r<F32, 4>(p, x, xfmt, ldx, y, yfmt, ldy, k, in_sel, in_sel_stride, in_scale, active);
}

template <class A, int KC, int R>
static int launch_contract_kc(Plan *p, const void *u, void *v, int k, const int *active) {
    if (R == 2 && p->b % 2 == 0) return launch_contract_impl<A, KC, R, true>(p, u, v, k, active);
    return launch_contract_impl<A, KC, R, false>(p, u, v, k, active);
}

// Launch width KC times rows per lane R is kept <= 8 accumulators per lane.
template <class A, int R>
static int launch_contract_r(Plan *p, const void *u, void *v, int k, const int *active) {
    constexpr int KM = (max_kc<A>() * R > 8) ? (8 / R > 0 ? 8 / R : 1) : max_kc<A>();
    if constexpr (KM >= 4) {
        if (k >= 3) return launch_contract_kc<A, 4, R>(p, u, v, k, active);
    }
    if constexpr (KM >= 2) {
        if (k >= 2) return launch_contract_kc<A, 2, R>(p, u, v, k, active);
    }
    return launch_contract_kc<A, 1, R>(p, u, v, k, active);
}

template <class A>
static int launch_contract(Plan *p, const void *u, void *v, int k, const int *active) {
    const int R = (p->b + 31) / 32;
    switch (R) {
        case 1: return launch_contract_r<A, 1>(p, u, v, k, active);
        case 2: return launch_contract_r<A, 2>(p, u, v, k, active);
        case 3: return launch_contract_r<A, 3>(p, u, v, k, active);
        case 4: return launch_contract_r<A, 4>(p, u, v, k, active);
        case 5: case 6: return launch_contract_r<A, 6>(p, u, v, k, active);
        default: return launch_contract_r<A, 8>(p, u, v, k, active);
    }
}

// ---------------------------------------------------------------------------
// Many right-hand sides (binary32): the per-bin block product is a complex GEMM
// V_k = G_k U_k with U_k of b x k.  CTA (tile, bin) stages the bin's spectrum
// block (column-major, as stored) and a 64-column tile of U (column-major, as
// stored) with two bulk copies, then thread (row p, column group g)
// accumulates its row over the tile's columns of group g; the vector entry of
// a column is a shared-memory broadcast.  Consecutive CTAs share a bin, so the
// spectrum block is re-read from L2.
// ---------------------------------------------------------------------------
constexpr int kMultiTile = 64;

template <int CPG>
__global__ void __launch_bounds__(256) contract_multi_kernel(const float2 *g0, long gbs, const float2 *u, float2 *v,
                                                              long ubs, int b, int k, int *err,
                                                              unsigned long long wait_ns) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 8);
    float2 *gs = reinterpret_cast<float2 *>(smem + 128);
    const uint32_t gbytes = round_up128((uint32_t)(b * b) * 8u);
    float2 *us = reinterpret_cast<float2 *>(smem + 128 + gbytes);
    const int bin = blockIdx.y, c0 = blockIdx.x * kMultiTile;
    const int nc = min(kMultiTile, k - c0);
    pdl_wait();
    if (threadIdx.x == 0) {
        *abort_flag = 0;
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t gb = round_up16((uint32_t)(b * b) * 8u);
        const uint32_t ub = round_up16((uint32_t)(nc * b) * 8u);
        mbar_arrive_expect_tx(bar, gb + ub);
        bulk_g2s(gs, g0 + (long)bin * gbs, gb, bar, l2_policy_evict_last());
        bulk_g2s(us, u + (long)bin * ubs + (long)c0 * b, ub, bar, l2_policy_evict_first());
    }
    const bool ok = mbar_wait_bounded(bar, 0, abort_flag, wait_ns);
    if (!ok) {
        if (threadIdx.x == 0) {
            atomicOr(err, DEVERR_TIMEOUT);
            mbar_wait_drain(bar, 0);
        }
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rw = (b + 31) / 32;                 // row warps
    const int cg = 8 / rw;                        // column groups
    const int wr = warp % rw, wg = warp / rw;
    const int p = wr * 32 + lane;
    if (wg < cg && p < b) {
        float2 acc[CPG];
#pragma unroll
        for (int j = 0; j < CPG; ++j) acc[j] = make_float2(0.f, 0.f);
        const int cbase = wg * CPG;
        for (int q = 0; q < b; ++q) {
            const float2 gq = gs[q * b + p];
#pragma unroll
            for (int j = 0; j < CPG; ++j) {
                const float2 x = us[(cbase + j) * b + q];     // broadcast within the warp
                acc[j].x = fmaf(gq.x, x.x, acc[j].x);
                acc[j].x = fmaf(-gq.y, x.y, acc[j].x);
                acc[j].y = fmaf(gq.x, x.y, acc[j].y);
                acc[j].y = fmaf(gq.y, x.x, acc[j].y);
            }
        }
#pragma unroll
        for (int j = 0; j < CPG; ++j)
            if (cbase + j < nc) gst(v + (long)bin * ubs + (long)(c0 + cbase + j) * b + p, acc[j]);
    }
    pdl_trigger();
}

// Same product for b <= 64 with a 4 x 4 register tile: thread (row group rg, column group cg) of the 256
// accumulates rows 2rg, 2rg+1, 32+2rg, 33+2rg of columns cg, cg+16, cg+32, cg+48 of the tile.  Per basis q it
// loads its two row pairs of the spectrum block (16-byte loads, consecutive across the warp's lanes, when b
// is even) and four vector entries (the two column groups of a warp are adjacent columns, on different
// banks): 6 shared loads per 64 FMAs.
__global__ void __launch_bounds__(256) contract_multi44_kernel(const float2 *g0, long gbs, const float2 *u,
                                                                float2 *v, long ubs, int b, int k, int *err,
                                                                unsigned long long wait_ns) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 8);
    float2 *gs = reinterpret_cast<float2 *>(smem + 128);
    const uint32_t gbytes = round_up128((uint32_t)(b * b) * 8u);
    float2 *us = reinterpret_cast<float2 *>(smem + 128 + gbytes);
    const int bin = blockIdx.y, c0 = blockIdx.x * kMultiTile;
    const int nc = min(kMultiTile, k - c0);
    pdl_wait();
    if (threadIdx.x == 0) {
        *abort_flag = 0;
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t gb = round_up16((uint32_t)(b * b) * 8u);
        const uint32_t ub = round_up16((uint32_t)(nc * b) * 8u);
        mbar_arrive_expect_tx(bar, gb + ub);
        bulk_g2s(gs, g0 + (long)bin * gbs, gb, bar, l2_policy_evict_last());
        bulk_g2s(us, u + (long)bin * ubs + (long)c0 * b, ub, bar, l2_policy_evict_first());
    }
    const bool ok = mbar_wait_bounded(bar, 0, abort_flag, wait_ns);
    if (!ok) {
        if (threadIdx.x == 0) {
            atomicOr(err, DEVERR_TIMEOUT);
            mbar_wait_drain(bar, 0);
        }
        return;
    }
    const int rg = threadIdx.x & 15, cg = threadIdx.x >> 4;
    const int pa = 2 * rg, pb = 32 + 2 * rg;                  // the thread's row pairs
    if (pa < b && cg < nc) {
        int prow[4] = {pa, pa + 1, pb, pb + 1};
        float2 acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[r][j] = make_float2(0.f, 0.f);
        const bool even = b % 2 == 0, hasb = pb < b;
        for (int q = 0; q < b; ++q) {
            float2 g[4];
            if (even) {
                const float4 a0 = *reinterpret_cast<const float4 *>(gs + q * b + pa);
                const float4 a1 = hasb ? *reinterpret_cast<const float4 *>(gs + q * b + pb)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                g[0] = make_float2(a0.x, a0.y);
                g[1] = make_float2(a0.z, a0.w);
                g[2] = make_float2(a1.x, a1.y);
                g[3] = make_float2(a1.z, a1.w);
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r) g[r] = prow[r] < b ? gs[q * b + prow[r]] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 x = us[(cg + 16 * j) * b + q];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    acc[r][j].x = fmaf(g[r].x, x.x, acc[r][j].x);
                    acc[r][j].x = fmaf(-g[r].y, x.y, acc[r][j].x);
                    acc[r][j].y = fmaf(g[r].x, x.y, acc[r][j].y);
                    acc[r][j].y = fmaf(g[r].y, x.x, acc[r][j].y);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int cc = cg + 16 * j;
            if (cc < nc)
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (prow[r] < b) gst(v + (long)bin * ubs + (long)(c0 + cc) * b + prow[r], acc[r][j]);
        }
    }
    pdl_trigger();
}

static int launch_contract_multi(Plan *p, const void *u, void *v, int k) {
    const int b = p->b;
    if (!p->ghat_hi) return set_error(p, BTTB_ERR_INVALID_ARG, "plan does not keep the binary32 spectrum");
    const int rw = (b + 31) / 32, cg = 8 / rw;     // b <= 128: rw in 1..4, cg in {8, 4, 2}
    const int cpg = kMultiTile / cg;                 // exactly covers the tile: 8, 16 or 32 columns
    const size_t smem = 128 + round_up128((uint32_t)(b * b) * 8u) + round_up128((uint32_t)(kMultiTile * b) * 8u);
    auto kern = b <= 64 ? contract_multi44_kernel
                        : (cpg == 8 ? contract_multi_kernel<8>
                                    : (cpg == 16 ? contract_multi_kernel<16> : contract_multi_kernel<32>));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_optin);
    if (e != cudaSuccess) return check_cuda(p, e, "multi-RHS smem attribute");
    const dim3 grid((k + kMultiTile - 1) / kMultiTile, (unsigned)p->bins);
    const int tok = prof_begin(p, BTTB_K_BLOCK_PRODUCT_PREC + BTTB_MV_FP32);
    e = launch_pdl(kern, grid, dim3(256), smem, p->stream, (const float2 *)p->ghat_hi, p->gbs, (const float2 *)u,
                   (float2 *)v, p->ubs, b, k, p->d_err, p->wait_ns);
    count_launch(p);
    prof_end(p, tok, (double)p->bins * ((double)b * b * 8 + 2.0 * k * b * 8));
    if (e != cudaSuccess) return check_cuda(p, e, "multi-RHS launch");
    return BTTB_OK;
}

// ---------------------------------------------------------------------------
// Many right-hand sides on the tensor cores (3xTF32).  The complex per-bin GEMM
// V_k = G_k U_k is one real GEMM: the 2b x 2b embedding [Gr -Gi; Gi Gr] times
// [Ur; Ui] (2b x k).  Every factor x is split into a TF32 head and a TF32 tail,
// x = hi + lo, and C += hi*lo' + lo*hi' + hi*hi' accumulates in binary32, which
// keeps binary32-level accuracy (the lo*lo' term is below binary32 rounding).
// CTA (64-column tile, bin), b <= 64: the embedding (up to 128 x 128, zero
// padded) and the real tile [Ur; Ui] are built in shared memory, row strides
// = 4 (mod 32) words so that the fragment loads are conflict-free; 8 warps in a
// 4 x 2 grid of 32 x 32 output blocks issue warp-level mma.sync m16n8k8 with
// TF32 inputs; the result is staged in shared memory and written back as
// complex columns.
// ---------------------------------------------------------------------------
constexpr int kTcTile = 64;

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
    hi = tf32_rna(x);
    lo = tf32_rna(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Row stride (floats) of the staged real operands: >= kp, = 4 (mod 32).
__host__ __device__ constexpr int tc_stride(int kp) { return ((kp + 27) / 32) * 32 + 4; }

__global__ void __launch_bounds__(256) contract_tc_kernel(const float2 *__restrict__ G, long gbs,
                                                          const float2 *__restrict__ U, float2 *__restrict__ V,
                                                          long ubs, int b, int k) {
    extern __shared__ __align__(16) float tcs[];
    const int twob = 2 * b;
    const int kp = (twob + 7) / 8 * 8;                   // K padded to the MMA depth
    const int st = tc_stride(kp);
    float *As = tcs;                                      // 128 rows x st (row r, column q')
    float *Bs = tcs + 128 * st;                           // kTcTile rows (columns n) x st (index q')
    const long bin = blockIdx.y;
    const int c0 = blockIdx.x * kTcTile;
    const int ncb = min(kTcTile, k - c0);
    pdl_wait();
    // zero the padding, then scatter the embedding and the tile
    for (int i = threadIdx.x; i < 128 * st; i += blockDim.x) {
        const int r = i / st, q = i - r * st;
        if (r >= twob || q >= twob) As[i] = 0.f;
    }
    for (int i = threadIdx.x; i < kTcTile * st; i += blockDim.x) {
        const int n = i / st, q = i - n * st;
        if (n >= ncb || q >= twob) Bs[i] = 0.f;
    }
    const float2 *gsrc = G + bin * gbs;
    for (int i = threadIdx.x; i < b * b; i += blockDim.x) {
        const int q = i / b, pr = i - q * b;              // column-major: entry (pr, q)
        const float2 g = gsrc[i];
        As[pr * st + q] = g.x;
        As[pr * st + q + b] = -g.y;
        As[(pr + b) * st + q] = g.y;
        As[(pr + b) * st + q + b] = g.x;
    }
    const float2 *usrc = U + bin * ubs + (long)c0 * b;
    for (int i = threadIdx.x; i < ncb * b; i += blockDim.x) {
        const int n = i / b, q = i - n * b;
        const float2 u = usrc[i];
        Bs[n * st + q] = u.x;
        Bs[n * st + q + b] = u.y;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int wm = warp >> 1, wn = warp & 1;
    float acc[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;
    const bool live = wm * 32 < twob;                     // warps whose rows are all padding skip the MMAs
    if (live) {
        for (int kb = 0; kb < kp; kb += 8) {
            uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const float *ar = As + (wm * 32 + mt * 16 + gid) * st + kb + tig;
                split_tf32(ar[0], ah[mt][0], al[mt][0]);
                split_tf32(ar[8 * st], ah[mt][1], al[mt][1]);
                split_tf32(ar[4], ah[mt][2], al[mt][2]);
                split_tf32(ar[8 * st + 4], ah[mt][3], al[mt][3]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const float *br = Bs + (wn * 32 + nt * 8 + gid) * st + kb + tig;
                split_tf32(br[0], bh[nt][0], bl[nt][0]);
                split_tf32(br[4], bh[nt][1], bl[nt][1]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    mma_tf32(acc[mt][nt], ah[mt], bl[nt]);
                    mma_tf32(acc[mt][nt], al[mt], bh[nt]);
                    mma_tf32(acc[mt][nt], ah[mt], bh[nt]);
                }
        }
    }
    __syncthreads();                                      // operands consumed: reuse the space for C
    float *Cs = tcs;                                      // kTcTile columns x (2b + 1)
    const int cst = twob + 1;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int r = wm * 32 + mt * 16 + gid, n = wn * 32 + nt * 8 + 2 * tig;
            if (r < twob) {
                Cs[n * cst + r] = acc[mt][nt][0];
                Cs[(n + 1) * cst + r] = acc[mt][nt][1];
            }
            if (r + 8 < twob) {
                Cs[n * cst + r + 8] = acc[mt][nt][2];
                Cs[(n + 1) * cst + r + 8] = acc[mt][nt][3];
            }
        }
    __syncthreads();
    pdl_trigger();
    float2 *vdst = V + bin * ubs + (long)c0 * b;
    for (int i = threadIdx.x; i < ncb * b; i += blockDim.x) {
        const int n = i / b, pr = i - n * b;
        vdst[i] = make_float2(Cs[n * cst + pr], Cs[n * cst + pr + b]);
    }
}

static size_t contract_tc_smem(int b) {
    const int kp = (2 * b + 7) / 8 * 8;
    return (size_t)(128 + kTcTile) * tc_stride(kp) * sizeof(float);
}

static int launch_contract_tc(Plan *p, const void *u, void *v, int k) {
    const int b = p->b;
    if (!p->ghat_hi) return set_error(p, BTTB_ERR_INVALID_ARG, "plan does not keep the binary32 spectrum");
    const size_t smem = contract_tc_smem(b);
    cudaError_t e = cudaFuncSetAttribute(contract_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)p->smem_optin);
    if (e != cudaSuccess) return check_cuda(p, e, "tensor-core product smem attribute");
    const dim3 grid((k + kTcTile - 1) / kTcTile, (unsigned)p->bins);
    const int tok = prof_begin(p, BTTB_K_BLOCK_PRODUCT_PREC + BTTB_MV_TC_3XTF32);
    e = launch_pdl(contract_tc_kernel, grid, dim3(256), smem, p->stream, (const float2 *)p->ghat_hi, p->gbs,
                   (const float2 *)u, (float2 *)v, p->ubs, b, k);
    count_launch(p);
    prof_end(p, tok, (double)p->bins * ((double)b * b * 8 + 2.0 * k * b * 8));
    if (e != cudaSuccess) return check_cuda(p, e, "tensor-core product launch");
    return BTTB_OK;
}

int contract_launch(Plan *p, int prec, const void *u, void *v, int k, const int *active) {
    // Tensor cores for a real per-bin GEMM (many columns, b <= 64); a GEMV (few columns) has no reuse.
    // Tensor cores for a real per-bin GEMM (many columns); a GEMV (few columns) has no reuse.  tcgen05 with
    // TMA-fed tiles when b is even and at most 64; the warp-level 3xTF32 form for odd b; binary32 otherwise.
    if (is_tc_prec(prec)) {
        if (tcgemm_fits(p, k)) return tcgemm_launch(p, prec == PREC_TCB ? 1 : 0, u, v, k);
        if (prec == PREC_TC && k >= kTcMinCols && p->b <= 64) return launch_contract_tc(p, u, v, k);
        prec = PREC_F32;
    }
    // Many right-hand sides in binary32: a tiled per-bin GEMM instead of k/4 passes over the spectrum.
    if (prec == PREC_F32 && k > 8 && p->b <= 128) return launch_contract_multi(p, u, v, k);
    switch (prec) {
        case PREC_F32: return launch_contract<F32>(p, u, v, k, active);
        case PREC_F64N: return launch_contract<F64N>(p, u, v, k, active);
        default: return launch_contract<DF64>(p, u, v, k, active);
    }
}

}  // namespace bttb
