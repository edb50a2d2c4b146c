// The middle of the product y = Z x (Sec. II-C, III-A) in one kernel for one to four columns: the
// level-2 (y) DFT of the padded vector, the per-bin block product v_k = G_k u_k of Eq. (multL) and the
// inverse level-2 DFT with the crop to ny rows.  The level-1 (x) transforms before and after it are the
// strided passes of fft.cu; together they are the 2-level blockwise FFT of App. B.
//
// The y transform of one column kx of the cell grid needs every row of that column, and the block
// product of a bin needs every basis index, so a thread-block cluster of Q CTAs takes one column kx.
// CTA r of the cluster owns the bases P_r (a share of the b) and the bins K_r (a share of the my values of
// ky), and
//   1. loads U[c][iy][kx][p] for p in P_r, iy < ny (the x pass's output), leaves rows iy >= ny zero
//      (Eq. (xc2)) and transforms along iy: Stockham stages in shared memory;
//   2. sends bin ky of its bases to the CTA that owns ky, through distributed shared memory;
//   3. forms v_k = G_k u_k for its bins, one warp per bin: lane l accumulates the rows l R .. l R + R - 1
//      over every column of the block, so a bin needs no reduction across warps.  Each warp streams its
//      bins' spectrum blocks (column-major chunks, the binary32 planes the precision reads) through a
//      private ring of shared-memory stages: lane 0 issues cp.async.bulk copies, an mbarrier per stage
//      counts the bytes in.  The spectrum does not depend on the x pass, so every warp fills the stages
//      of its ring that lie in the ring area before the programmatic-dependent-launch wait, and those
//      copies land while the x pass drains and steps 1-2 run; the y-transform buffers, free from the end
//      of step 2 to the start of step 4, hold the ring's other stages.  The per-lane accumulation is the
//      one of the block-product kernel (contract.cu), so the product has the bits of the strided-pass
//      route;
//   4. sends v_k of each basis back to the CTA that owns the basis;
//   5. transforms along ky (inverse, unnormalised: the 1/(mx my) is in the spectrum), keeps iy < ny and
//      stores V[c][iy][kx][p] for the inverse x pass.
// Every wait is bounded; a wait that runs out sets the plan's error word, the warp stops computing but
// the CTA keeps taking part in the cluster barriers, and every copy in flight is drained before exit.
#include <algorithm>

#include <cooperative_groups.h>

#include "arith.cuh"
#include "blockprod.cuh"
#include "fftcore.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace bttb {

constexpr int kYcWarps = 8;
constexpr int kYcThreads = kYcWarps * 32;
constexpr int kYcMaxStages = 8;                              // ring depth per warp
constexpr uint32_t kYcHead = 8u * kYcWarps * kYcMaxStages;   // mbarriers, then the abort flag

struct YcArgs {
    const void *U;                // x-pass output [c][iy][kx][p] (native format)
    void *V;                      // output, same layout, for the inverse x pass
    long plane;                   // column stride of U and V: ny*mx*b
    const void *g0, *g1;          // spectrum planes (g1: double-float low plane)
    long gbs;                     // bin stride of a plane
    const int *active;            // per-column flags of this group (may be null)
    int nx, ny, mx, my, b, kc;    // kc: columns of this launch
    int Q, pshare, kshare;        // cluster size, bases and bins per CTA (the last CTA may hold fewer)
    int Qc, nchunks, nstages;     // spectrum columns per stage, stages per bin, ring depth per warp
    int nfix;                     // stages per warp in the ring area (the rest in the y-transform buffers)
    uint32_t stage_bytes, off_g1; // bytes of one stage; offset of its low-plane part
    uint32_t off_tw, off_f0, off_f1, off_uh, off_ring;
    Fft2Side sy;
    const void *twy;
    int *err;
    unsigned long long wait_ns;
    int withhold;                 // test hook: warp 0 of CTA 0 withholds the arrival of its first stage
};

__host__ __device__ constexpr uint32_t yc_align(uint32_t x) { return (x + 127u) & ~127u; }
__host__ __device__ constexpr uint32_t yc_round16(uint32_t x) { return (x + 15u) & ~15u; }

// KC: columns per launch (compile time, kc <= KC); R: rows per lane (b <= 32 R); VEC: R = 2 with b even,
// row pairs loaded as one 16-byte word.
template <class A, int KC, int R, bool VEC>
__global__ void __launch_bounds__(kYcThreads, 2) ycontract_kernel(const YcArgs a) {
    namespace cg = cooperative_groups;
    using C = typename A::C;
    using GT = typename GElem<A>::T;
    constexpr int NPL = GElem<A>::planes;
    extern __shared__ __align__(128) unsigned char smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank();
    const int kx = blockIdx.x / a.Q;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = a.b, my = a.my, kc = a.kc, S = a.nstages;

    uint64_t *full = reinterpret_cast<uint64_t *>(smem) + warp * kYcMaxStages;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + kYcHead);
    C *tw = reinterpret_cast<C *>(smem + a.off_tw);
    C *F0 = reinterpret_cast<C *>(smem + a.off_f0);
    C *F1 = reinterpret_cast<C *>(smem + a.off_f1);
    C *Uh = reinterpret_cast<C *>(smem + a.off_uh);          // [kl][c][p]: u^ of my bins, then v^
    // stage s of this warp: the first nfix in the ring area, the others in the y-transform buffers
    // [off_f0, off_uh), which hold no live data during step 3
    auto stage = [&](int s) -> unsigned char * {
        return s < a.nfix ? smem + a.off_ring + ((size_t)warp * a.nfix + s) * a.stage_bytes
                          : smem + a.off_f0 + ((size_t)warp * (S - a.nfix) + (s - a.nfix)) * a.stage_bytes;
    };

    // shares: bases [plo, plo+np), bins [klo, klo+nk) of rank r (and of any rank o)
    auto p_lo = [&](int o) { return min(b, o * a.pshare); };
    auto p_n = [&](int o) { return min(b, (o + 1) * a.pshare) - p_lo(o); };
    auto k_lo = [&](int o) { return min(my, o * a.kshare); };
    const int plo = p_lo(r), np = p_n(r), klo = k_lo(r), nk = min(my, (r + 1) * a.kshare) - klo;
    const int nseq = kc * np;                                 // sequences of this CTA's y transforms
    // this warp's bins: kl = warp, warp + kYcWarps, ...; an item is one chunk of one of them
    const int nbw = warp < nk ? (nk - 1 - warp) / kYcWarps + 1 : 0;
    const int nitems = nbw * a.nchunks;

    if (threadIdx.x == 0) *abort_flag = 0;
    if (lane == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const uint64_t pol_stream = l2_policy_evict_first();
    const bool withheld0 = a.withhold && blockIdx.x == 0 && warp == 0;
    auto issue = [&](int it) {
        const int s = it % S;
        const int kl = warp + kYcWarps * (it / a.nchunks), ch = it % a.nchunks;
        const int q0 = ch * a.Qc, qn = min(a.Qc, b - q0);
        const uint32_t gbytes = yc_round16((uint32_t)(qn * b) * (uint32_t)sizeof(GT));
        const long goff = ((long)(klo + kl) * a.mx + kx) * a.gbs + (long)q0 * b;
        unsigned char *st = stage(s);
        if (withheld0 && it == 0) mbar_expect_tx(&full[s], gbytes * NPL);
        else mbar_arrive_expect_tx(&full[s], gbytes * NPL);
        bulk_g2s(st, reinterpret_cast<const GT *>(a.g0) + goff, gbytes, &full[s], pol_stream);
        if (NPL == 2) bulk_g2s(st + a.off_g1, reinterpret_cast<const GT *>(a.g1) + goff, gbytes, &full[s], pol_stream);
    };
    // the spectrum does not depend on the x pass: fill the ring area's stages before the dependency wait
    const int npre = min(a.nfix, nitems);
    if (lane == 0)
        for (int it = 0; it < npre; ++it) issue(it);
    for (int i = threadIdx.x; i < my + 5; i += blockDim.x) tw[i] = reinterpret_cast<const C *>(a.twy)[i];
    // every CTA of the cluster must have started before another writes into its shared memory: arrive
    // now, wait before the first exchange
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
    pdl_wait();

    bool any = true;
    if (a.active) {                                          // uniform over the cluster (same columns)
        any = false;
        for (int c = 0; c < kc; ++c) any |= a.active[c] != 0;
    }
    bool failed = false;
    int it = 0;                                               // this warp's first item not consumed
    if (any) {
        // ---- 1. load this CTA's bases of column kx and transform along iy
        const long ucol = (long)kx * b + plo;
        for (int idx = threadIdx.x; idx < my * nseq; idx += blockDim.x) {
            const int iy = idx / nseq, t = idx - iy * nseq;
            const int c = t / np, pl = t - c * np;
            C v = A::zero();
            if (iy < a.ny) v = load_vec<A, native_fmt<A>>(a.U, (long)c * a.plane + (long)iy * a.mx * b + ucol + pl);
            F0[idx] = v;
        }
        __syncthreads();
        const C *R1 = fft2_level<A, false>(F0, F1, tw, a.sy, nseq, nseq, 1);
        // ---- 2. bin ky of my bases to the CTA that owns ky
        asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
        for (int idx = threadIdx.x; idx < my * nseq; idx += blockDim.x) {
            const int ky = idx / nseq, t = idx - ky * nseq;
            const int c = t / np, pl = t - c * np;
            const int o = ky / a.kshare;
            C *dst = cl.map_shared_rank(Uh, o);
            const long di = (long)(ky - k_lo(o)) * kc * b + c * b + plo + pl;
            if (BTTB_ICHK(di, (long)a.kshare * kc * b)) dst[di] = R1[idx];
        }
        // the y-transform buffers take bulk copies from here on (async proxy after these generic accesses)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        cl.sync();
        if (lane == 0)
            for (int i = npre; i < min(S, nitems); ++i) issue(i);

        // ---- 3. block products of my bins, one warp per bin
        Acc<A> acc[KC][R];
        const int p0 = lane * R;
        for (; it < nitems; ++it) {
            const int s = it % S;
            const int kl = warp + kYcWarps * (it / a.nchunks), ch = it % a.nchunks;
            // a wait that ran out (or saw another warp's abort) ends the warp's loop; uniform over the warp
            const bool ok = mbar_wait_bounded(&full[s], (uint32_t)(it / S) & 1u, abort_flag, a.wait_ns);
            if (__any_sync(0xffffffffu, !ok)) {
                failed = true;
                break;
            }
            if (ch == 0) {
#pragma unroll
                for (int c = 0; c < KC; ++c)
#pragma unroll
                    for (int rr = 0; rr < R; ++rr) acc[c][rr].zero();
            }
            {
                const int q0 = ch * a.Qc, qn = min(a.Qc, b - q0);
                const unsigned char *st = stage(s);
                const GT *gs0 = reinterpret_cast<const GT *>(st) + p0;
                const GT *gs1 = reinterpret_cast<const GT *>(st + a.off_g1) + p0;
                const C *us = Uh + (long)kl * kc * b + q0;
                const bool us_ok = BTTB_ICHK((long)kl * kc * b + q0 + (long)(kc - 1) * b + (qn - 1),
                                             (long)a.kshare * kc * b);
                if (p0 < b && us_ok) {
#pragma unroll 2
                    for (int q = 0; q < qn; ++q) {
                        if constexpr (R == 2 && VEC) {
                            using PV = typename Pair<GT>::V;
                            const PV v0 = *reinterpret_cast<const PV *>(gs0 + q * b);
                            const PV v1 = NPL == 2 ? *reinterpret_cast<const PV *>(gs1 + q * b) : v0;
#pragma unroll
                            for (int c = 0; c < KC; ++c) {
                                if (c < kc) {
                                    const C u = us[c * b + q];
                                    acc[c][0].mac(Pair<GT>::lo(v0), Pair<GT>::lo(v1), u);
                                    acc[c][1].mac(Pair<GT>::hi(v0), Pair<GT>::hi(v1), u);
                                }
                            }
                        } else {
                            GT v0[R], v1[R];
#pragma unroll
                            for (int rr = 0; rr < R; ++rr) {
                                v0[rr] = p0 + rr < b ? gs0[q * b + rr] : GT{};
                                v1[rr] = NPL == 2 && p0 + rr < b ? gs1[q * b + rr] : v0[rr];
                            }
#pragma unroll
                            for (int c = 0; c < KC; ++c) {
                                if (c < kc) {
                                    const C u = us[c * b + q];
#pragma unroll
                                    for (int rr = 0; rr < R; ++rr) acc[c][rr].mac(v0[rr], v1[rr], u);
                                }
                            }
                        }
                    }
                }
            }
            // every lane is done with stage s (and, at a bin's end, with u^ of the bin) before the stage is
            // refilled and v^ overwrites u^
            __syncwarp();
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (ch == a.nchunks - 1) {
#pragma unroll
                for (int c = 0; c < KC; ++c)
#pragma unroll
                    for (int rr = 0; rr < R; ++rr)
                        if (c < kc && p0 + rr < b) Uh[(long)kl * kc * b + c * b + p0 + rr] = acc[c][rr].result();
            }
            if (lane == 0 && it + S < nitems) issue(it + S);
        }
        // a warp whose loop broke off drains its copies in flight (items it .. min(it + S, nitems) - 1, each
        // in its own stage; every earlier item completed its phase; a withheld arrival is supplied first)
        // before any CTA of the cluster writes into the y-transform buffers again
        if (failed && lane == 0) {
            atomicOr(a.err, DEVERR_TIMEOUT);
            for (int d = it; d < min(it + S, nitems); ++d) {
                if (withheld0 && d == 0) mbar_arrive(&full[d % S]);
                mbar_wait_drain(&full[d % S], (uint32_t)(d / S) & 1u);
            }
        }
        cl.sync();
        // ---- 4. v_k of each basis to the CTA that owns the basis
        for (int idx = threadIdx.x; idx < nk * kc * b; idx += blockDim.x) {
            const int kl = idx / (kc * b), rem = idx - kl * kc * b;
            const int c = rem / b, pr = rem - c * b;
            const int o = pr / a.pshare;
            const int npo = p_n(o);
            C *dst = cl.map_shared_rank(F0, o);
            const long di = (long)(klo + kl) * (kc * npo) + c * npo + (pr - p_lo(o));
            if (BTTB_ICHK(di, (long)my * kc * a.pshare)) dst[di] = Uh[idx];
        }
        cl.sync();
        // ---- 5. inverse transform along ky, crop to ny rows
        const C *R2 = fft2_level<A, true>(F0, F1, tw, a.sy, nseq, nseq, 1);
        pdl_trigger();
        for (int idx = threadIdx.x; idx < a.ny * nseq; idx += blockDim.x) {
            const int iy = idx / nseq, t = idx - iy * nseq;
            const int c = t / np, pl = t - c * np;
            store_vec<A, native_fmt<A>>(a.V, (long)c * a.plane + (long)iy * a.mx * b + ucol + pl, R2[idx]);
        }
    } else {
        pdl_trigger();
    }
    // with no active column the prefetched copies are still in flight: let them land (a withheld arrival
    // is supplied first) before the CTA's shared memory goes away
    if (!any && lane == 0) {
        for (int d = 0; d < npre; ++d) {
            if (withheld0 && d == 0) mbar_arrive(&full[d]);
            if (!mbar_wait_drain(&full[d], 0u)) atomicOr(a.err, DEVERR_TIMEOUT);
        }
    }
}

// ---------------------------------------------------------------- host side

template <class A, int KC>
static bool yc_layout(const Plan *p, int kc, int Q, YcShape &y) {
    using C = typename A::C;
    using GT = typename GElem<A>::T;
    constexpr int NPL = GElem<A>::planes;
    const int b = p->b, my = p->my;
    y.Q = Q;
    y.pshare = (b + Q - 1) / Q;
    y.kshare = (my + Q - 1) / Q;
    const uint32_t ce = sizeof(C);
    uint32_t off = yc_align(kYcHead + 16);
    y.off_tw = off;
    off = yc_align(off + (uint32_t)(my + 8) * ce);
    const uint32_t fbytes = (uint32_t)my * kc * y.pshare * ce;
    y.off_f0 = off;
    off = yc_align(off + fbytes);
    y.off_f1 = off;
    off = yc_align(off + fbytes);
    y.off_uh = off;
    off = yc_align(off + (uint32_t)y.kshare * kc * b * ce);
    y.off_ring = off;
    // per-warp rings: the largest chunk of whole spectrum columns (16-byte aligned starts, balanced over the
    // block) of which two stages per warp fit in what is left of a budget that lets two CTAs share an SM
    // (if such a stage holds at least 3 KB), else of the whole opt-in limit; then as many stages of that
    // size as fit there, plus those that fit in the y-transform buffers, kYcMaxStages at most
    const size_t optin = p->smem_optin > 0 ? (size_t)p->smem_optin : 227 * 1024;
    const size_t budget2 = (optin + 1024) / 2 - 1024;            // two CTAs (1 KB reserved each) per SM
    for (size_t budget : {budget2, optin}) {
        if (off >= budget) continue;
        const size_t per_warp = (budget - off) / kYcWarps;
        int qc = b;
        for (; qc >= 1; --qc) {
            if (qc < b && (qc * b) % 2) continue;
            if (2 * (size_t)yc_align((uint32_t)(qc * b * sizeof(GT))) * NPL <= per_warp) break;
        }
        if (qc < 1) continue;
        {
            const int nch = (b + qc - 1) / qc;
            int q2 = (b + nch - 1) / nch;
            if (q2 < b && (q2 * b) % 2) ++q2;
            if (q2 <= qc) qc = q2;
        }
        const uint32_t pb = yc_align((uint32_t)(qc * b * sizeof(GT)));
        const uint32_t stb = pb * NPL;
        if (budget == budget2 && stb < 3072 && qc < b) continue;
        const size_t nfix = std::min<size_t>(kYcMaxStages, per_warp / stb);
        const size_t per_f = (size_t)(y.off_uh - y.off_f0) / kYcWarps / stb;
        y.Qc = qc;
        y.nchunks = (b + qc - 1) / qc;
        y.off_g1 = pb;
        y.stage_bytes = stb;
        y.nfix = (int)nfix;
        y.nstages = (int)std::min<size_t>(kYcMaxStages, nfix + per_f);
        y.smem = off + (size_t)kYcWarps * nfix * stb;
        return true;
    }
    return false;
}

// The kernel instance for the plan's block size: rows per lane R = ceil(b/32) up to 4; four columns per
// launch only with R <= 2 (at most eight accumulators per lane).
using YcKernel = void (*)(YcArgs);
template <class A, int KC>
static YcKernel yc_kernel(int b) {
    const int R = (b + 31) / 32;
    if (R <= 1) return ycontract_kernel<A, KC, 1, false>;
    if (R == 2) return b % 2 == 0 ? ycontract_kernel<A, KC, 2, true> : ycontract_kernel<A, KC, 2, false>;
    if constexpr (KC == 1) {
        if (R == 3) return ycontract_kernel<A, 1, 3, false>;
        if (R == 4) return ycontract_kernel<A, 1, 4, false>;
    }
    return nullptr;
}

template <class A, int KC>
static cudaError_t yc_config(const Plan *p, const YcShape &y, cudaLaunchConfig_t &cfg, cudaLaunchAttribute *attr,
                             int ncols_groups) {
    cfg = {};
    cfg.gridDim = dim3(p->mx * y.Q, 1, 1);
    cfg.blockDim = dim3(kYcThreads);
    cfg.dynamicSmemBytes = y.smem;
    cfg.stream = p->stream;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = y.Q;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    (void)ncols_groups;
    const YcKernel kern = yc_kernel<A, KC>(p->b);
    if (!kern) return cudaErrorInvalidConfiguration;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_optin);
}

// Largest cluster size whose mx clusters are all resident at once (the occupancy API decides), so that
// every CTA streams its share of the spectrum from the start; false if none fits.
template <class A, int KC>
static bool yc_choose(Plan *p, int kc, YcShape &out) {
    const int qmax = std::min(8, std::min(p->b, p->my));
    for (int Q = qmax; Q >= 1; --Q) {
        if (p->yc_force_q && Q != p->yc_force_q) continue;
        YcShape y;
        if (!yc_layout<A, KC>(p, kc, Q, y)) continue;
        cudaLaunchConfig_t cfg;
        cudaLaunchAttribute attr[2];
        if (yc_config<A, KC>(p, y, cfg, attr, 1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        int nclus = 0;
        if (cudaOccupancyMaxActiveClusters(&nclus, yc_kernel<A, KC>(p->b), &cfg) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (nclus >= p->mx || (p->yc_force_q && nclus >= 1)) {   // a forced size may run in waves
            out = y;
            return true;
        }
    }
    return false;
}

template <class A, int KC>
static int yc_launch(Plan *p, const void *U, void *V, int kc, const int *active, const YcShape &y) {
    using GT = typename GElem<A>::T;
    constexpr int NPL = GElem<A>::planes;
    YcArgs a{};
    a.U = U;
    a.V = V;
    a.plane = (long)p->ny * p->mx * p->b;
    if constexpr (A::kind == 0) {
        a.g0 = p->ghat_hi;
        a.g1 = p->ghat_lo;
    } else {
        a.g0 = p->ghat_hi;
        a.g1 = nullptr;
    }
    a.gbs = p->gbs;
    a.active = active;
    a.nx = p->nx;
    a.ny = p->ny;
    a.mx = p->mx;
    a.my = p->my;
    a.b = p->b;
    a.kc = kc;
    a.Q = y.Q;
    a.pshare = y.pshare;
    a.kshare = y.kshare;
    a.Qc = y.Qc;
    a.nchunks = y.nchunks;
    a.nstages = y.nstages;
    a.nfix = y.nfix;
    a.stage_bytes = y.stage_bytes;
    a.off_g1 = y.off_g1;
    a.off_tw = y.off_tw;
    a.off_f0 = y.off_f0;
    a.off_f1 = y.off_f1;
    a.off_uh = y.off_uh;
    a.off_ring = y.off_ring;
    const FftPlan &fy = p->fy.M == p->my ? p->fy : p->fx;
    Fft2Side sd;
    sd.M = fy.M;
    sd.nst = fy.nst;
    {
        int ns = 1;
        for (int i = 0; i < fy.nst; ++i) {
            sd.radix[i] = fy.radix[i];
            sd.nsmagic[i] = ns == 1 ? 0u : (unsigned)((0x100000000ull + ns - 1) / ns);
            ns *= fy.radix[i];
        }
    }
    a.sy = sd;
    a.twy = A::kind == 0 ? (const void *)fy.tw_df : (const void *)fy.tw_f32;
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
    if (!a.g0 || (NPL == 2 && !a.g1) || !a.twy)
        return set_error(p, BTTB_ERR_INVALID_ARG, "plan does not keep the spectrum copy this precision reads");
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    cudaError_t e = yc_config<A, KC>(p, y, cfg, attr, 1);
    if (e != cudaSuccess) return check_cuda(p, e, "fused y-level product smem attribute");
    const int tok = prof_begin(p, BTTB_K_BLOCK_PRODUCT_PREC + (A::kind == 0 ? BTTB_MV_FP64 : BTTB_MV_FP32));
    e = cudaLaunchKernelEx(&cfg, yc_kernel<A, KC>(p->b), a);
    count_launch(p);
    if (e != cudaSuccess) return check_cuda(p, e, "fused y-level product launch");
    // algorithmic bytes: the spectrum planes once, U in and V out (the intermediates stay on chip)
    const double bins = (double)p->mx * p->my;
    prof_end(p, tok, bins * p->b * p->b * sizeof(GT) * NPL +
                         2.0 * kc * (double)p->ny * p->mx * p->b * sizeof(typename A::C));
    return check_cuda(p, cudaGetLastError(), "fused y-level product launch");
}

template <class A, int KC>
static YcShape &yc_shape(Plan *p, int k) {
    YcShape &y = p->yc[A::kind == 0 ? 1 : 0][k - 1];
    if (y.ok < 0) {
        YcShape t;
        t.ok = yc_choose<A, KC>(p, k, t) ? 1 : 0;
        y = t;
    }
    return y;
}

// Diagnostics (bttb_plan_debug): the cluster size and ring depth chosen, or for a given cluster size Q
// the number of clusters the occupancy API lets run at once (negative: that shape does not fit).
template <class A, int KC>
static int yc_probe(Plan *p, int k, int Q) {
    if (Q == 0) {
        const YcShape &y = yc_shape<A, KC>(p, k);
        return y.ok == 1 ? (y.Q | (y.nstages << 8)) : 0;
    }
    YcShape y;
    if (!yc_layout<A, KC>(p, k, Q, y)) return -1;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    if (yc_config<A, KC>(p, y, cfg, attr, 1) != cudaSuccess) {
        cudaGetLastError();
        return -2;
    }
    int nclus = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&nclus, yc_kernel<A, KC>(p->b), &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return -1000 - (int)e;
    }
    return nclus;
}

int ycontract_probe(Plan *p, int prec, int k, int Q) {
    if (k < 1 || k > 4) return -1;
    if (prec == PREC_DF64) return k == 1 ? yc_probe<DF64, 1>(p, k, Q) : yc_probe<DF64, 4>(p, k, Q);
    if (prec == PREC_F32) return k == 1 ? yc_probe<F32, 1>(p, k, Q) : yc_probe<F32, 4>(p, k, Q);
    return -1;
}

bool ycontract_fits(Plan *p, int prec, int k) {
    if (k < 1 || k > 4 || p->b > 128 || (k > 1 && p->b > 64)) return false;
    if (prec == PREC_DF64) return (k == 1 ? yc_shape<DF64, 1>(p, k) : yc_shape<DF64, 4>(p, k)).ok == 1;
    if (prec == PREC_F32) return (k == 1 ? yc_shape<F32, 1>(p, k) : yc_shape<F32, 4>(p, k)).ok == 1;
    return false;
}

int ycontract_launch(Plan *p, int prec, const void *U, void *V, int k, const int *active) {
    if (!ycontract_fits(p, prec, k)) return set_error(p, BTTB_ERR_INVALID_ARG, "fused y-level product does not fit");
    if (prec == PREC_DF64)
        return k == 1 ? yc_launch<DF64, 1>(p, U, V, k, active, p->yc[1][0]) : yc_launch<DF64, 4>(p, U, V, k, active, p->yc[1][k - 1]);
    return k == 1 ? yc_launch<F32, 1>(p, U, V, k, active, p->yc[0][0]) : yc_launch<F32, 4>(p, U, V, k, active, p->yc[0][k - 1]);
}

}  // namespace bttb
