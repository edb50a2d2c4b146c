// Batched mixed-radix FFT passes and the generator spectrum.
//
// The multilevel FFT of the paper (Sec. III-A, App. A/B) transforms, for
// every basis index, a sequence of cells along one level of the array with
// the other level held fixed.  In memory the basis index is the fastest, so a
// pass is a batch of strided 1-D transforms whose batch index is contiguous.
// One CTA takes P consecutive batch indices (P a power of two), stages the
// P interleaved sequences in shared memory (zero-padded to M, Eq. (xc2)),
// and runs a Stockham autosort FFT with radix 2/3/4/5 butterflies; consecutive
// threads work on consecutive batch indices, so every shared-memory access is
// conflict-free and every global access is a coalesced run of P elements.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include <cooperative_groups.h>

#include "arith.cuh"
#include "fftcore.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace bttb {

int smallest_5smooth(int n) {
    for (int m = n < 1 ? 1 : n;; ++m) {
        int r = m;
        for (int f : {2, 3, 5})
            while (r % f == 0) r /= f;
        if (r == 1) return m;
    }
}

static void split_df(long double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (long double)hi);
}

int fft_plan_init(Plan *p, FftPlan &f, int M) {
    f.M = M;
    f.nst = 0;
    int r = M;
    const int order[4] = {4, 2, 3, 5};
    for (int oi = 0; oi < 4; ++oi) {
        int R = order[oi];
        while (r % R == 0 && r > 1) {
            if (f.nst >= kMaxRadixStages) return set_error(p, BTTB_ERR_INVALID_ARG, "FFT length has too many factors");
            f.radix[f.nst++] = R;
            r /= R;
        }
    }
    if (r != 1) return set_error(p, BTTB_ERR_INVALID_ARG, "FFT length is not 5-smooth");
    const int ntab = M + 5;
    std::vector<double2> t64(ntab);
    std::vector<float4> tdf(ntab);
    std::vector<float2> t32(ntab);
    const long double two_pi = 6.283185307179586476925286766559005768L;
    std::vector<long double> re(ntab), im(ntab);
    for (int t = 0; t < M; ++t) {
        long double a = -two_pi * (long double)t / (long double)M;
        re[t] = cosl(a);
        im[t] = sinl(a);
    }
    const long double sq5 = sqrtl(5.0L);
    const long double consts[5] = {(sq5 - 1.0L) / 4.0L, -(sq5 + 1.0L) / 4.0L, sqrtl((5.0L + sq5) / 8.0L),
                                   sqrtl((5.0L - sq5) / 8.0L), sqrtl(3.0L) / 2.0L};
    for (int c = 0; c < 5; ++c) {
        re[M + c] = consts[c];
        im[M + c] = 0.0L;
    }
    for (int t = 0; t < ntab; ++t) {
        t64[t] = make_double2((double)re[t], (double)im[t]);
        float rh, rl, ih, il;
        split_df(re[t], rh, rl);
        split_df(im[t], ih, il);
        tdf[t] = make_float4(rh, ih, rl, il);
        t32[t] = make_float2(rh, ih);
    }
    cudaError_t e;
    if ((e = dev_malloc((void **)&f.tw_f64, ntab * sizeof(double2))) != cudaSuccess) return check_cuda(p, e, "twiddles");
    if ((e = dev_malloc((void **)&f.tw_df, ntab * sizeof(float4))) != cudaSuccess) return check_cuda(p, e, "twiddles");
    if ((e = dev_malloc((void **)&f.tw_f32, ntab * sizeof(float2))) != cudaSuccess) return check_cuda(p, e, "twiddles");
    cudaMemcpy(f.tw_f64, t64.data(), ntab * sizeof(double2), cudaMemcpyHostToDevice);
    cudaMemcpy(f.tw_df, tdf.data(), ntab * sizeof(float4), cudaMemcpyHostToDevice);
    e = cudaMemcpy(f.tw_f32, t32.data(), ntab * sizeof(float2), cudaMemcpyHostToDevice);
    return check_cuda(p, e, "twiddle upload");
}

void fft_plan_free(FftPlan &f) {
    cudaFree(f.tw_f64);
    cudaFree(f.tw_df);
    cudaFree(f.tw_f32);
    f.tw_f64 = nullptr;
    f.tw_df = nullptr;
    f.tw_f32 = nullptr;
}

// Whether an input format is the number system's own element or its leading part, so that the load is a
// plain copy (8 bytes for binary32, 16 for the others): then it can be an asynchronous copy.
template <class A, int INF>
constexpr bool async_copyable() {
    return (A::kind == 1 && (INF == FMT_C64 || INF == FMT_CDF)) || (A::kind == 0 && INF == FMT_CDF) ||
           (A::kind == 2 && INF == FMT_C128);
}

template <class A, int INF, int OUTF, bool INV>
__global__ void __launch_bounds__(kFftThreads) fft_pass_kernel(const FftPass a) {
    using C = typename A::C;
    using K = typename A::K;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *const buf0 = tw + (a.M + 8);                        // buffers buf0 + k*M*P, k < 2 (3 with a.cpb > 1)
    auto buf = [&](int k) { return buf0 + k * (a.M * a.P); };

    const int tid = threadIdx.x, nt = blockDim.x;
    const int o = blockIdx.x;
    const int p0 = blockIdx.y * a.P;
    const int P = a.P, lP = a.log2P, M = a.M;
    // the twiddles are constant: stage them before waiting for the preceding kernel
    const C *twg = reinterpret_cast<const C *>(a.tw);
    for (int i = tid; i < M + 5; i += nt) tw[i] = twg[i];
    pdl_wait();

    const int pp = tid & (P - 1), j0 = tid >> lP, jstep = nt >> lP;
    const long sel = a.in_sel ? (long)(*a.in_sel) * a.in_sel_stride : 0;

    // column c's M x P input: zero-padded beyond nin rows and pdim bases
    auto load_direct = [&](int c, C *dst) {
        const long ibase = (long)c * a.in_cs + (long)o * a.in_os + sel;
        const double scl = a.in_scale ? a.in_scale[c] : 1.0;
        for (int idx = tid; idx < M * P; idx += nt) {
            const int n = idx >> lP, q = idx & (P - 1), pi = p0 + q;
            C v = A::zero();
            if (n < a.nin && pi < a.pdim) {
                v = load_vec<A, INF>(a.in, ibase + (long)n * a.in_ns + pi);
                if (a.in_scale) v = scale_by<A>(v, scl);
            }
            dst[idx] = v;
        }
    };
    auto load_async = [&](int c, C *dst) {
        if constexpr (async_copyable<A, INF>()) {
            const long ibase = (long)c * a.in_cs + (long)o * a.in_os + sel;
            for (int idx = tid; idx < M * P; idx += nt) {
                const int n = idx >> lP, q = idx & (P - 1), pi = p0 + q;
                if (n < a.nin && pi < a.pdim) {
                    const long e = ibase + (long)n * a.in_ns + pi;
                    if constexpr (sizeof(C) == 8) {
                        // binary32: the element itself, or the leading (high) part of a double-float element
                        const char *src = reinterpret_cast<const char *>(a.in) + e * (INF == FMT_CDF ? 16 : 8);
                        cp_async8(dst + idx, src);
                    } else {
                        cp_async16(dst + idx, reinterpret_cast<const char *>(a.in) + e * 16);
                    }
                } else {
                    dst[idx] = A::zero();
                }
            }
        }
        cp_async_commit();
    };
    // (called after a barrier that follows the twiddle staging)
    auto stages = [&](C *src, C *dst) -> C * { return fft_pass_stages<A, INV>(a, src, dst, tw); };
    auto store = [&](int c, const C *res) {
        const long obase = (long)c * a.out_cs + (long)o * a.out_os;
        for (int idx = tid; idx < a.nout * P; idx += nt) {
            const int n = idx >> lP, q = idx & (P - 1), pi = p0 + q;
            if (pi < a.pdim) store_vec<A, OUTF>(a.out, obase + (long)n * a.out_ns + pi, res[idx]);
        }
    };

    const int cfirst = blockIdx.z * a.cpb, cend = min(cfirst + a.cpb, a.ncols);
    if (a.cpb == 1 || !async_copyable<A, INF>() || a.in_scale) {
        for (int c = cfirst; c < cend; ++c) {
            if (a.active && !a.active[c]) continue;         // finished column (uniform per CTA)
            load_direct(c, buf(0));
            __syncthreads();
            const C *res = stages(buf(0), buf(1));
            if (c == cend - 1) pdl_trigger();               // the next pass may start launching
            store(c, res);
            __syncthreads();                                // the buffers are reused by the next column
        }
        if (cfirst >= cend) pdl_trigger();
        return;
    }
    // several columns: input of column c+1 streams into the third buffer while column c is transformed
    int i = 0;                                              // column c: input buf(i), temporary buf(i+1)
    load_async(cfirst, buf(0));
    for (int c = cfirst; c < cend; ++c) {
        cp_async_wait<0>();
        __syncthreads();                                    // column c's input landed; column c-1 is stored
        C *in = buf(i), *tmp = buf(i == 2 ? 0 : i + 1), *nxt = buf(i == 0 ? 2 : i - 1);
        if (c + 1 < cend) load_async(c + 1, nxt);
        if (!a.active || a.active[c]) {                     // finished column (uniform per CTA)
            const C *res = stages(in, tmp);
            if (c == cend - 1) pdl_trigger();
            store(c, res);
        }
        i = i == 0 ? 2 : i - 1;
    }
    cp_async_wait<0>();
    pdl_trigger();
}

template <class A, int INF, int OUTF, bool INV>
static int launch_one(Plan *p, const FftPass &a) {
    using C = typename A::C;
    size_t smem = ((size_t)a.M + 8 + (a.cpb > 1 ? 3 : 2) * (size_t)a.M * a.P) * sizeof(C);
    auto kern = fft_pass_kernel<A, INF, OUTF, INV>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_optin);
        if (e != cudaSuccess) return check_cuda(p, e, "fft smem attribute");
    }
    dim3 grid(a.O, (a.pdim + a.P - 1) / a.P, (a.ncols + a.cpb - 1) / a.cpb);
    const int tok = prof_begin(p, BTTB_K_FFT);
    cudaError_t le = launch_pdl(kern, grid, dim3(kFftThreads), smem, p->stream, a);
    count_launch(p);
    if (le != cudaSuccess) return check_cuda(p, le, "fft pass launch");
    auto esz = [](int f) { return f == FMT_C128 ? 16.0 : (f == FMT_C64 ? 8.0 : 16.0); };
    prof_end(p, tok, (double)a.O * a.pdim * a.ncols * (a.nin * esz(INF) + a.nout * esz(OUTF)));
    return check_cuda(p, cudaGetLastError(), "fft pass launch");
}

template <class A>
static int dispatch_fmt(Plan *p, const FftPass &a, int infmt, int outfmt, bool inv) {
    constexpr int NF = native_fmt<A>;
    if (!inv) {
        if (outfmt != NF) return set_error(p, BTTB_ERR_INVALID_ARG, "forward pass writes native format only");
        switch (infmt) {
            case FMT_C128: return launch_one<A, FMT_C128, NF, false>(p, a);
            case FMT_C64: return launch_one<A, FMT_C64, NF, false>(p, a);
            default: return launch_one<A, FMT_CDF, NF, false>(p, a);
        }
    } else {
        if (infmt != NF) return set_error(p, BTTB_ERR_INVALID_ARG, "inverse pass reads native format only");
        switch (outfmt) {
            case FMT_C128: return launch_one<A, NF, FMT_C128, true>(p, a);
            case FMT_C64: return launch_one<A, NF, FMT_C64, true>(p, a);
            default: return launch_one<A, NF, FMT_CDF, true>(p, a);
        }
    }
}

static int choose_P(int M, int pdim, size_t elem, int pmax, int nbuf) {
    int P = 1;
    while (P < pmax && P < pdim) P <<= 1;
    while (P > 1 && ((size_t)M + 8 + nbuf * (size_t)M * P) * elem > 96 * 1024) P >>= 1;
    return P;
}

// Columns per CTA of a pass: one for few columns; with many, four, so that each CTA prefetches the next
// column's input while it transforms one (the grid still fills every SM many times over).
constexpr int kFftMultiCols = 4;
constexpr int kFftMultiMinCols = 32;

int fft_pass_prepare(Plan *p, FftPass &a, int prec, int pmax) {
    const FftPlan &f = (a.M == p->fx.M) ? p->fx : p->fy;
    if (f.M != a.M) return set_error(p, BTTB_ERR_INVALID_ARG, "no FFT plan for this length");
    a.nst = f.nst;
    {
        int ns = 1;
        for (int i = 0; i < f.nst; ++i) {
            a.radix[i] = f.radix[i];
            a.nsmagic[i] = ns == 1 ? 0u : (unsigned)((0x100000000ull + ns - 1) / ns);   // ceil(2^32 / Ns)
            ns *= f.radix[i];
        }
    }
    size_t elem = prec == PREC_F32 ? 8 : 16;
    if (a.cpb < 1) a.cpb = a.ncols >= kFftMultiMinCols ? kFftMultiCols : 1;
    a.P = choose_P(a.M, a.pdim, elem, pmax, a.cpb > 1 ? 3 : 2);
    a.log2P = 0;
    while ((1 << a.log2P) < a.P) ++a.log2P;
    switch (prec) {
        case PREC_F64N: a.tw = f.tw_f64; break;
        case PREC_F32: a.tw = f.tw_f32; break;
        default: a.tw = f.tw_df; break;
    }
    return BTTB_OK;
}

int fft_pass_launch(Plan *p, FftPass a, int prec, int infmt, int outfmt, bool inverse) {
    a.cpb = 0;
    const int rc = fft_pass_prepare(p, a, prec, p->fft_pmax);
    if (rc != BTTB_OK) return rc;
    if (a.O <= 0 || a.ncols <= 0 || a.pdim <= 0) return BTTB_OK;
    switch (prec) {
        case PREC_F64N: return dispatch_fmt<F64N>(p, a, infmt, outfmt, inverse);
        case PREC_F32: return dispatch_fmt<F32>(p, a, infmt, outfmt, inverse);
        default: return dispatch_fmt<DF64>(p, a, infmt, outfmt, inverse);
    }
}

// ---------------------------------------------------------------------------
// Both levels of the forward (or inverse) 2-level FFT in one kernel, for
// products of few vectors, where the two strided passes above are bound by
// their launch and memory latency rather than by bandwidth.  A cluster of Q
// CTAs takes one basis index p of one column.  For the forward transform CTA
// r loads its share of the ny nonzero rows, transforms them along kx (the x
// level, in shared memory [kx][row]), and sends every column kx to the CTA
// that owns it in the cluster's distributed shared memory; after one cluster
// barrier each CTA transforms its columns along iy (the y level, [kx][iy]
// with the iy stride rounded up to odd: conflict-free) and writes its bins.
// The inverse runs the same steps in reverse order.  The padding of Eq. (xc2)
// is the zero fill of the unused slots; the crop of Sec. II-C keeps the first
// nx, ny outputs.
// ---------------------------------------------------------------------------
struct Fft2Args {
    const void *in;
    void *out;
    long ld;                      // column stride of the cell-ordered vector (x for forward, y for inverse)
    long ubs;                     // spectrum side: element (bin, c, p) at bin*ubs + c*b + p
    const int *in_sel;            // forward only: input offset += (*in_sel) * in_sel_stride
    long in_sel_stride;
    const double *in_scale;       // forward only: per-column scale applied on load
    const int *active;
    int nx, ny, b, ms;            // ms: iy stride of a column share (my rounded up to odd)
    int xs, ncmax;                // row stride of a row share (ceil(ny/Q) rounded up to odd); widest column share
    Fft2Side sx, sy;
    const void *twx, *twy;
};

constexpr int kFft2Threads = 128;

// Forward: x (cell order, format INF) -> u^ (native).  Inverse: v^ (native) -> y (cell order, format OUTF).
// Launched with clusters of Q CTAs along x: CTA (p*Q + r, c) is rank r of the cluster for basis p, column c.
template <class A, int INF, int OUTF, bool INV>
__global__ void __launch_bounds__(kFft2Threads) fft2_fused_kernel(const Fft2Args a) {
    namespace cg = cooperative_groups;
    using C = typename A::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cl = cg::this_cluster();
    const int Q = (int)cl.num_blocks(), r = (int)cl.block_rank();
    const int mx = a.sx.M, my = a.sy.M, ms = a.ms, xs = a.xs, nx = a.nx, ny = a.ny, b = a.b;
    const int p = blockIdx.x / Q, c = blockIdx.y;
    // row share [rlo, rhi) of the ny nonzero rows, column share [clo, chi) of the mx columns
    const int rlo = r * ny / Q, nrow = (r + 1) * ny / Q - rlo;
    const int clo = r * mx / Q, ncol = (r + 1) * mx / Q - clo;
    C *twx = reinterpret_cast<C *>(smem_raw);
    C *twy = twx + (mx + 8);
    C *X0 = twy + (my + 8);                                // [kx][row of the share], stride xs
    C *X1 = X0 + mx * xs;
    C *Y0 = X1 + mx * xs;                                  // [column of the share][iy], stride ms
    C *Y1 = Y0 + a.ncmax * ms;
    for (int i = threadIdx.x; i < mx + 5; i += blockDim.x) twx[i] = reinterpret_cast<const C *>(a.twx)[i];
    for (int i = threadIdx.x; i < my + 5; i += blockDim.x) twy[i] = reinterpret_cast<const C *>(a.twy)[i];
    pdl_wait();
    if (a.active && !a.active[c]) return;                  // uniform over the cluster (same column)
    // every CTA of the cluster must have started before another writes into its shared memory: arrive now,
    // wait just before the exchange (long satisfied by then)
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
    if (!INV) {
        long ib = (long)c * a.ld + p;
        if (a.in_sel) ib += (long)(*a.in_sel) * a.in_sel_stride;
        const double scl = a.in_scale ? a.in_scale[c] : 1.0;
        for (int idx = threadIdx.x; idx < mx * nrow; idx += blockDim.x) {
            const int kx = idx / nrow, il = idx - kx * nrow;
            C v = A::zero();
            if (kx < nx) {
                v = load_vec<A, INF>(a.in, ib + ((long)(rlo + il) * nx + kx) * b);
                if (a.in_scale) v = scale_by<A>(v, scl);
            }
            X0[kx * xs + il] = v;
        }
        // the y level's padding rows of this CTA's columns (the exchange fills rows iy < ny)
        for (int idx = threadIdx.x; idx < ncol * ms; idx += blockDim.x)
            if (idx % ms >= ny) Y0[idx] = A::zero();
        __syncthreads();
        const C *R1 = fft2_level<A, false>(X0, X1, twx, a.sx, xs, nrow, 1);       // along kx, own rows
        asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
        for (int idx = threadIdx.x; idx < mx * nrow; idx += blockDim.x) {
            const int kx = idx / nrow, il = idx - kx * nrow;
            const int q = ((kx + 1) * Q - 1) / mx;                                  // owner of column kx
            C *dst = cl.map_shared_rank(Y0, q);
            const long di = (long)(kx - q * mx / Q) * ms + rlo + il;
            if (BTTB_ICHK(di, (long)a.ncmax * ms)) dst[di] = R1[kx * xs + il];
        }
        cl.sync();
        const C *R2 = fft2_level<A, false>(Y0, Y1, twy, a.sy, 1, ncol, ms);       // along iy, own columns
        pdl_trigger();
        for (int idx = threadIdx.x; idx < ncol * ms; idx += blockDim.x) {
            const int kl = idx / ms, ky = idx - kl * ms;
            if (ky < my)
                store_vec<A, native_fmt<A>>(a.out, ((long)ky * mx + clo + kl) * a.ubs + (long)c * b + p, R2[idx]);
        }
    } else {
        for (int idx = threadIdx.x; idx < ncol * ms; idx += blockDim.x) {
            const int kl = idx / ms, ky = idx - kl * ms;
            C v = A::zero();
            if (ky < my) v = load_vec<A, native_fmt<A>>(a.in, ((long)ky * mx + clo + kl) * a.ubs + (long)c * b + p);
            Y0[idx] = v;
        }
        __syncthreads();
        const C *R1 = fft2_level<A, true>(Y0, Y1, twy, a.sy, 1, ncol, ms);        // along ky, own columns
        asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
        for (int idx = threadIdx.x; idx < ncol * ny; idx += blockDim.x) {
            const int kl = idx / ny, iy = idx - kl * ny;
            const int q = ((iy + 1) * Q - 1) / ny;                                  // owner of row iy
            C *dst = cl.map_shared_rank(X0, q);
            const long di = (long)(clo + kl) * xs + iy - q * ny / Q;
            if (BTTB_ICHK(di, (long)mx * xs)) dst[di] = R1[kl * ms + iy];
        }
        cl.sync();
        const C *R2 = fft2_level<A, true>(X0, X1, twx, a.sx, xs, nrow, 1);        // along kx, own rows
        pdl_trigger();
        const long ob = (long)c * a.ld + p;
        for (int idx = threadIdx.x; idx < nrow * nx; idx += blockDim.x) {
            const int il = idx / nx, ix = idx - il * nx;
            store_vec<A, OUTF>(a.out, ob + ((long)(rlo + il) * nx + ix) * b, R2[ix * xs + il]);
        }
    }
}

static void fft2_side(const FftPlan &f, Fft2Side &sd) {
    sd.M = f.M;
    sd.nst = f.nst;
    int ns = 1;
    for (int i = 0; i < f.nst; ++i) {
        sd.radix[i] = f.radix[i];
        sd.nsmagic[i] = ns == 1 ? 0u : (unsigned)((0x100000000ull + ns - 1) / ns);
        ns *= f.radix[i];
    }
}

// CTAs per cluster of the fused FFT: up to 8 (the portable cluster size), no more than the grid lengths.
static int fft2_cluster(const Plan *p) { return std::max(1, std::min(8, std::min(p->mx, p->ny))); }

static void fft2_shape(const Plan *p, int &Q, int &ms, int &xs, int &ncmax) {
    Q = fft2_cluster(p);
    ms = p->my | 1;
    xs = ((p->ny + Q - 1) / Q) | 1;
    ncmax = (p->mx + Q - 1) / Q;
}

size_t fft2_fused_smem(const Plan *p, int prec) {
    const size_t elem = prec == PREC_F32 ? 8 : 16;
    int Q, ms, xs, ncmax;
    fft2_shape(p, Q, ms, xs, ncmax);
    return ((size_t)p->mx + 8 + p->my + 8 + 2 * (size_t)p->mx * xs + 2 * (size_t)ncmax * ms) * elem;
}

template <class A, int INF, int OUTF, bool INV>
static int launch_fused(Plan *p, const Fft2Args &a, int ncols, size_t smem) {
    auto kern = fft2_fused_kernel<A, INF, OUTF, INV>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_optin);
        if (e != cudaSuccess) return check_cuda(p, e, "fused fft smem attribute");
    }
    const int Q = fft2_cluster(p);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.b * Q, ncols);
    cfg.blockDim = dim3(kFft2Threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = p->stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = Q;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    const int tok = prof_begin(p, BTTB_K_FFT);
    cudaError_t le = cudaLaunchKernelEx(&cfg, kern, a);
    count_launch(p);
    if (le != cudaSuccess) return check_cuda(p, le, "fused fft launch");
    const double esz_in = INF == FMT_C64 ? 8.0 : 16.0, esz_out = OUTF == FMT_C64 ? 8.0 : 16.0;
    prof_end(p, tok, (double)ncols * a.b * ((double)a.nx * a.ny * esz_in + (double)a.sx.M * a.sy.M * esz_out));
    return check_cuda(p, cudaGetLastError(), "fused fft launch");
}

template <class A>
static int fused_dispatch(Plan *p, const Fft2Args &a, int ncols, int cellfmt, bool inv, size_t smem) {
    constexpr int NF = native_fmt<A>;
    if (!inv) {
        switch (cellfmt) {
            case FMT_C128: return launch_fused<A, FMT_C128, NF, false>(p, a, ncols, smem);
            case FMT_C64: return launch_fused<A, FMT_C64, NF, false>(p, a, ncols, smem);
            default: return launch_fused<A, FMT_CDF, NF, false>(p, a, ncols, smem);
        }
    }
    switch (cellfmt) {
        case FMT_C128: return launch_fused<A, NF, FMT_C128, true>(p, a, ncols, smem);
        case FMT_C64: return launch_fused<A, NF, FMT_C64, true>(p, a, ncols, smem);
        default: return launch_fused<A, NF, FMT_CDF, true>(p, a, ncols, smem);
    }
}

int fft2_fused_launch(Plan *p, const void *in, void *out, long ld, int ncols, int prec, int cellfmt, bool inverse,
                      const int *in_sel, long in_sel_stride, const double *in_scale, const int *active) {
    Fft2Args a{};
    a.in = in;
    a.out = out;
    a.ld = ld;
    a.ubs = p->ubs;
    a.in_sel = in_sel;
    a.in_sel_stride = in_sel_stride;
    a.in_scale = in_scale;
    a.active = active;
    a.nx = p->nx;
    a.ny = p->ny;
    a.b = p->b;
    int Q;
    fft2_shape(p, Q, a.ms, a.xs, a.ncmax);
    // with my == mx the plan keeps one set of tables (fx) and marks fy unused
    const FftPlan &fx = p->fx, &fy = p->fy.M == p->my ? p->fy : p->fx;
    if (fx.M != p->mx || fy.M != p->my)
        return set_error(p, BTTB_ERR_INVALID_ARG, "no FFT plan for the grid lengths");
    fft2_side(fx, a.sx);
    fft2_side(fy, a.sy);
    if (ncols <= 0) return BTTB_OK;
    const size_t smem = fft2_fused_smem(p, prec);
    switch (prec) {
        case PREC_F64N: a.twx = fx.tw_f64; a.twy = fy.tw_f64; break;
        case PREC_F32: a.twx = fx.tw_f32; a.twy = fy.tw_f32; break;
        default: a.twx = fx.tw_df; a.twy = fy.tw_df; break;
    }
    if (!a.twx || !a.twy) return set_error(p, BTTB_ERR_INVALID_ARG, "FFT twiddle tables missing");
    switch (prec) {
        case PREC_F64N: return fused_dispatch<F64N>(p, a, ncols, cellfmt, inverse, smem);
        case PREC_F32: return fused_dispatch<F32>(p, a, ncols, cellfmt, inverse, smem);
        default: return fused_dispatch<DF64>(p, a, ncols, cellfmt, inverse, smem);
    }
}

// ---------------------------------------------------------------------------
// Generator spectrum (one-time, binary64): Eq. (circL2) places T[i,j] at cell
// slot (i mod mx, j mod my); Eq. (multL) needs the 2-D DFT of that block
// column for each of the b*b entries.
// ---------------------------------------------------------------------------
__global__ void gen_check_kernel(const double2 *g, long count, int *err) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
        double2 v = g[i];
        if (!isfinite(v.x) || !isfinite(v.y)) atomicOr(err, DEVERR_NONFINITE);
    }
}

__global__ void gen_widen_kernel(const float2 *src, double2 *dst, long count) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
        dst[i] = make_double2(src[i].x, src[i].y);
}

// w[sy][sx][e] = T[i,j][e] at (sx, sy) = (i mod mx, j mod my), zero elsewhere.
__global__ void gen_scatter_kernel(const double2 *gen, double2 *w, int nx, int ny, int mx, int my, int bb) {
    const int sx = blockIdx.x, sy = blockIdx.y;
    int i = sx < nx ? sx : sx - mx;       // offsets 0..nx-1 then -(nx-1)..-1
    int j = sy < ny ? sy : sy - my;
    const bool on = (i > -nx && i < nx && j > -ny && j < ny);
    double2 *dst = w + ((long)sy * mx + sx) * bb;
    const double2 *src = on ? gen + ((long)(j + ny - 1) * (2 * nx - 1) + (i + nx - 1)) * bb : nullptr;
    for (int e = threadIdx.x; e < bb; e += blockDim.x) dst[e] = on ? src[e] : make_double2(0.0, 0.0);
}

// Scale by 1/(mx*my), transpose each bin to column-major, split into copies.
__global__ void gen_finish_kernel(const double2 *w, long bins, int b, long gbs, double scale, float2 *hi,
                                  float2 *lo, double2 *f64, int *err) {
    const long bin = blockIdx.x;
    const int bb = b * b;
    for (int e = threadIdx.x; e < bb; e += blockDim.x) {
        const int pr = e / b, q = e % b;           // source entry (p, q) row-major
        double2 v = w[bin * bb + e];
        v.x *= scale;
        v.y *= scale;
        if (!isfinite(v.x) || !isfinite(v.y)) atomicOr(err, DEVERR_NONFINITE);
        const long d = bin * gbs + (long)q * b + pr;
        if (f64) f64[d] = v;
        if (hi) {
            df r = df_from_double(v.x), i = df_from_double(v.y);
            hi[d] = make_float2(r.hi, i.hi);
            if (lo) lo[d] = make_float2(r.lo, i.lo);
        }
    }
}

int spectrum_compute(Plan *p, const void *gen, bttb_dtype dtype, int gen_is_host) {
    const int nx = p->nx, ny = p->ny, b = p->b, mx = p->mx, my = p->my;
    const long bb = (long)b * b;
    const long ngen = (long)(2 * nx - 1) * (2 * ny - 1) * bb;
    const long nw = p->bins * bb;
    double2 *g64 = nullptr, *w1 = nullptr, *w2 = nullptr;
    void *gtmp = nullptr;
    cudaError_t e;
    int rc = BTTB_OK;
    auto fail = [&](cudaError_t ee, const char *what) {
        rc = check_cuda(p, ee, what);
        return rc;
    };
    if ((e = dev_malloc((void **)&g64, ngen * sizeof(double2))) != cudaSuccess) { fail(e, "generator buffer"); goto done; }
    if ((e = dev_malloc((void **)&w1, nw * sizeof(double2))) != cudaSuccess) { fail(e, "spectrum workspace"); goto done; }
    if ((e = dev_malloc((void **)&w2, nw * sizeof(double2))) != cudaSuccess) { fail(e, "spectrum workspace"); goto done; }
    if (dtype == BTTB_C128) {
        e = cudaMemcpyAsync(g64, gen, ngen * sizeof(double2),
                            gen_is_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, p->stream);
        if (e != cudaSuccess) { fail(e, "generator copy"); goto done; }
    } else {
        const void *src = gen;
        if (gen_is_host) {
            if ((e = dev_malloc((void **)&gtmp, ngen * sizeof(float2))) != cudaSuccess) { fail(e, "generator copy"); goto done; }
            e = cudaMemcpyAsync(gtmp, gen, ngen * sizeof(float2), cudaMemcpyHostToDevice, p->stream);
            if (e != cudaSuccess) { fail(e, "generator copy"); goto done; }
            src = gtmp;
        }
        gen_widen_kernel<<<256, 256, 0, p->stream>>>((const float2 *)src, g64, ngen);
    }
    gen_check_kernel<<<256, 256, 0, p->stream>>>(g64, ngen, p->d_err);
    gen_scatter_kernel<<<dim3(mx, my), 256, 0, p->stream>>>(g64, w1, nx, ny, mx, my, (int)bb);
    count_launch(p, dtype == BTTB_C128 ? 2 : 3);
    if ((e = cudaGetLastError()) != cudaSuccess) { fail(e, "scatter"); goto done; }
    {
        // x level: transforms over sx for each (sy, entry)
        FftPass a{};
        a.in = w1; a.out = w2;
        a.in_cs = a.out_cs = 0;
        a.in_os = a.out_os = (long)mx * bb;
        a.in_ns = a.out_ns = bb;
        a.O = my; a.pdim = (int)bb; a.ncols = 1;
        a.nin = a.nout = mx; a.M = mx;
        if ((rc = fft_pass_launch(p, a, PREC_F64N, FMT_C128, FMT_C128, false)) != BTTB_OK) goto done;
        // y level: transforms over sy for each (kx, entry)
        FftPass c{};
        c.in = w2; c.out = w1;
        c.in_os = c.out_os = bb;
        c.in_ns = c.out_ns = (long)mx * bb;
        c.O = mx; c.pdim = (int)bb; c.ncols = 1;
        c.nin = c.nout = my; c.M = my;
        if ((rc = fft_pass_launch(p, c, PREC_F64N, FMT_C128, FMT_C128, false)) != BTTB_OK) goto done;
    }
    gen_finish_kernel<<<(unsigned)p->bins, 256, 0, p->stream>>>(w1, p->bins, b, p->gbs, 1.0 / ((double)mx * my),
                                                                 p->ghat_hi, p->ghat_lo, p->ghat_f64, p->d_err);
    count_launch(p);
    if ((e = cudaGetLastError()) != cudaSuccess) { fail(e, "spectrum finish"); goto done; }
    if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess) { fail(e, "spectrum sync"); goto done; }
done:
    cudaFree(g64);
    cudaFree(w1);
    cudaFree(w2);
    cudaFree(gtmp);
    return rc;
}

}  // namespace bttb
