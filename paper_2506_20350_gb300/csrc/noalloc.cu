// Allocation-free FP64 product for small arrays: bttb_matvec_noalloc.
//
// Some callers cannot call cudaMalloc at all -- a host application that only
// lets plug-ins use memory reserved at load time, code that runs while a CUDA
// graph is being captured, or a process whose allocator is owned by someone
// else.  They cannot create a plan, because a plan allocates its spectrum and
// workspace.  This entry point needs only the caller's generator blocks, input
// and output: the spectrum, its FFT work buffers, the twiddle tables, the
// product workspace and the device error word all live in one file-scope
// __device__ array of kNoAllocScratchBytes, which every GPU that loads the
// library holds until the process exits.
//
// The scratch array is shared by every call on a device and keeps the last
// call's contents.  Every buffer in it is fully rewritten before it is read;
// the device error word the kernels write into (non-finite spectrum entries,
// a bounded wait that ran out) is cleared by each call but never read back:
// the call does not synchronise, so it cannot report what the GPU finds.
// Calls that overlap on the GPU (two streams, or two host threads) race on
// the array: callers must serialise them.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (once per device, with that device current); make that
// first call before any stream capture begins.
#include <cmath>
#include <mutex>
#include <string>

#include "arith.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace bttb {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;      // 64 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static void *g_scratch_ptr[kNoAllocMaxDevices] = {};
static std::mutex g_scratch_mu;

static int scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kNoAllocMaxDevices) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "device ordinal too large");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return check_cuda(nullptr, e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return BTTB_OK;
}

// Twiddle tables exp(-2 pi i t / M) (binary64 sincospi) plus the five radix
// constants, in the three formats the FFT passes read.
__global__ void noalloc_twiddle_kernel(int M, double c1, double c2, double s1, double s2, double s3, double2 *t64,
                                       float4 *tdf, float2 *t32) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < M + 5; t += gridDim.x * blockDim.x) {
        double re, im;
        if (t < M) {
            double s, c;
            sincospi(-2.0 * (double)t / (double)M, &s, &c);
            re = c;
            im = s;
        } else {
            const double k[5] = {c1, c2, s1, s2, s3};
            re = k[t - M];
            im = 0.0;
        }
        t64[t] = make_double2(re, im);
        const df r = df_from_double(re), i = df_from_double(im);
        tdf[t] = make_float4(r.hi, i.hi, r.lo, i.lo);
        t32[t] = make_float2(r.hi, i.hi);
    }
}

// Copies of the spectrum kernels' work, on caller-provided buffers.
__global__ void noalloc_scatter_kernel(const double2 *gen, double2 *w, int nx, int ny, int mx, int my, int bb) {
    const int sx = blockIdx.x, sy = blockIdx.y;
    const int i = sx < nx ? sx : sx - mx;
    const int j = sy < ny ? sy : sy - my;
    const bool on = (i > -nx && i < nx && j > -ny && j < ny);
    double2 *dst = w + ((long)sy * mx + sx) * bb;
    const double2 *src = on ? gen + ((long)(j + ny - 1) * (2 * nx - 1) + (i + nx - 1)) * bb : nullptr;
    for (int e = threadIdx.x; e < bb; e += blockDim.x) dst[e] = on ? src[e] : make_double2(0.0, 0.0);
}

__global__ void noalloc_finish_kernel(const double2 *w, int b, long gbs, double scale, float2 *hi, float2 *lo,
                                      int *err) {
    const long bin = blockIdx.x;
    const int bb = b * b;
    for (int e = threadIdx.x; e < bb; e += blockDim.x) {
        const int pr = e / b, q = e % b;
        double2 v = w[bin * bb + e];
        v.x *= scale;
        v.y *= scale;
        if (!isfinite(v.x) || !isfinite(v.y)) atomicOr(err, DEVERR_NONFINITE);
        const long d = bin * gbs + (long)q * b + pr;
        const df r = df_from_double(v.x), i = df_from_double(v.y);
        hi[d] = make_float2(r.hi, i.hi);
        lo[d] = make_float2(r.lo, i.lo);
    }
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int fill_fft_plan(FftPlan &f, int M, unsigned char *&cur) {
    f.M = M;
    f.nst = 0;
    int r = M;
    const int order[4] = {4, 2, 3, 5};
    for (int oi = 0; oi < 4; ++oi)
        while (r % order[oi] == 0 && r > 1) {
            f.radix[f.nst++] = order[oi];
            r /= order[oi];
        }
    f.tw_f64 = reinterpret_cast<double2 *>(cur);
    cur += align256((M + 5) * sizeof(double2));
    f.tw_df = reinterpret_cast<float4 *>(cur);
    cur += align256((M + 5) * sizeof(float4));
    f.tw_f32 = reinterpret_cast<float2 *>(cur);
    cur += align256((M + 5) * sizeof(float2));
    return r == 1 ? BTTB_OK : BTTB_ERR_INVALID_ARG;
}

}  // namespace bttb

using namespace bttb;

extern "C" int bttb_matvec_noalloc(int nx, int ny, int b, const void *gen, const void *x, void *y, int nrhs,
                                   long ld, void *cuda_stream) {
    if (nx < 1 || ny < 1 || b < 1 || nrhs < 0 || nx > 1024 || ny > 1024 || b > 256)
        return set_error(nullptr, BTTB_ERR_INVALID_ARG, "bttb_matvec_noalloc: bad sizes");
    if (nrhs == 0) return BTTB_OK;
    if (!gen || !x || !y) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "bttb_matvec_noalloc: NULL pointer");
    if (ld < (long)nx * ny * b) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "bttb_matvec_noalloc: ld < N");

    Plan p;    // a plan-shaped view of the scratch array; owns nothing
    p.nx = nx;
    p.ny = ny;
    p.b = b;
    p.max_rhs = nrhs;
    p.n = (long)nx * ny * b;
    p.mx = smallest_5smooth(2 * nx - 1);
    p.my = smallest_5smooth(2 * ny - 1);
    p.bins = (long)p.mx * p.my;
    p.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    p.gbs = ((long)b * b + 1) / 2 * 2;
    p.ubs = ((long)nrhs * b + 1) / 2 * 2;

    // Scratch layout and the size check (before touching the device).
    auto tw_tables = [](int M) {
        return align256((M + 5) * sizeof(double2)) + align256((M + 5) * sizeof(float4)) +
               align256((M + 5) * sizeof(float2));
    };
    const size_t tw_bytes = tw_tables(p.mx) + (p.my != p.mx ? tw_tables(p.my) : 0);
    const size_t w_bytes = align256((size_t)p.bins * p.gbs * sizeof(double2));
    const size_t ws_bytes = align256((size_t)p.bins * p.ubs * 16);
    const size_t need = 256 + tw_bytes + 2 * w_bytes + 2 * ws_bytes;
    if (need > kNoAllocScratchBytes)
        return set_error(nullptr, BTTB_ERR_INVALID_ARG,
                         "bttb_matvec_noalloc: problem needs " + std::to_string(need) +
                             " bytes of scratch, above the fixed " + std::to_string(kNoAllocScratchBytes) +
                             " (use a plan)");

    cudaError_t e = cudaGetDevice(&p.dev);
    if (e != cudaSuccess) return check_cuda(nullptr, e, "cudaGetDevice");
    void *base = nullptr;
    int rc = scratch_address(p.dev, &base);
    if (rc != BTTB_OK) return rc;
    cudaDeviceGetAttribute(&p.nsm, cudaDevAttrMultiProcessorCount, p.dev);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p.dev);
    p.smem_optin = (size_t)optin;

    check_track(base, kNoAllocScratchBytes);
    check_track(gen, (size_t)(2 * nx - 1) * (2 * ny - 1) * b * b * 16);
    check_track_cols(x, nrhs, ld, p.n, 16);
    check_track_cols(y, nrhs, ld, p.n, 16);
    unsigned char *cur = static_cast<unsigned char *>(base);
    p.d_err = reinterpret_cast<int *>(cur);
    p.d_gbar = reinterpret_cast<unsigned long long *>(cur + 16);   // monotonic: never cleared
    cur += 256;
    fill_fft_plan(p.fx, p.mx, cur);
    if (p.my == p.mx) {
        p.fy = p.fx;
        p.fy.M = -1;
    } else {
        fill_fft_plan(p.fy, p.my, cur);
    }
    double2 *w1 = reinterpret_cast<double2 *>(cur);
    cur += w_bytes;
    double2 *w2 = reinterpret_cast<double2 *>(cur);
    cur += w_bytes;
    p.wsA = cur;
    cur += ws_bytes;
    p.wsB = cur;
    // The spectrum planes reuse w2 once the y-level transform has left it.
    p.ghat_hi = reinterpret_cast<float2 *>(w2);
    p.ghat_lo = reinterpret_cast<float2 *>(w2) + (size_t)p.bins * p.gbs;

    cudaStream_t st = p.stream;
    cudaMemsetAsync(p.d_err, 0, sizeof(int), st);
    const long double sq5 = sqrtl(5.0L);
    const double kc[5] = {(double)((sq5 - 1.0L) / 4.0L), (double)(-(sq5 + 1.0L) / 4.0L),
                          (double)sqrtl((5.0L + sq5) / 8.0L), (double)sqrtl((5.0L - sq5) / 8.0L),
                          (double)(sqrtl(3.0L) / 2.0L)};
    noalloc_twiddle_kernel<<<4, 256, 0, st>>>(p.mx, kc[0], kc[1], kc[2], kc[3], kc[4], p.fx.tw_f64, p.fx.tw_df,
                                              p.fx.tw_f32);
    if (p.my != p.mx)
        noalloc_twiddle_kernel<<<4, 256, 0, st>>>(p.my, kc[0], kc[1], kc[2], kc[3], kc[4], p.fy.tw_f64, p.fy.tw_df,
                                                  p.fy.tw_f32);
    const long bb = (long)b * b;
    noalloc_scatter_kernel<<<dim3(p.mx, p.my), 256, 0, st>>>(reinterpret_cast<const double2 *>(gen), w1, nx, ny,
                                                             p.mx, p.my, (int)bb);
    if ((e = cudaGetLastError()) != cudaSuccess) return check_cuda(nullptr, e, "no-alloc spectrum launch");
    FftPass a{};
    a.in = w1; a.out = w2;
    a.in_os = a.out_os = (long)p.mx * bb;
    a.in_ns = a.out_ns = bb;
    a.O = p.my; a.pdim = (int)bb; a.ncols = 1;
    a.nin = a.nout = p.mx; a.M = p.mx;
    if ((rc = fft_pass_launch(&p, a, PREC_F64N, FMT_C128, FMT_C128, false)) != BTTB_OK) return rc;
    FftPass c{};
    c.in = w2; c.out = w1;
    c.in_os = c.out_os = bb;
    c.in_ns = c.out_ns = (long)p.mx * bb;
    c.O = p.mx; c.pdim = (int)bb; c.ncols = 1;
    c.nin = c.nout = p.my; c.M = p.my;
    if ((rc = fft_pass_launch(&p, c, PREC_F64N, FMT_C128, FMT_C128, false)) != BTTB_OK) return rc;
    noalloc_finish_kernel<<<(unsigned)p.bins, 256, 0, st>>>(w1, b, p.gbs, 1.0 / ((double)p.mx * p.my), p.ghat_hi,
                                                            p.ghat_lo, p.d_err);
    if ((e = cudaGetLastError()) != cudaSuccess) return check_cuda(nullptr, e, "no-alloc spectrum launch");
    return matvec_run(&p, x, FMT_C128, ld, y, FMT_C128, ld, nrhs, PREC_DF64);
}
