// Learned Fourier-domain correction to the block-Jacobi preconditioner,
// M(r) = P_K^{-1} r + f(r), used inside flexible GMRES.  For a column r:
//   r^ = FFT2(pad r)/s                      (s = sqrt(mx my), the product's FFT passes)
//   h_k = B_k r^_k                          per bin, B_k in C^{R x b}       (encode)
//   g = h + conv3(relu(conv2(relu(conv1(h)))))   3x3 circular convolutions over
//                                           the (ky, kx) grid, h read as 2R real channels
//   z^_k = A_k g_k                          per bin, A_k in C^{b x R}       (decode)
//   f(r) = crop(IFFT2(z^))/s
// Weights are stored in binary32 (master, updated by Adam) and read by every
// kernel from a bfloat16 copy; activations and accumulation are binary32.
// Training minimises mean_c ||P_K^{-1} r_c + f(r_c) - e_c||^2/||e_c||^2 over
// (residual, exact correction) pairs; gradients of complex weights are
// dL/dRe + i dL/dIm.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

#include "arith.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace bttb {

struct Learned {
    Plan *p = nullptr;
    int R = 0, C = 0, b = 0, mx = 0, my = 0, maxcols = 0;
    long bins = 0, n = 0, ubs = 0;
    float scale = 1.f;                         // 1/sqrt(bins)
    long oB = 0, oA = 0, oW1 = 0, oc1 = 0, oW2 = 0, oc2 = 0, oW3 = 0, oc3 = 0, count = 0;
    float *master = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
    __nv_bfloat16 *wbf = nullptr;
    long step = 0;
    float2 *ubuf = nullptr, *rh = nullptr, *zh = nullptr, *zs = nullptr, *dz = nullptr, *bjr = nullptr;
    float *hc = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *dg = nullptr, *dx = nullptr, *dh = nullptr;
    float *wpart = nullptr, *colred = nullptr;
    __nv_bfloat16 *wtb = nullptr;      // one convolution's weights in the tensor-core layout
    long wpart_len = 0;
    size_t bytes = 0;
};

// ------------------------------------------------------------------ kernels

__device__ __forceinline__ float bf(const __nv_bfloat16 *w, long i) { return __bfloat162float(w[i]); }

constexpr int kEncCols = 16;

// hc[c][bin][2r, 2r+1] = scale * sum_p B[bin][r][p] rh[bin][c][p]
// Shared layouts keep a warp's reads on distinct banks: B as [p][r] with row
// stride R+1, the staged columns with row stride b+1.
__global__ void __launch_bounds__(256) lp_encode_kernel(const __nv_bfloat16 *Bw, const float2 *rh, long ubs, float *hc,
                                                        int nc, int b, int R, long bins, float scale) {
    extern __shared__ __align__(16) float2 sm2[];
    const int bst = R + 1, xst = b + 1;
    float2 *Bs = sm2;                    // b*bst
    float2 *xs = sm2 + (long)b * bst;    // kEncCols*xst
    const long bin = blockIdx.x;
    const int c0 = blockIdx.y * kEncCols;
    const int ncb = min(kEncCols, nc - c0);
    for (int i = threadIdx.x; i < R * b; i += blockDim.x) {
        const long o = (bin * R * b + i) * 2;
        const int r = i / b, q = i - r * b;
        Bs[q * bst + r] = make_float2(bf(Bw, o), bf(Bw, o + 1));
    }
    for (int i = threadIdx.x; i < ncb * b; i += blockDim.x) {
        const int cl = i / b;
        xs[cl * xst + (i - cl * b)] = rh[bin * ubs + (long)c0 * b + i];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ncb * R; t += blockDim.x) {
        const int cl = t / R, r = t % R;
        float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
        const float2 *xr = xs + cl * xst;
        int q = 0;
        for (; q + 1 < b; q += 2) {
            const float2 w = Bs[q * bst + r], x = xr[q];
            const float2 w2 = Bs[(q + 1) * bst + r], x2 = xr[q + 1];
            ar = fmaf(w.x, x.x, fmaf(-w.y, x.y, ar));
            ai = fmaf(w.x, x.y, fmaf(w.y, x.x, ai));
            br = fmaf(w2.x, x2.x, fmaf(-w2.y, x2.y, br));
            bi = fmaf(w2.x, x2.y, fmaf(w2.y, x2.x, bi));
        }
        if (q < b) {
            const float2 w = Bs[q * bst + r], x = xr[q];
            ar = fmaf(w.x, x.x, fmaf(-w.y, x.y, ar));
            ai = fmaf(w.x, x.y, fmaf(w.y, x.x, ai));
        }
        float *o = hc + ((long)(c0 + cl) * bins + bin) * 2 * R + 2 * r;
        o[0] = (ar + br) * scale;
        o[1] = (ai + bi) * scale;
    }
}

// zh[bin][c][p] = scale * sum_r A[bin][p][r] g[c][bin][r], g = hc + a3 (as complex).
// A staged as [r][p] with row stride b+1.
__global__ void __launch_bounds__(256) lp_decode_kernel(const __nv_bfloat16 *Aw, const float *hc, const float *a3,
                                                        float2 *zh, long ubs, int nc, int b, int R, long bins,
                                                        float scale) {
    extern __shared__ __align__(16) float2 sm2[];
    const int ast = b + 1;
    float2 *As = sm2;                    // R*ast
    float2 *gs = sm2 + (long)R * ast;    // kEncCols*R
    const long bin = blockIdx.x;
    const int c0 = blockIdx.y * kEncCols;
    const int ncb = min(kEncCols, nc - c0);
    for (int i = threadIdx.x; i < b * R; i += blockDim.x) {
        const long o = (bin * b * R + i) * 2;
        const int pr = i / R, r = i - pr * R;
        As[r * ast + pr] = make_float2(bf(Aw, o), bf(Aw, o + 1));
    }
    for (int i = threadIdx.x; i < ncb * R; i += blockDim.x) {
        const long o = ((long)(c0 + i / R) * bins + bin) * 2 * R + 2 * (i % R);
        gs[i] = make_float2(hc[o] + a3[o], hc[o + 1] + a3[o + 1]);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ncb * b; t += blockDim.x) {
        const int cl = t / b, pr = t % b;
        float ar = 0.f, ai = 0.f;
        for (int r = 0; r < R; ++r) {
            const float2 w = As[r * ast + pr], g = gs[cl * R + r];
            ar = fmaf(w.x, g.x, fmaf(-w.y, g.y, ar));
            ai = fmaf(w.x, g.y, fmaf(w.y, g.x, ai));
        }
        zh[bin * ubs + (long)(c0 + cl) * b + pr] = make_float2(ar * scale, ai * scale);
    }
}

// Row stride (bfloat16 entries) of the tensor-core weight layout: >= 9*Ci and
// = 8 (mod 64), i.e. 4 (mod 32) words, so that fragment loads are conflict-free.
__host__ __device__ constexpr int conv_kst(int ci) { return ((9 * ci + 55) / 64) * 64 + 8; }

// Wb[co][tap*Ci + ci] = W[co][ci][tap]                 (forward: W is [Co][Ci][9])
// Wb[co][tap*Ci + ci] = W[ci][co][8 - tap]             (flip = 1, data gradient: W is [Ci][Co][9])
// for the convolution with Ci inputs and Co outputs; padding entries are zero.
__global__ void lp_wtb_kernel(const __nv_bfloat16 *W, __nv_bfloat16 *Wb, int Co, int Ci, int flip) {
    const int kst = conv_kst(Ci);
    const int total = Co * kst;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int co = i / kst, k = i - co * kst;
        __nv_bfloat16 v = __float2bfloat16_rn(0.f);
        if (k < 9 * Ci) {
            const int tap = k / Ci, ci = k - tap * Ci;
            v = flip ? W[((long)ci * Co + co) * 9 + (8 - tap)] : W[((long)co * Ci + ci) * 9 + tap];
        }
        Wb[i] = v;
    }
}

// Circular 3x3 convolution over the (ky, kx) grid of every column, on the
// tensor cores:
//   out[n][co] = bias[co] + sum_{tap, ci} W(co, ci, tap) * in(nb(n, tap))[ci],
// nb(n, tap) the neighbour (y + tap/3 - 1, x + tap%3 - 1) mod (my, mx) of
// position n in its column, in = relu(X) when relu_in; the result is zeroed
// where mask[n][co] <= 0 when a mask is given (the ReLU derivative of the
// backward pass).  An implicit GEMM: M = positions (tiles of kConvTP), N = CO,
// K = 9 taps x Ci.  The bfloat16 weights (the B operand, exact) stay in shared
// memory; per tap the kConvTP neighbour rows (Ci binary32 values each) are
// copied in with 16-byte cp.async, double-buffered across taps, through a
// per-tile table of neighbour rows.  Each binary32 activation enters the
// mma.sync m16n8k16 (bf16 inputs, binary32 accumulation) as three bfloat16
// terms, x = hi + mid + lo, and the weights are bfloat16 already, so the
// products carry binary32 accuracy (split-BF16x3).  Warp w owns 16 positions x
// all CO channels.
constexpr int kConvTP = 128;

// x = hi + mid + lo with three bfloat16 terms (24 significant bits: the
// binary32 value up to its last bit or so), for a pair of activations.
__device__ __forceinline__ void split3_bf16x2(float a, float b, uint32_t &hi, uint32_t &mid, uint32_t &lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const float ra = a - hf.x, rb = b - hf.y;
    const __nv_bfloat162 m = __floats2bfloat162_rn(ra, rb);
    const float2 mf = __bfloat1622float2(m);
    const __nv_bfloat162 l = __floats2bfloat162_rn(ra - mf.x, rb - mf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    mid = *reinterpret_cast<const uint32_t *>(&m);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int CO>
__global__ void __launch_bounds__(256, 1) lp_conv_kernel(const float *X, int Ci, int relu_in,
                                                         const __nv_bfloat16 *Wb, const float *bias, float *out,
                                                         long npos, int my, int mx, long bins, const float *mask) {
    constexpr int TP = kConvTP;
    constexpr int NT = CO / 8;
    extern __shared__ __align__(16) unsigned char lsm_raw[];
    const int kst = conv_kst(Ci);
    const int xstride = Ci + 4;                                      // floats per staged row
    __nv_bfloat16 *ws = reinterpret_cast<__nv_bfloat16 *>(lsm_raw); // CO * kst
    float *xs0 = reinterpret_cast<float *>(lsm_raw + (((size_t)CO * kst * 2 + 15) & ~(size_t)15));
    int *nbr0 = reinterpret_cast<int *>(xs0 + 2 * TP * xstride);    // 2 tables of 9*TP rows
    const long ntiles = (npos + TP - 1) / TP;
    if ((long)blockIdx.x >= ntiles) return;
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(Wb);
        uint4 *dst = reinterpret_cast<uint4 *>(ws);
        for (int i = threadIdx.x; i < CO * kst / 8; i += blockDim.x) dst[i] = src[i];
    }
    // neighbour rows of tile t (row = c*bins + yy*mx + xx, -1 past the end)
    auto build_table = [&](long t, int *tab) {
        for (int pl = threadIdx.x; pl < TP; pl += blockDim.x) {
            const long n = t * TP + pl;
            if (n < npos) {
                const long c = n / bins;
                const int pos = (int)(n - c * bins);
                const int y = pos / mx, x = pos - y * mx;
                const int ym = y == 0 ? my - 1 : y - 1, yp = y == my - 1 ? 0 : y + 1;
                const int xm = x == 0 ? mx - 1 : x - 1, xp = x == mx - 1 ? 0 : x + 1;
                const int base = (int)(c * bins);
                const int ys[3] = {ym, y, yp}, xs3[3] = {xm, x, xp};
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) tab[tap * TP + pl] = base + ys[tap / 3] * mx + xs3[tap % 3];
            } else {
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) tab[tap * TP + pl] = -1;
            }
        }
    };
    const int cshift = 31 - __clz(Ci / 4);     // Ci/4 is a power of two
    const int cmask = Ci / 4 - 1;
    auto stage = [&](const int *tab, int tap, float *dst) {
        for (int i = threadIdx.x; i < TP * (Ci / 4); i += blockDim.x) {
            const int pl = i >> cshift, ch = i & cmask;
            const int row = tab[tap * TP + pl];
            float *d = dst + pl * xstride + ch * 4;
            if (row >= 0) cp_async16(d, X + (long)row * Ci + ch * 4);
            else *reinterpret_cast<float4 *>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        cp_async_commit();
    };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gid = lane >> 2, tig = lane & 3;
    int buf = 0, tb = 0;
    build_table(blockIdx.x, nbr0);
    __syncthreads();
    stage(nbr0, 0, xs0);
    for (long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long tn = t + gridDim.x;
        int *tab = nbr0 + tb * 9 * TP, *tabn = nbr0 + (tb ^ 1) * 9 * TP;
        if (tn < ntiles) build_table(tn, tabn);       // read first at tap 8, after two barriers
        float acc[NT][4];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            if (tap < 8) stage(tab, tap + 1, xs0 + (buf ^ 1) * TP * xstride);
            else if (tn < ntiles) stage(tabn, 0, xs0 + (buf ^ 1) * TP * xstride);
            else cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
            const float *xr0 = xs0 + buf * TP * xstride + (warp * 16 + gid) * xstride + 2 * tig;
            const float *xr1 = xr0 + 8 * xstride;
            const __nv_bfloat16 *wr = ws + gid * kst + tap * Ci + 2 * tig;
#pragma unroll 1
            for (int kc = 0; kc < Ci; kc += 16) {
                float2 v00 = *reinterpret_cast<const float2 *>(xr0 + kc);
                float2 v10 = *reinterpret_cast<const float2 *>(xr1 + kc);
                float2 v01 = *reinterpret_cast<const float2 *>(xr0 + kc + 8);
                float2 v11 = *reinterpret_cast<const float2 *>(xr1 + kc + 8);
                if (relu_in) {
                    v00 = make_float2(fmaxf(v00.x, 0.f), fmaxf(v00.y, 0.f));
                    v10 = make_float2(fmaxf(v10.x, 0.f), fmaxf(v10.y, 0.f));
                    v01 = make_float2(fmaxf(v01.x, 0.f), fmaxf(v01.y, 0.f));
                    v11 = make_float2(fmaxf(v11.x, 0.f), fmaxf(v11.y, 0.f));
                }
                uint32_t ah[4], am[4], al[4];
                split3_bf16x2(v00.x, v00.y, ah[0], am[0], al[0]);
                split3_bf16x2(v10.x, v10.y, ah[1], am[1], al[1]);
                split3_bf16x2(v01.x, v01.y, ah[2], am[2], al[2]);
                split3_bf16x2(v11.x, v11.y, ah[3], am[3], al[3]);
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const __nv_bfloat16 *wn = wr + nt * 8 * kst + kc;
                    const uint32_t b0 = *reinterpret_cast<const uint32_t *>(wn);
                    const uint32_t b1 = *reinterpret_cast<const uint32_t *>(wn + 8);
                    mma_bf16(acc[nt], al, b0, b1);              // smallest terms first
                    mma_bf16(acc[nt], am, b0, b1);
                    mma_bf16(acc[nt], ah, b0, b1);
                }
            }
            __syncthreads();
            buf ^= 1;
        }
        tb ^= 1;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const long n = t * TP + warp * 16 + gid + half * 8;
            if (n >= npos) continue;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int co = nt * 8 + 2 * tig;
                float2 o = make_float2(acc[nt][2 * half], acc[nt][2 * half + 1]);
                if (bias) {
                    o.x += bias[co];
                    o.y += bias[co + 1];
                }
                if (mask) {
                    const float2 mv = *reinterpret_cast<const float2 *>(mask + n * CO + co);
                    if (!(mv.x > 0.f)) o.x = 0.f;
                    if (!(mv.y > 0.f)) o.y = 0.f;
                }
                *reinterpret_cast<float2 *>(out + n * CO + co) = o;
            }
        }
    }
    cp_async_wait<0>();
}

// Partial weight gradients of one convolution over a chunk of positions, one tap
// per CTA row (blockIdx.y):
//   wpart[chunk][co][ci*9 + tap] = sum_{n in chunk} dA[n][co] * in(nb(n, tap))[ci]
//   wpart[chunk][co][Ci*9]       = sum_{n in chunk} dA[n][co]        (bias, tap 0 only)
// in = relu(X) when relu_in.  A GEMM per CTA, M = Co, N = Ci, K = the chunk's
// positions, on the tensor cores (mma.sync m16n8k16, bfloat16 inputs, binary32
// accumulation): tiles of kWgTile positions (input rows of the tap and dA rows)
// are copied in with cp.async, double-buffered; each binary32 operand enters as
// two bfloat16 terms, x = hi + lo, and the product as hi*hi + hi*lo + lo*hi (the
// dropped lo*lo and the remainders are below 2^-16 relative per product).  Warp w
// owns the 16 x 8 output tiles w, w + 8, ... (one row block of Co, so its A
// fragment is loaded once per step).
constexpr int kWgTile = 64;
constexpr int kWgChunks = 96;       // position chunks (x 9 taps) of a weight-gradient launch
constexpr int kWgThreads = 256;

// x = hi + lo with two bfloat16 terms, for a pair of values (packed low half first).
__device__ __forceinline__ void split2_bf16x2(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

__global__ void __launch_bounds__(kWgThreads) lp_wgrad_kernel(const float *X, int Ci, int relu_in, const float *dA,
                                                              int Co, long npos, long chunk_len, int my, int mx,
                                                              long bins, float *wpart) {
    extern __shared__ __align__(16) float gsm[];
    const int xs_stride = Ci + 4, ds_stride = Co + 4;
    const int buf_floats = kWgTile * (xs_stride + ds_stride);
    const int chunk = blockIdx.x, tap = blockIdx.y;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const long n0 = (long)chunk * chunk_len;
    const long n1 = min(npos, n0 + chunk_len);
    const int xch = Ci / 4, dch = Co / 4;
    auto stage = [&](long nb, float *dst) {
        float *xs = dst, *ds = dst + kWgTile * xs_stride;
        for (int i = threadIdx.x; i < kWgTile * (xch + dch); i += blockDim.x) {
            const int pl = i / (xch + dch), q = i - pl * (xch + dch);
            const long n = nb + pl;
            float *d = q < xch ? xs + pl * xs_stride + q * 4 : ds + pl * ds_stride + (q - xch) * 4;
            if (n < n1) {
                if (q < xch) {
                    const long c = n / bins;
                    const int pos = (int)(n - c * bins);
                    const int y = pos / mx, x = pos - y * mx;
                    int yy = y + dy, xx = x + dx;
                    yy += yy < 0 ? my : 0;
                    yy -= yy >= my ? my : 0;
                    xx += xx < 0 ? mx : 0;
                    xx -= xx >= mx ? mx : 0;
                    cp_async16(d, X + (c * bins + (long)yy * mx + xx) * Ci + q * 4);
                } else {
                    cp_async16(d, dA + n * Co + (q - xch) * 4);
                }
            } else {
                *reinterpret_cast<float4 *>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        cp_async_commit();
    };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int MT = Co / 16, NTt = Ci / 8, T = MT * NTt;       // MT divides 8: a warp keeps one row block
    const int mt = warp % MT;
    int ntile = 0, nts[4];
    for (int t = warp; t < T && ntile < 4; t += kWgThreads / 32) nts[ntile++] = t / MT;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[i][e] = 0.f;
    float bacc = 0.f;
    const bool do_bias = tap == 0 && (int)threadIdx.x < Co;
    int buf = 0;
    if (n0 < n1) stage(n0, gsm);
    for (long nb = n0; nb < n1; nb += kWgTile) {
        if (nb + kWgTile < n1) stage(nb + kWgTile, gsm + (buf ^ 1) * buf_floats);
        else cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const float *xs = gsm + buf * buf_floats;
        const float *ds = xs + kWgTile * xs_stride;
        if (ntile > 0) {
#pragma unroll
            for (int k0 = 0; k0 < kWgTile; k0 += 16) {
                // A (Co x K): rows co = 16 mt + gid (+8), columns k = k0 + 2 tig (+1, +8, +9)
                const float *dr = ds + (k0 + 2 * tig) * ds_stride + mt * 16 + gid;
                uint32_t ah[4], al[4];
                split2_bf16x2(dr[0], dr[ds_stride], ah[0], al[0]);
                split2_bf16x2(dr[8], dr[ds_stride + 8], ah[1], al[1]);
                split2_bf16x2(dr[8 * ds_stride], dr[9 * ds_stride], ah[2], al[2]);
                split2_bf16x2(dr[8 * ds_stride + 8], dr[9 * ds_stride + 8], ah[3], al[3]);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (i < ntile) {
                        // B (K x Ci): rows k = k0 + 2 tig (+1, +8, +9), column ci = 8 nt + gid
                        const float *xr = xs + (k0 + 2 * tig) * xs_stride + nts[i] * 8 + gid;
                        float v0 = xr[0], v1 = xr[xs_stride], v2 = xr[8 * xs_stride], v3 = xr[9 * xs_stride];
                        if (relu_in) {
                            v0 = fmaxf(v0, 0.f);
                            v1 = fmaxf(v1, 0.f);
                            v2 = fmaxf(v2, 0.f);
                            v3 = fmaxf(v3, 0.f);
                        }
                        uint32_t bh0, bl0, bh1, bl1;
                        split2_bf16x2(v0, v1, bh0, bl0);
                        split2_bf16x2(v2, v3, bh1, bl1);
                        mma_bf16(acc[i], al, bh0, bh1);           // smallest terms first
                        mma_bf16(acc[i], ah, bl0, bl1);
                        mma_bf16(acc[i], ah, bh0, bh1);
                    }
                }
            }
        }
        if (do_bias)
            for (int pl = 0; pl < kWgTile; ++pl) bacc += ds[pl * ds_stride + threadIdx.x];
        __syncthreads();
        buf ^= 1;
    }
    cp_async_wait<0>();
    const int K = Ci * 9 + 1;
    for (int i = 0; i < ntile; ++i) {
        const int ci = nts[i] * 8 + 2 * tig;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float *row = wpart + ((long)chunk * Co + mt * 16 + gid + 8 * half) * K;
            row[ci * 9 + tap] = acc[i][2 * half];
            row[(ci + 1) * 9 + tap] = acc[i][2 * half + 1];
        }
    }
    if (do_bias) wpart[((long)chunk * Co + threadIdx.x) * K + Ci * 9] = bacc;
}

// grad[oW + co*Ci*9 + k] = sum_chunks wpart (k < Ci*9); grad[oc + co] = bias column
__global__ void lp_wgrad_reduce_kernel(const float *wpart, int nchunks, int Co, int Ci, float *gW, float *gc) {
    const int K = Ci * 9 + 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Co * K; i += gridDim.x * blockDim.x) {
        const int co = i / K, k = i % K;
        float s = 0.f;
        for (int ch = 0; ch < nchunks; ++ch) s += wpart[((long)ch * Co + co) * K + k];
        if (k < Ci * 9) gW[(long)co * Ci * 9 + k] = s;
        else gc[co] = s;
    }
}

constexpr int kBwdCols = 32;

// dA[bin][p][r] = scale * sum_c dzh[bin][c][p] conj(g[c][bin][r]);
// dg[c][bin][2r..] = scale * sum_p conj(A[bin][p][r]) dzh[bin][c][p].
// Columns are taken kBwdCols at a time; each thread owns the same dA entries
// across chunks and accumulates them in place.
__global__ void __launch_bounds__(256) lp_decode_bwd_kernel(const __nv_bfloat16 *Aw, const float *hc, const float *a3,
                                                            const float2 *dzh, long ubs, int nc, int b, int R,
                                                            long bins, float scale, float *gA, float *dg) {
    extern __shared__ __align__(16) float2 sm2[];
    float2 *As = sm2;                       // b*R
    float2 *ds = As + (long)b * R;          // kBwdCols*b
    float2 *gs = ds + (long)kBwdCols * b;   // kBwdCols*R
    const long bin = blockIdx.x;
    for (int i = threadIdx.x; i < b * R; i += blockDim.x) {
        const long o = (bin * b * R + i) * 2;
        As[i] = make_float2(bf(Aw, o), bf(Aw, o + 1));
    }
    for (int c0 = 0; c0 < nc; c0 += kBwdCols) {
        const int ncb = min(kBwdCols, nc - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < ncb * b; i += blockDim.x) ds[i] = dzh[bin * ubs + (long)c0 * b + i];
        for (int i = threadIdx.x; i < ncb * R; i += blockDim.x) {
            const long o = ((long)(c0 + i / R) * bins + bin) * 2 * R + 2 * (i % R);
            gs[i] = make_float2(hc[o] + a3[o], hc[o + 1] + a3[o + 1]);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < b * R; t += blockDim.x) {
            const int pr = t / R, r = t % R;
            float ar = 0.f, ai = 0.f;
            for (int c = 0; c < ncb; ++c) {
                const float2 d = ds[c * b + pr], g = gs[c * R + r];
                ar = fmaf(d.x, g.x, fmaf(d.y, g.y, ar));          // d * conj(g)
                ai = fmaf(d.y, g.x, fmaf(-d.x, g.y, ai));
            }
            float *o = gA + (bin * b * R + t) * 2;
            o[0] = (c0 ? o[0] : 0.f) + ar * scale;
            o[1] = (c0 ? o[1] : 0.f) + ai * scale;
        }
        for (int t = threadIdx.x; t < ncb * R; t += blockDim.x) {
            const int c = t / R, r = t % R;
            float ar = 0.f, ai = 0.f;
            for (int pr = 0; pr < b; ++pr) {
                const float2 w = As[pr * R + r], d = ds[c * b + pr];
                ar = fmaf(w.x, d.x, fmaf(w.y, d.y, ar));          // conj(w) * d
                ai = fmaf(w.x, d.y, fmaf(-w.y, d.x, ai));
            }
            float *o = dg + ((long)(c0 + c) * bins + bin) * 2 * R + 2 * r;
            o[0] = ar * scale;
            o[1] = ai * scale;
        }
    }
}

// dB[bin][r][p] = scale * sum_c dh[c][bin][r] conj(rh[bin][c][p]), columns in chunks.
__global__ void __launch_bounds__(256) lp_encode_bwd_kernel(const float *dh, const float2 *rh, long ubs, int nc, int b,
                                                            int R, long bins, float scale, float *gB) {
    extern __shared__ __align__(16) float2 sm2[];
    float2 *xs = sm2;                       // kBwdCols*b
    float2 *hs = xs + (long)kBwdCols * b;   // kBwdCols*R
    const long bin = blockIdx.x;
    for (int c0 = 0; c0 < nc; c0 += kBwdCols) {
        const int ncb = min(kBwdCols, nc - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < ncb * b; i += blockDim.x) xs[i] = rh[bin * ubs + (long)c0 * b + i];
        for (int i = threadIdx.x; i < ncb * R; i += blockDim.x) {
            const long o = ((long)(c0 + i / R) * bins + bin) * 2 * R + 2 * (i % R);
            hs[i] = make_float2(dh[o], dh[o + 1]);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < R * b; t += blockDim.x) {
            const int r = t / b, pr = t % b;
            float ar = 0.f, ai = 0.f;
            for (int c = 0; c < ncb; ++c) {
                const float2 d = hs[c * R + r], x = xs[c * b + pr];
                ar = fmaf(d.x, x.x, fmaf(d.y, x.y, ar));
                ai = fmaf(d.y, x.x, fmaf(-d.x, x.y, ai));
            }
            float *o = gB + (bin * R * b + t) * 2;
            o[0] = (c0 ? o[0] : 0.f) + ar * scale;
            o[1] = (c0 ? o[1] : 0.f) + ai * scale;
        }
    }
}

// Per column: colred[c] = (sum |e|^2, sum |q - e|^2) with q = bjr + z.
__global__ void __launch_bounds__(256) lp_colnorm_kernel(const float2 *bjr, const float2 *z, const float2 *e, long lde,
                                                         long n, float *colred) {
    __shared__ float s0[256], s1[256];
    const int c = blockIdx.x;
    float a = 0.f, d = 0.f;
    for (long i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 ev = e[(long)c * lde + i], q0 = bjr[(long)c * n + i], q1 = z[(long)c * n + i];
        const float dr = q0.x + q1.x - ev.x, di = q0.y + q1.y - ev.y;
        a = fmaf(ev.x, ev.x, fmaf(ev.y, ev.y, a));
        d = fmaf(dr, dr, fmaf(di, di, d));
    }
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = d;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) {
            s0[threadIdx.x] += s0[threadIdx.x + st];
            s1[threadIdx.x] += s1[threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        colred[2 * c] = s0[0];
        colred[2 * c + 1] = s1[0];
    }
}

// dz = 2 (bjr + z - e) / ||e||^2 / nc
__global__ void lp_dz_kernel(const float2 *bjr, const float2 *z, const float2 *e, long lde, long n, int nc,
                             const float *colred, float2 *dz) {
    const int c = blockIdx.y;
    const float k = 2.f / (colred[2 * c] * (float)nc);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float2 ev = e[(long)c * lde + i], q0 = bjr[(long)c * n + i], q1 = z[(long)c * n + i];
        dz[(long)c * n + i] = make_float2(k * (q0.x + q1.x - ev.x), k * (q0.y + q1.y - ev.y));
    }
}

__global__ void lp_add_channels_kernel(float *dst, const float *src, long count) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
        dst[i] += src[i];
}

// out (native df64 or binary32 complex) += z
template <int FMT>
__global__ void lp_add_out_kernel(void *out, long ldo, const float2 *z, long n, int nc) {
    const int c = blockIdx.y;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float2 zv = z[(long)c * n + i];
        if constexpr (FMT == FMT_CDF) {
            float4 &o = reinterpret_cast<float4 *>(out)[(long)c * ldo + i];
            const df r = df_add(df{o.x, o.z}, df{zv.x, 0.f}), q = df_add(df{o.y, o.w}, df{zv.y, 0.f});
            o = make_float4(r.hi, q.hi, r.lo, q.lo);
        } else if constexpr (FMT == FMT_C64) {
            float2 &o = reinterpret_cast<float2 *>(out)[(long)c * ldo + i];
            o = make_float2(o.x + zv.x, o.y + zv.y);
        } else {
            double2 &o = reinterpret_cast<double2 *>(out)[(long)c * ldo + i];
            o = make_double2(o.x + zv.x, o.y + zv.y);
        }
    }
}

__global__ void lp_adam_kernel(float *w, const float *g, float *m, float *v, long count, float lr, float b1, float b2,
                               float eps, float c1, float c2, __nv_bfloat16 *wbf) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        wbf[i] = __float2bfloat16_rn(wi);
    }
}

__global__ void lp_to_bf16_kernel(const float *w, __nv_bfloat16 *wbf, long count) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
        wbf[i] = __float2bfloat16_rn(w[i]);
}

// ------------------------------------------------------------------ host side

static int fft_fwd(Plan *p, Learned *L, const void *in, int infmt, long ld, int nc, float2 *out) {
    FftPass a{};
    const int nx = p->nx, ny = p->ny, b = p->b, mx = p->mx, my = p->my;
    const long plane = (long)ny * mx * b;
    a.in = in; a.out = L->ubuf;
    a.in_cs = ld; a.in_os = (long)nx * b; a.in_ns = b;
    a.out_cs = plane; a.out_os = (long)mx * b; a.out_ns = b;
    a.O = ny; a.pdim = b; a.ncols = nc; a.nin = nx; a.nout = mx; a.M = mx;
    int rc = fft_pass_launch(p, a, PREC_F32, infmt, FMT_C64, false);
    if (rc != BTTB_OK) return rc;
    FftPass c{};
    c.in = L->ubuf; c.out = out;
    c.in_cs = plane; c.in_os = b; c.in_ns = (long)mx * b;
    c.out_cs = b; c.out_os = L->ubs; c.out_ns = (long)mx * L->ubs;
    c.O = mx; c.pdim = b; c.ncols = nc; c.nin = ny; c.nout = my; c.M = my;
    return fft_pass_launch(p, c, PREC_F32, FMT_C64, FMT_C64, false);
}

static int fft_inv(Plan *p, Learned *L, const float2 *in, int nc, void *out, int outfmt, long ld) {
    const int nx = p->nx, ny = p->ny, b = p->b, mx = p->mx, my = p->my;
    const long plane = (long)ny * mx * b;
    FftPass d{};
    d.in = in; d.out = L->ubuf;
    d.in_cs = b; d.in_os = L->ubs; d.in_ns = (long)mx * L->ubs;
    d.out_cs = plane; d.out_os = b; d.out_ns = (long)mx * b;
    d.O = mx; d.pdim = b; d.ncols = nc; d.nin = my; d.nout = ny; d.M = my;
    int rc = fft_pass_launch(p, d, PREC_F32, FMT_C64, FMT_C64, true);
    if (rc != BTTB_OK) return rc;
    FftPass e{};
    e.in = L->ubuf; e.out = out;
    e.in_cs = plane; e.in_os = (long)mx * b; e.in_ns = b;
    e.out_cs = ld; e.out_os = (long)nx * b; e.out_ns = b;
    e.O = ny; e.pdim = b; e.ncols = nc; e.nin = mx; e.nout = nx; e.M = mx;
    return fft_pass_launch(p, e, PREC_F32, FMT_C64, outfmt, true);
}

template <int CO>
static size_t conv_smem(int Ci) {
    return (((size_t)CO * conv_kst(Ci) * 2 + 15) & ~(size_t)15) +
           (2 * (size_t)kConvTP * (Ci + 4) + 2 * 9 * (size_t)kConvTP) * sizeof(float);
}

template <int CO>
static int conv_launch_co(Plan *p, Learned *L, const float *X, int Ci, int relu_in, const float *bias, float *out,
                          int nc, const float *mask) {
    const size_t smem = conv_smem<CO>(Ci);
    cudaFuncSetAttribute(lp_conv_kernel<CO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_optin);
    const long npos = (long)nc * L->bins;
    const long ntiles = (npos + kConvTP - 1) / kConvTP;
    const long blocks = std::min<long>(ntiles, p->nsm);
    lp_conv_kernel<CO><<<(unsigned)blocks, 256, smem, p->stream>>>(X, Ci, relu_in, L->wtb, bias, out, npos, L->my,
                                                                   L->mx, L->bins, mask);
    return BTTB_OK;
}

static int conv_launch(Plan *p, Learned *L, const float *X, int Ci, int relu_in, const __nv_bfloat16 *W,
                       const float *bias, float *out, int Co, int nc, int flip, const float *mask) {
    // flip = 1: data gradient (W is [Ci][Co][9], the forward convolution from Co to Ci channels)
    lp_wtb_kernel<<<64, 256, 0, p->stream>>>(W, L->wtb, Co, Ci, flip);
    if (Co == 64) conv_launch_co<64>(p, L, X, Ci, relu_in, bias, out, nc, mask);
    else if (Co == 32) conv_launch_co<32>(p, L, X, Ci, relu_in, bias, out, nc, mask);
    else conv_launch_co<16>(p, L, X, Ci, relu_in, bias, out, nc, mask);
    count_launch(p, 2);
    return check_cuda(p, cudaGetLastError(), "learned conv launch");
}

static int wgrad_launch(Plan *p, Learned *L, const float *X, int Ci, int relu_in, const float *dA, int Co, int nc,
                        float *gW, float *gc) {
    const long npos = (long)nc * L->bins;
    const int nchunks = (int)std::min<long>(kWgChunks, (npos + kWgTile - 1) / kWgTile);
    const long chunk_len = ((npos + nchunks - 1) / nchunks + kWgTile - 1) / kWgTile * kWgTile;
    const int nch = (int)((npos + chunk_len - 1) / chunk_len);
    const size_t smem = 2 * (size_t)kWgTile * (Ci + Co + 8) * sizeof(float);
    cudaFuncSetAttribute(lp_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_optin);
    lp_wgrad_kernel<<<dim3(nch, 9), kWgThreads, smem, p->stream>>>(X, Ci, relu_in, dA, Co, npos, chunk_len, L->my,
                                                                      L->mx, L->bins, L->wpart);
    const int K = Ci * 9 + 1;
    lp_wgrad_reduce_kernel<<<(Co * K + 255) / 256, 256, 0, p->stream>>>(L->wpart, nch, Co, Ci, gW, gc);
    count_launch(p, 2);
    return check_cuda(p, cudaGetLastError(), "learned weight-gradient launch");
}

// Forward f(r) into L->zs ([c][N] binary32); keeps the activations.
static int learned_forward(Learned *L, const void *r, int rfmt, long ld, int nc) {
    Plan *p = L->p;
    const int R = L->R, C = L->C, b = L->b;
    int rc = fft_fwd(p, L, r, rfmt, ld, nc, L->rh);
    if (rc != BTTB_OK) return rc;
    const __nv_bfloat16 *wB = L->wbf + L->oB, *wA = L->wbf + L->oA;
    const dim3 eg((unsigned)L->bins, (nc + kEncCols - 1) / kEncCols);
    cudaFuncSetAttribute(lp_encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_optin);
    cudaFuncSetAttribute(lp_decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_optin);
    lp_encode_kernel<<<eg, 256, (size_t)(b * (R + 1) + kEncCols * (b + 1)) * sizeof(float2), p->stream>>>(
        wB, L->rh, L->ubs, L->hc, nc, b, R, L->bins, L->scale);
    count_launch(p);
    if ((rc = conv_launch(p, L, L->hc, 2 * R, 0, L->wbf + L->oW1, L->master + L->oc1, L->a1, C, nc, 0, nullptr)))
        return rc;
    if ((rc = conv_launch(p, L, L->a1, C, 1, L->wbf + L->oW2, L->master + L->oc2, L->a2, C, nc, 0, nullptr))) return rc;
    if ((rc = conv_launch(p, L, L->a2, C, 1, L->wbf + L->oW3, L->master + L->oc3, L->a3, 2 * R, nc, 0, nullptr)))
        return rc;
    lp_decode_kernel<<<eg, 256, (size_t)(R * (b + 1) + kEncCols * R) * sizeof(float2), p->stream>>>(
        wA, L->hc, L->a3, L->zh, L->ubs, nc, b, R, L->bins, L->scale);
    count_launch(p);
    return fft_inv(p, L, L->zh, nc, L->zs, FMT_C64, L->n);
}

// Loss and gradients (into L->grad) for pairs (r, e) given as complex64 [c][ld].
static int learned_backward(Learned *L, const void *r, const void *e, long ld, int nc, double *loss) {
    Plan *p = L->p;
    const int R = L->R, C = L->C, b = L->b;
    int rc = learned_forward(L, r, FMT_C64, ld, nc);
    if (rc != BTTB_OK) return rc;
    if ((rc = block_jacobi_run(p, r, FMT_C64, ld, L->bjr, FMT_C64, L->n, nc)) != BTTB_OK) return rc;
    lp_colnorm_kernel<<<nc, 256, 0, p->stream>>>(L->bjr, L->zs, (const float2 *)e, ld, L->n, L->colred);
    const int vg = (int)std::min<long>((L->n + 255) / 256, 256);
    lp_dz_kernel<<<dim3(vg, nc), 256, 0, p->stream>>>(L->bjr, L->zs, (const float2 *)e, ld, L->n, nc, L->colred, L->dz);
    count_launch(p, 2);
    if ((rc = fft_fwd(p, L, L->dz, FMT_C64, L->n, nc, L->zh)) != BTTB_OK) return rc;       // zh <- FFT(pad dz)
    const size_t dsm = (size_t)(b * R + kBwdCols * (b + R)) * sizeof(float2);
    cudaFuncSetAttribute(lp_decode_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_optin);
    lp_decode_bwd_kernel<<<(unsigned)L->bins, 256, dsm, p->stream>>>(L->wbf + L->oA, L->hc, L->a3, L->zh, L->ubs, nc,
                                                                     b, R, L->bins, L->scale, L->grad + L->oA, L->dg);
    count_launch(p);
    // conv3: da3 = dg
    if ((rc = wgrad_launch(p, L, L->a2, C, 1, L->dg, 2 * R, nc, L->grad + L->oW3, L->grad + L->oc3))) return rc;
    if ((rc = conv_launch(p, L, L->dg, 2 * R, 0, L->wbf + L->oW3, nullptr, L->dx, C, nc, 1, L->a2))) return rc;
    // conv2: da2 = dx (masked)
    if ((rc = wgrad_launch(p, L, L->a1, C, 1, L->dx, C, nc, L->grad + L->oW2, L->grad + L->oc2))) return rc;
    if ((rc = conv_launch(p, L, L->dx, C, 0, L->wbf + L->oW2, nullptr, L->dh, C, nc, 1, L->a1))) return rc;
    // conv1: da1 = dh (masked, stored in dh), input hc
    if ((rc = wgrad_launch(p, L, L->hc, 2 * R, 0, L->dh, C, nc, L->grad + L->oW1, L->grad + L->oc1))) return rc;
    if ((rc = conv_launch(p, L, L->dh, C, 0, L->wbf + L->oW1, nullptr, L->dx, 2 * R, nc, 1, nullptr))) return rc;
    const long nch = (long)nc * L->bins * 2 * R;
    lp_add_channels_kernel<<<256, 256, 0, p->stream>>>(L->dx, L->dg, nch);          // dh_total = dg + conv1^T(da1)
    const size_t esm = (size_t)kBwdCols * (b + R) * sizeof(float2);
    cudaFuncSetAttribute(lp_encode_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_optin);
    lp_encode_bwd_kernel<<<(unsigned)L->bins, 256, esm, p->stream>>>(L->dx, L->rh, L->ubs, nc, b, R, L->bins, L->scale,
                                                                     L->grad + L->oB);
    count_launch(p, 2);
    if (loss) {
        std::vector<float> cr(2 * nc);
        cudaError_t e2 = cudaMemcpyAsync(cr.data(), L->colred, sizeof(float) * 2 * nc, cudaMemcpyDeviceToHost, p->stream);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(p->stream);
        if (e2 != cudaSuccess) return check_cuda(p, e2, "learned loss");
        double s = 0.0;
        for (int c = 0; c < nc; ++c) s += (double)cr[2 * c + 1] / (double)cr[2 * c];
        *loss = s / nc;
    }
    return check_cuda(p, cudaGetLastError(), "learned backward");
}

// z = P_K^{-1} x + f(x) for the product's / GMRES's vectors (any VecFmt).
int learned_max_cols(const Learned *L) { return L->maxcols; }

int learned_apply_run(Plan *p, const void *x, int xfmt, long ldx, void *z, int zfmt, long ldz, int nc) {
    Learned *L = p->learned;
    if (!L) return set_error(p, BTTB_ERR_INVALID_ARG, "no learned preconditioner attached to the plan");
    if (nc > L->maxcols) return set_error(p, BTTB_ERR_INVALID_ARG, "more columns than the learned workspace holds");
    int rc = learned_forward(L, x, xfmt, ldx, nc);
    if (rc != BTTB_OK) return rc;
    if ((rc = block_jacobi_run(p, x, xfmt, ldx, z, zfmt, ldz, nc)) != BTTB_OK) return rc;
    const int vg = (int)std::min<long>((L->n + 255) / 256, 256);
    if (zfmt == FMT_CDF) lp_add_out_kernel<FMT_CDF><<<dim3(vg, nc), 256, 0, p->stream>>>(z, ldz, L->zs, L->n, nc);
    else if (zfmt == FMT_C64) lp_add_out_kernel<FMT_C64><<<dim3(vg, nc), 256, 0, p->stream>>>(z, ldz, L->zs, L->n, nc);
    else lp_add_out_kernel<FMT_C128><<<dim3(vg, nc), 256, 0, p->stream>>>(z, ldz, L->zs, L->n, nc);
    count_launch(p);
    return check_cuda(p, cudaGetLastError(), "learned apply");
}

void learned_free(Learned *L) {
    if (!L) return;
    cudaFree(L->master); cudaFree(L->grad); cudaFree(L->m1); cudaFree(L->m2); cudaFree(L->wbf);
    cudaFree(L->ubuf); cudaFree(L->rh); cudaFree(L->zh); cudaFree(L->zs); cudaFree(L->dz); cudaFree(L->bjr);
    cudaFree(L->hc); cudaFree(L->a1); cudaFree(L->a2); cudaFree(L->a3); cudaFree(L->dg); cudaFree(L->dx);
    cudaFree(L->dh); cudaFree(L->wtb); cudaFree(L->wpart); cudaFree(L->colred);
    delete L;
}

}  // namespace bttb

using namespace bttb;

struct bttb_learned_s {
    Learned *L;
};

extern "C" {

int bttb_learned_create(bttb_learned *out, bttb_plan plan, int rank, int channels, int max_cols,
                        unsigned long long seed) {
    if (!out || !plan) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "out or plan is NULL");
    *out = nullptr;
    if ((rank != 8 && rank != 16 && rank != 32) || (channels != 16 && channels != 32 && channels != 64) ||
        max_cols < 1 || max_cols > 256)
        return set_error(nullptr, BTTB_ERR_INVALID_ARG,
                         "need rank in {8, 16, 32}, channels in {16, 32, 64}, 1 <= max_cols <= 256");
    Plan &p = plan->p;
    if (!p.ghat_hi) return set_error(&p, BTTB_ERR_INVALID_ARG, "the plan needs the binary32 spectrum copy");
    Learned *L = new (std::nothrow) Learned();
    if (!L) return set_error(&p, BTTB_ERR_OOM, "host allocation failed");
    L->p = &p;
    L->R = rank;
    L->C = channels;
    L->b = p.b;
    L->mx = p.mx;
    L->my = p.my;
    L->bins = p.bins;
    L->n = p.n;
    L->maxcols = max_cols;
    L->scale = 1.f / std::sqrt((float)p.bins);
    L->ubs = ((long)max_cols * p.b + 1) / 2 * 2;
    const long bins = p.bins;
    const int b = p.b, R = rank, C = channels;
    long o = 0;
    L->oB = o; o += bins * R * b * 2;
    L->oA = o; o += bins * b * R * 2;
    L->oW1 = o; o += (long)C * 2 * R * 9;
    L->oc1 = o; o += C;
    L->oW2 = o; o += (long)C * C * 9;
    L->oc2 = o; o += C;
    L->oW3 = o; o += (long)2 * R * C * 9;
    L->oc3 = o; o += 2 * R;
    L->count = o;
    bool ok = true;
    auto alloc = [&](auto **ptr, size_t bytes) {
        if (!ok) return;
        if (dev_malloc((void **)ptr, bytes) != cudaSuccess) ok = false;
        L->bytes += bytes;
    };
    alloc(&L->master, sizeof(float) * o);
    alloc(&L->grad, sizeof(float) * o);
    alloc(&L->m1, sizeof(float) * o);
    alloc(&L->m2, sizeof(float) * o);
    alloc(&L->wbf, sizeof(__nv_bfloat16) * o);
    const long nc = max_cols;
    alloc(&L->ubuf, sizeof(float2) * nc * p.ny * p.mx * b);
    alloc(&L->rh, sizeof(float2) * bins * L->ubs);
    alloc(&L->zh, sizeof(float2) * bins * L->ubs);
    alloc(&L->zs, sizeof(float2) * nc * p.n);
    alloc(&L->dz, sizeof(float2) * nc * p.n);
    alloc(&L->bjr, sizeof(float2) * nc * p.n);
    const long pos = nc * bins;
    alloc(&L->hc, sizeof(float) * pos * 2 * R);
    alloc(&L->a1, sizeof(float) * pos * C);
    alloc(&L->a2, sizeof(float) * pos * C);
    alloc(&L->a3, sizeof(float) * pos * 2 * R);
    alloc(&L->dg, sizeof(float) * pos * 2 * R);
    alloc(&L->dx, sizeof(float) * pos * std::max(C, 2 * R));
    alloc(&L->dh, sizeof(float) * pos * C);
    alloc(&L->wtb, sizeof(__nv_bfloat16) * (size_t)std::max(C, 2 * R) * conv_kst(std::max(C, 2 * R)));
    const long mc = std::max(C, 2 * R);
    L->wpart_len = (long)kWgChunks * mc * (mc * 9 + 1);
    alloc(&L->wpart, sizeof(float) * L->wpart_len);
    alloc(&L->colred, sizeof(float) * 2 * nc);
    if (!ok) {
        learned_free(L);
        return set_error(&p, BTTB_ERR_OOM, "learned preconditioner allocation failed");
    }
    // Seeded initialisation: small per-bin maps (the correction starts near zero), He-scaled convolutions.
    std::vector<float> w(o, 0.f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    const float sab = 0.01f / std::sqrt((float)b);
    for (long i = L->oB; i < L->oA + bins * b * R * 2; ++i) w[i] = sab * nd(rng);
    auto he = [&](long off, long cnt, int fan_in) {
        const float s = 0.5f * std::sqrt(2.f / (float)fan_in);
        for (long i = off; i < off + cnt; ++i) w[i] = s * nd(rng);
    };
    he(L->oW1, (long)C * 2 * R * 9, 2 * R * 9);
    he(L->oW2, (long)C * C * 9, C * 9);
    he(L->oW3, (long)2 * R * C * 9, C * 9);
    cudaMemcpy(L->master, w.data(), sizeof(float) * o, cudaMemcpyHostToDevice);
    cudaMemset(L->m1, 0, sizeof(float) * o);
    cudaMemset(L->m2, 0, sizeof(float) * o);
    cudaMemset(L->grad, 0, sizeof(float) * o);
    lp_to_bf16_kernel<<<256, 256>>>(L->master, L->wbf, o);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        learned_free(L);
        return check_cuda(&p, e, "learned init");
    }
    bttb_learned h = new bttb_learned_s{L};
    *out = h;
    return BTTB_OK;
}

long bttb_learned_param_count(bttb_learned l) { return l ? l->L->count : 0; }

int bttb_learned_params(bttb_learned l, float *host, int to_host) {
    if (!l || !host) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "NULL argument");
    Learned *L = l->L;
    cudaError_t e = cudaStreamSynchronize(L->p->stream);
    if (e != cudaSuccess) return check_cuda(L->p, e, "params sync");
    if (to_host) {
        e = cudaMemcpy(host, L->master, sizeof(float) * L->count, cudaMemcpyDeviceToHost);
    } else {
        e = cudaMemcpy(L->master, host, sizeof(float) * L->count, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            lp_to_bf16_kernel<<<256, 256, 0, L->p->stream>>>(L->master, L->wbf, L->count);
            e = cudaStreamSynchronize(L->p->stream);
        }
    }
    return check_cuda(L->p, e, "params copy");
}

int bttb_learned_apply(bttb_learned l, const void *r, void *z, int ncols, long ld, bttb_dtype dtype) {
    if (!l || !r || !z) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "NULL argument");
    Learned *L = l->L;
    if (ncols < 1 || ncols > L->maxcols || ld < L->n) return set_error(L->p, BTTB_ERR_INVALID_ARG, "bad ncols or ld");
    if (!L->p->bj_ready) return set_error(L->p, BTTB_ERR_SINGULAR, "block-Jacobi part unavailable (singular T[0,0])");
    Plan *p = L->p;
    Learned *saved = p->learned;
    p->learned = L;
    const int fmt = dtype == BTTB_C128 ? FMT_C128 : FMT_C64;
    check_track_cols(r, ncols, ld, L->n, dtype == BTTB_C128 ? 16 : 8);
    check_track_cols(z, ncols, ld, L->n, dtype == BTTB_C128 ? 16 : 8);
    const int rc = learned_apply_run(p, r, fmt, ld, z, fmt, ld, ncols);
    p->learned = saved;
    return rc;
}

int bttb_learned_gradients(bttb_learned l, const void *r, const void *e, int ncols, long ld, float *grad_host,
                           double *loss_host) {
    if (!l || !r || !e) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "NULL argument");
    Learned *L = l->L;
    if (ncols < 1 || ncols > L->maxcols || ld < L->n) return set_error(L->p, BTTB_ERR_INVALID_ARG, "bad ncols or ld");
    if (!L->p->bj_ready) return set_error(L->p, BTTB_ERR_SINGULAR, "block-Jacobi part unavailable (singular T[0,0])");
    check_track_cols(r, ncols, ld, L->n, 8);
    check_track_cols(e, ncols, ld, L->n, 8);
    int rc = learned_backward(L, r, e, ld, ncols, loss_host);
    if (rc != BTTB_OK) return rc;
    if (grad_host) {
        cudaError_t e2 = cudaStreamSynchronize(L->p->stream);
        if (e2 == cudaSuccess) e2 = cudaMemcpy(grad_host, L->grad, sizeof(float) * L->count, cudaMemcpyDeviceToHost);
        if (e2 != cudaSuccess) return check_cuda(L->p, e2, "gradient copy");
    }
    return BTTB_OK;
}

int bttb_learned_train_step(bttb_learned l, const void *r, const void *e, int ncols, long ld, float lr,
                            double *loss_host) {
    int rc = bttb_learned_gradients(l, r, e, ncols, ld, nullptr, loss_host);
    if (rc != BTTB_OK) return rc;
    Learned *L = l->L;
    L->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)L->step), c2 = 1.f - std::pow(b2, (float)L->step);
    lp_adam_kernel<<<1024, 256, 0, L->p->stream>>>(L->master, L->grad, L->m1, L->m2, L->count, lr, b1, b2, 1e-8f, c1,
                                                   c2, L->wbf);
    count_launch(L->p);
    return check_cuda(L->p, cudaGetLastError(), "learned Adam step");
}

int bttb_plan_set_learned(bttb_plan plan, bttb_learned l) {
    if (!plan) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "plan is NULL");
    if (l && l->L->p != &plan->p) return set_error(&plan->p, BTTB_ERR_INVALID_ARG, "learned object belongs to another plan");
    plan->p.learned = l ? l->L : nullptr;
    gmres_free(&plan->p);                      // drop captured cycles that referenced the old preconditioner
    return BTTB_OK;
}

int bttb_learned_destroy(bttb_learned l) {
    if (!l) return BTTB_OK;
    if (l->L->p->learned == l->L) {
        l->L->p->learned = nullptr;
        gmres_free(l->L->p);
    }
    cudaStreamSynchronize(l->L->p->stream);
    learned_free(l->L);
    delete l;
    return BTTB_OK;
}

}  // extern "C"
