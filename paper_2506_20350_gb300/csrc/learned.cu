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
    float *wt = nullptr, *wpart = nullptr, *colred = nullptr;
    long wpart_len = 0;
    size_t bytes = 0;
};

// ------------------------------------------------------------------ kernels

__device__ __forceinline__ float bf(const __nv_bfloat16 *w, long i) { return __bfloat162float(w[i]); }

constexpr int kEncCols = 16;

// hc[c][bin][2r, 2r+1] = scale * sum_p B[bin][r][p] rh[bin][c][p]
__global__ void __launch_bounds__(256) lp_encode_kernel(const __nv_bfloat16 *Bw, const float2 *rh, long ubs, float *hc,
                                                        int nc, int b, int R, long bins, float scale) {
    extern __shared__ __align__(16) float2 sm2[];
    float2 *Bs = sm2;                    // R*b
    float2 *xs = sm2 + (long)R * b;      // kEncCols*b
    const long bin = blockIdx.x;
    const int c0 = blockIdx.y * kEncCols;
    const int ncb = min(kEncCols, nc - c0);
    for (int i = threadIdx.x; i < R * b; i += blockDim.x) {
        const long o = (bin * R * b + i) * 2;
        Bs[i] = make_float2(bf(Bw, o), bf(Bw, o + 1));
    }
    for (int i = threadIdx.x; i < ncb * b; i += blockDim.x) xs[i] = rh[bin * ubs + (long)(c0 + i / b) * b + i % b];
    __syncthreads();
    for (int t = threadIdx.x; t < ncb * R; t += blockDim.x) {
        const int cl = t / R, r = t % R;
        float ar = 0.f, ai = 0.f;
        for (int q = 0; q < b; ++q) {
            const float2 w = Bs[r * b + q], x = xs[cl * b + q];
            ar = fmaf(w.x, x.x, fmaf(-w.y, x.y, ar));
            ai = fmaf(w.x, x.y, fmaf(w.y, x.x, ai));
        }
        float *o = hc + ((long)(c0 + cl) * bins + bin) * 2 * R + 2 * r;
        o[0] = ar * scale;
        o[1] = ai * scale;
    }
}

// zh[bin][c][p] = scale * sum_r A[bin][p][r] g[c][bin][r], g = hc + a3 (as complex)
__global__ void __launch_bounds__(256) lp_decode_kernel(const __nv_bfloat16 *Aw, const float *hc, const float *a3,
                                                        float2 *zh, long ubs, int nc, int b, int R, long bins,
                                                        float scale) {
    extern __shared__ __align__(16) float2 sm2[];
    float2 *As = sm2;                    // b*R
    float2 *gs = sm2 + (long)b * R;      // kEncCols*R
    const long bin = blockIdx.x;
    const int c0 = blockIdx.y * kEncCols;
    const int ncb = min(kEncCols, nc - c0);
    for (int i = threadIdx.x; i < b * R; i += blockDim.x) {
        const long o = (bin * b * R + i) * 2;
        As[i] = make_float2(bf(Aw, o), bf(Aw, o + 1));
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
            const float2 w = As[pr * R + r], g = gs[cl * R + r];
            ar = fmaf(w.x, g.x, fmaf(-w.y, g.y, ar));
            ai = fmaf(w.x, g.y, fmaf(w.y, g.x, ai));
        }
        zh[bin * ubs + (long)(c0 + cl) * b + pr] = make_float2(ar * scale, ai * scale);
    }
}

// Wt[(ci*9 + tap)*Co + co] = W[co][ci][tap]            (forward layout)
// Wt[(co*9 + tap)*Ci + ci] = W[co][ci][8 - tap]        (flip = 1: data-gradient layout)
__global__ void lp_wt_kernel(const __nv_bfloat16 *W, float *Wt, int Co, int Ci, int flip) {
    const int total = Co * Ci * 9;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int co = i / (Ci * 9), ci = (i / 9) % Ci, tap = i % 9;
        const float v = bf(W, i);
        if (!flip) Wt[((long)ci * 9 + tap) * Co + co] = v;
        else Wt[((long)co * 9 + (8 - tap)) * Ci + ci] = v;
    }
}

// out[n][co] = (bias ? bias[co] : 0) + sum_{ci, tap} Wt[(ci*9+tap)*Co + co] * in(neighbour(n, tap))[ci],
// in = relu(X) when relu_in; the result is multiplied by (mask[n][co] > 0) when mask is given.
__global__ void __launch_bounds__(256) lp_conv_kernel(const float *X, int Ci, int relu_in, const float *Wt,
                                                      const float *bias, float *out, int Co, long npos, int my,
                                                      int mx, long bins, const float *mask) {
    extern __shared__ __align__(16) float wsm[];        // Ci*9*Co
    for (int i = threadIdx.x; i < Ci * 9 * Co; i += blockDim.x) wsm[i] = Wt[i];
    __syncthreads();
    const int P = blockDim.x / Co;
    const int pl = threadIdx.x / Co, co = threadIdx.x % Co;
    if (pl >= P) return;
    for (long n = (long)blockIdx.x * P + pl; n < npos; n += (long)gridDim.x * P) {
        const long c = n / bins, pos = n % bins;
        const int y = (int)(pos / mx), x = (int)(pos % mx);
        float acc = bias ? bias[co] : 0.f;
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            const int yy = (y + tap / 3 - 1 + my) % my, xx = (x + tap % 3 - 1 + mx) % mx;
            const float *xr = X + (c * bins + (long)yy * mx + xx) * Ci;
            const float *wr = wsm + (long)tap * Co + co;
#pragma unroll 8
            for (int ci = 0; ci < Ci; ++ci) {
                float v = xr[ci];
                if (relu_in) v = fmaxf(v, 0.f);
                acc = fmaf(wr[(long)ci * 9 * Co], v, acc);
            }
        }
        if (mask && !(mask[n * Co + co] > 0.f)) acc = 0.f;
        out[n * Co + co] = acc;
    }
}

// Partial weight gradients of one convolution over a chunk of positions:
// wpart[chunk][co][k], k = ci*9 + tap for k < Ci*9 and k = Ci*9 for the bias:
//   sum_n dA[n][co] * in(neighbour(n, tap))[ci]   (in = relu(X) when relu_in).
constexpr int kWgChunk = 512;
constexpr int kWgStep = 32;

__global__ void __launch_bounds__(256) lp_wgrad_kernel(const float *X, int Ci, int relu_in, const float *dA, int Co,
                                                       long npos, int my, int mx, long bins, float *wpart) {
    __shared__ float das[kWgStep][64];
    __shared__ float xcs[kWgStep][64];
    const int K = Ci * 9 + 1;
    const int chunk = blockIdx.x, ktile = blockIdx.y * 64;
    const int TCO = Co / 16;                          // co per thread (Co = 64 -> 4, 32 -> 2)
    const int tco = threadIdx.x / 16, tk = threadIdx.x % 16;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[a][k] = 0.f;
    const long n0 = (long)chunk * kWgChunk;
    for (int s = 0; s < kWgChunk; s += kWgStep) {
        __syncthreads();
        for (int i = threadIdx.x; i < kWgStep * 64; i += blockDim.x) {
            const int np = i / 64, j = i % 64;
            const long n = n0 + s + np;
            // dA rows (Co values, zero beyond)
            das[np][j] = (n < npos && j < Co) ? dA[n * Co + j] : 0.f;
            // columns of the unfolded input for this k tile
            const int k = ktile + j;
            float v = 0.f;
            if (n < npos && k < K) {
                if (k == Ci * 9) {
                    v = 1.f;
                } else {
                    const int ci = k / 9, tap = k % 9;
                    const long c = n / bins, pos = n % bins;
                    const int y = (int)(pos / mx), x = (int)(pos % mx);
                    const int yy = (y + tap / 3 - 1 + my) % my, xx = (x + tap % 3 - 1 + mx) % mx;
                    v = X[(c * bins + (long)yy * mx + xx) * Ci + ci];
                    if (relu_in) v = fmaxf(v, 0.f);
                }
            }
            xcs[np][j] = v;
        }
        __syncthreads();
        for (int np = 0; np < kWgStep; ++np) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                if (a < TCO) {
                    const float d = das[np][tco * TCO + a];
#pragma unroll
                    for (int k = 0; k < 4; ++k) acc[a][k] = fmaf(d, xcs[np][tk * 4 + k], acc[a][k]);
                }
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int co = tco * TCO + a, kk = ktile + tk * 4 + k;
            if (a < TCO && kk < K) wpart[((long)chunk * Co + co) * K + kk] = acc[a][k];
        }
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

static int conv_launch(Plan *p, Learned *L, const float *X, int Ci, int relu_in, const __nv_bfloat16 *W,
                       const float *bias, float *out, int Co, int nc, int flip, const float *mask) {
    // flip = 1: data gradient (input channels Co of W, output channels Ci of W)
    const int wCo = flip ? Ci : Co, wCi = flip ? Co : Ci;
    lp_wt_kernel<<<64, 256, 0, p->stream>>>(W, L->wt, wCo, wCi, flip);
    const size_t smem = (size_t)Ci * 9 * Co * sizeof(float);
    cudaFuncSetAttribute(lp_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_optin);
    const long npos = (long)nc * L->bins;
    const int P = 256 / Co;
    long blocks = (npos + P - 1) / P;
    if (blocks > (long)p->nsm * 8) blocks = (long)p->nsm * 8;
    lp_conv_kernel<<<(unsigned)blocks, 256, smem, p->stream>>>(X, Ci, relu_in, L->wt, bias, out, Co, npos, L->my, L->mx,
                                                               L->bins, mask);
    count_launch(p, 2);
    return check_cuda(p, cudaGetLastError(), "learned conv launch");
}

static int wgrad_launch(Plan *p, Learned *L, const float *X, int Ci, int relu_in, const float *dA, int Co, int nc,
                        float *gW, float *gc) {
    const long npos = (long)nc * L->bins;
    const int nchunks = (int)((npos + kWgChunk - 1) / kWgChunk);
    const int K = Ci * 9 + 1;
    const dim3 grid(nchunks, (K + 63) / 64);
    lp_wgrad_kernel<<<grid, 256, 0, p->stream>>>(X, Ci, relu_in, dA, Co, npos, L->my, L->mx, L->bins, L->wpart);
    lp_wgrad_reduce_kernel<<<(Co * K + 255) / 256, 256, 0, p->stream>>>(L->wpart, nchunks, Co, Ci, gW, gc);
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
    lp_encode_kernel<<<eg, 256, (size_t)(R * b + kEncCols * b) * sizeof(float2), p->stream>>>(
        wB, L->rh, L->ubs, L->hc, nc, b, R, L->bins, L->scale);
    count_launch(p);
    if ((rc = conv_launch(p, L, L->hc, 2 * R, 0, L->wbf + L->oW1, L->master + L->oc1, L->a1, C, nc, 0, nullptr)))
        return rc;
    if ((rc = conv_launch(p, L, L->a1, C, 1, L->wbf + L->oW2, L->master + L->oc2, L->a2, C, nc, 0, nullptr))) return rc;
    if ((rc = conv_launch(p, L, L->a2, C, 1, L->wbf + L->oW3, L->master + L->oc3, L->a3, 2 * R, nc, 0, nullptr)))
        return rc;
    lp_decode_kernel<<<eg, 256, (size_t)(b * R + kEncCols * R) * sizeof(float2), p->stream>>>(
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
    cudaFree(L->dh); cudaFree(L->wt); cudaFree(L->wpart); cudaFree(L->colred);
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
    if (rank < 8 || rank > 32 || rank % 8 != 0 || (channels != 16 && channels != 32 && channels != 64) ||
        max_cols < 1 || max_cols > 256)
        return set_error(nullptr, BTTB_ERR_INVALID_ARG,
                         "need rank in {8, 16, 24, 32}, channels in {16, 32, 64}, 1 <= max_cols <= 256");
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
        if (cudaMalloc((void **)ptr, bytes) != cudaSuccess) ok = false;
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
    alloc(&L->wt, sizeof(float) * (size_t)std::max(C, 2 * R) * 9 * C);
    const long nchunks = (pos + kWgChunk - 1) / kWgChunk;
    const long mc = std::max(C, 2 * R);
    L->wpart_len = nchunks * mc * (mc * 9 + 1);
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
