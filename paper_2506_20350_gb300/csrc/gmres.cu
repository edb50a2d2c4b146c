// Restarted (flexible) GMRES(m) on the device, one Krylov space per column
// (Sec. III-C hands the fast product to GMRES; a multi-column right-hand side
// is solved column by column in lockstep, one batched product per step).
//
// Per Arnoldi step j, for every column still active:
//   z_j = M^{-1} v_j (right preconditioner, stored: flexible GMRES)
//   w   = Z z_j                          (product in the cycle's precision)
//   h   = V_j^H w ; w -= V_j h           (classical Gram-Schmidt, twice)
//   beta = ||w|| ; Givens rotations of the Hessenberg column ; v_{j+1} = w/beta
// Every cycle starts from the true residual r = V - Z x computed with the FP64
// product, so a cycle whose inner products are binary32 is one step of
// iterative refinement (GMRES-IR).  All vectors, inner products and updates
// are double-float (48-bit); Hessenberg, rotations and the triangular solve
// are binary64 scalars.  Converged columns are masked.
#include <algorithm>
#include <cmath>
#include <vector>

#include "arith.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace bttb {

struct GmresWork {
    int m = 0, k = 0;
    long n = 0;
    bool flex = false;
    int NB = 0, nblk = 0;
    float4 *X = nullptr, *Vb = nullptr, *Zb = nullptr, *W = nullptr, *R = nullptr, *Vin = nullptr;
    double2 *H = nullptr, *hacc = nullptr, *gv = nullptr, *sn = nullptr;
    float4 *hco = nullptr, *ycoef = nullptr, *part = nullptr;
    double *cs = nullptr, *beta2 = nullptr, *vnorm = nullptr, *inv_beta = nullptr, *target = nullptr;
    int *active = nullptr, *steps = nullptr, *bdown = nullptr, *mlimit = nullptr, *d_j = nullptr, *d_any = nullptr;
    double2 *io = nullptr;        // staging for host_io
    int *h_any = nullptr;         // pinned
    size_t bytes = 0;
};

constexpr int kVecThreads = 256;

// ------------------------------------------------------------------ kernels

__global__ void cvt_in_kernel(const double2 *in, long ld, float4 *out, long n) {
    const int c = blockIdx.y;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        out[(long)c * n + i] = F64N::to_cdf(in[(long)c * ld + i]);
}

__global__ void cvt_out_kernel(const float4 *in, double2 *out, long ld, long n) {
    const int c = blockIdx.y;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        out[(long)c * ld + i] = DF64::to_c128(DF64::from_cdf(in[(long)c * n + i]));
}

__global__ void fill_zero_kernel(float4 *x, long count) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
        x[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ void warp_reduce_dacc(dacc &a) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        dacc o;
        o.S = __shfl_xor_sync(0xffffffffu, a.S, off);
        o.s = __shfl_xor_sync(0xffffffffu, a.s, off);
        dacc_add(a, o);
    }
}

// part[(c*maxcnt + i)*nblk + blk] = sum over the block's chunk of conj(B_i[n]) w[n]
// for i < cnt, cnt = (*cnt_dev + 1) or cnt_fixed.  B_i of column c at
// basis + i*bs_i + c*bs_c.
__global__ void __launch_bounds__(kVecThreads) dots_partial_kernel(const float4 *basis, long bs_i, long bs_c,
                                                                   const int *cnt_dev, int cnt_fixed,
                                                                   const float4 *w, long n, int NB, int nblk,
                                                                   int maxcnt, float4 *part, const int *active) {
    extern __shared__ __align__(16) float4 wsm[];
    const int c = blockIdx.y, blk = blockIdx.x;
    if (active && !active[c]) return;
    const int cnt = cnt_dev ? (*cnt_dev + 1) : cnt_fixed;
    const long n0 = (long)blk * NB;
    const int len = (int)min((long)NB, n - n0);
    for (int e = threadIdx.x; e < len; e += blockDim.x) wsm[e] = w[(long)c * n + n0 + e];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < cnt; i += nw) {
        const float4 *bv = basis + (long)i * bs_i + (long)c * bs_c + n0;
        dacc re{0.f, 0.f}, im{0.f, 0.f};
        for (int e = lane; e < len; e += 32) {
            const float4 v = bv[e], x = wsm[e];
            // conj(v) x = (vr xr + vi xi) + i (vr xi - vi xr)
            dacc_mac(re, v.x, v.z, x.x, x.z);
            dacc_mac(re, v.y, v.w, x.y, x.w);
            dacc_mac(im, v.x, v.z, x.y, x.w);
            dacc_mac(im, -v.y, -v.w, x.x, x.z);
        }
        warp_reduce_dacc(re);
        warp_reduce_dacc(im);
        if (lane == 0) {
            df r = dacc_result(re), q = dacc_result(im);
            part[((long)c * maxcnt + i) * nblk + blk] = make_float4(r.hi, q.hi, r.lo, q.lo);
        }
    }
}

// mode 0: hco = sum, hacc = sum ; mode 1: hco = sum, hacc += sum ; mode 2: out_real[c] = Re(sum)
__global__ void dots_reduce_kernel(const float4 *part, int nblk, const int *cnt_dev, int cnt_fixed, int maxcnt,
                                   float4 *hco, double2 *hacc, int mode, double *out_real, const int *active) {
    const int i = blockIdx.x, c = blockIdx.y, lane = threadIdx.x;
    if (active && !active[c]) return;
    const int cnt = cnt_dev ? (*cnt_dev + 1) : cnt_fixed;
    if (i >= cnt) return;
    const float4 *pp = part + ((long)c * maxcnt + i) * nblk;
    dacc re{0.f, 0.f}, im{0.f, 0.f};
    for (int e = lane; e < nblk; e += 32) {
        const float4 v = pp[e];
        dacc_add(re, dacc{v.x, v.z});
        dacc_add(im, dacc{v.y, v.w});
    }
    warp_reduce_dacc(re);
    warp_reduce_dacc(im);
    if (lane == 0) {
        df r = dacc_result(re), q = dacc_result(im);
        if (mode == 2) {
            out_real[c] = df_to_double(r);
        } else {
            hco[(long)c * maxcnt + i] = make_float4(r.hi, q.hi, r.lo, q.lo);
            const double2 v = make_double2(df_to_double(r), df_to_double(q));
            double2 &h = hacc[(long)c * maxcnt + i];
            if (mode == 0) h = v;
            else h = make_double2(h.x + v.x, h.y + v.y);
        }
    }
}

// w[c][n] += sgn * sum_{i < cnt} B_i[c][n] coef[c][i], with cnt = *cnt_dev + 1,
// or cnt_col[c] per column when cnt_col is given.
__global__ void __launch_bounds__(kVecThreads) update_kernel(const float4 *basis, long bs_i, long bs_c,
                                                             const int *cnt_dev, const int *cnt_col,
                                                             const float4 *coef, int maxcnt, float4 *w, long n,
                                                             float sgn, const int *active) {
    extern __shared__ __align__(16) float4 csm[];
    const int c = blockIdx.y;
    if (active && !active[c]) return;
    const int cnt = cnt_col ? cnt_col[c] : (*cnt_dev + 1);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        float4 h = coef[(long)c * maxcnt + i];
        csm[i] = make_float4(sgn * h.x, sgn * h.y, sgn * h.z, sgn * h.w);
    }
    __syncthreads();
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const float4 x = w[(long)c * n + e];
        dacc re{x.x, x.z}, im{x.y, x.w};
        for (int i = 0; i < cnt; ++i) {
            const float4 v = basis[(long)i * bs_i + (long)c * bs_c + e];
            const float4 h = csm[i];
            // v h = (vr hr - vi hi) + i (vr hi + vi hr)
            dacc_mac(re, v.x, v.z, h.x, h.z);
            dacc_mac(re, -v.y, -v.w, h.y, h.w);
            dacc_mac(im, v.x, v.z, h.y, h.w);
            dacc_mac(im, v.y, v.w, h.x, h.z);
        }
        df r = dacc_result(re), q = dacc_result(im);
        w[(long)c * n + e] = make_float4(r.hi, q.hi, r.lo, q.lo);
    }
}

// Vb[*d_j][c] = W[c] * inv_beta[c]
__global__ void scale_kernel(const float4 *w, float4 *vb, long bs_i, long bs_c, const int *d_j,
                             const double *inv_beta, long n, const int *active) {
    const int c = blockIdx.y;
    if (active && !active[c]) return;
    const df s = df_from_double(inv_beta[c]);
    float4 *dst = vb + (long)(*d_j) * bs_i + (long)c * bs_c;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const float4 x = w[(long)c * n + e];
        const df r = df_mul(df{x.x, x.z}, s), q = df_mul(df{x.y, x.w}, s);
        dst[e] = make_float4(r.hi, q.hi, r.lo, q.lo);
    }
}

// R = Vin - ZX
__global__ void resid_kernel(const float4 *vin, const float4 *zx, float4 *r, long count) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < count; e += (long)gridDim.x * blockDim.x) {
        const float4 a = vin[e], b = zx[e];
        const df re = df_sub(df{a.x, a.z}, df{b.x, b.z}), im = df_sub(df{a.y, a.w}, df{b.y, b.w});
        r[e] = make_float4(re.hi, im.hi, re.lo, im.lo);
    }
}

// Start of a cycle: g = (beta0, 0, ...), inv_beta = 1/beta0, j = 0.
__global__ void cycle_start_kernel(const double *beta2, double2 *gv, double *inv_beta, int m, int k,
                                   const int *active, int *d_j) {
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if (!active[c]) continue;
        const double b0 = sqrt(beta2[c]);
        double2 *g = gv + (long)c * (m + 1);
        g[0] = make_double2(b0, 0.0);
        for (int i = 1; i <= m; ++i) g[i] = make_double2(0.0, 0.0);
        inv_beta[c] = 1.0 / b0;
    }
    if (threadIdx.x == 0) *d_j = 0;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 conj2(double2 a) { return make_double2(a.x, -a.y); }

// One Givens step per active column (binary64 scalars); advances j.
__global__ void givens_kernel(double2 *H, const double2 *hacc, const double *beta2, double *cs, double2 *sn,
                              double2 *gv, int *active, int *steps, int *bdown, const int *mlimit,
                              const double *target, double *inv_beta, int m, int k, int *d_j, int *d_any,
                              int *err) {
    const int j = *d_j;
    int any = 0;
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if (!active[c]) continue;
        double2 *Hc = H + (long)c * (m + 1) * m;
        const double2 *ha = hacc + (long)c * (m + 1);
        double2 *g = gv + (long)c * (m + 1);
        double *csc = cs + (long)c * m;
        double2 *snc = sn + (long)c * m;
        const double beta = sqrt(fmax(beta2[c], 0.0));
        double zn = beta * beta;
        for (int i = 0; i <= j; ++i) {
            const double2 h = ha[i];
            Hc[i + (long)j * (m + 1)] = h;
            zn += h.x * h.x + h.y * h.y;
        }
        zn = sqrt(zn);
        if (!isfinite(zn)) {
            atomicOr(err, DEVERR_NONFINITE);
            active[c] = 0;
            continue;
        }
        for (int i = 0; i < j; ++i) {
            const double2 a0 = Hc[i + (long)j * (m + 1)], a1 = Hc[i + 1 + (long)j * (m + 1)];
            const double2 s = snc[i];
            const double2 t0 = make_double2(csc[i] * a0.x + (s.x * a1.x - s.y * a1.y),
                                            csc[i] * a0.y + (s.x * a1.y + s.y * a1.x));
            const double2 cs_ = conj2(s);
            const double2 t1 = make_double2(-(cs_.x * a0.x - cs_.y * a0.y) + csc[i] * a1.x,
                                            -(cs_.x * a0.y + cs_.y * a0.x) + csc[i] * a1.y);
            Hc[i + (long)j * (m + 1)] = t0;
            Hc[i + 1 + (long)j * (m + 1)] = t1;
        }
        const double2 a = Hc[j + (long)j * (m + 1)];
        const double aa = hypot(a.x, a.y);
        const double rho = hypot(aa, beta);
        double c_;
        double2 s_;
        if (aa == 0.0) {
            c_ = 0.0;
            s_ = make_double2(1.0, 0.0);
        } else {
            c_ = aa / rho;
            s_ = make_double2(a.x / aa * beta / rho, a.y / aa * beta / rho);
        }
        csc[j] = c_;
        snc[j] = s_;
        Hc[j + (long)j * (m + 1)] = make_double2(c_ * a.x + s_.x * beta, c_ * a.y + s_.y * beta);
        const double2 gj = g[j];
        const double2 ms = conj2(s_);
        g[j + 1] = make_double2(-(ms.x * gj.x - ms.y * gj.y), -(ms.x * gj.y + ms.y * gj.x));
        g[j] = make_double2(c_ * gj.x, c_ * gj.y);
        steps[c] = j + 1;
        const bool bd = !(beta > 1e-14 * zn);
        if (bd) bdown[c] = 1;
        const double est = hypot(g[j + 1].x, g[j + 1].y);
        const bool done = bd || est <= target[c] || (j + 1) >= mlimit[c];
        if (done) {
            active[c] = 0;
        } else {
            inv_beta[c] = 1.0 / beta;
            any = 1;
        }
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        *d_j = j + 1;
        *d_any = any;
    }
}

// y = H^{-1} g (upper triangular, steps[c] x steps[c]), stored as double-float.
__global__ void finish_kernel(const double2 *H, const double2 *gv, const int *steps, float4 *ycoef, int m, int k,
                              const int *was_active) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < k; c += gridDim.x * blockDim.x) {
        if (!was_active[c]) continue;
        const int kk = steps[c];
        const double2 *Hc = H + (long)c * (m + 1) * m;
        const double2 *g = gv + (long)c * (m + 1);
        double2 y[201];
        for (int i = kk - 1; i >= 0; --i) {
            double2 s = g[i];
            for (int l = i + 1; l < kk; ++l) {
                const double2 t = cmul(Hc[i + (long)l * (m + 1)], y[l]);
                s.x -= t.x;
                s.y -= t.y;
            }
            const double2 d = Hc[i + (long)i * (m + 1)];
            const double dd = d.x * d.x + d.y * d.y;
            y[i] = dd > 0.0 ? make_double2((s.x * d.x + s.y * d.y) / dd, (s.y * d.x - s.x * d.y) / dd)
                            : make_double2(0.0, 0.0);
        }
        for (int i = 0; i < kk; ++i) ycoef[(long)c * (m + 1) + i] = F64N::to_cdf(y[i]);
    }
}

// ------------------------------------------------------------------ host side

static void free_work(GmresWork *g) {
    if (!g) return;
    cudaFree(g->X); cudaFree(g->Vb); cudaFree(g->Zb); cudaFree(g->W); cudaFree(g->R); cudaFree(g->Vin);
    cudaFree(g->H); cudaFree(g->hacc); cudaFree(g->gv); cudaFree(g->sn); cudaFree(g->hco); cudaFree(g->ycoef);
    cudaFree(g->part); cudaFree(g->cs); cudaFree(g->beta2); cudaFree(g->vnorm); cudaFree(g->inv_beta);
    cudaFree(g->target); cudaFree(g->active); cudaFree(g->steps); cudaFree(g->bdown); cudaFree(g->mlimit);
    cudaFree(g->d_j); cudaFree(g->d_any); cudaFree(g->io);
    cudaFreeHost(g->h_any);
    delete g;
}

void gmres_free(Plan *p) {
    if (p->gw) p->bytes_held -= p->gw->bytes;
    free_work(p->gw);
    p->gw = nullptr;
}

static int ensure_work(Plan *p, int m, int k, bool flex, bool host_io) {
    GmresWork *g = p->gw;
    if (g && g->m == m && g->k >= k && (g->flex || !flex) && (!host_io || g->io)) return BTTB_OK;
    gmres_free(p);
    g = new GmresWork();
    g->m = m;
    g->k = k;
    g->n = p->n;
    g->flex = flex;
    g->NB = k <= 4 ? 256 : 1024;
    g->nblk = (int)((p->n + g->NB - 1) / g->NB);
    const long n = p->n;
    size_t total = 0;
    bool ok = true;
    auto alloc = [&](auto **ptr, size_t bytes) {
        if (!ok) return;
        if (cudaMalloc((void **)ptr, bytes) != cudaSuccess) ok = false;
        total += bytes;
    };
    alloc(&g->X, sizeof(float4) * k * n);
    alloc(&g->Vb, sizeof(float4) * (size_t)(m + 1) * k * n);
    if (flex) alloc(&g->Zb, sizeof(float4) * (size_t)m * k * n);
    alloc(&g->W, sizeof(float4) * k * n);
    alloc(&g->R, sizeof(float4) * k * n);
    alloc(&g->Vin, sizeof(float4) * k * n);
    alloc(&g->H, sizeof(double2) * (size_t)k * (m + 1) * m);
    alloc(&g->hacc, sizeof(double2) * (size_t)k * (m + 1));
    alloc(&g->gv, sizeof(double2) * (size_t)k * (m + 1));
    alloc(&g->sn, sizeof(double2) * (size_t)k * m);
    alloc(&g->hco, sizeof(float4) * (size_t)k * (m + 1));
    alloc(&g->ycoef, sizeof(float4) * (size_t)k * (m + 1));
    alloc(&g->part, sizeof(float4) * (size_t)k * (m + 1) * g->nblk);
    alloc(&g->cs, sizeof(double) * (size_t)k * m);
    alloc(&g->beta2, sizeof(double) * k);
    alloc(&g->vnorm, sizeof(double) * k);
    alloc(&g->inv_beta, sizeof(double) * k);
    alloc(&g->target, sizeof(double) * k);
    alloc(&g->active, sizeof(int) * k);
    alloc(&g->steps, sizeof(int) * k);
    alloc(&g->bdown, sizeof(int) * k);
    alloc(&g->mlimit, sizeof(int) * k);
    alloc(&g->d_j, sizeof(int));
    alloc(&g->d_any, sizeof(int));
    if (host_io) alloc(&g->io, sizeof(double2) * k * n);
    if (ok && cudaMallocHost((void **)&g->h_any, sizeof(int)) != cudaSuccess) ok = false;
    g->bytes = total;
    p->gw = g;
    p->bytes_held += total;
    if (!ok) {
        gmres_free(p);
        return set_error(p, BTTB_ERR_OOM, "GMRES workspace allocation failed");
    }
    return BTTB_OK;
}

// ||col||^2 of the k columns of x ([c][n] double-float) into g->beta2.
static int norm2_cols(Plan *p, GmresWork *g, const float4 *x, int k, const int *active) {
    dim3 grid(g->nblk, k);
    dots_partial_kernel<<<grid, kVecThreads, g->NB * sizeof(float4), p->stream>>>(
        x, 0, p->n, nullptr, 1, x, p->n, g->NB, g->nblk, g->m + 1, g->part, active);
    count_launch(p);
    dots_reduce_kernel<<<dim3(1, k), 32, 0, p->stream>>>(g->part, g->nblk, nullptr, 1, g->m + 1, nullptr, nullptr, 2,
                                                          g->beta2, active);
    count_launch(p);
    return check_cuda(p, cudaGetLastError(), "norm launch");
}

int gmres_solve(Plan *p, const void *V, void *I, int k, long ld, const bttb_gmres_opts *o,
                bttb_col_result *out) {
    const int m = o->restart;
    const bool flex = o->pc == BTTB_PC_BLOCK_JACOBI;
    const int inner = o->inner;
    int rc = ensure_work(p, m, k, flex, o->host_io != 0);
    if (rc != BTTB_OK) return rc;
    GmresWork *g = p->gw;
    const long n = p->n;
    const long bs_i = (long)k * n, bs_c = n;    // basis layout [i][c][n]
    cudaStream_t st = p->stream;
    cudaError_t e;
    const int vgrid = (int)std::min<long>((n + kVecThreads - 1) / kVecThreads, 1024);

    // Inputs: V -> Vin (double-float), I (x0) -> X
    const double2 *Vd = reinterpret_cast<const double2 *>(V);
    long ldv = ld;
    if (o->host_io) {
        e = cudaMemcpy2DAsync(g->io, n * sizeof(double2), V, ld * sizeof(double2), n * sizeof(double2), k,
                              cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return check_cuda(p, e, "copy V to device");
        Vd = g->io;
        ldv = n;
    }
    cvt_in_kernel<<<dim3(vgrid, k), kVecThreads, 0, st>>>(Vd, ldv, g->Vin, n);
    count_launch(p);
    if (o->use_x0) {
        const double2 *Xd = reinterpret_cast<const double2 *>(I);
        long ldx = ld;
        if (o->host_io) {
            e = cudaMemcpy2DAsync(g->io, n * sizeof(double2), I, ld * sizeof(double2), n * sizeof(double2), k,
                                  cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return check_cuda(p, e, "copy I to device");
            Xd = g->io;
            ldx = n;
        }
        cvt_in_kernel<<<dim3(vgrid, k), kVecThreads, 0, st>>>(Xd, ldx, g->X, n);
        count_launch(p);
    } else {
        fill_zero_kernel<<<1024, kVecThreads, 0, st>>>(g->X, (long)k * n);
        count_launch(p);
    }
    if ((rc = norm2_cols(p, g, g->Vin, k, nullptr)) != BTTB_OK) return rc;
    std::vector<double> vn2(k), vnorm(k), b2(k), relres(k, 0.0), tgt(k);
    std::vector<int> status(k, BTTB_OK), total(k, 0), cycles(k, 0), act(k), mlim(k), stp(k), bd(k);
    e = cudaMemcpyAsync(vn2.data(), g->beta2, sizeof(double) * k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return check_cuda(p, e, "norm of V");
    for (int c = 0; c < k; ++c) vnorm[c] = std::sqrt(vn2[c]);
    std::vector<char> done(k, 0);
    int hist_n = 0;
    const int max_iters = o->max_iters;
    int dev_err = 0;

    for (int cycle = 0;; ++cycle) {
        // True residual with the FP64 product.
        if ((rc = matvec_run(p, g->X, FMT_CDF, n, g->W, FMT_CDF, n, k, PREC_DF64)) != BTTB_OK) return rc;
        resid_kernel<<<1024, kVecThreads, 0, st>>>(g->Vin, g->W, g->R, (long)k * n);
        count_launch(p);
        if ((rc = norm2_cols(p, g, g->R, k, nullptr)) != BTTB_OK) return rc;
        e = cudaMemcpyAsync(b2.data(), g->beta2, sizeof(double) * k, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&dev_err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return check_cuda(p, e, "residual norm");
        if (dev_err & DEVERR_TIMEOUT) return set_error(p, BTTB_ERR_TIMEOUT, "a device pipeline wait timed out");
        bool any = false;
        for (int c = 0; c < k; ++c) {
            if (done[c]) { act[c] = 0; continue; }
            relres[c] = vnorm[c] > 0.0 ? std::sqrt(b2[c]) / vnorm[c] : 0.0;
            if (!std::isfinite(relres[c])) {
                status[c] = BTTB_ERR_NONFINITE;
                done[c] = 1;
            } else if (relres[c] <= o->tol || vnorm[c] == 0.0) {
                status[c] = BTTB_OK;
                done[c] = 1;
            } else if (total[c] >= max_iters) {
                status[c] = BTTB_NOT_CONVERGED;
                done[c] = 1;
            } else if (cycle > 0 && bd[c] && stp[c] == 0) {
                status[c] = BTTB_BREAKDOWN;
                done[c] = 1;
            }
            act[c] = done[c] ? 0 : 1;
            if (act[c]) {
                any = true;
                mlim[c] = std::min(m, max_iters - total[c]);
                const double b0 = std::sqrt(b2[c]);
                double t = 0.9 * o->tol * vnorm[c];
                if (inner == BTTB_MV_FP32) t = std::max(t, 1e-5 * b0);
                tgt[c] = t;
                cycles[c] += 1;
            }
        }
        if (o->history && hist_n < o->history_len) o->history[hist_n++] = relres[0];
        if (!any) break;
        cudaMemcpyAsync(g->active, act.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(g->mlimit, mlim.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(g->target, tgt.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(g->bdown, 0, sizeof(int) * k, st);
        cudaMemsetAsync(g->steps, 0, sizeof(int) * k, st);
        cycle_start_kernel<<<1, 256, 0, st>>>(g->beta2, g->gv, g->inv_beta, m, k, g->active, g->d_j);
        count_launch(p);
        scale_kernel<<<dim3(vgrid, k), kVecThreads, 0, st>>>(g->R, g->Vb, bs_i, bs_c, g->d_j, g->inv_beta, n,
                                                             g->active);
        count_launch(p);
        for (int step = 0; step < m; ++step) {
            const float4 *src = g->Vb;
            if (flex) {
                rc = block_jacobi_run(p, g->Vb, FMT_CDF, n, g->Zb, FMT_CDF, n, k, g->d_j, bs_i);
                if (rc != BTTB_OK) return rc;
                src = g->Zb;
            }
            rc = matvec_run(p, src, FMT_CDF, n, g->W, FMT_CDF, n, k, inner, g->d_j, bs_i);
            if (rc != BTTB_OK) return rc;
            for (int pass = 0; pass < 2; ++pass) {
                dots_partial_kernel<<<dim3(g->nblk, k), kVecThreads, g->NB * sizeof(float4), st>>>(
                    g->Vb, bs_i, bs_c, g->d_j, 0, g->W, n, g->NB, g->nblk, m + 1, g->part, g->active);
                count_launch(p);
                dots_reduce_kernel<<<dim3(m + 1, k), 32, 0, st>>>(g->part, g->nblk, g->d_j, 0, m + 1, g->hco, g->hacc,
                                                                   pass, nullptr, g->active);
                count_launch(p);
                update_kernel<<<dim3(vgrid, k), kVecThreads, (m + 1) * sizeof(float4), st>>>(
                    g->Vb, bs_i, bs_c, g->d_j, nullptr, g->hco, m + 1, g->W, n, -1.f, g->active);
                count_launch(p);
            }
            if ((rc = norm2_cols(p, g, g->W, k, g->active)) != BTTB_OK) return rc;
            givens_kernel<<<1, 256, 0, st>>>(g->H, g->hacc, g->beta2, g->cs, g->sn, g->gv, g->active, g->steps,
                                             g->bdown, g->mlimit, g->target, g->inv_beta, m, k, g->d_j, g->d_any,
                                             p->d_err);
            count_launch(p);
            scale_kernel<<<dim3(vgrid, k), kVecThreads, 0, st>>>(g->W, g->Vb, bs_i, bs_c, g->d_j, g->inv_beta, n,
                                                                 g->active);
            count_launch(p);
            e = cudaMemcpyAsync(g->h_any, g->d_any, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return check_cuda(p, e, "Arnoldi step");
            if (!*g->h_any) break;
        }
        // x += Z_basis y over the steps each column took in this cycle.
        cudaMemcpyAsync(g->active, act.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st);
        finish_kernel<<<(k + 127) / 128, 128, 0, st>>>(g->H, g->gv, g->steps, g->ycoef, m, k, g->active);
        count_launch(p);
        update_kernel<<<dim3(vgrid, k), kVecThreads, (m + 1) * sizeof(float4), st>>>(
            flex ? g->Zb : g->Vb, bs_i, bs_c, nullptr, g->steps, g->ycoef, m + 1, g->X, n, 1.f, g->active);
        count_launch(p);
        e = cudaMemcpyAsync(stp.data(), g->steps, sizeof(int) * k, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(bd.data(), g->bdown, sizeof(int) * k, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return check_cuda(p, e, "cycle end");
        for (int c = 0; c < k; ++c)
            if (act[c]) total[c] += stp[c];
    }

    // Output
    double2 *Id = reinterpret_cast<double2 *>(I);
    long ldo = ld;
    if (o->host_io) {
        Id = g->io;
        ldo = n;
    }
    cvt_out_kernel<<<dim3(vgrid, k), kVecThreads, 0, st>>>(g->X, Id, ldo, n);
    count_launch(p);
    if (o->host_io) {
        e = cudaMemcpy2DAsync(I, ld * sizeof(double2), g->io, n * sizeof(double2), n * sizeof(double2), k,
                              cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return check_cuda(p, e, "copy I to host");
    }
    e = cudaMemcpyAsync(&dev_err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return check_cuda(p, e, "solve end");
    int worst = BTTB_OK;
    for (int c = 0; c < k; ++c) {
        if (out) {
            out[c].status = status[c];
            out[c].iters = total[c];
            out[c].cycles = cycles[c];
            out[c].relres_true = relres[c];
        }
        if (status[c] < 0) worst = std::min(worst, status[c]);
        else if (worst >= 0) worst = std::max(worst, status[c]);
    }
    if (dev_err & DEVERR_TIMEOUT) return set_error(p, BTTB_ERR_TIMEOUT, "a device pipeline wait timed out");
    if (worst == BTTB_ERR_NONFINITE) return set_error(p, BTTB_ERR_NONFINITE, "non-finite residual");
    return worst;
}

}  // namespace bttb
