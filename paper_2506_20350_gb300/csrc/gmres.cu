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
    int *act_cycle = nullptr;     // columns active at the start of the cycle
    unsigned *counters = nullptr; // 3k per-column arrival counters + 1 global (fused step kernels)
    int *d_any_step = nullptr;    // largest step + 1 after which some column continued
    size_t bytes = 0;
    // Captured restart cycle (graph mode).
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t cycle_exec = nullptr;
    int graph_inner = -1;
    bool graph_prof = false;
    long launches_per_cycle = 0;
    std::vector<Plan::GraphRec> grecs;
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

// One Givens step of column c by one warp (binary64 scalars).  The lanes stage
// the Hessenberg column and the earlier rotations in shared memory (3m+2
// double2 at `wsm`), lane 0 applies the rotations in order from there.
// Returns (on every lane) whether the column continues.
__device__ int givens_column(int c, int j, int m, double2 *wsm, double2 *H, const double2 *hacc,
                             const double *beta2, double *cs, double2 *sn, double2 *gv, int *active, int *steps,
                             int *bdown, const int *mlimit, const double *target, double *inv_beta, int *err) {
    const int lane = threadIdx.x & 31;
    double2 *hcol = wsm;                                        // m+1 entries
    double2 *snw = hcol + (m + 1);                              // m entries
    double *csw = reinterpret_cast<double *>(snw + m);          // m entries
    double2 *Hc = H + (long)c * (m + 1) * m;
    const double2 *ha = hacc + (long)c * (m + 1);
    double zn2 = 0.0;
    for (int i = lane; i <= j; i += 32) {
        const double2 h = ha[i];
        hcol[i] = h;
        zn2 += h.x * h.x + h.y * h.y;
    }
    for (int i = lane; i < j; i += 32) {
        snw[i] = sn[(long)c * m + i];
        csw[i] = cs[(long)c * m + i];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) zn2 += __shfl_xor_sync(0xffffffffu, zn2, off);
    __syncwarp();
    int cont = 0;
    if (lane == 0) {
        const double beta = sqrt(fmax(beta2[c], 0.0));
        const double zn = sqrt(zn2 + beta * beta);
        if (!isfinite(zn)) {
            atomicOr(err, DEVERR_NONFINITE);
            active[c] = 0;
        } else {
            for (int i = 0; i < j; ++i) {
                const double2 a0 = hcol[i], a1 = hcol[i + 1], s = snw[i];
                const double ci = csw[i];
                hcol[i] = make_double2(ci * a0.x + (s.x * a1.x - s.y * a1.y), ci * a0.y + (s.x * a1.y + s.y * a1.x));
                // -conj(s) a0 + c a1
                hcol[i + 1] = make_double2(-(s.x * a0.x + s.y * a0.y) + ci * a1.x,
                                           -(s.x * a0.y - s.y * a0.x) + ci * a1.y);
            }
            const double2 a = hcol[j];
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
            cs[(long)c * m + j] = c_;
            sn[(long)c * m + j] = s_;
            hcol[j] = make_double2(c_ * a.x + s_.x * beta, c_ * a.y + s_.y * beta);
            double2 *g = gv + (long)c * (m + 1);
            const double2 gj = g[j];
            // g[j+1] = -conj(s) g[j] ; g[j] = c g[j]
            g[j + 1] = make_double2(-(s_.x * gj.x + s_.y * gj.y), -(s_.x * gj.y - s_.y * gj.x));
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
                cont = 1;
            }
        }
    }
    __syncwarp();
    for (int i = lane; i <= j; i += 32) Hc[i + (long)j * (m + 1)] = hcol[i];
    return __shfl_sync(0xffffffffu, cont, 0);
}

// ---------------------------------------------------------------------------
// Fused Arnoldi-step kernels.  One CTA = 256 consecutive entries of one
// column; grid (nblk, k).  Partial sums of a column are combined by the last
// CTA of that column to arrive (per-column counter, fixed summation order).
// ---------------------------------------------------------------------------
constexpr int kStepNB = 256;
constexpr int kStepWarps = kStepNB / 32;

// Per-CTA partial dots conj(B_i) . x over the CTA's chunk for i < cnt, x staged
// in xs; warp w takes i = w, w+8, ...  Result to part[(c*maxcnt + i)*nblk + blk].
__device__ __forceinline__ void cta_dots(const float4 *basis, long bs_i, long boff, const float4 *xs, int len,
                                         int cnt, float4 *part, long pbase, int nblk, int blk) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < cnt; i += kStepWarps) {
        const float4 *bv = basis + (long)i * bs_i + boff;
        dacc re{0.f, 0.f}, im{0.f, 0.f};
#pragma unroll 4
        for (int e = lane; e < len; e += 32) {
            const float4 v = bv[e], x = xs[e];
            dacc_mac(re, v.x, v.z, x.x, x.z);
            dacc_mac(re, v.y, v.w, x.y, x.w);
            dacc_mac(im, v.x, v.z, x.y, x.w);
            dacc_mac(im, -v.y, -v.w, x.x, x.z);
        }
        warp_reduce_dacc(re);
        warp_reduce_dacc(im);
        if (lane == 0) {
            const df r = dacc_result(re), q = dacc_result(im);
            part[(pbase + i) * nblk + blk] = make_float4(r.hi, q.hi, r.lo, q.lo);
        }
    }
}

// Last CTA of column c: sum the partials of i < cnt in block order.
// mode 0: hco = h, hacc = h ; mode 1: hco = h, hacc += h ; mode 2: beta2 = Re h_0
__device__ __forceinline__ void last_cta_reduce(const float4 *part, long pbase, int nblk, int cnt, int mode,
                                                float4 *hco, double2 *hacc, double *beta2, int c) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < cnt; i += kStepWarps) {
        const float4 *pp = part + (pbase + i) * nblk;
        dacc re{0.f, 0.f}, im{0.f, 0.f};
        for (int e = lane; e < nblk; e += 32) {
            const float4 v = __ldcg(pp + e);
            dacc_add(re, dacc{v.x, v.z});
            dacc_add(im, dacc{v.y, v.w});
        }
        warp_reduce_dacc(re);
        warp_reduce_dacc(im);
        if (lane == 0) {
            const df r = dacc_result(re), q = dacc_result(im);
            if (mode == 2) {
                beta2[c] = df_to_double(r);
            } else {
                hco[pbase + i] = make_float4(r.hi, q.hi, r.lo, q.lo);
                const double2 v = make_double2(df_to_double(r), df_to_double(q));
                double2 &h = hacc[pbase + i];
                h = mode == 0 ? v : make_double2(h.x + v.x, h.y + v.y);
            }
        }
    }
}

// Returns true in every thread of the CTA that arrives last for column c.
__device__ __forceinline__ bool arrive_last(unsigned *counter, int nblk) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(counter, 1u);
        s_last = (prev == (unsigned)nblk - 1);
        if (s_last) *counter = 0u;                 // ready for the next use
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// w -= sum_{i<cnt} B_i h_i for this thread's entry (compensated), returns the new value.
__device__ __forceinline__ float4 cta_update_entry(const float4 *basis, long bs_i, long boff, const float4 *hs,
                                                   int cnt, float4 x) {
    dacc re{x.x, x.z}, im{x.y, x.w};
#pragma unroll 8
    for (int i = 0; i < cnt; ++i) {
        const float4 v = basis[(long)i * bs_i + boff];
        const float4 h = hs[i];                     // already negated
        dacc_mac(re, v.x, v.z, h.x, h.z);
        dacc_mac(re, -v.y, -v.w, h.y, h.w);
        dacc_mac(im, v.x, v.z, h.y, h.w);
        dacc_mac(im, v.y, v.w, h.x, h.z);
    }
    const df r = dacc_result(re), q = dacc_result(im);
    return make_float4(r.hi, q.hi, r.lo, q.lo);
}

struct StepArgs {
    const float4 *Vb;      // basis [i][c][n]
    float4 *W;             // [c][n]
    long n, bs_i, bs_c;
    int m, k, nblk;
    float4 *part;          // [c][m+1][nblk]
    float4 *hco;           // [c][m+1]
    double2 *hacc;         // [c][m+1]
    double *beta2;
    unsigned *cnt_a, *cnt_b, *cnt_c, *cnt_d;    // per-column arrival counters (cnt_d: one)
    int *active;
    int *d_j, *d_any_step;
    // Givens
    double2 *H, *gv, *sn;
    double *cs, *inv_beta;
    int *steps, *bdown;
    const int *mlimit;
    const double *target;
    int *err;
};

// (A) first Gram-Schmidt pass: h = V_j^H w
__global__ void __launch_bounds__(kStepNB) step_dots_kernel(const StepArgs a) {
    __shared__ float4 xs[kStepNB];
    const int c = blockIdx.y, blk = blockIdx.x;
    if (!a.active[c]) return;
    const int cnt = *a.d_j + 1;
    const long n0 = (long)blk * kStepNB;
    const int len = (int)min((long)kStepNB, a.n - n0);
    if ((int)threadIdx.x < len) xs[threadIdx.x] = a.W[(long)c * a.n + n0 + threadIdx.x];
    __syncthreads();
    const long pbase = (long)c * (a.m + 1);
    cta_dots(a.Vb, a.bs_i, (long)c * a.bs_c + n0, xs, len, cnt, a.part, pbase, a.nblk, blk);
    if (!arrive_last(a.cnt_a + c, a.nblk)) return;
    last_cta_reduce(a.part, pbase, a.nblk, cnt, 0, a.hco, a.hacc, nullptr, c);
}

// (B) w -= V h (first pass), then the second pass h2 = V^H w
__global__ void __launch_bounds__(kStepNB) step_update_dots_kernel(const StepArgs a) {
    __shared__ float4 xs[kStepNB];
    extern __shared__ __align__(16) float4 hs[];          // m+1
    const int c = blockIdx.y, blk = blockIdx.x;
    if (!a.active[c]) return;
    const int cnt = *a.d_j + 1;
    const long pbase = (long)c * (a.m + 1);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const float4 h = a.hco[pbase + i];
        hs[i] = make_float4(-h.x, -h.y, -h.z, -h.w);
    }
    __syncthreads();
    const long n0 = (long)blk * kStepNB;
    const int len = (int)min((long)kStepNB, a.n - n0);
    const int t = threadIdx.x;
    if (t < len) {
        const long e = (long)c * a.n + n0 + t;
        const float4 x = cta_update_entry(a.Vb, a.bs_i, (long)c * a.bs_c + n0 + t, hs, cnt, a.W[e]);
        a.W[e] = x;
        xs[t] = x;
    }
    __syncthreads();
    cta_dots(a.Vb, a.bs_i, (long)c * a.bs_c + n0, xs, len, cnt, a.part, pbase, a.nblk, blk);
    if (!arrive_last(a.cnt_b + c, a.nblk)) return;
    last_cta_reduce(a.part, pbase, a.nblk, cnt, 1, a.hco, a.hacc, nullptr, c);
}

// (C) w -= V h2, beta^2 = ||w||^2, then (last CTA of the column) one Givens step
__global__ void __launch_bounds__(kStepNB) step_update_norm_givens_kernel(const StepArgs a) {
    __shared__ float4 xs[kStepNB];
    extern __shared__ __align__(16) float4 dyn[];          // hs: m+1 float4, then Givens scratch
    const int c = blockIdx.y, blk = blockIdx.x;
    if (!a.active[c]) return;
    const int j = *a.d_j, cnt = j + 1;
    const long pbase = (long)c * (a.m + 1);
    float4 *hs = dyn;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const float4 h = a.hco[pbase + i];
        hs[i] = make_float4(-h.x, -h.y, -h.z, -h.w);
    }
    __syncthreads();
    const long n0 = (long)blk * kStepNB;
    const int len = (int)min((long)kStepNB, a.n - n0);
    const int t = threadIdx.x;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t < len) {
        const long e = (long)c * a.n + n0 + t;
        x = cta_update_entry(a.Vb, a.bs_i, (long)c * a.bs_c + n0 + t, hs, cnt, a.W[e]);
        a.W[e] = x;
    }
    xs[t] = x;
    __syncthreads();
    cta_dots(xs - (long)0, 0, 0, xs, len, 1, a.part, pbase, a.nblk, blk);   // ||w||^2 partial (i = 0)
    if (!arrive_last(a.cnt_c + c, a.nblk)) return;
    last_cta_reduce(a.part, pbase, a.nblk, 1, 2, nullptr, nullptr, a.beta2, c);
    __syncthreads();
    if (threadIdx.x < 32) {
        double2 *wsm = reinterpret_cast<double2 *>(dyn + (a.m + 1));
        const int cont = givens_column(c, j, a.m, wsm, a.H, a.hacc, a.beta2, a.cs, a.sn, a.gv, a.active, a.steps,
                                       a.bdown, a.mlimit, a.target, a.inv_beta, a.err);
        if (threadIdx.x == 0 && cont) atomicMax(a.d_any_step, j + 1);
    }
}

// (D) v_{j+1} = w / beta for continuing columns; the last CTA overall advances j.
__global__ void __launch_bounds__(kStepNB) step_scale_advance_kernel(const StepArgs a) {
    const int c = blockIdx.y, blk = blockIdx.x;
    const int j = *a.d_j;
    if (a.active[c]) {
        const df s = df_from_double(a.inv_beta[c]);
        const long n0 = (long)blk * kStepNB;
        const long e = n0 + threadIdx.x;
        if (e < a.n) {
            const float4 x = a.W[(long)c * a.n + e];
            const df r = df_mul(df{x.x, x.z}, s), q = df_mul(df{x.y, x.w}, s);
            const_cast<float4 *>(a.Vb)[(long)(j + 1) * a.bs_i + (long)c * a.bs_c + e] =
                make_float4(r.hi, q.hi, r.lo, q.lo);
        }
    }
    if (arrive_last(a.cnt_d, a.nblk * a.k)) {
        if (threadIdx.x == 0) *a.d_j = j + 1;
    }
}

// y = H^{-1} g (upper triangular, steps[c] x steps[c]) for column c = blockIdx.x,
// stored as double-float.  Column-oriented back substitution: one diagonal
// division per step, the remaining right-hand side updated in parallel.
constexpr int kFinishThreads = 128;

__global__ void __launch_bounds__(kFinishThreads) finish_kernel(const double2 *H, const double2 *gv,
                                                                const int *steps, float4 *ycoef, int m,
                                                                const int *was_active) {
    extern __shared__ __align__(16) unsigned char fsm[];
    const int c = blockIdx.x;
    if (!was_active[c]) return;
    const int kk = steps[c];
    double2 *rhs = reinterpret_cast<double2 *>(fsm);              // m+1
    const double2 *Hc = H + (long)c * (m + 1) * m;
    const double2 *g = gv + (long)c * (m + 1);
    for (int i = threadIdx.x; i < kk; i += blockDim.x) rhs[i] = g[i];
    __syncthreads();
    for (int i = kk - 1; i >= 0; --i) {
        const double2 d = Hc[i + (long)i * (m + 1)];
        const double dd = d.x * d.x + d.y * d.y;
        const double2 s = rhs[i];
        const double2 yi = dd > 0.0 ? make_double2((s.x * d.x + s.y * d.y) / dd, (s.y * d.x - s.x * d.y) / dd)
                                    : make_double2(0.0, 0.0);
        for (int l = threadIdx.x; l < i; l += blockDim.x) {
            const double2 t = cmul(Hc[l + (long)i * (m + 1)], yi);
            rhs[l] = make_double2(rhs[l].x - t.x, rhs[l].y - t.y);
        }
        if (threadIdx.x == 0) ycoef[(long)c * (m + 1) + i] = F64N::to_cdf(yi);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host side

static void drop_graph(GmresWork *g) {
    if (g->cycle_exec) cudaGraphExecDestroy(g->cycle_exec);
    g->cycle_exec = nullptr;
    for (auto &r : g->grecs) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    g->grecs.clear();
}

static void free_work(GmresWork *g) {
    if (!g) return;
    drop_graph(g);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    cudaFree(g->X); cudaFree(g->Vb); cudaFree(g->Zb); cudaFree(g->W); cudaFree(g->R); cudaFree(g->Vin);
    cudaFree(g->H); cudaFree(g->hacc); cudaFree(g->gv); cudaFree(g->sn); cudaFree(g->hco); cudaFree(g->ycoef);
    cudaFree(g->part); cudaFree(g->cs); cudaFree(g->beta2); cudaFree(g->vnorm); cudaFree(g->inv_beta);
    cudaFree(g->target); cudaFree(g->active); cudaFree(g->steps); cudaFree(g->bdown); cudaFree(g->mlimit);
    cudaFree(g->d_j); cudaFree(g->d_any); cudaFree(g->io); cudaFree(g->act_cycle);
    cudaFree(g->counters); cudaFree(g->d_any_step);
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
    if (g && g->m == m && g->k == k && (g->flex || !flex) && (!host_io || g->io)) return BTTB_OK;
    gmres_free(p);
    g = new GmresWork();
    g->m = m;
    g->k = k;
    g->n = p->n;
    g->flex = flex;
    g->NB = kStepNB;
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
    alloc(&g->act_cycle, sizeof(int) * k);
    alloc(&g->steps, sizeof(int) * k);
    alloc(&g->bdown, sizeof(int) * k);
    alloc(&g->mlimit, sizeof(int) * k);
    alloc(&g->d_j, sizeof(int));
    alloc(&g->d_any, sizeof(int));
    alloc(&g->counters, sizeof(unsigned) * (3 * (size_t)k + 1));
    alloc(&g->d_any_step, sizeof(int));
    if (ok && cudaMemset(g->counters, 0, sizeof(unsigned) * (3 * (size_t)k + 1)) != cudaSuccess) ok = false;
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

// One Arnoldi step for every active column, on p->stream (captured or not):
// [block-Jacobi], the product, then the four fused Gram-Schmidt/Givens kernels.
static int arnoldi_step(Plan *p, GmresWork *g, int inner) {
    const int m = g->m, k = g->k;
    const long n = p->n, bs_i = (long)k * n;
    cudaStream_t st = p->stream;
    int rc;
    const float4 *src = g->Vb;
    if (g->flex) {
        rc = block_jacobi_run(p, g->Vb, FMT_CDF, n, g->Zb, FMT_CDF, n, k, g->d_j, bs_i, g->active);
        if (rc != BTTB_OK) return rc;
        src = g->Zb;
    }
    rc = matvec_run(p, src, FMT_CDF, n, g->W, FMT_CDF, n, k, inner, g->d_j, bs_i, nullptr, g->active);
    if (rc != BTTB_OK) return rc;
    StepArgs a{};
    a.Vb = g->Vb;
    a.W = g->W;
    a.n = n;
    a.bs_i = bs_i;
    a.bs_c = n;
    a.m = m;
    a.k = k;
    a.nblk = g->nblk;
    a.part = g->part;
    a.hco = g->hco;
    a.hacc = g->hacc;
    a.beta2 = g->beta2;
    a.cnt_a = g->counters;
    a.cnt_b = g->counters + k;
    a.cnt_c = g->counters + 2 * k;
    a.cnt_d = g->counters + 3 * k;
    a.active = g->active;
    a.d_j = g->d_j;
    a.d_any_step = g->d_any_step;
    a.H = g->H;
    a.gv = g->gv;
    a.sn = g->sn;
    a.cs = g->cs;
    a.inv_beta = g->inv_beta;
    a.steps = g->steps;
    a.bdown = g->bdown;
    a.mlimit = g->mlimit;
    a.target = g->target;
    a.err = p->d_err;
    const dim3 grid(g->nblk, k);
    const size_t hs_bytes = (size_t)(m + 1) * sizeof(float4);
    step_dots_kernel<<<grid, kStepNB, 0, st>>>(a);
    step_update_dots_kernel<<<grid, kStepNB, hs_bytes, st>>>(a);
    step_update_norm_givens_kernel<<<grid, kStepNB, hs_bytes + (size_t)(3 * m + 2) * sizeof(double2), st>>>(a);
    step_scale_advance_kernel<<<grid, kStepNB, 0, st>>>(a);
    count_launch(p, 4);
    return check_cuda(p, cudaGetLastError(), "Arnoldi step launch");
}

// Back substitution and x += (preconditioned) basis * y for the columns of this cycle.
static int cycle_finish(Plan *p, GmresWork *g) {
    const int m = g->m, k = g->k;
    const long n = p->n, bs_i = (long)k * n, bs_c = n;
    const int vgrid = (int)std::min<long>((n + kVecThreads - 1) / kVecThreads, 1024);
    finish_kernel<<<k, kFinishThreads, (m + 1) * sizeof(double2), p->stream>>>(g->H, g->gv, g->steps, g->ycoef, m,
                                                                               g->act_cycle);
    count_launch(p);
    update_kernel<<<dim3(vgrid, k), kVecThreads, (m + 1) * sizeof(float4), p->stream>>>(
        g->flex ? g->Zb : g->Vb, bs_i, bs_c, nullptr, g->steps, g->ycoef, m + 1, g->X, n, 1.f, g->act_cycle);
    count_launch(p);
    return check_cuda(p, cudaGetLastError(), "cycle finish launch");
}

// Capture m Arnoldi steps and the cycle finish into one executable graph.
static int build_cycle_graph(Plan *p, GmresWork *g, int inner) {
    drop_graph(g);
    cudaError_t e;
    if (!g->cap_stream && (e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return check_cuda(p, e, "capture stream");
    cudaStream_t saved = p->stream;
    const long launches0 = p->launches;
    p->stream = g->cap_stream;
    p->sink = &g->grecs;
    if ((e = cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeRelaxed)) != cudaSuccess) {
        p->stream = saved;
        p->sink = nullptr;
        return check_cuda(p, e, "begin capture");
    }
    int rc = BTTB_OK;
    for (int step = 0; step < g->m && rc == BTTB_OK; ++step) {
        p->sink_step = step;
        rc = arnoldi_step(p, g, inner);
    }
    p->sink_step = g->m;
    if (rc == BTTB_OK) rc = cycle_finish(p, g);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(g->cap_stream, &graph);
    p->stream = saved;
    p->sink = nullptr;
    g->launches_per_cycle = p->launches - launches0;
    p->launches = launches0;
    if (rc != BTTB_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return check_cuda(p, e, "end capture");
    e = cudaGraphInstantiate(&g->cycle_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return check_cuda(p, e, "graph instantiate");
    g->graph_inner = inner;
    g->graph_prof = p->prof;
    return BTTB_OK;
}

int gmres_solve(Plan *p, const void *V, void *I, int k, long ld, const bttb_gmres_opts *o,
                bttb_col_result *out) {
    const int m = o->restart;
    const bool flex = o->pc == BTTB_PC_BLOCK_JACOBI;
    const int inner = o->inner;
    const bool use_graph = !(o->flags & BTTB_GMRES_NO_GRAPH);
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
    std::vector<int> status(k, BTTB_OK), total(k, 0), cycles(k, 0), act(k), mlim(k), stp(k, 0), bd(k, 0);
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
        cudaMemcpyAsync(g->act_cycle, act.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(g->mlimit, mlim.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(g->target, tgt.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(g->bdown, 0, sizeof(int) * k, st);
        cudaMemsetAsync(g->steps, 0, sizeof(int) * k, st);
        cudaMemsetAsync(g->d_any_step, 0, sizeof(int), st);
        cycle_start_kernel<<<1, 256, 0, st>>>(g->beta2, g->gv, g->inv_beta, m, k, g->active, g->d_j);
        count_launch(p);
        scale_kernel<<<dim3(vgrid, k), kVecThreads, 0, st>>>(g->R, g->Vb, bs_i, bs_c, g->d_j, g->inv_beta, n,
                                                             g->active);
        count_launch(p);
        if (use_graph) {
            if (!g->cycle_exec || g->graph_inner != inner || g->graph_prof != p->prof)
                if ((rc = build_cycle_graph(p, g, inner)) != BTTB_OK) return rc;
            if ((e = cudaGraphLaunch(g->cycle_exec, st)) != cudaSuccess) return check_cuda(p, e, "graph launch");
            p->launches += g->launches_per_cycle;
        } else {
            for (int step = 0; step < m; ++step) {
                if ((rc = arnoldi_step(p, g, inner)) != BTTB_OK) return rc;
                e = cudaMemcpyAsync(g->h_any, g->d_any_step, sizeof(int), cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) return check_cuda(p, e, "Arnoldi step");
                if (*g->h_any < step + 1) break;              // no column continued after this step
            }
            if ((rc = cycle_finish(p, g)) != BTTB_OK) return rc;
        }
        e = cudaMemcpyAsync(stp.data(), g->steps, sizeof(int) * k, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(bd.data(), g->bdown, sizeof(int) * k, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return check_cuda(p, e, "cycle end");
        int maxsteps = 0;
        for (int c = 0; c < k; ++c)
            if (act[c]) {
                total[c] += stp[c];
                maxsteps = std::max(maxsteps, stp[c]);
            }
        if (use_graph && p->prof) {
            // Timed launches of the steps that did work (later steps exited at once).
            for (const auto &r : g->grecs) {
                if (r.step >= maxsteps && r.step < m) continue;
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) continue;
                if (r.kid >= 0 && r.kid < Plan::kMaxKid) {
                    p->acc_ms[r.kid] += ms;
                    p->acc_bytes[r.kid] += r.bytes;
                    p->acc_n[r.kid] += 1;
                }
            }
        }
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
