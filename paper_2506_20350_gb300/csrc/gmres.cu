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
// iterative refinement (GMRES-IR).  Vectors, inner products, updates, the
// Hessenberg matrix, the rotations and the triangular solve are all
// double-float (48-bit significand) on the binary32 pipes: scalar binary64
// code is slow on this GPU.  Converged columns are masked.
#include <algorithm>
#include <cmath>
#include <vector>

#include "arith.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace bttb {

struct GmresWork {
    int m = 0, k = 0;             // Krylov dimension, Krylov columns
    long n = 0;                   // Krylov vector length
    int kp = 0;                   // product columns (k, or the k user columns of one global Krylov column)
    long np = 0;                  // product vector length (N)
    bool glob = false;            // global GMRES: one Krylov column over all kp user columns
    int *act_prod = nullptr;      // per product column copy of the global column's active flag
    bool dcgs = false;            // delayed CGS2 (unpreconditioned cycles) instead of CGS2
    float4 *U = nullptr;          // delayed CGS2: the not yet reorthogonalised vector u_j [k][n]
    float4 *cco = nullptr, *hpre = nullptr;   // [k][m+1]: update coefficients; [2][k][m+1] preliminary column
    float4 *Horig = nullptr;      // [k][(m+1)*m] Hessenberg columns before the rotations
    bool flex = false;            // Zb allocated
    int pc = BTTB_PC_NONE;        // preconditioner of the current solve
    int NB = 0, nblk = 0;
    float4 *X = nullptr, *Vb = nullptr, *Zb = nullptr, *W = nullptr, *R = nullptr, *Vin = nullptr;
    // Hessenberg [c][(m+1)*m] column-major, accumulated CGS coefficients [c][m+1],
    // rotation sines [c][m] and right-hand side [c][m+1]: complex double-float;
    // rotation cosines [c][m]: real double-float.
    float4 *H = nullptr, *hacc = nullptr, *gv = nullptr, *sn = nullptr;
    float2 *cs = nullptr;
    float4 *hco = nullptr, *ycoef = nullptr, *part = nullptr;
    double *beta2 = nullptr, *vnorm = nullptr, *inv_beta = nullptr, *target = nullptr;
    unsigned long long *cmax = nullptr;   // per user column: largest |Re|, |Im| of V (binary64 bits)
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
    int graph_pc = -1;
    int graph_dcgs = -1;
    int graph_prof = 0;
    long launches_per_cycle = 0;
    std::vector<Plan::GraphRec> grecs;
};

constexpr int kVecThreads = 256;

// ------------------------------------------------------------------ kernels

// Input scaling.  Double-float numbers have binary32's exponent range, so a right-hand side whose entries
// lie far from 1 (below ~1e-19 its squared norm underflows, above ~1e19 it overflows) cannot be solved as
// given.  Each column c of V (and of the initial guess) is therefore multiplied by 2^-e_c, e_c the binary64
// exponent of the column's largest |Re| or |Im|, before the conversion, and the solution by 2^e_c after it.
// Scaling by a power of two is exact and commutes with every rounding of the solver, so the iterates are
// the same as for the unscaled column whenever that one stays in range; the relative residual does not
// change.  Global GMRES uses one exponent for all columns (its Frobenius inner products mix them).
//
// cmax[c * cstride] = largest |Re|, |Im| of column c as binary64 bits: for non-negative doubles the integer
// order is the numeric order and a NaN sorts above +Inf, so one NaN makes the column's maximum NaN.
__global__ void colmax_kernel(const double2 *in, long ld, long n, unsigned long long *cmax, int cstride) {
    const int c = blockIdx.y;
    unsigned long long m = 0ull;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double2 v = in[(long)c * ld + i];
        m = max(m, (unsigned long long)__double_as_longlong(fabs(v.x)));
        m = max(m, (unsigned long long)__double_as_longlong(fabs(v.y)));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0 && m != 0ull) atomicMax(cmax + (long)c * cstride, m);
}

// e_c of a column maximum; zero and non-finite columns stay unscaled (the norm check reports the latter).
__device__ __forceinline__ int col_exponent(unsigned long long bits) {
    const double m = __longlong_as_double((long long)bits);
    return (m > 0.0 && isfinite(m)) ? ilogb(m) : 0;
}

__global__ void cvt_in_kernel(const double2 *in, long ld, float4 *out, long n, const unsigned long long *cmax,
                              int cstride) {
    const int c = blockIdx.y;
    const int e = col_exponent(cmax[(long)c * cstride]);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double2 v = in[(long)c * ld + i];
        out[(long)c * n + i] = F64N::to_cdf(make_double2(ldexp(v.x, -e), ldexp(v.y, -e)));
    }
}

// I = 2^e_c X; a column whose V is exactly zero has the solution zero, whatever the initial guess.
__global__ void cvt_out_kernel(const float4 *in, double2 *out, long ld, long n, const unsigned long long *cmax,
                               int cstride) {
    const int c = blockIdx.y;
    const unsigned long long bits = cmax[(long)c * cstride];
    const int e = col_exponent(bits);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double2 v = DF64::to_c128(DF64::from_cdf(in[(long)c * n + i]));
        out[(long)c * ld + i] = bits == 0ull ? make_double2(0.0, 0.0) : make_double2(ldexp(v.x, e), ldexp(v.y, e));
    }
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

// Sum of n partials {re.hi, im.hi, re.lo, im.lo} by one warp: each lane issues its loads eight at
// a time before adding them (in the same per-lane order as a plain loop), then the warp reduces.
__device__ __forceinline__ void warp_sum_partials(const float4 *pp, int n, dacc &re, dacc &im) {
    const int lane = threadIdx.x & 31;
    re = dacc{0.f, 0.f};
    im = dacc{0.f, 0.f};
    for (int e0 = lane; e0 < n; e0 += 32 * 8) {
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + 32 * u;
            v[u] = e < n ? gldcg(pp + e) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            dacc_add(re, dacc{v[u].x, v[u].z});
            dacc_add(im, dacc{v[u].y, v[u].w});
        }
    }
    warp_reduce_dacc(re);
    warp_reduce_dacc(im);
}

// ||x_c||^2 partials: part[c*pstride + blk] over the block's chunk of NB entries.
__global__ void __launch_bounds__(kVecThreads) norm_partial_kernel(const float4 *x, long n, int NB, int nblk,
                                                                   long pstride, float4 *part) {
    __shared__ dacc red[kVecThreads / 32];
    const int c = blockIdx.y, blk = blockIdx.x;
    const long n0 = (long)blk * NB;
    const int len = (int)min((long)NB, n - n0);
    dacc acc{0.f, 0.f};
    for (int e = threadIdx.x; e < len; e += blockDim.x) {
        const float4 v = x[(long)c * n + n0 + e];
        dacc_mac(acc, v.x, v.z, v.x, v.z);
        dacc_mac(acc, v.y, v.w, v.y, v.w);
    }
    warp_reduce_dacc(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        dacc t = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) dacc_add(t, red[w]);
        const df r = dacc_result(t);
        gst(part + (long)c * pstride + blk, make_float4(r.hi, 0.f, r.lo, 0.f));
    }
}

// beta2[c] = sum of the column's partials (one warp per column).
__global__ void norm_final_kernel(const float4 *part, int nblk, long pstride, double *beta2) {
    const int c = blockIdx.x, lane = threadIdx.x;
    dacc acc, unused;
    warp_sum_partials(part + (long)c * pstride, nblk, acc, unused);
    if (lane == 0) beta2[c] = df_to_double(dacc_result(acc));
}

// w[c][n] += sgn * sum_{i < cnt_col[c]} B_i[c][n] coef[c][i]
// x += z (double-float) for the columns active in the cycle.
__global__ void add_active_kernel(float4 *x, const float4 *z, long n, const int *active) {
    const int c = blockIdx.y;
    if (active && !active[c]) return;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const float4 a = x[(long)c * n + e], b = z[(long)c * n + e];
        const df r = df_add(df{a.x, a.z}, df{b.x, b.z}), q = df_add(df{a.y, a.w}, df{b.y, b.w});
        x[(long)c * n + e] = make_float4(r.hi, q.hi, r.lo, q.lo);
    }
}

__global__ void __launch_bounds__(kVecThreads) update_kernel(const float4 *basis, long bs_i, long bs_c,
                                                             const int *cnt_col, const float4 *coef, int maxcnt,
                                                             float4 *w, long n, float sgn, const int *active) {
    extern __shared__ __align__(16) float4 csm[];
    const int c = blockIdx.y;
    if (active && !active[c]) return;
    const int cnt = cnt_col[c];
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        float4 h = coef[(long)c * maxcnt + i];
        csm[i] = make_float4(sgn * h.x, sgn * h.y, sgn * h.z, sgn * h.w);
    }
    __syncthreads();
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const float4 x = w[(long)c * n + e];
        dacc re{x.x, x.z}, im{x.y, x.w};
        for (int i = 0; i < cnt; ++i) {
            const float4 v = gld(basis + (long)i * bs_i + (long)c * bs_c + e);
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

// Vb[j][c] = W[c] * inv_beta[c]
__global__ void scale_kernel(const float4 *w, float4 *vb, long bs_i, long bs_c, int j,
                             const double *inv_beta, long n, const int *active) {
    const int c = blockIdx.y;
    if (active && !active[c]) return;
    const df s = df_from_double(inv_beta[c]);
    float4 *dst = vb + (long)j * bs_i + (long)c * bs_c;
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
// Global GMRES: every product column follows the one Krylov column's flag.
__global__ void bcast_active_kernel(const int *active, int *act_prod, int kp) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kp; i += gridDim.x * blockDim.x) act_prod[i] = active[0];
}

__global__ void cycle_start_kernel(const double *beta2, float4 *gv, double *inv_beta, int m, int k,
                                   const int *active) {
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if (!active[c]) continue;
        const double b0 = sqrt(beta2[c]);
        float4 *g = gv + (long)c * (m + 1);
        const df r = df_from_double(b0);
        g[0] = make_float4(r.hi, 0.f, r.lo, 0.f);
        for (int i = 1; i <= m; ++i) g[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        inv_beta[c] = 1.0 / b0;
    }
}

// Shuffle a double-float complex value (8 floats) within the warp.
__device__ __forceinline__ dfc shfl_up_dfc(dfc v, int d) {
    return dfc{df{__shfl_up_sync(0xffffffffu, v.re.hi, d), __shfl_up_sync(0xffffffffu, v.re.lo, d)},
               df{__shfl_up_sync(0xffffffffu, v.im.hi, d), __shfl_up_sync(0xffffffffu, v.im.lo, d)}};
}
__device__ __forceinline__ dfc shfl_dfc(dfc v, int src) {
    return dfc{df{__shfl_sync(0xffffffffu, v.re.hi, src), __shfl_sync(0xffffffffu, v.re.lo, src)},
               df{__shfl_sync(0xffffffffu, v.im.hi, src), __shfl_sync(0xffffffffu, v.im.lo, src)}};
}

// One Givens step of column c by one warp, in double-float.  The earlier
// rotations G_0 .. G_{j-1} act on the new Hessenberg column h as
//   out_i = c_i t_i + s_i h_{i+1},   t_{i+1} = -conj(s_i) t_i + c_i h_{i+1},
// t_0 = h_0, out_j = t_j: an affine recurrence for t, so the warp composes the
// maps t -> alpha t + beta with a prefix scan (each lane first composes its own
// run of consecutive rotations) instead of applying them one after another.
// Lane 0 then forms the new rotation.  Returns (on every lane) whether the
// column continues.  Scratch `wsm`: 4m+4 float4.
__device__ int givens_column(int c, int j, int m, float4 *wsm, float4 *H, const float4 *ha, double beta2,
                             float2 *cs, float4 *sn, float4 *gv, int *active, int *steps, int *bdown,
                             const int *mlimit, const double *target, double *inv_beta, int *err) {
    const int lane = threadIdx.x & 31;
    float4 *hcol = wsm;                                         // m+1 entries
    float4 *snw = hcol + (m + 1);                               // m entries
    float2 *csw = reinterpret_cast<float2 *>(snw + m);          // m entries (m float4 reserved)
    float4 *hout = snw + 2 * m;                                 // m+1 entries
    float4 *Hc = H + (long)c * (m + 1) * m;
    float zn2 = 0.f;
    for (int i = lane; i <= j; i += 32) {
        const float4 h = gld(ha + i);
        hcol[i] = h;
        zn2 += h.x * h.x + h.y * h.y;
    }
    for (int i = lane; i < j; i += 32) {
        snw[i] = gld(sn + (long)c * m + i);
        csw[i] = gld(cs + (long)c * m + i);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) zn2 += __shfl_xor_sync(0xffffffffu, zn2, off);
    __syncwarp();
    if (j > 0) {
        const int per = (j + 31) / 32;                          // rotations per lane
        const int i0 = min(lane * per, j), i1 = min(i0 + per, j);
        const dfc zero{df{0.f, 0.f}, df{0.f, 0.f}};
        dfc al{df{1.f, 0.f}, df{0.f, 0.f}}, be = zero;          // composition of this lane's maps
        for (int i = i0; i < i1; ++i) {
            const dfc si = dfc_load(*reinterpret_cast<const cdf *>(&snw[i]));
            const df ci{csw[i].x, csw[i].y};
            const dfc hn = dfc_load(*reinterpret_cast<const cdf *>(&hcol[i + 1]));
            const dfc ai = dfc_neg(dfc_conj(si));
            be = dfc_add(dfc_mul(ai, be), dfc_scale(hn, ci));
            al = dfc_mul(ai, al);
        }
        // inclusive scan over lanes: lane L holds the maps of lanes 0..L composed
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const dfc ao = shfl_up_dfc(al, d), bo = shfl_up_dfc(be, d);
            if (lane >= d) {
                be = dfc_add(dfc_mul(al, bo), be);
                al = dfc_mul(al, ao);
            }
        }
        // t at the start of this lane's run: the exclusive prefix applied to h_0
        dfc ea = shfl_up_dfc(al, 1), eb = shfl_up_dfc(be, 1);
        const dfc h0 = dfc_load(*reinterpret_cast<const cdf *>(&hcol[0]));
        dfc t = lane == 0 ? h0 : dfc_add(dfc_mul(ea, h0), eb);
        for (int i = i0; i < i1; ++i) {
            const dfc si = dfc_load(*reinterpret_cast<const cdf *>(&snw[i]));
            const df ci{csw[i].x, csw[i].y};
            const dfc hn = dfc_load(*reinterpret_cast<const cdf *>(&hcol[i + 1]));
            *reinterpret_cast<cdf *>(&hout[i]) = dfc_store(dfc_add(dfc_scale(t, ci), dfc_mul(si, hn)));
            t = dfc_add(dfc_mul(dfc_neg(dfc_conj(si)), t), dfc_scale(hn, ci));
        }
        // t_j from the full composition (lane 31)
        const dfc ta = shfl_dfc(al, 31), tb = shfl_dfc(be, 31);
        __syncwarp();
        for (int i = lane; i < j; i += 32) hcol[i] = hout[i];
        if (lane == 0) *reinterpret_cast<cdf *>(&hcol[j]) = dfc_store(dfc_add(dfc_mul(ta, h0), tb));
        __syncwarp();
    }
    int cont = 0;
    if (lane == 0) {
        const df beta = df_sqrt(df_from_double(fmax(beta2, 0.0)));
        const float zn = sqrtf(zn2 + beta.hi * beta.hi);
        if (!isfinite(zn) || !isfinite(beta.hi)) {
            atomicOr(err, DEVERR_NONFINITE);
            active[c] = 0;
        } else {
            const dfc a = dfc_load(*reinterpret_cast<const cdf *>(&hcol[j]));
            const df aa2 = dfc_abs2(a);
            const df rho = df_sqrt(df_add(aa2, df_mul(beta, beta)));
            df c_;
            dfc s_;
            if (!(aa2.hi > 0.f)) {
                c_ = df{0.f, 0.f};
                s_ = dfc{df{1.f, 0.f}, df{0.f, 0.f}};
            } else {
                const df aa = df_sqrt(aa2);
                const df inv_rho = df_recip(rho);
                c_ = df_mul(aa, inv_rho);
                s_ = dfc_scale(a, df_mul(df_mul(beta, inv_rho), df_recip(aa)));   // (a/|a|) beta/rho
            }
            gst(cs + (long)c * m + j, make_float2(c_.hi, c_.lo));
            gst(reinterpret_cast<cdf *>(sn + (long)c * m + j), dfc_store(s_));
            // new diagonal c a + s beta
            const dfc hj = dfc_add(dfc_scale(a, c_), dfc_scale(s_, beta));
            *reinterpret_cast<cdf *>(&hcol[j]) = dfc_store(hj);
            float4 *g = gv + (long)c * (m + 1);
            const dfc gj = dfc_load(gld(reinterpret_cast<const cdf *>(g + j)));
            const dfc gj1 = dfc_neg(dfc_mul(dfc_conj(s_), gj));         // g[j+1] = -conj(s) g[j]
            gst(reinterpret_cast<cdf *>(g + j + 1), dfc_store(gj1));
            gst(reinterpret_cast<cdf *>(g + j), dfc_store(dfc_scale(gj, c_)));
            steps[c] = j + 1;
            const bool bd = !(beta.hi > 1e-14f * zn);
            if (bd) bdown[c] = 1;
            const double est = sqrt(df_to_double(dfc_abs2(gj1)));
            const bool done = bd || est <= target[c] || (j + 1) >= mlimit[c];
            if (done) {
                active[c] = 0;
            } else {
                if (inv_beta) inv_beta[c] = 1.0 / df_to_double(beta);
                cont = 1;
            }
        }
    }
    __syncwarp();
    for (int i = lane; i <= j; i += 32) gst(Hc + i + (long)j * (m + 1), hcol[i]);
    return __shfl_sync(0xffffffffu, cont, 0);
}

// ---------------------------------------------------------------------------
// Arnoldi-step kernels.  Partial sums of a column are combined by the last CTA
// of that column to arrive (per-column counter, fixed summation order).
// ---------------------------------------------------------------------------
constexpr int kStepNB = 256;

// Returns true in every thread of the CTA that arrives last on `counter`.
__device__ __forceinline__ bool arrive_last(unsigned *counter, int total) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(counter, 1u);
        s_last = (prev == (unsigned)total - 1);
        if (s_last) *counter = 0u;                 // ready for the next use
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// Gram-Schmidt dots: the grid is sized for step j (static in the captured
// graph): warp t of the launch takes work item t = (basis vector i, chunk of
// kDotNE entries), i = t / nblk_dot, so the warps of a CTA read consecutive
// chunks of one vector; a lane issues all of its loads before it accumulates.
// Every CTA of an active column arrives on the column's counter; the last one
// sums the partials in chunk order: mode 0 sets hco = hacc = h, mode 1 sets
// hco = h and adds h to hacc.
constexpr int kDotNE = 256;
constexpr int kDotIW = 8;
constexpr int kDotVB = 8;        // vector-major reduction: vectors per shared-memory round
constexpr int kDotPL = kDotNE / 32;         // entries per lane

struct StepArgs {
    const float4 *Vb;      // basis [i][c][n]
    float4 *W;             // [c][n]
    long n, bs_i, bs_c;
    int m, k;
    int dot_sub;           // kDotNE-entry pieces per dots chunk (1, more for very long vectors)
    int nblk_dot, ich;     // dots: chunks per vector; CTAs of the launch
    int nblk_vec;          // update / scale grid (kStepNB entries per CTA)
    float4 *part;          // [c][m+1][nblk_dot] (dots), reused as [c][nblk_vec] (norm)
    long pstride;          // (m+1)*max(nblk_dot, nblk_vec) per column
    float4 *hco;           // [c][m+1]
    float4 *hacc;          // [c][m+1]
    unsigned *cnt_a, *cnt_b, *cnt_c, *cnt_d;
    int *active;
    int *d_any_step;
    float4 *H, *gv, *sn;
    float2 *cs;
    double *inv_beta;
    int *steps, *bdown;
    const int *mlimit;
    const double *target;
    int *err;
};

// Pass 0 forms its coefficients in binary32 from the hi parts (the double-float
// second pass projects out whatever they miss, so h = h1 + h2 keeps full
// accuracy); pass 1 is double-float throughout.
__global__ void __launch_bounds__(kDotIW * 32) step_dots_kernel(const StepArgs a, int mode, unsigned *counter,
                                                                 int j) {
    const int c = blockIdx.y;
    pdl_wait();
    if (!a.active[c]) return;
    const int cnt = j + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long t = (long)blockIdx.x * kDotIW + warp;
    const int i = (int)(t / a.nblk_dot), blk = (int)(t - (long)i * a.nblk_dot);
    float4 *part = a.part + (long)c * a.pstride;
    if (i < cnt) {
        float re = 0.f, im = 0.f, re1 = 0.f, im1 = 0.f;                       // mode 0
        dacc re0{0.f, 0.f}, im0{0.f, 0.f}, dre1{0.f, 0.f}, dim1{0.f, 0.f};    // mode 1
        for (int sc = 0; sc < a.dot_sub; ++sc) {
            const long n0 = ((long)blk * a.dot_sub + sc) * kDotNE;
            const int len = (int)max(0L, min((long)kDotNE, a.n - n0));
            const float4 *bv = a.Vb + (long)i * a.bs_i + (long)c * a.bs_c + n0;
            const float4 *xv = a.W + (long)c * a.n + n0;
            float4 v[kDotPL], x[kDotPL];
#pragma unroll
            for (int q = 0; q < kDotPL; ++q) {
                const int e = lane + 32 * q;
                v[q] = e < len ? bv[e] : make_float4(0.f, 0.f, 0.f, 0.f);
                x[q] = e < len ? xv[e] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if (mode == 0) {
#pragma unroll
                for (int q = 0; q < kDotPL; q += 2) {
                    re = fmaf(v[q].x, x[q].x, fmaf(v[q].y, x[q].y, re));
                    im = fmaf(v[q].x, x[q].y, fmaf(-v[q].y, x[q].x, im));
                    re1 = fmaf(v[q + 1].x, x[q + 1].x, fmaf(v[q + 1].y, x[q + 1].y, re1));
                    im1 = fmaf(v[q + 1].x, x[q + 1].y, fmaf(-v[q + 1].y, x[q + 1].x, im1));
                }
            } else {
#pragma unroll
                for (int q = 0; q < kDotPL; q += 2) {
                    dacc_mac(re0, v[q].x, v[q].z, x[q].x, x[q].z);
                    dacc_mac(re0, v[q].y, v[q].w, x[q].y, x[q].w);
                    dacc_mac(im0, v[q].x, v[q].z, x[q].y, x[q].w);
                    dacc_mac(im0, -v[q].y, -v[q].w, x[q].x, x[q].z);
                    dacc_mac(dre1, v[q + 1].x, v[q + 1].z, x[q + 1].x, x[q + 1].z);
                    dacc_mac(dre1, v[q + 1].y, v[q + 1].w, x[q + 1].y, x[q + 1].w);
                    dacc_mac(dim1, v[q + 1].x, v[q + 1].z, x[q + 1].y, x[q + 1].w);
                    dacc_mac(dim1, -v[q + 1].y, -v[q + 1].w, x[q + 1].x, x[q + 1].z);
                }
            }
        }
        if (mode == 0) {
            re += re1;
            im += im1;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                re += __shfl_xor_sync(0xffffffffu, re, off);
                im += __shfl_xor_sync(0xffffffffu, im, off);
            }
            if (lane == 0) gst(part + (long)i * a.nblk_dot + blk, make_float4(re, im, 0.f, 0.f));
        } else {
            dacc_add(re0, dre1);
            dacc_add(im0, dim1);
            warp_reduce_dacc(re0);
            warp_reduce_dacc(im0);
            if (lane == 0) {
                const df r = dacc_result(re0), q = dacc_result(im0);
                gst(part + (long)i * a.nblk_dot + blk, make_float4(r.hi, q.hi, r.lo, q.lo));
            }
        }
    }
    pdl_trigger();
    if (!arrive_last(counter + c, (int)gridDim.x)) return;
    for (int ii = warp; ii < cnt; ii += kDotIW) {
        dacc re, im;
        warp_sum_partials(part + (long)ii * a.nblk_dot, a.nblk_dot, re, im);
        if (lane == 0) {
            const df r = dacc_result(re), q = dacc_result(im);
            const long hidx = (long)c * (a.m + 1) + ii;
            a.hco[hidx] = make_float4(r.hi, q.hi, r.lo, q.lo);
            if (mode == 0) {
                a.hacc[hidx] = make_float4(r.hi, q.hi, r.lo, q.lo);
            } else {
                const float4 o = a.hacc[hidx];
                const df nr = df_add(df{o.x, o.z}, r), ni = df_add(df{o.y, o.w}, q);
                a.hacc[hidx] = make_float4(nr.hi, ni.hi, nr.lo, ni.lo);
            }
        }
    }
}

// w -= sum_{i<cnt} B_i h_i for this thread's entry (compensated), returns the
// new value.  The basis entries are loaded UB at a time, all loads of a batch
// issued before its accumulations: a deep batch when few columns leave the GPU
// short of warps, a shallow one (fewer registers, more warps) otherwise.
// T32: binary32 FMAs (the first CGS pass of a solve with binary32 products; the second pass, compensated
// double-float, removes what it leaves in span(V), as in the delayed-CGS2 update).
template <int UB, bool T32 = false>
__device__ __forceinline__ float4 cta_update_entry(const float4 *basis, long bs_i, long boff, const float4 *hs,
                                                   int cnt, float4 x) {
    dacc re{x.x, x.z}, im{x.y, x.w};
    float fr = __fadd_rn(x.x, x.z), fi = __fadd_rn(x.y, x.w);
    for (int i0 = 0; i0 < cnt; i0 += UB) {
        float4 v[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u)
            if (i0 + u < cnt) v[u] = gld(basis + (long)(i0 + u) * bs_i + boff);
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            if (i0 + u < cnt) {
                const float4 h = hs[i0 + u];              // already negated
                if constexpr (T32) {
                    fr = fmaf(v[u].x, h.x, fr);
                    fr = fmaf(-v[u].y, h.y, fr);
                    fi = fmaf(v[u].x, h.y, fi);
                    fi = fmaf(v[u].y, h.x, fi);
                } else {
                    dacc_mac(re, v[u].x, v[u].z, h.x, h.z);
                    dacc_mac(re, -v[u].y, -v[u].w, h.y, h.w);
                    dacc_mac(im, v[u].x, v[u].z, h.y, h.w);
                    dacc_mac(im, v[u].y, v[u].w, h.x, h.z);
                }
            }
        }
    }
    if constexpr (T32) return make_float4(fr, fi, 0.f, 0.f);
    const df r = dacc_result(re), q = dacc_result(im);
    return make_float4(r.hi, q.hi, r.lo, q.lo);
}

// w -= V h (one entry per thread).  With `last` set (second pass) the kernel
// also forms ||w||^2 and the last CTA of the column runs its Givens step.
template <int UB, bool T32>
__global__ void __launch_bounds__(kStepNB) step_update_kernel(const StepArgs a, int last, int j) {
    extern __shared__ __align__(16) float4 dyn[];          // hs: m+1, then Givens scratch 4m+4
    __shared__ dacc red[kStepNB / 32];
    const int c = blockIdx.y, blk = blockIdx.x;
    pdl_wait();
    if (!a.active[c]) return;
    const int cnt = j + 1;
    float4 *hs = dyn;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const float4 h = a.hco[(long)c * (a.m + 1) + i];
        hs[i] = make_float4(-h.x, -h.y, -h.z, -h.w);
    }
    __syncthreads();
    const long e = (long)blk * kStepNB + threadIdx.x;
    dacc nrm{0.f, 0.f};
    if (e < a.n) {
        float4 &wv = a.W[(long)c * a.n + e];
        const float4 x = cta_update_entry<UB, T32>(a.Vb, a.bs_i, (long)c * a.bs_c + e, hs, cnt, wv);
        wv = x;
        dacc_mac(nrm, x.x, x.z, x.x, x.z);
        dacc_mac(nrm, x.y, x.w, x.y, x.w);
    }
    pdl_trigger();
    if (!last) return;
    warp_reduce_dacc(nrm);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = nrm;
    __syncthreads();
    float4 *part = a.part + (long)c * a.pstride;
    if (threadIdx.x == 0) {
        dacc t = red[0];
        for (int w = 1; w < kStepNB / 32; ++w) dacc_add(t, red[w]);
        const df r = dacc_result(t);
        gst(part + blk, make_float4(r.hi, 0.f, r.lo, 0.f));
    }
    if (!arrive_last(a.cnt_c + c, a.nblk_vec)) return;
    if (warp == 0) {
        dacc t, unused;
        warp_sum_partials(part, a.nblk_vec, t, unused);
        const double beta2 = df_to_double(dacc_result(t));
        const int cont = givens_column(c, j, a.m, dyn + (a.m + 1), a.H, a.hacc + (long)c * (a.m + 1), beta2, a.cs,
                                       a.sn, a.gv, a.active,
                                       a.steps, a.bdown, a.mlimit, a.target, a.inv_beta, a.err);
        if (lane == 0 && cont) atomicMax(a.d_any_step, j + 1);
    }
}

// v_{j+1} = w / beta for continuing columns.
__global__ void __launch_bounds__(kStepNB) step_scale_kernel(const StepArgs a, int j) {
    const int c = blockIdx.y, blk = blockIdx.x;
    pdl_wait();
    if (a.active[c]) {
        const df s = df_from_double(a.inv_beta[c]);
        const long e = (long)blk * kStepNB + threadIdx.x;
        if (e < a.n) {
            const float4 x = gld(a.W + (long)c * a.n + e);
            const df r = df_mul(df{x.x, x.z}, s), q = df_mul(df{x.y, x.w}, s);
            gst(const_cast<float4 *>(a.Vb) + (long)(j + 1) * a.bs_i + (long)c * a.bs_c + e,
                make_float4(r.hi, q.hi, r.lo, q.lo));
        }
    }
    pdl_trigger();
}


// ---------------------------------------------------------------------------
// Delayed CGS2 for unpreconditioned cycles: one reduction and one update per
// step instead of two of each.  The step applies the operator to u_j, the
// previous step's vector after one Gram-Schmidt pass (not yet reorthogonalised
// or normalised), x = A u_j, and in one reduction forms
//   s = Q_{j-1}^H u_j,  t = Q_{j-1}^H x,  alpha = u_j^H u_j,  tau = u_j^H x.
// The reorthogonalised q_j = (u_j - Q s)/nu, nu^2 = alpha - |s|^2, closes
// Hessenberg column j-1 (its entries gain s, its subdiagonal is nu), and since
// A Q_{j-1} = Q_j H, A q_j = (x - Q_j H s)/nu: the coefficients of A q_j on Q_j
// are c = [t; (tau - s^H t)/nu], the preliminary column j is (c - H s)/nu, and
//   u_{j+1} = (x - Q_{j-1} t - q_j c_j)/nu.
// The update writes q_j and u_{j+1} in one pass over the basis.  A closing
// reduction without x finalises the last column of the cycle.  t (and tau) are
// first-pass Gram-Schmidt coefficients: the reduction forms them in binary32,
// and the next step's reorthogonalisation s, formed in double-float like alpha
// and like the update itself, measures and removes what they miss (the closed
// Hessenberg column is the coefficients used plus that correction), so the
// Arnoldi relation holds to double-float accuracy.
// ---------------------------------------------------------------------------
__device__ __forceinline__ df warp_sum_df(df v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        v = df_add(v, df{__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off)});
    return v;
}
__device__ __forceinline__ dfc warp_sum_dfc(dfc v) { return dfc{warp_sum_df(v.re), warp_sum_df(v.im)}; }

struct DcgsArgs {
    const float4 *Vb;     // basis q_0 .. q_{j-1}, [i][c][n]
    float4 *U;            // u_j on entry to the update, u_{j+1} on exit, [c][n]
    const float4 *X;      // x = A u_j, [c][n]
    long n, bs_i, bs_c;
    int m, k;
    int dot_sub, nblk_dot, ich, nblk_vec;
    int cmajor;           // 1: a CTA covers its chunks for every vector (u, x read once; many columns)
    int vgrp;             // vector-major: basis vectors per CTA
    int fused;            // vector-major: the update kernel's CTAs sum the partials and close the column
    int dsm_last;         // float4 slots of dynamic shared memory used by the last CTA (stages follow)
    float4 *part;
    long pstride;
    float4 *sco, *cco, *hpre, *Horig, *hcol;   // [c][m+1] x 4, Horig [c][(m+1)*m]
    double *nu2;          // [c]: subdiagonal^2 of the column the update kernel's Givens CTA closes
    unsigned *cnt;
    int *active, *d_any_step;
    float4 *H, *gv, *sn;
    float2 *cs;
    double *inv_beta;
    int *steps, *bdown;
    const int *mlimit;
    const double *target;
    int *err;
    unsigned long long wait_ns;   // bound of every pipeline wait
};

// Sums four per-lane accumulators over the warp by a reduce-scatter butterfly: at offset 16 each half keeps
// two of them, at offset 8 each quarter keeps one, offsets 4, 2, 1 finish it.  Lanes 0-7 return the sum of
// a, 8-15 of b, 16-23 of c, 24-31 of d (12 shuffles of pairs and 6 merges instead of 40 and 20).
__device__ __forceinline__ dacc warp_reduce_scatter4(dacc a, dacc b, dacc c, dacc d, int lane) {
    const bool hi16 = lane & 16;
    dacc k0 = hi16 ? c : a, k1 = hi16 ? d : b;
    const dacc s0 = hi16 ? a : c, s1 = hi16 ? b : d;
    dacc_add(k0, dacc{__shfl_xor_sync(0xffffffffu, s0.S, 16), __shfl_xor_sync(0xffffffffu, s0.s, 16)});
    dacc_add(k1, dacc{__shfl_xor_sync(0xffffffffu, s1.S, 16), __shfl_xor_sync(0xffffffffu, s1.s, 16)});
    const bool hi8 = lane & 8;
    dacc k = hi8 ? k1 : k0;
    const dacc sd = hi8 ? k0 : k1;
    dacc_add(k, dacc{__shfl_xor_sync(0xffffffffu, sd.S, 8), __shfl_xor_sync(0xffffffffu, sd.s, 8)});
#pragma unroll
    for (int off = 4; off > 0; off >>= 1)
        dacc_add(k, dacc{__shfl_xor_sync(0xffffffffu, k.S, off), __shfl_xor_sync(0xffffffffu, k.s, off)});
    return k;
}

// Roles of the closing work of a delayed-CGS2 step (dcgs_tail).
enum TailRole : int {
    TAIL_LAST = 0,     // the reduction's last CTA: all of it (the update kernel then reads the coefficients)
    TAIL_COEF = 1,     // an update CTA of the few-column layout: the coefficients s, t, c_j and 1/nu only
    TAIL_HESS = 2,     // that layout's first extra update CTA: close column j-1, H s, the preliminary column j
    TAIL_GIVENS = 3,   // its second extra update CTA: close column j-1 in shared memory, its Givens step
};

// The closing work of step j of column c once every partial sum is in `part` (npart per quantity; slot q
// holds s_q for q <= j, slot m+1+q holds t_q): the sums, nu and s^H t, then per role c_j = (tau - s^H t)/nu,
// the close of Hessenberg column j-1 (preliminary entries + s, subdiagonal nu), H s and the preliminary
// column j, and the Givens step of column j-1.  Every role sums in the same order, so every CTA gets the
// same bits.  The preliminary column is double-buffered by step parity (step j reads buffer (j-1) mod 2 and
// writes buffer j mod 2), so the two extra CTAs of the few-column layout need no ordering between them.
// Shared memory `dsm`: DcgsArgs::dsm_last float4 slots; on return s is at dsm[0..j-1] and t at
// dsm[m+1..m+1+j] with t_j replaced by c_j.
__device__ void dcgs_tail(const DcgsArgs &a, int c, int j, int has_x, int npart, const float4 *part, float4 *dsm,
                          int role, df *nu_out, df *inu_out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = a.m;
    float4 *ssm = dsm, *tsm = dsm + (m + 1);
    float4 *gscr = dsm + 2 * (m + 1);
    float4 *hs = gscr + (4 * m + 4);
    // the 2(j+1) sums (s_q for q <= j, then t): T consecutive lanes per sum (a power of two up to 32, as
    // many as the block's threads allow), lane t adding the partials t, t+T, ... in order (eight loads in
    // flight; a partial past the end adds an exact zero), then a fixed xor tree over the T lanes
    {
        const int nsum = 2 * (j + 1);
        int T = 1;
        while (T < 32 && 2 * T * nsum <= (int)blockDim.x) T <<= 1;
        const int spp = (int)blockDim.x / T, t = lane & (T - 1);
        for (int q0 = 0; q0 < nsum; q0 += spp) {
            const int q = q0 + (int)threadIdx.x / T;
            dacc re{0.f, 0.f}, im{0.f, 0.f};
            if (q < nsum) {
                const float4 *pp = part + (long)(q <= j ? q : (m + 1) + (q - j - 1)) * npart;
                for (int e = t; e < npart; e += 8 * T) {
                    float4 v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        v[u] = e + u * T < npart ? gldcg(pp + e + u * T) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        dacc_add(re, dacc{v[u].x, v[u].z});
                        dacc_add(im, dacc{v[u].y, v[u].w});
                    }
                }
            }
            for (int off = T >> 1; off > 0; off >>= 1) {
                const dacc ro{__shfl_xor_sync(0xffffffffu, re.S, off), __shfl_xor_sync(0xffffffffu, re.s, off)};
                const dacc io{__shfl_xor_sync(0xffffffffu, im.S, off), __shfl_xor_sync(0xffffffffu, im.s, off)};
                dacc_add(re, ro);
                dacc_add(im, io);
            }
            if (t == 0 && q < nsum) {
                const df r = dacc_result(re), z = dacc_result(im);
                (q <= j ? ssm[q] : tsm[q - j - 1]) = make_float4(r.hi, z.hi, r.lo, z.lo);
            }
        }
    }
    __syncthreads();
    // nu^2 = alpha - |s|^2 (alpha = u^H u is the real part of slot j) by warp 0, and
    // s^H t for c_j by warp 1, each a strided sum and a fixed-order warp reduction
    __shared__ float4 s_nu;                               // {nu.hi, 1/nu.hi, nu.lo, 1/nu.lo}
    __shared__ float4 s_sht;                              // s^H t
    if (warp == 0) {
        df acc{0.f, 0.f};
        for (int q = lane; q < j; q += 32) acc = df_add(acc, dfc_abs2(dfc_load(*reinterpret_cast<const cdf *>(&ssm[q]))));
        acc = warp_sum_df(acc);
        if (lane == 0) {
            df nu2 = df_sub(df{ssm[j].x, ssm[j].z}, acc);
            if (!(nu2.hi > 0.f)) nu2 = df{0.f, 0.f};
            const df nu = df_sqrt(nu2);
            const df inu = nu.hi > 0.f ? df_recip(nu) : df{0.f, 0.f};
            s_nu = make_float4(nu.hi, inu.hi, nu.lo, inu.lo);
        }
    } else if (warp == 1 && has_x && role != TAIL_GIVENS) {
        dfc acc{df{0.f, 0.f}, df{0.f, 0.f}};
        for (int q = lane; q < j; q += 32)
            acc = dfc_add(acc, dfc_mul(dfc_conj(dfc_load(*reinterpret_cast<const cdf *>(&ssm[q]))),
                                       dfc_load(*reinterpret_cast<const cdf *>(&tsm[q]))));
        acc = warp_sum_dfc(acc);
        if (lane == 0) {
            const cdf st = dfc_store(acc);
            s_sht = make_float4(st.rh, st.ih, st.rl, st.il);
        }
    }
    __syncthreads();
    const df nu{s_nu.x, s_nu.z}, inu{s_nu.y, s_nu.w};
    *nu_out = nu;
    *inu_out = inu;
    // c_j = (tau - s^H t)/nu in place of t_j
    auto put_cj = [&]() {
        const dfc cj = dfc_sub(dfc_load(*reinterpret_cast<const cdf *>(&tsm[j])),
                               dfc_load(*reinterpret_cast<const cdf *>(&s_sht)));
        const cdf st = dfc_store(dfc_scale(cj, inu));
        tsm[j] = make_float4(st.rh, st.ih, st.rl, st.il);
    };
    if (role == TAIL_COEF) {
        if (threadIdx.x == 0 && has_x) put_cj();
        __syncthreads();
        return;
    }
    const float4 *hp = a.hpre + ((long)((j + 1) & 1) * a.k + c) * (m + 1);   // step j-1's preliminary column
    float4 *hw = a.hpre + ((long)(j & 1) * a.k + c) * (m + 1);               // this step's
    float4 *Hoc = a.Horig + (long)c * (m + 1) * m;
    if (role == TAIL_GIVENS) {
        // the closed column j-1 in shared memory only, then its Givens step by warp 0
        if (j >= 1) {
            float4 *fc = hs;
            for (int q = threadIdx.x; q < j; q += blockDim.x) {
                const cdf st = dfc_store(dfc_add(dfc_load(gld(reinterpret_cast<const cdf *>(hp + q))),
                                                 dfc_load(*reinterpret_cast<const cdf *>(&ssm[q]))));
                fc[q] = make_float4(st.rh, st.ih, st.rl, st.il);
            }
            __syncthreads();
            if (warp == 0) {
                const int cont = givens_column(c, j - 1, m, gscr, a.H, fc, df_to_double(df_mul(nu, nu)), a.cs, a.sn,
                                               a.gv, a.active, a.steps, a.bdown, a.mlimit, a.target, nullptr, a.err);
                if (lane == 0 && cont) atomicMax(a.d_any_step, j + 1);
            }
        } else if (threadIdx.x == 0) {
            atomicMax(a.d_any_step, 1);
        }
        return;
    }
    // H s (rows 0..j) from the unrotated columns 0..j-1 (column q has rows 0..q+1): thread (row r, group g)
    // sums the columns q = g, g+G, ... of row r; the G partial sums of a row are added in group order after
    const int R = j + 1;
    const int G = max(1, min(j, (int)blockDim.x / R));   // no more groups than columns
    float4 *hpart = hs + (m + 1);                         // R*G partial sums (hs itself holds column j-1 first)
    auto hs_partials = [&]() {
        const int tt = (int)threadIdx.x;
        if (tt < R * G) {
            const int r = tt % R, gq = tt / R;
            dfc acc{df{0.f, 0.f}, df{0.f, 0.f}};
#pragma unroll 4
            for (int q = max(r - 1, 0) + ((gq - max(r - 1, 0) % G) % G + G) % G; q < j; q += G)
                acc = dfc_add(acc, dfc_mul(dfc_load(gld(reinterpret_cast<const cdf *>(Hoc + (long)q * (m + 1) + r))),
                                           dfc_load(*reinterpret_cast<const cdf *>(&ssm[q]))));
            const cdf st = dfc_store(acc);
            sst(hpart + gq * R + r, make_float4(st.rh, st.ih, st.rl, st.il));
        }
        if (threadIdx.x == 0) put_cj();
    };
    if (j >= 1) {
        // close column j-1: entries hpre + s (rows 0..j-1), subdiagonal nu
        float4 *fc = hs;                                  // the closed column, rows 0..j-1
        for (int q = threadIdx.x; q < j; q += blockDim.x) {
            const cdf st = dfc_store(dfc_add(dfc_load(gld(reinterpret_cast<const cdf *>(hp + q))),
                                             dfc_load(*reinterpret_cast<const cdf *>(&ssm[q]))));
            fc[q] = make_float4(st.rh, st.ih, st.rl, st.il);
            gst(Hoc + (long)(j - 1) * (m + 1) + q, fc[q]);
        }
        if (threadIdx.x == 0) gst(Hoc + (long)(j - 1) * (m + 1) + j, make_float4(nu.hi, 0.f, nu.lo, 0.f));
        if (!has_x) {
            // the cycle's last close (role TAIL_LAST): its Givens step here
            __syncthreads();
            if (warp == 0) {
                const double nu2d = df_to_double(df_mul(nu, nu));
                givens_column(c, j - 1, m, gscr, a.H, fc, nu2d, a.cs, a.sn, a.gv, a.active, a.steps, a.bdown,
                              a.mlimit, a.target, a.inv_beta, a.err);
            }
            return;
        }
        if (role == TAIL_LAST) {
            // the Givens step of column j-1 runs in the update kernel's extra CTA, beside the update
            float4 *hc = a.hcol + (long)c * (m + 1);
            for (int q = threadIdx.x; q < j; q += blockDim.x) gst(hc + q, fc[q]);
            if (threadIdx.x == 0) {
                a.nu2[c] = df_to_double(df_mul(nu, nu));
                a.inv_beta[c] = df_to_double(inu);
            }
        }
        __syncthreads();
        hs_partials();
        __syncthreads();
    } else {
        if (threadIdx.x == 0) a.inv_beta[c] = df_to_double(inu);
        if (!has_x) return;
        hs_partials();
        __syncthreads();
    }
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        dfc acc = dfc_load(*reinterpret_cast<const cdf *>(&hpart[r]));
        for (int gq = 1; gq < G; ++gq) acc = dfc_add(acc, dfc_load(*reinterpret_cast<const cdf *>(&hpart[gq * R + r])));
        const cdf st = dfc_store(acc);
        hs[r] = make_float4(st.rh, st.ih, st.rl, st.il);
    }
    __syncthreads();
    for (int r = threadIdx.x; r <= j; r += blockDim.x) {
        const long o = (long)c * (m + 1) + r;
        if (role == TAIL_LAST) {
            if (r < j) gst(a.sco + o, ssm[r]);
            gst(a.cco + o, tsm[r]);
        }
        const dfc hpj = dfc_scale(dfc_sub(dfc_load(*reinterpret_cast<const cdf *>(&tsm[r])),
                                          dfc_load(*reinterpret_cast<const cdf *>(&hs[r]))), inu);
        const cdf st = dfc_store(hpj);
        gst(hw + r, make_float4(st.rh, st.ih, st.rl, st.il));
    }
}

// CM: the chunk-major layout (a.cmajor), a separate instance (the chunk-major one holds u and x in
// registers).  Both are sized for two CTAs per SM, the vector-major grid's target.
template <bool CM>
__global__ void __launch_bounds__(kDotIW * 32, 2) dcgs_dots_kernel(const DcgsArgs a, int j, int has_x) {
    extern __shared__ __align__(16) float4 dsm[];      // s, t: 2(m+1); Givens scratch 4m+4; Hs: m+1; partials
    const int c = blockIdx.y;
    pdl_wait();
    if (!a.active[c]) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cpv = (a.nblk_dot + kDotIW - 1) / kDotIW;
    float4 *part = a.part + (long)c * a.pstride;
    const int npart = CM ? a.nblk_dot : cpv;               // partials per quantity for the last CTA
    if constexpr (CM) {
        // chunk-major: CTA = chunk group blockIdx.x, warp w takes chunk blockIdx.x*kDotIW + w for every
        // vector i <= j.  The warp keeps its entries of u and x in registers and streams the basis chunks
        // through two shared-memory stages (bulk copies on an mbarrier each): q_{i+1} lands while q_i is
        // used.  One partial per warp and quantity.
        float4 *stg = dsm + a.dsm_last + (long)warp * 2 * kDotNE;
        uint64_t *bar = reinterpret_cast<uint64_t *>(dsm + a.dsm_last + kDotIW * 2 * kDotNE) + 2 * warp;
        __shared__ int s_abort;
        if (threadIdx.x == 0) s_abort = 0;
        if (lane == 0) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            fence_mbar_init();
        }
        __syncthreads();
        const int blk = blockIdx.x * kDotIW + warp;
        if (blk < a.nblk_dot) {
            const long n0 = (long)blk * kDotNE;
            const int len = (int)min((long)kDotNE, a.n - n0);
            const float4 *uv = a.U + (long)c * a.n + n0;
            const float4 *xv = a.X + (long)c * a.n + n0;
            const float4 *qb = a.Vb + (long)c * a.bs_c + n0;
            const uint64_t pol = l2_policy_evict_first();
            auto issue = [&](int i) {
                mbar_arrive_expect_tx(&bar[i & 1], (uint32_t)len * 16u);
                bulk_g2s(stg + (i & 1) * kDotNE, qb + (long)i * a.bs_i, (uint32_t)len * 16u, &bar[i & 1], pol);
            };
            if (lane == 0 && j > 0) issue(0);
            float4 u[kDotPL], x[kDotPL];
#pragma unroll
            for (int r = 0; r < kDotPL; ++r) {
                const int e = lane + 32 * r;
                const bool in = e < len;
                u[r] = in ? gld(uv + e) : make_float4(0.f, 0.f, 0.f, 0.f);
                x[r] = in && has_x ? gld(xv + e) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            bool failed = false;
            int issued = j > 0 ? 0 : -1, waited = -1;     // lane 0's view of the copies
            for (int i = 0; i <= j; ++i) {
                float4 q[kDotPL];
                if (i < j) {
                    if (lane == 0 && !failed && i + 1 < j) {
                        issue(i + 1);                     // its stage was released at the end of step i-1
                        issued = i + 1;
                    }
                    if (!failed) {
                        if (mbar_wait_bounded(&bar[i & 1], (uint32_t)(i >> 1) & 1u, &s_abort, a.wait_ns)) {
                            waited = i;
                        } else {
                            failed = true;
                            if (lane == 0) atomicOr(a.err, DEVERR_TIMEOUT);
                        }
                    }
                    const float4 *sq = stg + (i & 1) * kDotNE;
#pragma unroll
                    for (int r = 0; r < kDotPL; ++r) {
                        const int e = lane + 32 * r;
                        q[r] = !failed && e < len ? sq[e] : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < kDotPL; ++r) q[r] = u[r];
                }
                dacc sr{0.f, 0.f}, si{0.f, 0.f};
                float ftr = 0.f, fti = 0.f;
#pragma unroll
                for (int r = 0; r < kDotPL; ++r) {
                    dacc_mac(sr, q[r].x, q[r].z, u[r].x, u[r].z);
                    dacc_mac(sr, q[r].y, q[r].w, u[r].y, u[r].w);
                    dacc_mac(si, q[r].x, q[r].z, u[r].y, u[r].w);
                    dacc_mac(si, -q[r].y, -q[r].w, u[r].x, u[r].z);
                    ftr = fmaf(q[r].x, x[r].x, ftr);             // t: first-pass coefficients, binary32
                    ftr = fmaf(q[r].y, x[r].y, ftr);
                    fti = fmaf(q[r].x, x[r].y, fti);
                    fti = fmaf(-q[r].y, x[r].x, fti);
                }
                dacc tr{ftr, 0.f}, ti{fti, 0.f};
                // every lane has read stage i&1 before lane 0 refills it (next step)
                __syncwarp();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                // reduce-scatter of the four sums: lanes 0-7 end with Re s, 8-15 Im s, 16-23 Re t, 24-31 Im t
                const dacc tot = warp_reduce_scatter4(sr, si, tr, ti, lane);
                const dacc oth{__shfl_down_sync(0xffffffffu, tot.S, 8), __shfl_down_sync(0xffffffffu, tot.s, 8)};
                if ((lane & 15) == 0) {
                    const df re = dacc_result(tot), im = dacc_result(oth);
                    gst(part + (long)(lane == 0 ? i : a.m + 1 + i) * npart + blk, make_float4(re.hi, im.hi, re.lo, im.lo));
                }
            }
            if (lane == 0)                                 // copies still in flight after a failed wait
                for (int d = waited + 1; d <= issued; ++d) mbar_wait_drain(&bar[d & 1], (uint32_t)(d >> 1) & 1u);
        }
    } else {
        // vector-major: CTA (group vg of a.vgrp vectors, group cb of kDotIW chunks); warp w takes chunk
        // cb*kDotIW + w of each vector of its group in turn, so u and x come from L1 after the first one and
        // the grid stays within about one wave.  The CTAs of one chunk group are adjacent (vg fastest).  The
        // warps' sums of up to kDotVB vectors wait in shared memory for one barrier, after which the CTA's
        // partials of those vectors are formed (warp order) together.
        const int ngrp = (j + 1 + a.vgrp - 1) / a.vgrp;
        const int cb = blockIdx.x / ngrp, vg = blockIdx.x - cb * ngrp;
        const int blk = cb * kDotIW + warp;
        const int ilo = vg * a.vgrp, ihi = min(j + 1, (vg + 1) * a.vgrp);
        __shared__ dacc cred[kDotVB][4][kDotIW];
        for (int i0 = ilo; i0 < ihi; i0 += kDotVB) {
            const int nb = min(kDotVB, ihi - i0);
            for (int i = i0; i < i0 + nb; ++i) {
                dacc sr{0.f, 0.f}, si{0.f, 0.f}, tr{0.f, 0.f}, ti{0.f, 0.f};
                if (blk < a.nblk_dot) {
                    // i < j: (q_i, u) and (q_i, x); i == j: (u, u) and (u, x)
                    const float4 *uv = a.U + (long)c * a.n;
                    const float4 *xv = a.X + (long)c * a.n;
                    const float4 *qv = i < j ? a.Vb + (long)i * a.bs_i + (long)c * a.bs_c : uv;
                    for (int sc = 0; sc < a.dot_sub; ++sc) {
                        const long n0 = ((long)blk * a.dot_sub + sc) * kDotNE;
                        const int len = (int)max(0L, min((long)kDotNE, a.n - n0));
                        float4 q[kDotPL], u[kDotPL], x[kDotPL];
#pragma unroll
                        for (int r = 0; r < kDotPL; ++r) {
                            const int e = lane + 32 * r;
                            const bool in = e < len;
                            q[r] = in ? gld(qv + n0 + e) : make_float4(0.f, 0.f, 0.f, 0.f);
                            u[r] = in ? gld(uv + n0 + e) : make_float4(0.f, 0.f, 0.f, 0.f);
                            x[r] = in && has_x ? gld(xv + n0 + e) : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                        float ftr = 0.f, fti = 0.f;
#pragma unroll
                        for (int r = 0; r < kDotPL; ++r) {
                            // conj(q) u compensated; conj(q) x (first-pass coefficients t) in binary32
                            dacc_mac(sr, q[r].x, q[r].z, u[r].x, u[r].z);
                            dacc_mac(sr, q[r].y, q[r].w, u[r].y, u[r].w);
                            dacc_mac(si, q[r].x, q[r].z, u[r].y, u[r].w);
                            dacc_mac(si, -q[r].y, -q[r].w, u[r].x, u[r].z);
                            ftr = fmaf(q[r].x, x[r].x, ftr);
                            ftr = fmaf(q[r].y, x[r].y, ftr);
                            fti = fmaf(q[r].x, x[r].y, fti);
                            fti = fmaf(-q[r].y, x[r].x, fti);
                        }
                        dacc_add(tr, dacc{ftr, 0.f});
                        dacc_add(ti, dacc{fti, 0.f});
                    }
                    warp_reduce_dacc(sr);
                    warp_reduce_dacc(si);
                    warp_reduce_dacc(tr);
                    warp_reduce_dacc(ti);
                }
                if (lane == 0) {
                    cred[i - i0][0][warp] = sr;
                    cred[i - i0][1][warp] = si;
                    cred[i - i0][2][warp] = tr;
                    cred[i - i0][3][warp] = ti;
                }
            }
            __syncthreads();
            // lane (vector v, quantity qn) of warp 0 sums the warps in warp order; the lanes of Re s and Re t
            // write the partials with their neighbours' Im s and Im t
            static_assert(4 * kDotVB == 32, "one warp forms the partials of a round");
            if (warp == 0) {
                const int v = lane >> 2, qn = lane & 3;
                dacc acc = cred[v][qn][0];                // rows v >= nb hold stale sums, never stored
                for (int w = 1; w < kDotIW; ++w) dacc_add(acc, cred[v][qn][w]);
                const df r = dacc_result(acc);
                const float rh = __shfl_sync(0xffffffffu, r.hi, lane ^ 1);
                const float rl = __shfl_sync(0xffffffffu, r.lo, lane ^ 1);
                if (v < nb && (qn == 0 || qn == 2)) {
                    const int i = i0 + v;
                    gst(part + (long)(qn == 0 ? i : a.m + 1 + i) * cpv + cb, make_float4(r.hi, rh, r.lo, rl));
                }
            }
            __syncthreads();                              // cred is reused by the group's next vectors
        }
    }
    pdl_trigger();
    // few-column layout: the update kernel closes the column (its CTAs sum the partials themselves)
    if (a.fused && has_x) return;
    if (!arrive_last(a.cnt + c, (int)gridDim.x)) return;
    df nu_, inu_;
    dcgs_tail(a, c, j, has_x, npart, part, dsm, TAIL_LAST, &nu_, &inu_);
}

// q_j = (u_j - Q s)/nu and u_{j+1} = (x - Q t - q_j c_j)/nu, one entry per thread, the basis
// entries loaded UB at a time and shared by both sums.
static_assert(kStepNB == kDotIW * 32, "the update kernel's CTAs run the reduction tail with its warp count");
// T32: the products of this solve are binary32 (the inner solve of GMRES-IR), so the first-pass part
// u_{j+1} = (x - Q t - q_j c_j)/nu is formed in binary32 FMAs: x itself carries binary32 errors, t is a
// binary32 first-pass coefficient, and the next step's reorthogonalisation (s = Q^H u_{j+1}, compensated
// double-float) removes what this pass leaves in span(Q).  q_j stays double-float.
template <int UB, bool T32>
__global__ void __launch_bounds__(kStepNB, 2) dcgs_update_kernel(const DcgsArgs a, int j) {
    extern __shared__ __align__(16) float4 csm[];        // -s: j entries, -c: j+1 entries; Givens scratch
    const int c = blockIdx.y, blk = blockIdx.x;
    pdl_wait();
    if (!a.active[c]) return;
    df inu_f{0.f, 0.f};
    if (a.fused) {
        // few-column layout: every CTA sums the column's partials itself (the same order everywhere, so
        // every CTA gets the same coefficients); the two extra CTAs close column j-1 and write the
        // preliminary column j, and run the Givens step of column j-1 -- both off the update's path
        const int cpv = (a.nblk_dot + kDotIW - 1) / kDotIW;
        const int role = blk < a.nblk_vec ? TAIL_COEF : blk == a.nblk_vec ? TAIL_HESS : TAIL_GIVENS;
        df nu_;
        dcgs_tail(a, c, j, 1, cpv, a.part + (long)c * a.pstride, csm, role, &nu_, &inu_f);
        if (role != TAIL_COEF) return;
        // -s and -c in place of s and t
        for (int q = threadIdx.x; q <= j; q += blockDim.x) {
            if (q < j) {
                const float4 v = csm[q];
                csm[q] = make_float4(-v.x, -v.y, -v.z, -v.w);
            }
            const float4 w = csm[a.m + 1 + q];
            csm[a.m + 1 + q] = make_float4(-w.x, -w.y, -w.z, -w.w);
        }
        __syncthreads();
    } else if (blk == a.nblk_vec) {
        // the extra CTA: Givens step of column j-1 (closed by the reduction), off the update's path
        if (j >= 1 && threadIdx.x < 32) {
            const int cont = givens_column(c, j - 1, a.m, csm, a.H, a.hcol + (long)c * (a.m + 1), a.nu2[c], a.cs,
                                           a.sn, a.gv, a.active, a.steps, a.bdown, a.mlimit, a.target, nullptr,
                                           a.err);
            if (threadIdx.x == 0 && cont) atomicMax(a.d_any_step, j + 1);
        } else if (j == 0 && threadIdx.x == 0) {
            atomicMax(a.d_any_step, 1);
        }
        return;
    }
    float4 *sn_ = csm, *cn_ = csm + (a.m + 1);
    if (!a.fused) {
        for (int q = threadIdx.x; q <= j; q += blockDim.x) {
            const long o = (long)c * (a.m + 1) + q;
            if (q < j) {
                const float4 v = gld(a.sco + o);
                sn_[q] = make_float4(-v.x, -v.y, -v.z, -v.w);
            }
            const float4 w = gld(a.cco + o);
            cn_[q] = make_float4(-w.x, -w.y, -w.z, -w.w);
        }
        __syncthreads();
    }
    const long e = (long)blk * kStepNB + threadIdx.x;
    if (e < a.n) {
        const float4 u = gld(a.U + (long)c * a.n + e), x = gld(a.X + (long)c * a.n + e);
        dacc qr{u.x, u.z}, qi{u.y, u.w}, xr{x.x, x.z}, xi{x.y, x.w};
        float fr = __fadd_rn(x.x, x.z), fi = __fadd_rn(x.y, x.w);       // T32: x in binary32
        const float4 *basis = a.Vb + (long)c * a.bs_c + e;
        for (int i0 = 0; i0 < j; i0 += UB) {
            float4 v[UB];
#pragma unroll
            for (int r = 0; r < UB; ++r)
                if (i0 + r < j) v[r] = gld(basis + (long)(i0 + r) * a.bs_i);
#pragma unroll
            for (int r = 0; r < UB; ++r) {
                if (i0 + r < j) {
                    const float4 h = sn_[i0 + r], g = cn_[i0 + r];
                    dacc_mac(qr, v[r].x, v[r].z, h.x, h.z);
                    dacc_mac(qr, -v[r].y, -v[r].w, h.y, h.w);
                    dacc_mac(qi, v[r].x, v[r].z, h.y, h.w);
                    dacc_mac(qi, v[r].y, v[r].w, h.x, h.z);
                    if constexpr (T32) {
                        fr = fmaf(v[r].x, g.x, fr);
                        fr = fmaf(-v[r].y, g.y, fr);
                        fi = fmaf(v[r].x, g.y, fi);
                        fi = fmaf(v[r].y, g.x, fi);
                    } else {
                        dacc_mac(xr, v[r].x, v[r].z, g.x, g.z);
                        dacc_mac(xr, -v[r].y, -v[r].w, g.y, g.w);
                        dacc_mac(xi, v[r].x, v[r].z, g.y, g.w);
                        dacc_mac(xi, v[r].y, v[r].w, g.x, g.z);
                    }
                }
            }
        }
        const df inu = a.fused ? inu_f : df_from_double(a.inv_beta[c]);
        const df q0 = df_mul(dacc_result(qr), inu), q1 = df_mul(dacc_result(qi), inu);
        const float4 g = cn_[j];
        float4 un;
        if constexpr (T32) {
            fr = fmaf(q0.hi, g.x, fr);
            fr = fmaf(-q1.hi, g.y, fr);
            fi = fmaf(q0.hi, g.y, fi);
            fi = fmaf(q1.hi, g.x, fi);
            un = make_float4(__fmul_rn(fr, inu.hi), __fmul_rn(fi, inu.hi), 0.f, 0.f);
        } else {
            dacc_mac(xr, q0.hi, q0.lo, g.x, g.z);
            dacc_mac(xr, -q1.hi, -q1.lo, g.y, g.w);
            dacc_mac(xi, q0.hi, q0.lo, g.y, g.w);
            dacc_mac(xi, q1.hi, q1.lo, g.x, g.z);
            const df x0 = df_mul(dacc_result(xr), inu), x1 = df_mul(dacc_result(xi), inu);
            un = make_float4(x0.hi, x1.hi, x0.lo, x1.lo);
        }
        gst(const_cast<float4 *>(a.Vb) + (long)j * a.bs_i + (long)c * a.bs_c + e, make_float4(q0.hi, q1.hi, q0.lo, q1.lo));
        gst(a.U + (long)c * a.n + e, un);
    }
    pdl_trigger();
}

// y = H^{-1} g (upper triangular, steps[c] x steps[c]) for column c = blockIdx.x,
// in double-float.  Column-oriented back substitution: one diagonal division
// per step, the remaining right-hand side updated in parallel.
constexpr int kFinishThreads = 128;

__global__ void __launch_bounds__(kFinishThreads) finish_kernel(const float4 *H, const float4 *gv,
                                                                const int *steps, float4 *ycoef, int m,
                                                                const int *was_active) {
    extern __shared__ __align__(16) float4 rhs[];              // m+1
    __shared__ float4 ysh;
    const int c = blockIdx.x;
    if (!was_active[c]) return;
    const int kk = steps[c];
    const float4 *Hc = H + (long)c * (m + 1) * m;
    const float4 *g = gv + (long)c * (m + 1);
    for (int i = threadIdx.x; i < kk; i += blockDim.x) rhs[i] = g[i];
    __syncthreads();
    for (int i = kk - 1; i >= 0; --i) {
        if (threadIdx.x == 0) {
            const dfc d = dfc_load(gld(reinterpret_cast<const cdf *>(Hc + i + (long)i * (m + 1))));
            const dfc sv = dfc_load(*reinterpret_cast<const cdf *>(&rhs[i]));
            const df dd = dfc_abs2(d);
            dfc yi{df{0.f, 0.f}, df{0.f, 0.f}};
            if (dd.hi > 0.f) yi = dfc_scale(dfc_mul(sv, dfc_conj(d)), df_recip(dd));
            const cdf yc = dfc_store(yi);
            ysh = make_float4(yc.rh, yc.ih, yc.rl, yc.il);
            gst(ycoef + (long)c * (m + 1) + i, ysh);
        }
        __syncthreads();
        const dfc yi = dfc_load(*reinterpret_cast<const cdf *>(&ysh));
        for (int l = threadIdx.x; l < i; l += blockDim.x) {
            const dfc t = dfc_mul(dfc_load(gld(reinterpret_cast<const cdf *>(Hc + l + (long)i * (m + 1)))), yi);
            const dfc r = dfc_sub(dfc_load(*reinterpret_cast<const cdf *>(&rhs[l])), t);
            *reinterpret_cast<cdf *>(&rhs[l]) = dfc_store(r);
        }
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
    cudaFree(g->counters); cudaFree(g->d_any_step); cudaFree(g->act_prod);
    cudaFree(g->U); cudaFree(g->cco); cudaFree(g->hpre); cudaFree(g->Horig); cudaFree(g->cmax);
    cudaFreeHost(g->h_any);
    delete g;
}

void gmres_free(Plan *p) {
    if (p->gw) p->bytes_held -= p->gw->bytes;
    free_work(p->gw);
    p->gw = nullptr;
}

static long norm_pstride(int m, long len) {
    // dots: two slots (s and t of delayed CGS2) per basis vector and chunk; norms: one per block
    return std::max(2L * (m + 1) * ((len + kDotNE - 1) / kDotNE), (len + kStepNB - 1) / kStepNB);
}

// Workspace for k Krylov columns of length n; the product sees kp columns of
// length np (kp = k, np = n, or one global column: k = 1, n = kp * np).
static int ensure_work(Plan *p, int m, int k, long nv, int kp, bool flex, bool host_io) {
    GmresWork *g = p->gw;
    if (g && g->m == m && g->k == k && g->n == nv && g->kp == kp && (g->flex || !flex) && (!host_io || g->io))
        return BTTB_OK;
    gmres_free(p);
    g = new GmresWork();
    g->m = m;
    g->k = k;
    g->n = nv;
    g->kp = kp;
    g->np = p->n;
    g->glob = (k == 1 && kp > 1);
    g->flex = flex;
    g->NB = kStepNB;
    g->nblk = (int)((nv + g->NB - 1) / g->NB);                 // update / scale / norm grid
    const long pstride = std::max(norm_pstride(m, nv) * k, norm_pstride(m, p->n) * kp);
    const long n = nv;
    const int ks = std::max(k, kp);                             // per-column scalars (user norms need kp)
    size_t total = 0;
    bool ok = true;
    auto alloc = [&](auto **ptr, size_t bytes) {
        if (!ok) return;
        if (dev_malloc((void **)ptr, bytes) != cudaSuccess) ok = false;
        total += bytes;
    };
    alloc(&g->X, sizeof(float4) * k * n);
    alloc(&g->Vb, sizeof(float4) * (size_t)(m + 1) * k * n);
    if (flex) alloc(&g->Zb, sizeof(float4) * (size_t)m * k * n);
    alloc(&g->W, sizeof(float4) * k * n);
    alloc(&g->R, sizeof(float4) * k * n);
    alloc(&g->Vin, sizeof(float4) * k * n);
    alloc(&g->H, sizeof(float4) * (size_t)k * (m + 1) * m);
    alloc(&g->hacc, sizeof(float4) * (size_t)k * (m + 1));
    alloc(&g->gv, sizeof(float4) * (size_t)k * (m + 1));
    alloc(&g->sn, sizeof(float4) * (size_t)k * m);
    alloc(&g->hco, sizeof(float4) * (size_t)k * (m + 1));
    alloc(&g->cco, sizeof(float4) * (size_t)k * (m + 1));
    alloc(&g->hpre, sizeof(float4) * 2 * (size_t)k * (m + 1));   // two buffers, by step parity
    alloc(&g->Horig, sizeof(float4) * (size_t)k * (m + 1) * m);
    alloc(&g->U, sizeof(float4) * k * n);
    alloc(&g->ycoef, sizeof(float4) * (size_t)k * (m + 1));
    alloc(&g->part, sizeof(float4) * (size_t)pstride);
    alloc(&g->cs, sizeof(float2) * (size_t)k * m);
    alloc(&g->beta2, sizeof(double) * ks);
    alloc(&g->act_prod, sizeof(int) * kp);
    alloc(&g->cmax, sizeof(unsigned long long) * kp);
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

// ||col||^2 of the ncols columns of x ([c][len] double-float) into g->beta2.
static int norm2_cols(Plan *p, GmresWork *g, const float4 *x, int ncols, long len) {
    const long pstride = norm_pstride(g->m, len);
    const int nblk = (int)((len + kStepNB - 1) / kStepNB);
    norm_partial_kernel<<<dim3(nblk, ncols), kVecThreads, 0, p->stream>>>(x, len, kStepNB, nblk, pstride, g->part);
    norm_final_kernel<<<ncols, 32, 0, p->stream>>>(g->part, nblk, pstride, g->beta2);
    count_launch(p, 2);
    return check_cuda(p, cudaGetLastError(), "norm launch");
}

// One Arnoldi step for every active column, on p->stream (captured or not):
// [block-Jacobi], the product, then the four fused Gram-Schmidt/Givens kernels.
static int arnoldi_step(Plan *p, GmresWork *g, int inner, int j) {
    const int m = g->m, k = g->k, kp = g->kp;
    const long n = g->n, np = g->np, bs_i = (long)k * n;
    cudaStream_t st = p->stream;
    int rc;
    const float4 *src = g->Vb;
    const int *pact = g->active;                 // product-column flags
    if (g->glob) {
        bcast_active_kernel<<<(kp + 255) / 256, 256, 0, st>>>(g->active, g->act_prod, kp);
        count_launch(p);
        pact = g->act_prod;
    }
    if (g->pc == BTTB_PC_BLOCK_JACOBI) {
        rc = block_jacobi_run(p, g->Vb + (long)j * bs_i, FMT_CDF, np, g->Zb + (long)j * bs_i, FMT_CDF, np, kp,
                              nullptr, 0, pact);
        if (rc != BTTB_OK) return rc;
        src = g->Zb;
    } else if (g->pc == BTTB_PC_LEARNED) {
        rc = learned_apply_run(p, g->Vb + (long)j * bs_i, FMT_CDF, np, g->Zb + (long)j * bs_i, FMT_CDF, np, kp);
        if (rc != BTTB_OK) return rc;
        src = g->Zb;
    }
    rc = matvec_run(p, src + (long)j * bs_i, FMT_CDF, np, g->W, FMT_CDF, np, kp, inner, nullptr, 0, nullptr, pact);
    if (rc != BTTB_OK) return rc;
    StepArgs a{};
    a.Vb = g->Vb;
    a.W = g->W;
    a.n = n;
    a.bs_i = bs_i;
    a.bs_c = n;
    a.m = m;
    a.k = k;
    a.dot_sub = 1;
    while ((n + (long)kDotNE * a.dot_sub - 1) / ((long)kDotNE * a.dot_sub) > 4096) a.dot_sub <<= 1;
    a.nblk_dot = (int)((n + (long)kDotNE * a.dot_sub - 1) / ((long)kDotNE * a.dot_sub));
    a.ich = (int)(((long)a.nblk_dot * (j + 1) + kDotIW - 1) / kDotIW);
    a.nblk_vec = g->nblk;
    a.part = g->part;
    a.pstride = norm_pstride(m, n);
    a.hco = g->hco;
    a.hacc = g->hacc;
    a.cnt_a = g->counters;
    a.cnt_b = g->counters + k;
    a.cnt_c = g->counters + 2 * k;
    a.cnt_d = g->counters + 3 * k;
    a.active = g->active;
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
    const dim3 dgrid(a.ich, k), vgrid(a.nblk_vec, k);
    const size_t hs_bytes = (size_t)(m + 1) * sizeof(float4);
    const size_t upd_smem = hs_bytes + (size_t)(4 * m + 4) * sizeof(float4);
    int tok;
    for (int pass = 0; pass < 2; ++pass) {
        tok = prof_begin(p, 3);
        launch_pdl(step_dots_kernel, dgrid, dim3(kDotIW * 32), 0, st, a, pass, pass == 0 ? a.cnt_a : a.cnt_b, j);
        prof_end(p, tok, 0.0);
        tok = prof_begin(p, pass == 0 ? 4 : 5);
        // the first pass in binary32 FMAs when the products are binary32 (the second pass corrects it)
        const bool t32 = pass == 0 && fft_prec_of(inner) == PREC_F32;
        const bool deep = !p->in_batch && (long)a.nblk_vec * k < 4L * p->nsm;
        auto ukern = deep ? (t32 ? step_update_kernel<16, true> : step_update_kernel<16, false>)
                          : (t32 ? step_update_kernel<4, true> : step_update_kernel<4, false>);
        launch_pdl(ukern, vgrid, dim3(kStepNB), upd_smem, st, a, pass, j);
        prof_end(p, tok, 0.0);
    }
    tok = prof_begin(p, 6);
    launch_pdl(step_scale_kernel, vgrid, dim3(kStepNB), 0, st, a, j);
    prof_end(p, tok, 0.0);
    count_launch(p, 5);
    return check_cuda(p, cudaGetLastError(), "Arnoldi step launch");
}


static DcgsArgs dcgs_args(Plan *p, GmresWork *g, int j) {
    DcgsArgs a{};
    const long n = g->n;
    a.Vb = g->Vb;
    a.U = g->U;
    a.X = g->W;
    a.n = n;
    a.bs_i = (long)g->k * n;
    a.bs_c = n;
    a.m = g->m;
    a.k = g->k;
    a.dot_sub = 1;
    while ((n + (long)kDotNE * a.dot_sub - 1) / ((long)kDotNE * a.dot_sub) > 4096) a.dot_sub <<= 1;
    a.nblk_dot = (int)((n + (long)kDotNE * a.dot_sub - 1) / ((long)kDotNE * a.dot_sub));
    {
        const long cpv = (a.nblk_dot + kDotIW - 1) / kDotIW;
        // many columns of one-piece chunks: each CTA covers all vectors of its chunk group and keeps u and x
        // in registers; otherwise a CTA per (vector, chunk group) for parallelism
        a.cmajor = a.dot_sub == 1 && cpv * g->k >= 2L * p->nsm;
        // vector-major: enough vectors per CTA that the grid is about two CTAs per SM
        const long want = 2L * p->nsm;
        const long tot = cpv * (long)(j + 1) * g->k;
        a.vgrp = a.cmajor ? 1 : (int)std::max<long>(1, std::min<long>(j + 1, (tot + want - 1) / want));
        a.ich = (int)(a.cmajor ? cpv : cpv * ((j + 1 + a.vgrp - 1) / a.vgrp));
        a.fused = a.cmajor ? 0 : 1;
    }
    a.dsm_last = 7 * g->m + 7 + kDotIW * 32 + g->m + 1;
    a.nblk_vec = g->nblk;
    a.part = g->part;
    a.pstride = norm_pstride(g->m, n);
    a.sco = g->hco;
    a.cco = g->cco;
    a.hpre = g->hpre;
    a.Horig = g->Horig;
    a.hcol = g->hacc;
    a.nu2 = g->beta2;
    a.cnt = g->counters;
    a.active = g->active;
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
    a.wait_ns = p->wait_ns;
    return a;
}

// Dynamic shared memory above 48 KB needs the kernel's opt-in; the limit covers static and dynamic
// shared memory together, so a restart length whose scratch does not fit is an argument error.
template <typename K>
static int dcgs_smem_optin(Plan *p, K kern, size_t smem, const char *what) {
    if (smem <= 48 * 1024) return BTTB_OK;
    cudaFuncAttributes fa{};
    cudaError_t ea = cudaFuncGetAttributes(&fa, kern);
    if (ea == cudaSuccess && smem + fa.sharedSizeBytes > p->smem_optin)
        return set_error(p, BTTB_ERR_INVALID_ARG, "restart length too large for the delayed CGS2 shared memory");
    if (ea == cudaSuccess)
        ea = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(p->smem_optin - fa.sharedSizeBytes));
    return ea == cudaSuccess ? BTTB_OK : check_cuda(p, ea, what);
}

static int dcgs_dots_launch(Plan *p, GmresWork *g, int j, int has_x) {
    const DcgsArgs a = dcgs_args(p, g, j);
    // last-CTA scratch, then (chunk-major) two basis stages per warp and their mbarriers
    const size_t smem = (size_t)a.dsm_last * sizeof(float4) +
                        (a.cmajor ? (size_t)kDotIW * 2 * kDotNE * sizeof(float4) + kDotIW * 2 * sizeof(uint64_t) : 0);
    int rc = a.cmajor ? dcgs_smem_optin(p, dcgs_dots_kernel<true>, smem, "delayed CGS2 reduction shared memory")
                      : dcgs_smem_optin(p, dcgs_dots_kernel<false>, smem, "delayed CGS2 reduction shared memory");
    if (rc != BTTB_OK) return rc;
    const int tok = prof_begin(p, 3);
    cudaError_t e = a.cmajor
        ? launch_pdl(dcgs_dots_kernel<true>, dim3(a.ich, g->k), dim3(kDotIW * 32), smem, p->stream, a, j, has_x)
        : launch_pdl(dcgs_dots_kernel<false>, dim3(a.ich, g->k), dim3(kDotIW * 32), smem, p->stream, a, j, has_x);
    prof_end(p, tok, 0.0);
    count_launch(p);
    if (e != cudaSuccess) return check_cuda(p, e, "delayed CGS2 reduction launch");
    return BTTB_OK;
}

// One Arnoldi step with delayed CGS2 (unpreconditioned): x = A u_j, the reduction
// (which closes column j-1 and runs its Givens step), then the update.
static int arnoldi_step_dcgs(Plan *p, GmresWork *g, int inner, int j) {
    const int kp = g->kp;
    const long np = g->np;
    cudaStream_t st = p->stream;
    const int *pact = g->active;
    if (g->glob) {
        bcast_active_kernel<<<(kp + 255) / 256, 256, 0, st>>>(g->active, g->act_prod, kp);
        count_launch(p);
        pact = g->act_prod;
    }
    // x = A u_j, or x = A P_K^{-1} u_j with block-Jacobi (fixed, linear: plain right preconditioning)
    const float4 *src = g->U;
    int rc;
    if (g->pc == BTTB_PC_BLOCK_JACOBI) {
        if ((rc = block_jacobi_run(p, g->U, FMT_CDF, np, g->Zb, FMT_CDF, np, kp, nullptr, 0, pact)) != BTTB_OK)
            return rc;
        src = g->Zb;
    }
    rc = matvec_run(p, src, FMT_CDF, np, g->W, FMT_CDF, np, kp, inner, nullptr, 0, nullptr, pact);
    if (rc != BTTB_OK) return rc;
    if ((rc = dcgs_dots_launch(p, g, j, 1)) != BTTB_OK) return rc;
    const DcgsArgs a = dcgs_args(p, g, j);
    // coefficients / Givens scratch; with the fused close, the reduction tail's scratch
    const size_t smem = (size_t)(a.fused ? a.dsm_last : std::max(2 * g->m + 2, 4 * g->m + 4)) * sizeof(float4);
    const dim3 vgrid(a.nblk_vec + (a.fused ? 2 : 1), g->k);   // + the Givens CTA (+ the Hessenberg CTA)
    // basis entries loaded eight at a time for a lone plan (the few-column grid is latency-bound, the
    // many-column one streams the basis from HBM: both want the loads in flight), four in a batch, whose
    // arrays' kernels share the SMs
    const bool wide = !p->in_batch;
    const bool t32 = fft_prec_of(inner) == PREC_F32;          // binary32 products: binary32 first pass
    auto kern = wide ? (t32 ? dcgs_update_kernel<8, true> : dcgs_update_kernel<8, false>)
                     : (t32 ? dcgs_update_kernel<4, true> : dcgs_update_kernel<4, false>);
    if ((rc = dcgs_smem_optin(p, kern, smem, "delayed CGS2 update shared memory")) != BTTB_OK) return rc;
    const int tok = prof_begin(p, 4);
    cudaError_t e = launch_pdl(kern, vgrid, dim3(kStepNB), smem, st, a, j);
    prof_end(p, tok, 0.0);
    count_launch(p);
    if (e != cudaSuccess) return check_cuda(p, e, "delayed CGS2 update launch");
    return check_cuda(p, cudaGetLastError(), "Arnoldi step launch");
}

// Back substitution and x += (preconditioned) basis * y for the columns of this cycle.
static int cycle_finish(Plan *p, GmresWork *g) {
    const int m = g->m, k = g->k;
    const long n = g->n, bs_i = (long)k * n, bs_c = n;
    if (g->dcgs) {
        // close the cycle's last column (a reduction without x)
        const int rc = dcgs_dots_launch(p, g, m, 0);
        if (rc != BTTB_OK) return rc;
    }
    const int vgrid = (int)std::min<long>((n + kVecThreads - 1) / kVecThreads, 1024);
    finish_kernel<<<k, kFinishThreads, (m + 1) * sizeof(double2), p->stream>>>(g->H, g->gv, g->steps, g->ycoef, m,
                                                                               g->act_cycle);
    count_launch(p);
    if (g->dcgs && g->pc == BTTB_PC_BLOCK_JACOBI) {
        // x += P_K^{-1} (Q y): Q y into R (free until the next cycle's residual), then the preconditioner
        fill_zero_kernel<<<1024, kVecThreads, 0, p->stream>>>(g->R, (long)k * n);
        update_kernel<<<dim3(vgrid, k), kVecThreads, (m + 1) * sizeof(float4), p->stream>>>(
            g->Vb, bs_i, bs_c, g->steps, g->ycoef, m + 1, g->R, n, 1.f, g->act_cycle);
        count_launch(p, 2);
        const int rc = block_jacobi_run(p, g->R, FMT_CDF, g->np, g->Zb, FMT_CDF, g->np, g->kp, nullptr, 0,
                                        g->glob ? nullptr : g->act_cycle);
        if (rc != BTTB_OK) return rc;
        add_active_kernel<<<dim3(vgrid, k), kVecThreads, 0, p->stream>>>(g->X, g->Zb, n, g->act_cycle);
        count_launch(p);
    } else {
        update_kernel<<<dim3(vgrid, k), kVecThreads, (m + 1) * sizeof(float4), p->stream>>>(
            g->pc != BTTB_PC_NONE ? g->Zb : g->Vb, bs_i, bs_c, g->steps, g->ycoef, m + 1, g->X, n, 1.f,
            g->act_cycle);
        count_launch(p);
    }
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
        rc = g->dcgs ? arnoldi_step_dcgs(p, g, inner, step) : arnoldi_step(p, g, inner, step);
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
    g->graph_pc = g->pc;
    g->graph_dcgs = g->dcgs;
    g->graph_prof = p->prof;
    return BTTB_OK;
}

int gmres_solve(Plan *p, const void *V, void *I, int k, long ld, const bttb_gmres_opts *o,
                bttb_col_result *out) {
    const int m = o->restart;
    const bool flex = o->pc != BTTB_PC_NONE;
    const int inner = o->inner;
    const bool use_graph = !(o->flags & BTTB_GMRES_NO_GRAPH);
    // Global GMRES (Sec. III-C, Eq. (ZIVvec)): one Krylov space for vec(I), Frobenius inner products.
    const bool glob = (o->flags & BTTB_GMRES_GLOBAL) && k > 1;
    const long n = p->n;                         // user / product vector length
    const int kg = glob ? 1 : k;                 // Krylov columns
    const long nv = glob ? (long)k * n : n;      // Krylov vector length
    int rc = ensure_work(p, m, kg, nv, k, flex, o->host_io != 0);
    if (rc != BTTB_OK) return rc;
    GmresWork *g = p->gw;
    g->pc = o->pc;
    // delayed CGS2 unless the preconditioner is the learned (nonlinear) one, which needs flexible GMRES
    g->dcgs = (o->pc == BTTB_PC_NONE || o->pc == BTTB_PC_BLOCK_JACOBI) && !(o->flags & BTTB_GMRES_CGS2);
    const long bs_i = (long)kg * nv, bs_c = nv;  // basis layout [i][c][nv]
    cudaStream_t st = p->stream;
    cudaError_t e;
    const int vgrid = (int)std::min<long>((n + kVecThreads - 1) / kVecThreads, 1024);
    const int kgrid = (int)std::min<long>((nv + kVecThreads - 1) / kVecThreads, 1024);

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
    // column exponents of V (one for all columns in global GMRES), then V and x0 scaled by them
    const int cstride = glob ? 0 : 1;
    if ((e = cudaMemsetAsync(g->cmax, 0, sizeof(unsigned long long) * k, st)) != cudaSuccess)
        return check_cuda(p, e, "column scale");
    colmax_kernel<<<dim3(std::min(vgrid, 64), k), kVecThreads, 0, st>>>(Vd, ldv, n, g->cmax, cstride);
    cvt_in_kernel<<<dim3(vgrid, k), kVecThreads, 0, st>>>(Vd, ldv, g->Vin, n, g->cmax, cstride);
    count_launch(p, 2);
    if ((e = cudaGetLastError()) != cudaSuccess) return check_cuda(p, e, "input conversion");
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
        cvt_in_kernel<<<dim3(vgrid, k), kVecThreads, 0, st>>>(Xd, ldx, g->X, n, g->cmax, cstride);
        count_launch(p);
    } else {
        fill_zero_kernel<<<1024, kVecThreads, 0, st>>>(g->X, (long)k * n);
        count_launch(p);
    }
    if ((rc = norm2_cols(p, g, g->Vin, k, n)) != BTTB_OK) return rc;
    std::vector<double> vn2(k), vnorm(k), b2(k), relres(k, 0.0), tgt(kg);
    std::vector<int> status(k, BTTB_OK), cycles(k, 0);
    std::vector<int> total(kg, 0), act(kg), mlim(kg), stp(kg, 0), bd(kg, 0);   // per Krylov column
    e = cudaMemcpyAsync(vn2.data(), g->beta2, sizeof(double) * k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return check_cuda(p, e, "norm of V");
    double vmin = INFINITY;
    for (int c = 0; c < k; ++c) {
        vnorm[c] = std::sqrt(vn2[c]);
        if (vnorm[c] > 0.0) vmin = std::min(vmin, vnorm[c]);
    }
    std::vector<char> done(k, 0);
    int hist_n = 0;
    const int max_iters = o->max_iters;
    int dev_err = 0;

    for (int cycle = 0;; ++cycle) {
        // True residual with the FP64 product, per user column.
        if ((rc = matvec_run(p, g->X, FMT_CDF, n, g->W, FMT_CDF, n, k, PREC_DF64)) != BTTB_OK) return rc;
        resid_kernel<<<1024, kVecThreads, 0, st>>>(g->Vin, g->W, g->R, (long)k * n);
        count_launch(p);
        if ((rc = norm2_cols(p, g, g->R, k, n)) != BTTB_OK) return rc;
        e = cudaMemcpyAsync(b2.data(), g->beta2, sizeof(double) * k, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&dev_err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return check_cuda(p, e, "residual norm");
        if (dev_err & DEVERR_TIMEOUT) return set_error(p, BTTB_ERR_TIMEOUT, "a device pipeline wait timed out");
        bool any = false;
        if (!glob) {
            for (int c = 0; c < k; ++c) {
                if (done[c]) { act[c] = 0; continue; }
                relres[c] = vnorm[c] == 0.0 ? 0.0 : std::sqrt(b2[c]) / vnorm[c];   // NaN for a non-finite V
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
                    if (inner == BTTB_MV_FP32 || inner == BTTB_MV_TC_3XTF32 || inner == BTTB_MV_TC_BF16X3) t = std::max(t, 1e-5 * b0);
                    tgt[c] = t;
                    cycles[c] += 1;
                }
            }
        } else {
            // Every column stays in the one Krylov space until all meet tol; the cycle's target on the
            // Frobenius norm, tol * min_c ||V_c||, bounds every column's residual by tol ||V_c||.
            double f2 = 0.0;
            bool all_ok = true, bad = false;
            for (int c = 0; c < k; ++c) {
                relres[c] = vnorm[c] == 0.0 ? 0.0 : std::sqrt(b2[c]) / vnorm[c];   // NaN for a non-finite V
                if (!std::isfinite(relres[c])) bad = true;
                if (!(relres[c] <= o->tol) && vnorm[c] != 0.0) all_ok = false;
                f2 += b2[c];
            }
            int fin = -1;                                 // status for every column when the solve ends
            if (bad) fin = BTTB_ERR_NONFINITE;
            else if (all_ok) fin = BTTB_OK;
            else if (total[0] >= max_iters) fin = BTTB_NOT_CONVERGED;
            else if (cycle > 0 && bd[0] && stp[0] == 0) fin = BTTB_BREAKDOWN;
            if (fin != -1) {
                for (int c = 0; c < k; ++c) {
                    status[c] = fin;
                    if ((fin == BTTB_NOT_CONVERGED || fin == BTTB_BREAKDOWN) && relres[c] <= o->tol)
                        status[c] = BTTB_OK;
                    if (fin == BTTB_ERR_NONFINITE && std::isfinite(relres[c])) status[c] = BTTB_NOT_CONVERGED;
                }
                act[0] = 0;
            } else {
                any = true;
                act[0] = 1;
                mlim[0] = std::min(m, max_iters - total[0]);
                double t = 0.9 * o->tol * (std::isfinite(vmin) ? vmin : 0.0);
                if (inner == BTTB_MV_FP32 || inner == BTTB_MV_TC_3XTF32 || inner == BTTB_MV_TC_BF16X3) t = std::max(t, 1e-5 * std::sqrt(f2));
                tgt[0] = t;
                for (int c = 0; c < k; ++c) cycles[c] += 1;
                e = cudaMemcpyAsync(g->beta2, &f2, sizeof(double), cudaMemcpyHostToDevice, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);     // f2 is a host stack value
                if (e != cudaSuccess) return check_cuda(p, e, "Frobenius norm");
            }
        }
        if (o->history && hist_n < o->history_len) o->history[hist_n++] = relres[0];
        if (!any) break;
        e = cudaMemcpyAsync(g->active, act.data(), sizeof(int) * kg, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->act_cycle, act.data(), sizeof(int) * kg, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->mlimit, mlim.data(), sizeof(int) * kg, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->target, tgt.data(), sizeof(double) * kg, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(g->bdown, 0, sizeof(int) * kg, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(g->steps, 0, sizeof(int) * kg, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(g->d_any_step, 0, sizeof(int), st);
        if (e != cudaSuccess) return check_cuda(p, e, "cycle set-up");
        cycle_start_kernel<<<1, 256, 0, st>>>(g->beta2, g->gv, g->inv_beta, m, kg, g->active);
        count_launch(p);
        // the first basis vector r/beta: into the basis (CGS2) or as u_0 (delayed CGS2)
        scale_kernel<<<dim3(kgrid, kg), kVecThreads, 0, st>>>(g->R, g->dcgs ? g->U : g->Vb, g->dcgs ? bs_c : bs_i,
                                                              bs_c, 0, g->inv_beta, nv, g->active);
        count_launch(p);
        if (use_graph) {
            if (!g->cycle_exec || g->graph_inner != inner || g->graph_pc != g->pc || g->graph_prof != p->prof ||
                g->graph_dcgs != (int)g->dcgs)
                if ((rc = build_cycle_graph(p, g, inner)) != BTTB_OK) return rc;
            if ((e = cudaGraphLaunch(g->cycle_exec, st)) != cudaSuccess) return check_cuda(p, e, "graph launch");
            p->launches += g->launches_per_cycle;
        } else {
            for (int step = 0; step < m; ++step) {
                rc = g->dcgs ? arnoldi_step_dcgs(p, g, inner, step) : arnoldi_step(p, g, inner, step);
                if (rc != BTTB_OK) return rc;
                e = cudaMemcpyAsync(g->h_any, g->d_any_step, sizeof(int), cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) return check_cuda(p, e, "Arnoldi step");
                if (*g->h_any < step + 1) break;              // no column continued after this step
            }
            if ((rc = cycle_finish(p, g)) != BTTB_OK) return rc;
        }
        e = cudaMemcpyAsync(stp.data(), g->steps, sizeof(int) * kg, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(bd.data(), g->bdown, sizeof(int) * kg, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return check_cuda(p, e, "cycle end");
        int maxsteps = 0;
        for (int c = 0; c < kg; ++c)
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
    cvt_out_kernel<<<dim3(vgrid, k), kVecThreads, 0, st>>>(g->X, Id, ldo, n, g->cmax, cstride);
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
            out[c].iters = total[glob ? 0 : c];
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
