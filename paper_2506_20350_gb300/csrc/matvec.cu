// The multilevel-FFT product y = Z x (Sec. II-C and III-A) as five
// stream-ordered passes over the plan workspace:
//   1. pad + forward FFT along the cells of each row      x  -> U  (ny rows kept)
//   2. forward FFT along the rows of each column          U  -> u^ (all my rows)
//   3. per-bin block product (contract.cu)                u^ -> v^
//   4. inverse FFT along the rows, crop to ny rows        v^ -> V
//   5. inverse FFT along the cells, crop to nx cells      V  -> y
// Passes 1/2 together are the forward 2-level blockwise FFT of App. B (the
// padding of Eq. (xc2) is implicit: the zero slots are never read, the pass
// zero-fills them on chip); passes 4/5 are its inverse with the crop of
// Sec. II-C.  The 1/(mx my) of the inverse is folded into the stored spectrum.
//
// Layouts (elements of the precision's native complex type):
//   U, V : [c][iy][kx][p]         at c*ny*mx*b + iy*mx*b + kx*b + p
//   u^,v^: [bin][c][p]            at (ky*mx + kx)*ubs + c*b + p
#include <algorithm>
#include <cmath>
#include <vector>

#include "arith.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace bttb {

static int native_of(int prec) {
    return prec == PREC_F64N ? FMT_C128 : ((prec == PREC_F32 || is_tc_prec(prec)) ? FMT_C64 : FMT_CDF);
}

// Few columns.  ROUTE_FUSED_Y: the x pass, then the y-level transforms and the block product in one
// cluster kernel (ycontract.cu: the transformed vectors never leave the chip), then the inverse x pass.
// ROUTE_FUSED_FFT2: both FFT levels in one cluster kernel each way around the block product (no U / V
// round trip).  ROUTE_PASSES: four strided passes around the block product (also every product of more
// than kFusedFftMaxCols columns).  The automatic choice takes the fused y-level form where its shares fit
// on chip with every cluster resident; otherwise the fused two-level FFT for the double-float and binary64
// products and for plans that run beside other arrays' kernels in a batch, and the four passes for a lone
// binary32 product (they overlap better with their neighbours under programmatic dependent launch).
int product_route(Plan *p, int nrhs, int prec) {
    const bool few = nrhs <= kFusedFftMaxCols;
    const int fprec = fft_prec_of(prec);
    const int yprec = is_tc_prec(prec) ? PREC_F32 : prec;       // below kTcMinCols the TC forms are binary32
    const bool y_ok = few && (yprec == PREC_DF64 || yprec == PREC_F32) && ycontract_fits(p, yprec, nrhs);
    const bool f2_ok = few && fft2_fused_smem(p, fprec) <= p->smem_optin / 2;
    const bool pk_ok = few && product_persistent_fits(p, yprec, nrhs);
    int route = (prec == PREC_DF64 || prec == PREC_F64N) ? p->route_df : p->route_f32;
    if (route == ROUTE_PERSISTENT && !pk_ok) route = ROUTE_AUTO;
    if (route == ROUTE_FUSED_Y && !y_ok) route = ROUTE_AUTO;
    if (route == ROUTE_FUSED_FFT2 && !f2_ok) route = ROUTE_AUTO;
    if (route == ROUTE_AUTO)
        route = (f2_ok && (fprec != PREC_F32 || p->in_batch)) ? ROUTE_FUSED_FFT2 : ROUTE_PASSES;
    return route;
}

int matvec_run(Plan *p, const void *x, int xfmt, long ldx, void *y, int yfmt, long ldy, int nrhs, int prec,
               const int *in_sel, long in_sel_stride, const double *in_scale, const int *active) {
    const int nx = p->nx, ny = p->ny, b = p->b, mx = p->mx, my = p->my;
    const int NF = native_of(prec);
    const int fprec = fft_prec_of(prec);
    const long plane = (long)ny * mx * b;
    int rc;
    const int route = product_route(p, nrhs, prec);
    const int yprec = is_tc_prec(prec) ? PREC_F32 : prec;

    if (route == ROUTE_PERSISTENT)
        return product_persistent_launch(p, x, xfmt, ldx, y, yfmt, ldy, nrhs, yprec, in_sel, in_sel_stride, in_scale,
                                         active);
    if (route == ROUTE_FUSED_FFT2) {
        if ((rc = fft2_fused_launch(p, x, p->wsA, ldx, nrhs, fprec, xfmt, false, in_sel, in_sel_stride, in_scale,
                                    active)) != BTTB_OK)
            return rc;
        if ((rc = contract_launch(p, prec, p->wsA, p->wsB, nrhs, active)) != BTTB_OK) return rc;
        return fft2_fused_launch(p, p->wsB, y, ldy, nrhs, fprec, yfmt, true, nullptr, 0, nullptr, active);
    }

    FftPass a{};
    a.in = x; a.out = p->wsB;
    a.in_cs = ldx; a.in_os = (long)nx * b; a.in_ns = b;
    a.out_cs = plane; a.out_os = (long)mx * b; a.out_ns = b;
    a.in_sel = in_sel; a.in_sel_stride = in_sel_stride; a.in_scale = in_scale; a.active = active;
    a.O = ny; a.pdim = b; a.ncols = nrhs;
    a.nin = nx; a.nout = mx; a.M = mx;
    if ((rc = fft_pass_launch(p, a, fprec, xfmt, NF, false)) != BTTB_OK) return rc;

    FftPass e{};
    e.in = p->wsA; e.out = y;
    e.in_cs = plane; e.in_os = (long)mx * b; e.in_ns = b;
    e.out_cs = ldy; e.out_os = (long)nx * b; e.out_ns = b;
    e.O = ny; e.pdim = b; e.ncols = nrhs; e.active = active;
    e.nin = mx; e.nout = nx; e.M = mx;
    if (route == ROUTE_FUSED_Y) {
        if ((rc = ycontract_launch(p, yprec, p->wsB, p->wsA, nrhs, active)) != BTTB_OK) return rc;
        return fft_pass_launch(p, e, fprec, NF, yfmt, true);
    }

    FftPass c{};
    c.in = p->wsB; c.out = p->wsA;
    c.in_cs = plane; c.in_os = b; c.in_ns = (long)mx * b;
    c.out_cs = b; c.out_os = p->ubs; c.out_ns = (long)mx * p->ubs;
    c.O = mx; c.pdim = b; c.ncols = nrhs; c.active = active;
    c.nin = ny; c.nout = my; c.M = my;
    if ((rc = fft_pass_launch(p, c, fprec, NF, NF, false)) != BTTB_OK) return rc;

    if ((rc = contract_launch(p, prec, p->wsA, p->wsB, nrhs, active)) != BTTB_OK) return rc;

    FftPass d{};
    d.in = p->wsB; d.out = p->wsA;
    d.in_cs = b; d.in_os = p->ubs; d.in_ns = (long)mx * p->ubs;
    d.out_cs = plane; d.out_os = b; d.out_ns = (long)mx * b;
    d.O = mx; d.pdim = b; d.ncols = nrhs; d.active = active;
    d.nin = my; d.nout = ny; d.M = my;
    if ((rc = fft_pass_launch(p, d, fprec, NF, NF, true)) != BTTB_OK) return rc;
    return fft_pass_launch(p, e, fprec, NF, yfmt, true);
}

// ---------------------------------------------------------------------------
// Block-Jacobi preconditioner P_K (Sec. III-B): every cell's b-block is
// multiplied by R_0^{-1}, R_0 = T[0,0].  The inverse is formed once on the
// host from an LU factorisation with partial pivoting (binary64) and applied
// in binary32 as a batched b x b GEMV: it only steers the Krylov space of a
// flexible GMRES, which stores the preconditioned vectors it used.
// ---------------------------------------------------------------------------
constexpr int kBjThreads = 256;

// R_0^{-1} is stored column-major with the rows padded to bq = 4*ceil(b/4)
// (entry (p, q) at q*bq + p, zero rows beyond b), so the four rows a thread
// owns are one 32-byte load.  Thread (row group rg, cell group cg) computes
// rows 4rg .. 4rg+3 of CC consecutive cells: per basis q it loads four entries
// of R_0^{-1} and CC entries of x for 4*CC complex multiply-adds.  With CC = 4
// the CTA stages R_0^{-1} in shared memory; with CC = 1 (few cells: small CTAs
// that fill every SM) it reads R_0^{-1} through L1.
template <int INF, int OUTF, int CC>
__global__ void __launch_bounds__(kBjThreads) bj_apply_kernel(const float2 *rinv, const void *x, long ldx, void *z,
                                                               long ldz, int b, int ncells, int ncg,
                                                               const int *in_sel, long in_sel_stride,
                                                               int rinv_in_smem, const int *active) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int bq = (b + 3) & ~3;
    const int xst = b + 1;                                    // padded row stride of the staged cells
    const int cpb = ncg * CC;
    float2 *rsm = reinterpret_cast<float2 *>(smem_raw);      // b*bq (when staged)
    float2 *xs = rsm + (rinv_in_smem ? (long)b * bq : 0);    // cpb*xst
    const float2 *rs = rinv_in_smem ? rsm : rinv;
    const int c = blockIdx.y;
    pdl_wait();
    if (active && !active[c]) return;
    const int cell0 = blockIdx.x * cpb;
    const int nc = min(cpb, ncells - cell0);
    if (rinv_in_smem) {
        const float4 *src = reinterpret_cast<const float4 *>(rinv);
        float4 *dst = reinterpret_cast<float4 *>(rsm);
        for (int i = threadIdx.x; i < b * bq / 2; i += blockDim.x) dst[i] = src[i];
    }
    long xoff = (long)c * ldx + (long)cell0 * b;
    if (in_sel) xoff += (long)(*in_sel) * in_sel_stride;
    for (int i = threadIdx.x; i < nc * b; i += blockDim.x) {
        const int cl = i / b;
        xs[cl * xst + (i - cl * b)] = load_vec<F32, INF>(x, xoff + i);
    }
    __syncthreads();
    const int nrg = bq / 4;
    const int rg = threadIdx.x % nrg, cg = threadIdx.x / nrg;
    if (cg >= ncg) return;
    const int r0 = rg * 4;
    float2 acc[CC][4];
#pragma unroll
    for (int u = 0; u < CC; ++u)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[u][r] = make_float2(0.f, 0.f);
    const float2 *xv = xs + (long)cg * CC * xst;
    for (int q = 0; q < b; ++q) {
        const float4 g01 = *reinterpret_cast<const float4 *>(rs + (long)q * bq + r0);
        const float4 g23 = *reinterpret_cast<const float4 *>(rs + (long)q * bq + r0 + 2);
        const float2 g[4] = {make_float2(g01.x, g01.y), make_float2(g01.z, g01.w), make_float2(g23.x, g23.y),
                             make_float2(g23.z, g23.w)};
#pragma unroll
        for (int u = 0; u < CC; ++u) {
            const float2 v = xv[u * xst + q];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                acc[u][r].x = fmaf(g[r].x, v.x, acc[u][r].x);
                acc[u][r].x = fmaf(-g[r].y, v.y, acc[u][r].x);
                acc[u][r].y = fmaf(g[r].x, v.y, acc[u][r].y);
                acc[u][r].y = fmaf(g[r].y, v.x, acc[u][r].y);
            }
        }
    }
    long zoff = (long)c * ldz + (long)cell0 * b;
    if (in_sel) zoff += (long)(*in_sel) * in_sel_stride;       // same selected column slot on output
#pragma unroll
    for (int u = 0; u < CC; ++u) {
        const int cl = cg * CC + u;
        if (cl >= nc) continue;
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (r0 + r < b) store_vec<F32, OUTF>(z, zoff + (long)cl * b + r0 + r, acc[u][r]);
    }
}

template <int INF, int OUTF>
static int bj_launch(Plan *p, const void *x, long ldx, void *z, long ldz, int nrhs, const int *in_sel,
                     long in_sel_stride, const int *active) {
    const int b = p->b, ncells = p->nx * p->ny;
    const int bq = (b + 3) & ~3, nrg = bq / 4;
    const int gmax = kBjThreads / nrg;                          // cell groups per CTA at most (b <= 256: >= 4)
    const long want = 2L * p->nsm;                              // CTAs that fill every SM twice over
    const long total = (long)ncells * nrhs;
    const size_t r_bytes = (size_t)b * bq * sizeof(float2);
    // Four cells per thread when there are cells enough for full CTAs everywhere and R_0^{-1} fits on chip.
    const bool wide = total >= 4L * want * gmax && r_bytes + (size_t)4 * gmax * (b + 1) * sizeof(float2) <= 160 * 1024;
    const int CC = wide ? 4 : 1;
    long ncg = (total + want * CC - 1) / (want * CC);
    if (ncg > gmax) ncg = gmax;
    if (ncg < 1) ncg = 1;
    const int cpb = (int)ncg * CC;
    const int in_smem = wide ? 1 : 0;
    const size_t smem = (in_smem ? r_bytes : 0) + (size_t)cpb * (b + 1) * sizeof(float2);
    auto kern = wide ? bj_apply_kernel<INF, OUTF, 4> : bj_apply_kernel<INF, OUTF, 1>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_optin);
        if (e != cudaSuccess) return check_cuda(p, e, "block-Jacobi smem attribute");
    }
    dim3 grid((ncells + cpb - 1) / cpb, nrhs);
    cudaError_t le = launch_pdl(kern, grid, dim3(nrg * (int)ncg), smem, p->stream, (const float2 *)p->bj_inv, x, ldx,
                                z, ldz, b, ncells, (int)ncg, in_sel, in_sel_stride, in_smem, active);
    count_launch(p);
    if (le != cudaSuccess) return check_cuda(p, le, "block-Jacobi launch");
    return check_cuda(p, cudaGetLastError(), "block-Jacobi launch");
}

int block_jacobi_run(Plan *p, const void *x, int xfmt, long ldx, void *z, int zfmt, long ldz, int nrhs,
                     const int *in_sel, long in_sel_stride, const int *active) {
    if (!p->bj_ready) return set_error(p, BTTB_ERR_NO_GENERATORS, "block-Jacobi needs bttb_set_generators first");
#define BJ_CASE(I, O)                                     \
    if (xfmt == I && zfmt == O) return bj_launch<I, O>(p, x, ldx, z, ldz, nrhs, in_sel, in_sel_stride, active);
    BJ_CASE(FMT_C128, FMT_C128)
    BJ_CASE(FMT_C64, FMT_C64)
    BJ_CASE(FMT_CDF, FMT_CDF)
#undef BJ_CASE
    return set_error(p, BTTB_ERR_INVALID_ARG, "block-Jacobi: unsupported format pair");
}

// LU with partial pivoting of the b x b self block (binary64), then its
// inverse column by column; singular pivots are reported, not divided by.
int block_jacobi_setup(Plan *p, const double2 *t00) {
    const int b = p->b;
    std::vector<double> ar(2L * b * b);
    for (long i = 0; i < (long)b * b; ++i) {
        ar[2 * i] = t00[i].x;
        ar[2 * i + 1] = t00[i].y;
    }
    auto A = [&](int r, int c) -> double * { return &ar[2 * ((long)r * b + c)]; };
    std::vector<int> piv(b);
    double amax = 0.0;
    for (long i = 0; i < (long)b * b; ++i) amax = std::max(amax, std::hypot(ar[2 * i], ar[2 * i + 1]));
    for (int k = 0; k < b; ++k) {
        int pk = k;
        double best = std::hypot(A(k, k)[0], A(k, k)[1]);
        for (int i = k + 1; i < b; ++i) {
            double v = std::hypot(A(i, k)[0], A(i, k)[1]);
            if (v > best) { best = v; pk = i; }
        }
        piv[k] = pk;
        if (!(best > 1e-300) || best < 1e-15 * amax) {
            p->bj_ready = false;
            return set_error(p, BTTB_ERR_SINGULAR, "block-Jacobi: T[0,0] is singular to working precision");
        }
        if (pk != k)
            for (int j = 0; j < b; ++j) std::swap(A(k, j)[0], A(pk, j)[0]), std::swap(A(k, j)[1], A(pk, j)[1]);
        const double dr = A(k, k)[0], di = A(k, k)[1], dd = dr * dr + di * di;
        for (int i = k + 1; i < b; ++i) {
            double *l = A(i, k);
            const double lr = (l[0] * dr + l[1] * di) / dd, li = (l[1] * dr - l[0] * di) / dd;
            l[0] = lr;
            l[1] = li;
            for (int j = k + 1; j < b; ++j) {
                double *t = A(i, j);
                const double *u = A(k, j);
                t[0] -= lr * u[0] - li * u[1];
                t[1] -= lr * u[1] + li * u[0];
            }
        }
    }
    const int bq = (b + 3) & ~3;                                // rows padded to a multiple of 4
    std::vector<float2> inv((long)b * bq, make_float2(0.f, 0.f));
    std::vector<double> col(2 * b);
    for (int e = 0; e < b; ++e) {
        // solve R_0 x = e_e: permute, forward with unit L, back with U
        for (int i = 0; i < b; ++i) col[2 * i] = col[2 * i + 1] = 0.0;
        col[2 * e] = 1.0;
        for (int k = 0; k < b; ++k)
            if (piv[k] != k) std::swap(col[2 * k], col[2 * piv[k]]), std::swap(col[2 * k + 1], col[2 * piv[k] + 1]);
        for (int i = 0; i < b; ++i)
            for (int k = 0; k < i; ++k) {
                const double *l = A(i, k);
                col[2 * i] -= l[0] * col[2 * k] - l[1] * col[2 * k + 1];
                col[2 * i + 1] -= l[0] * col[2 * k + 1] + l[1] * col[2 * k];
            }
        for (int i = b - 1; i >= 0; --i) {
            double sr = col[2 * i], si = col[2 * i + 1];
            for (int k = i + 1; k < b; ++k) {
                const double *u = A(i, k);
                sr -= u[0] * col[2 * k] - u[1] * col[2 * k + 1];
                si -= u[0] * col[2 * k + 1] + u[1] * col[2 * k];
            }
            const double dr = A(i, i)[0], di = A(i, i)[1], dd = dr * dr + di * di;
            col[2 * i] = (sr * dr + si * di) / dd;
            col[2 * i + 1] = (si * dr - sr * di) / dd;
        }
        for (int i = 0; i < b; ++i) inv[(long)e * bq + i] = make_float2((float)col[2 * i], (float)col[2 * i + 1]);
    }
    if (!p->bj_inv) {
        cudaError_t e = dev_malloc((void **)&p->bj_inv, (size_t)b * bq * sizeof(float2));
        if (e != cudaSuccess) return check_cuda(p, e, "block-Jacobi buffer");
        p->bytes_held += (size_t)b * bq * sizeof(float2);
    }
    cudaError_t e = cudaMemcpy(p->bj_inv, inv.data(), (size_t)b * bq * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return check_cuda(p, e, "block-Jacobi upload");
    p->bj_ready = true;
    return BTTB_OK;
}

}  // namespace bttb
