// The per-bin block product for many right-hand sides on the fifth-generation tensor cores (tcgen05):
// V_k = G_k U_k (Eq. (multL) for a block of columns, Sec. III-C: the columns of I_M transformed together).
//
// The complex b x b by b x n product is one real GEMM.  With complex entries interleaved (re, im), the
// transformed vectors of a bin are a real 2b x n matrix B, column c holding 2b consecutive floats (the
// stored layout of u^), and G_k becomes the real 2b x 2b matrix A with the 2 x 2 block
// [[Re g, -Im g], [Im g, Re g]] at (2p, 2q); D = A B is v^ in the same interleaved layout.  A (M = 128:
// rows beyond 2b are zero) stays in shared memory for all column tiles of its bin; B tiles of 32 columns
// come in by TMA (cp.async.bulk.tensor, 128-byte swizzle, zero fill beyond 2b and beyond the last column).
// Each factor x is split into two terms x = hi + lo, and D = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulates
// in binary32 in tensor memory (the lo*lo term is below binary32 rounding for TF32 terms):
//   3xTF32       : hi = x with its 13 low mantissa bits cleared (exact in TF32), lo = x - hi (exact);
//   split-BF16x3 : hi = bf16(x), lo = bf16(x - hi), both rounded to nearest (about 2^-17 relative per term).
//
// Warp roles in a persistent CTA (one per SM; bins dealt out round robin, each bin's column tiles in turn):
//   warp 0   : TMA producer of the B tiles (two buffers);
//   warp 1   : owns the tensor memory (two 32-column accumulators) and one thread issues the MMAs;
//   warps 2-5: build A_hi / A_lo of each bin from the binary32 spectrum block, split each B tile, and move
//              each finished accumulator from tensor memory to v^ (warp w reads TMEM lanes 32 (w mod 4) ..).
// The stages are linked by mbarriers; every wait is bounded.  A wait that runs out sets the error word and
// the abort flag; every role then stops, the copies and MMAs in flight are waited for (bounded), and the
// tensor memory is released before the CTA exits.
#include <cuda_bf16.h>

#include "arith.cuh"
#include "internal.h"
#include "ptx.cuh"
#include "tc.cuh"

namespace bttb {

constexpr int kTgN = 32;                  // columns per tile (MMA N)
constexpr int kTgThreads = 192;
constexpr uint32_t kTgTmemCols = 64;      // two accumulators of kTgN binary32 columns

template <int FMT> struct TgLayout;
template <> struct TgLayout<kTcFmtTF32> {
    static constexpr uint32_t kA = 4 * 16384;                 // one operand copy of A: 4 K blocks of 128 rows x 128 B
    static constexpr uint32_t kRaw = 4 * 4096;                // a raw binary32 B tile: 4 K blocks of 32 rows
    static constexpr uint32_t kB = kRaw;                      // B_hi is the raw tile split in place
    static constexpr uint32_t oAhi = 0, oAlo = kA, oRaw = 2 * kA, oBlo = oRaw + 2 * kRaw, oCtl = oBlo + 2 * kB;
};
template <> struct TgLayout<kTcFmtBF16> {
    static constexpr uint32_t kA = 2 * 16384;                 // 2 K blocks of 64 bf16
    static constexpr uint32_t kRaw = 4 * 4096;
    static constexpr uint32_t kB = 2 * 4096;
    static constexpr uint32_t oAhi = 0, oAlo = kA, oRaw = 2 * kA, oBhi = oRaw + 2 * kRaw, oBlo = oBhi + 2 * kB,
                              oCtl = oBlo + 2 * kB;
};

struct TgArgs {
    const float2 *G;      // binary32 spectrum (hi plane), bin k's block column-major at k*gbs
    long gbs;
    float *v;             // v^ as binary32 pairs: bin*2*ubs + c*2b + row
    long ubs;
    int b, k, nbins, ntiles, nkb_raw, nks;
    int *err;
    unsigned long long wait_ns;
};

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

template <int FMT>
__global__ void __launch_bounds__(kTgThreads, 1) tcgemm_kernel(const __grid_constant__ CUtensorMap map, const TgArgs a) {
    using L = TgLayout<FMT>;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t base_u32 = (smem_u32(smem_raw) + 1023u) & ~1023u;   // 1024-byte aligned swizzle atoms
    unsigned char *sm = smem_raw + (base_u32 - smem_u32(smem_raw));
    uint64_t *b_full = reinterpret_cast<uint64_t *>(sm + L::oCtl);
    uint64_t *split_done = b_full + 2, *mma_done = b_full + 4, *d_free = b_full + 6, *a_ready = b_full + 8;
    uint64_t *drain = b_full + 9;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + L::oCtl + 96);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + L::oCtl + 100);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = a.b, twob = 2 * b;
    const int nbin_cta = blockIdx.x < a.nbins ? (a.nbins - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int items = nbin_cta * a.ntiles;

    if (threadIdx.x == 0) {
        *abort_flag = 0;
        for (int i = 0; i < 2; ++i) {
            mbar_init(&b_full[i], 1);
            mbar_init(&split_done[i], 4);
            mbar_init(&mma_done[i], 1);
            mbar_init(&d_free[i], 4);
        }
        mbar_init(a_ready, 4);
        mbar_init(drain, 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, kTgTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    pdl_wait();

    auto binof = [&](int i) { return (int)blockIdx.x + (i / a.ntiles) * (int)gridDim.x; };
    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(a.err, DEVERR_TIMEOUT);
    };

    if (warp == 0) {
        // ---------------------------------------------------------------- TMA producer
        int issued = 0;
        if (lane == 0) {
            for (int i = 0; i < items; ++i) {
                const int buf = i & 1;
                if (i >= 2 && !mbar_wait_bounded(&mma_done[buf], (uint32_t)((i - 2) >> 1) & 1u, abort_flag, a.wait_ns)) {
                    fail();
                    break;
                }
                if (*abort_flag) break;
                const int t = i % a.ntiles;
                unsigned char *dst = sm + L::oRaw + buf * L::kRaw;
                mbar_arrive_expect_tx(&b_full[buf], (uint32_t)a.nkb_raw * 4096u);
                for (int kb = 0; kb < a.nkb_raw; ++kb)
                    tma_load_3d(dst + kb * 4096, &map, kb * 32, t * kTgN, binof(i), &b_full[buf]);
                issued = i + 1;
            }
            // copies that may still be in flight: the last two issued tiles, each in its own buffer
            if (*abort_flag)
                for (int d = issued > 2 ? issued - 2 : 0; d < issued; ++d)
                    mbar_wait_drain(&b_full[d & 1], (uint32_t)(d >> 1) & 1u);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc_idesc(FMT, 128, kTgN);
            const uint32_t sAhi = base_u32 + L::oAhi, sAlo = base_u32 + L::oAlo;
            int done_items = 0;
            for (int i = 0; i < items; ++i) {
                const int buf = i & 1, t = i % a.ntiles;
                if (t == 0 && !mbar_wait_bounded(a_ready, (uint32_t)(i / a.ntiles) & 1u, abort_flag, a.wait_ns)) {
                    fail();
                    break;
                }
                if (!mbar_wait_bounded(&split_done[buf], (uint32_t)(i >> 1) & 1u, abort_flag, a.wait_ns) ||
                    (i >= 2 && !mbar_wait_bounded(&d_free[buf], (uint32_t)((i - 2) >> 1) & 1u, abort_flag, a.wait_ns))) {
                    fail();
                    break;
                }
                tc_fence_after();
                uint32_t sBhi, sBlo;
                if constexpr (FMT == kTcFmtTF32) {
                    sBhi = base_u32 + L::oRaw + buf * L::kRaw;
                    sBlo = base_u32 + L::oBlo + buf * L::kB;
                } else {
                    sBhi = base_u32 + TgLayout<kTcFmtBF16>::oBhi + buf * L::kB;
                    sBlo = base_u32 + L::oBlo + buf * L::kB;
                }
                const uint32_t d = tmem + (uint32_t)buf * kTgN;
                for (int s = 0; s < a.nks; ++s) {
                    const uint32_t offA = (uint32_t)(s >> 2) * 16384u + (uint32_t)(s & 3) * 32u;
                    const uint32_t offB = (uint32_t)(s >> 2) * 4096u + (uint32_t)(s & 3) * 32u;
                    const uint64_t ah = tc_smem_desc(sAhi + offA, 1024), al = tc_smem_desc(sAlo + offA, 1024);
                    const uint64_t bh = tc_smem_desc(sBhi + offB, 1024), bl = tc_smem_desc(sBlo + offB, 1024);
                    if constexpr (FMT == kTcFmtTF32) {
                        tc_mma_tf32(d, ah, bl, idesc, s > 0 ? 1u : 0u);
                        tc_mma_tf32(d, al, bh, idesc, 1u);
                        tc_mma_tf32(d, ah, bh, idesc, 1u);
                    } else {
                        tc_mma_f16(d, ah, bl, idesc, s > 0 ? 1u : 0u);
                        tc_mma_f16(d, al, bh, idesc, 1u);
                        tc_mma_f16(d, ah, bh, idesc, 1u);
                    }
                }
                tc_commit(&mma_done[buf]);
                done_items = i + 1;
            }
            // every MMA issued has completed before the tensor memory is released
            if (*abort_flag && done_items > 0) {
                tc_commit(drain);
                mbar_wait_drain(drain, 0u);
            }
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- workers: A, B split, epilogue
        const int wi = threadIdx.x - 64;                   // 0..127
        const int qw = warp & 3;                           // TMEM lane quarter this warp may read
        bool failed = false;
        auto epilogue = [&](int j) {
            const int buf = j & 1;
            if (!failed && !mbar_wait_bounded(&mma_done[buf], (uint32_t)(j >> 1) & 1u, abort_flag, a.wait_ns)) {
                fail();
                failed = true;
            }
            failed = __any_sync(0xffffffffu, failed);
            if (failed) return;
            tc_fence_after();
            float v0[16], v1[16];
            const uint32_t ta = tmem + ((uint32_t)(32 * qw) << 16) + (uint32_t)buf * kTgN;
            tmem_ld16(ta, v0);
            tmem_ld16(ta + 16, v1);
            tmem_ld_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&d_free[buf]);
            const int r = 32 * qw + lane, t = j % a.ntiles;
            if (r < twob) {
                float *dst = a.v + (long)binof(j) * 2 * a.ubs + r;
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    if (t * kTgN + c < a.k) gst(dst + (long)(t * kTgN + c) * twob, v0[c]);
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    if (t * kTgN + 16 + c < a.k) gst(dst + (long)(t * kTgN + 16 + c) * twob, v1[c]);
            }
        };
        auto build_a = [&](int bin) {
            // row m of A from row p = m/2 of the spectrum block (entry (p, q) at q*b + p)
            const int m = wi, p = m >> 1, odd = m & 1;
            const float2 *g = a.G + (long)bin * a.gbs + p;
            constexpr int EB = FMT == kTcFmtTF32 ? 32 : 64;     // elements per K block
            constexpr int EC = FMT == kTcFmtTF32 ? 4 : 8;       // elements per 16-byte chunk
            constexpr int NKB = FMT == kTcFmtTF32 ? 4 : 2;
            for (int kb = 0; kb < NKB; ++kb)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float x[EC];
#pragma unroll
                    for (int e = 0; e < EC; e += 2) {
                        const int q = (kb * EB + j * EC + e) >> 1;
                        float2 gq = make_float2(0.f, 0.f);
                        if (m < twob && q < b && BTTB_GCHK(g + (long)q * b, sizeof(float2))) gq = __ldg(g + (long)q * b);
                        x[e] = odd ? gq.y : gq.x;
                        x[e + 1] = odd ? gq.x : -gq.y;
                    }
                    const uint32_t off = (uint32_t)kb * 16384u + (uint32_t)m * 128u + ((uint32_t)(j ^ (m & 7)) << 4);
                    if constexpr (FMT == kTcFmtTF32) {
                        float4 hi, lo;
                        hi.x = tf32_hi(x[0]); hi.y = tf32_hi(x[1]); hi.z = tf32_hi(x[2]); hi.w = tf32_hi(x[3]);
                        lo = make_float4(x[0] - hi.x, x[1] - hi.y, x[2] - hi.z, x[3] - hi.w);
                        *reinterpret_cast<float4 *>(sm + L::oAhi + off) = hi;
                        *reinterpret_cast<float4 *>(sm + L::oAlo + off) = lo;
                    } else {
                        __nv_bfloat16 h[8], l[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            h[e] = __float2bfloat16_rn(x[e]);
                            l[e] = __float2bfloat16_rn(x[e] - __bfloat162float(h[e]));
                        }
                        *reinterpret_cast<uint4 *>(sm + L::oAhi + off) = *reinterpret_cast<const uint4 *>(h);
                        *reinterpret_cast<uint4 *>(sm + L::oAlo + off) = *reinterpret_cast<const uint4 *>(l);
                    }
                }
        };
        auto split_b = [&](int buf) {
            unsigned char *raw = sm + L::oRaw + buf * L::kRaw;
            if constexpr (FMT == kTcFmtTF32) {
                float4 *hv = reinterpret_cast<float4 *>(raw);
                float4 *lv = reinterpret_cast<float4 *>(sm + L::oBlo + buf * L::kB);
                for (int idx = wi; idx < a.nkb_raw * 256; idx += 128) {       // 16-byte chunks
                    const float4 x = hv[idx];
                    float4 hi;
                    hi.x = tf32_hi(x.x); hi.y = tf32_hi(x.y); hi.z = tf32_hi(x.z); hi.w = tf32_hi(x.w);
                    hv[idx] = hi;
                    lv[idx] = make_float4(x.x - hi.x, x.y - hi.y, x.z - hi.z, x.w - hi.w);
                }
            } else {
                unsigned char *bh = sm + TgLayout<kTcFmtBF16>::oBhi + buf * L::kB;
                unsigned char *bl = sm + L::oBlo + buf * L::kB;
                for (int idx = wi; idx < 2 * kTgN * 8; idx += 128) {         // (row n, bf16 block kb, chunk j)
                    const int n = idx >> 4, kb = (idx >> 3) & 1, j = idx & 7;
                    const int k0 = kb * 64 + j * 8;                           // 8 consecutive K of row n
                    const int rb = k0 >> 5, rc = (k0 & 31) >> 2;              // raw block and chunk
                    const float4 x0 = *reinterpret_cast<const float4 *>(raw + rb * 4096 + n * 128 + ((rc ^ (n & 7)) << 4));
                    const float4 x1 =
                        *reinterpret_cast<const float4 *>(raw + rb * 4096 + n * 128 + (((rc + 1) ^ (n & 7)) << 4));
                    const float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                    __nv_bfloat16 h[8], l[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        h[e] = __float2bfloat16_rn(x[e]);
                        l[e] = __float2bfloat16_rn(x[e] - __bfloat162float(h[e]));
                    }
                    const uint32_t off = (uint32_t)kb * 4096u + (uint32_t)n * 128u + ((uint32_t)(j ^ (n & 7)) << 4);
                    *reinterpret_cast<uint4 *>(bh + off) = *reinterpret_cast<const uint4 *>(h);
                    *reinterpret_cast<uint4 *>(bl + off) = *reinterpret_cast<const uint4 *>(l);
                }
            }
        };
        for (int i = 0; i < items && !failed; ++i) {
            const int buf = i & 1, t = i % a.ntiles;
            if (t == 0) {
                if (i > 0) epilogue(i - 1);                // every MMA of the previous bin has completed
                if (failed) break;
                build_a(binof(i));
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(a_ready);
            }
            if (!mbar_wait_bounded(&b_full[buf], (uint32_t)(i >> 1) & 1u, abort_flag, a.wait_ns)) {
                fail();
                failed = true;
            }
            failed = __any_sync(0xffffffffu, failed);
            if (failed) break;
            split_b(buf);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&split_done[buf]);
            if (t != 0) epilogue(i - 1);
        }
        if (items > 0 && !failed) epilogue(items - 1);
    }
    pdl_trigger();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kTgTmemCols);
    }
}

// ---------------------------------------------------------------- host side

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

bool tcgemm_fits(const Plan *p, int k) {
    return p->b % 2 == 0 && 2 * p->b <= 128 && k >= kTcMinCols && p->ubs % 2 == 0 && encode_fn() != nullptr;
}

int tcgemm_launch(Plan *p, int fmt_bf16, const void *u, void *v, int k) {
    if (!tcgemm_fits(p, k)) return set_error(p, BTTB_ERR_INVALID_ARG, "tensor-core product: b must be even and <= 64");
    if (!p->ghat_hi) return set_error(p, BTTB_ERR_INVALID_ARG, "plan does not keep the binary32 spectrum");
    const int b = p->b;
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * b), (cuuint64_t)k, (cuuint64_t)p->bins};
    const cuuint64_t strides[2] = {(cuuint64_t)b * 8, (cuuint64_t)p->ubs * 8};
    const cuuint32_t box[3] = {32, (cuuint32_t)kTgN, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult cr = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(u), dims, strides, box,
                                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return set_error(p, BTTB_ERR_CUDA, "cuTensorMapEncodeTiled failed for the product tile map");
    TgArgs a{};
    a.G = p->ghat_hi;
    a.gbs = p->gbs;
    a.v = reinterpret_cast<float *>(v);
    a.ubs = p->ubs;
    a.b = b;
    a.k = k;
    a.nbins = (int)p->bins;
    a.ntiles = (k + kTgN - 1) / kTgN;
    a.nkb_raw = (2 * b + 31) / 32;
    a.nks = fmt_bf16 ? (2 * b + 15) / 16 : (2 * b + 7) / 8;
    a.err = p->d_err;
    a.wait_ns = p->wait_ns;
    const size_t smem = (fmt_bf16 ? TgLayout<kTcFmtBF16>::oCtl : TgLayout<kTcFmtTF32>::oCtl) + 256 + 1024;
    auto kern = fmt_bf16 ? tcgemm_kernel<kTcFmtBF16> : tcgemm_kernel<kTcFmtTF32>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return check_cuda(p, e, "tensor-core product smem attribute");
    const int grid = (int)std::min<long>(p->bins, p->nsm);
    const int tok = prof_begin(p, BTTB_K_BLOCK_PRODUCT_PREC + (fmt_bf16 ? BTTB_MV_TC_BF16X3 : BTTB_MV_TC_3XTF32));
    e = launch_pdl(kern, dim3(grid), dim3(kTgThreads), smem, p->stream, map, a);
    count_launch(p);
    if (e != cudaSuccess) return check_cuda(p, e, "tensor-core product launch");
    prof_end(p, tok, (double)p->bins * ((double)b * b * 8 + 2.0 * k * b * 8));
    return check_cuda(p, cudaGetLastError(), "tensor-core product launch");
}

}  // namespace bttb
