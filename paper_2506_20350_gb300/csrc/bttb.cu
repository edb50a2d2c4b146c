// C ABI of libbttb: plan lifecycle, argument checks and error reporting.
// The arithmetic lives in fft.cu, contract.cu, matvec.cu and gmres.cu.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "arith.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace bttb {

static thread_local std::string g_last_error = "no error";

int set_error(Plan *, int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int check_cuda(Plan *p, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return BTTB_OK;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return set_error(p, e == cudaErrorMemoryAllocation ? BTTB_ERR_OOM : BTTB_ERR_CUDA, m);
}

constexpr int kSinkToken = 1 << 30;

int prof_begin(Plan *p, int kid) {
    if (!p->prof) return -1;
    if (p->sink) {
        if (kid < BTTB_K_BLOCK_PRODUCT_PREC && p->prof < 2) return -1;   // level 1: only the block product in graphs
        Plan::GraphRec r{nullptr, nullptr, kid, 0.0, p->sink_step};
        if (cudaEventCreate(&r.e0) != cudaSuccess || cudaEventCreate(&r.e1) != cudaSuccess) return -1;
        // External: captured as an event-record node that timestamps every replay
        cudaEventRecordWithFlags(r.e0, p->stream, cudaEventRecordExternal);
        p->sink->push_back(r);
        return kSinkToken + (int)p->sink->size() - 1;
    }
    if (p->ev_used + 2 > (int)p->ev_pool.size()) {
        for (int i = 0; i < 64; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            p->ev_pool.push_back(e);
        }
    }
    const int e0 = p->ev_used, e1 = p->ev_used + 1;
    p->ev_used += 2;
    cudaEventRecord(p->ev_pool[e0], p->stream);
    p->recs.push_back(Plan::ProfRec{e0, e1, kid, 0.0});
    return (int)p->recs.size() - 1;
}

void prof_end(Plan *p, int token, double bytes) {
    if (token < 0 || !p->prof) return;
    if (token >= kSinkToken) {
        Plan::GraphRec &r = (*p->sink)[token - kSinkToken];
        r.bytes = bytes;
        cudaEventRecordWithFlags(r.e1, p->stream, cudaEventRecordExternal);
        return;
    }
    Plan::ProfRec &r = p->recs[token];
    r.bytes = bytes;
    cudaEventRecord(p->ev_pool[r.ev1], p->stream);
}

static bool prec_enabled(const Plan &p, int prec) {
    switch (prec) {
        case BTTB_MV_FP64: return p.ghat_hi && p.ghat_lo;
        case BTTB_MV_FP32: return p.ghat_hi != nullptr;
        case BTTB_MV_FP64_NATIVE: return p.ghat_f64 != nullptr;
        case BTTB_MV_TC_3XTF32:
        case BTTB_MV_TC_BF16X3: return p.ghat_hi != nullptr;
        default: return false;
    }
}

static void plan_release(Plan &p) {
    gmres_free(&p);
    for (cudaEvent_t e : p.ev_pool) cudaEventDestroy(e);
    p.ev_pool.clear();
    fft_plan_free(p.fx);
    fft_plan_free(p.fy);
    cudaFree(p.ghat_hi);
    cudaFree(p.ghat_lo);
    cudaFree(p.ghat_f64);
    cudaFree(p.bj_inv);
    cudaFree(p.wsA);
    cudaFree(p.wsB);
    cudaFree(p.d_err);
    p.ghat_hi = p.ghat_lo = nullptr;
    p.ghat_f64 = nullptr;
    p.bj_inv = nullptr;
    p.wsA = p.wsB = nullptr;
    p.d_err = nullptr;
    p.d_gbar = nullptr;
}

}  // namespace bttb

using namespace bttb;

extern "C" {

int bttb_plan_create(bttb_plan *out, int nx, int ny, int b, int max_rhs, unsigned prec_mask, void *cuda_stream) {
    if (!out) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || b < 1 || max_rhs < 1 || nx > 1024 || ny > 1024 || b > 256 || max_rhs > 4096)
        return set_error(nullptr, BTTB_ERR_INVALID_ARG,
                         "sizes must satisfy 1 <= nx, ny <= 1024, 1 <= b <= 256, 1 <= max_rhs <= 4096");
    if (prec_mask == 0) prec_mask = (1u << BTTB_MV_FP64) | (1u << BTTB_MV_FP32);
    if (prec_mask & ~((1u << BTTB_MV_FP64) | (1u << BTTB_MV_FP32) | (1u << BTTB_MV_FP64_NATIVE) |
                      (1u << BTTB_MV_TC_3XTF32) | (1u << BTTB_MV_TC_BF16X3)))
        return set_error(nullptr, BTTB_ERR_INVALID_ARG, "unknown bit in prec_mask");
    bttb_plan h = new (std::nothrow) bttb_plan_s();
    if (!h) return set_error(nullptr, BTTB_ERR_OOM, "host allocation failed");
    Plan &p = h->p;
    p.nx = nx;
    p.ny = ny;
    p.b = b;
    p.max_rhs = max_rhs;
    p.prec_mask = prec_mask;
    p.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    p.n = (long)nx * ny * b;
    p.mx = smallest_5smooth(2 * nx - 1);
    p.my = smallest_5smooth(2 * ny - 1);
    p.bins = (long)p.mx * p.my;
    int rc = BTTB_OK;
    cudaError_t e;
    auto bail = [&](int code) {
        plan_release(p);
        delete h;
        return code;
    };
    if (p.mx > kMaxM || p.my > kMaxM) return bail(set_error(nullptr, BTTB_ERR_INVALID_ARG, "FFT grid too large"));
    if ((e = cudaGetDevice(&p.dev)) != cudaSuccess) return bail(check_cuda(nullptr, e, "cudaGetDevice"));
    cudaDeviceGetAttribute(&p.nsm, cudaDevAttrMultiProcessorCount, p.dev);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p.dev);
    p.smem_optin = (size_t)optin;
    if ((rc = fft_plan_init(&p, p.fx, p.mx)) != BTTB_OK) return bail(rc);
    if (p.my == p.mx) {
        p.fy = p.fx;                       // share tables; freed once
        p.fy.tw_f64 = nullptr;
        p.fy.tw_df = nullptr;
        p.fy.tw_f32 = nullptr;
        p.fy.M = -1;                       // lookups fall back to fx when my == mx
    } else if ((rc = fft_plan_init(&p, p.fy, p.my)) != BTTB_OK) {
        return bail(rc);
    }
    p.gbs = ((long)b * b + 1) / 2 * 2;
    const size_t gplane = (size_t)p.bins * p.gbs;
    auto alloc = [&](void **ptr, size_t bytes, const char *what) -> int {
        cudaError_t ee = dev_malloc(ptr, bytes);
        if (ee != cudaSuccess) return check_cuda(&p, ee, what);
        p.bytes_held += bytes;
        return BTTB_OK;
    };
    if (prec_mask & ((1u << BTTB_MV_FP64) | (1u << BTTB_MV_FP32) | (1u << BTTB_MV_TC_3XTF32) | (1u << BTTB_MV_TC_BF16X3)))
        if ((rc = alloc((void **)&p.ghat_hi, gplane * sizeof(float2), "spectrum hi plane")) != BTTB_OK) return bail(rc);
    if (prec_mask & (1u << BTTB_MV_FP64))
        if ((rc = alloc((void **)&p.ghat_lo, gplane * sizeof(float2), "spectrum lo plane")) != BTTB_OK) return bail(rc);
    if (prec_mask & (1u << BTTB_MV_FP64_NATIVE))
        if ((rc = alloc((void **)&p.ghat_f64, gplane * sizeof(double2), "spectrum binary64 copy")) != BTTB_OK)
            return bail(rc);
    p.ubs = ((long)max_rhs * b + 1) / 2 * 2;
    p.ws_bytes = (size_t)p.bins * p.ubs * 16;
    if ((rc = alloc(&p.wsA, p.ws_bytes, "product workspace")) != BTTB_OK) return bail(rc);
    if ((rc = alloc(&p.wsB, p.ws_bytes, "product workspace")) != BTTB_OK) return bail(rc);
    if ((rc = alloc((void **)&p.d_err, 64, "error word")) != BTTB_OK) return bail(rc);
    if ((e = cudaMemset(p.d_err, 0, 64)) != cudaSuccess) return bail(check_cuda(&p, e, "error word"));
    p.d_gbar = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(p.d_err) + 16);
    *out = h;
    return BTTB_OK;
}

int bttb_plan_grid(bttb_plan plan, int *mx, int *my) {
    if (!plan) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "plan is NULL");
    if (mx) *mx = plan->p.mx;
    if (my) *my = plan->p.my;
    return BTTB_OK;
}

int bttb_set_generators(bttb_plan plan, const void *gen, bttb_dtype dtype, int gen_is_host) {
    if (!plan || !gen) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "plan or gen is NULL");
    if (dtype != BTTB_C64 && dtype != BTTB_C128) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "bad dtype");
    Plan &p = plan->p;
    p.have_gen = false;
    if (!gen_is_host) {
        // A device generator buffer may have been produced on any stream.
        cudaError_t e0 = cudaDeviceSynchronize();
        if (e0 != cudaSuccess) return check_cuda(&p, e0, "set_generators: device synchronise");
    }
    if (!gen_is_host)
        check_track(gen, (size_t)(2 * p.nx - 1) * (2 * p.ny - 1) * p.b * p.b * (dtype == BTTB_C128 ? 16 : 8));
    cudaMemsetAsync(p.d_err, 0, sizeof(int), p.stream);
    int rc = spectrum_compute(&p, gen, dtype, gen_is_host);
    if (rc != BTTB_OK) return rc;
    int err = 0;
    cudaError_t e = cudaMemcpy(&err, p.d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return check_cuda(&p, e, "error word");
    if (err & DEVERR_NONFINITE) {
        cudaMemset(p.d_err, 0, sizeof(int));
        return set_error(&p, BTTB_ERR_NONFINITE, "generators or their spectrum hold NaN/Inf");
    }
    // Self block T[0,0] for the block-Jacobi preconditioner.
    const int b = p.b;
    const long off = ((long)(p.ny - 1) * (2 * p.nx - 1) + (p.nx - 1)) * b * b;
    std::vector<double2> t00((size_t)b * b);
    if (dtype == BTTB_C128) {
        const double2 *src = reinterpret_cast<const double2 *>(gen) + off;
        if (gen_is_host) std::memcpy(t00.data(), src, sizeof(double2) * b * b);
        else if ((e = cudaMemcpy(t00.data(), src, sizeof(double2) * b * b, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return check_cuda(&p, e, "T[0,0] copy");
    } else {
        std::vector<float2> tf((size_t)b * b);
        const float2 *src = reinterpret_cast<const float2 *>(gen) + off;
        if (gen_is_host) std::memcpy(tf.data(), src, sizeof(float2) * b * b);
        else if ((e = cudaMemcpy(tf.data(), src, sizeof(float2) * b * b, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return check_cuda(&p, e, "T[0,0] copy");
        for (long i = 0; i < (long)b * b; ++i) t00[i] = make_double2(tf[i].x, tf[i].y);
    }
    block_jacobi_setup(&p, t00.data());   // failure only disables the preconditioner
    p.have_gen = true;
    return BTTB_OK;
}

int bttb_matvec(bttb_plan plan, const void *x, void *y, int nrhs, long ld, bttb_dtype dtype, bttb_mv_prec prec) {
    if (!plan) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = plan->p;
    if (!p.have_gen) return set_error(&p, BTTB_ERR_NO_GENERATORS, "bttb_set_generators has not succeeded");
    if (nrhs < 0 || nrhs > p.max_rhs) return set_error(&p, BTTB_ERR_INVALID_ARG, "nrhs out of range [0, max_rhs]");
    if (nrhs == 0) return BTTB_OK;
    if (!x || !y) return set_error(&p, BTTB_ERR_INVALID_ARG, "x or y is NULL");
    if (ld < p.n) return set_error(&p, BTTB_ERR_INVALID_ARG, "ld < N");
    if (dtype != BTTB_C64 && dtype != BTTB_C128) return set_error(&p, BTTB_ERR_INVALID_ARG, "bad dtype");
    if (!prec_enabled(p, prec)) return set_error(&p, BTTB_ERR_INVALID_ARG, "precision not enabled in this plan");
    const int fmt = dtype == BTTB_C128 ? FMT_C128 : FMT_C64;
    check_track_cols(x, nrhs, ld, p.n, dtype == BTTB_C128 ? 16 : 8);
    check_track_cols(y, nrhs, ld, p.n, dtype == BTTB_C128 ? 16 : 8);
    return matvec_run(&p, x, fmt, ld, y, fmt, ld, nrhs, (int)prec);
}

int bttb_block_jacobi_apply(bttb_plan plan, const void *x, void *z, int nrhs, long ld, bttb_dtype dtype) {
    if (!plan) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = plan->p;
    if (!p.have_gen) return set_error(&p, BTTB_ERR_NO_GENERATORS, "bttb_set_generators has not succeeded");
    if (!p.bj_ready) return set_error(&p, BTTB_ERR_SINGULAR, "T[0,0] is singular: no block-Jacobi preconditioner");
    if (nrhs < 0 || ld < p.n || (nrhs > 0 && (!x || !z)))
        return set_error(&p, BTTB_ERR_INVALID_ARG, "bad nrhs, ld or pointer");
    if (nrhs == 0) return BTTB_OK;
    const int fmt = dtype == BTTB_C128 ? FMT_C128 : FMT_C64;
    check_track_cols(x, nrhs, ld, p.n, dtype == BTTB_C128 ? 16 : 8);
    check_track_cols(z, nrhs, ld, p.n, dtype == BTTB_C128 ? 16 : 8);
    return block_jacobi_run(&p, x, fmt, ld, z, fmt, ld, nrhs);
}

int bttb_gmres_solve(bttb_plan plan, const void *V, void *I, int nrhs, long ld, const bttb_gmres_opts *opts,
                     bttb_col_result *out_host) {
    if (!plan || !opts) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "plan or opts is NULL");
    Plan &p = plan->p;
    if (!p.have_gen) return set_error(&p, BTTB_ERR_NO_GENERATORS, "bttb_set_generators has not succeeded");
    if (nrhs < 1 || nrhs > p.max_rhs) return set_error(&p, BTTB_ERR_INVALID_ARG, "nrhs out of range [1, max_rhs]");
    if (!V || !I || ld < p.n) return set_error(&p, BTTB_ERR_INVALID_ARG, "bad V, I or ld");
    if (!(opts->tol > 0.0) || opts->restart < 1 || opts->restart > 200 || opts->max_iters < 0)
        return set_error(&p, BTTB_ERR_INVALID_ARG, "need tol > 0, 1 <= restart <= 200, max_iters >= 0");
    if (opts->pc != BTTB_PC_NONE && opts->pc != BTTB_PC_BLOCK_JACOBI && opts->pc != BTTB_PC_LEARNED)
        return set_error(&p, BTTB_ERR_INVALID_ARG, "unknown preconditioner");
    if (opts->pc != BTTB_PC_NONE && !p.bj_ready)
        return set_error(&p, BTTB_ERR_SINGULAR, "T[0,0] is singular: no block-Jacobi preconditioner");
    if (opts->pc == BTTB_PC_LEARNED && (!p.learned || nrhs > learned_max_cols(p.learned)))
        return set_error(&p, BTTB_ERR_INVALID_ARG,
                         "BTTB_PC_LEARNED needs an attached learned object with max_cols >= nrhs");
    if (!prec_enabled(p, opts->inner)) return set_error(&p, BTTB_ERR_INVALID_ARG, "inner precision not enabled");
    if (!prec_enabled(p, BTTB_MV_FP64))
        return set_error(&p, BTTB_ERR_INVALID_ARG, "GMRES needs the FP64 (double-float) spectrum for its residuals");
    if (!opts->host_io) {
        check_track_cols(V, nrhs, ld, p.n, 16);
        check_track_cols(I, nrhs, ld, p.n, 16);
    }
    cudaMemsetAsync(p.d_err, 0, sizeof(int), p.stream);
    return gmres_solve(&p, V, I, nrhs, ld, opts, out_host);
}

int bttb_get_spectrum_bin(bttb_plan plan, int ky, int kx, double *out_host) {
    if (!plan || !out_host) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "plan or out is NULL");
    Plan &p = plan->p;
    if (!p.have_gen) return set_error(&p, BTTB_ERR_NO_GENERATORS, "bttb_set_generators has not succeeded");
    if (ky < 0 || ky >= p.my || kx < 0 || kx >= p.mx) return set_error(&p, BTTB_ERR_INVALID_ARG, "bin out of range");
    const int b = p.b;
    const long bin = (long)ky * p.mx + kx;
    cudaError_t e = cudaStreamSynchronize(p.stream);
    if (e != cudaSuccess) return check_cuda(&p, e, "sync");
    std::vector<double2> v((size_t)b * b);
    if (p.ghat_f64) {
        e = cudaMemcpy(v.data(), p.ghat_f64 + bin * p.gbs, sizeof(double2) * b * b, cudaMemcpyDeviceToHost);
    } else {
        std::vector<float2> hi((size_t)b * b), lo((size_t)b * b, make_float2(0.f, 0.f));
        e = cudaMemcpy(hi.data(), p.ghat_hi + bin * p.gbs, sizeof(float2) * b * b, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && p.ghat_lo)
            e = cudaMemcpy(lo.data(), p.ghat_lo + bin * p.gbs, sizeof(float2) * b * b, cudaMemcpyDeviceToHost);
        for (long i = 0; i < (long)b * b; ++i)
            v[i] = make_double2((double)hi[i].x + lo[i].x, (double)hi[i].y + lo[i].y);
    }
    if (e != cudaSuccess) return check_cuda(&p, e, "spectrum copy");
    for (int pr = 0; pr < b; ++pr)
        for (int q = 0; q < b; ++q) {
            const double2 t = v[(size_t)q * b + pr];      // stored column-major
            out_host[2 * ((size_t)pr * b + q)] = t.x;
            out_host[2 * ((size_t)pr * b + q) + 1] = t.y;
        }
    return BTTB_OK;
}

int bttb_profile(bttb_plan plan, int enable) {
    if (!plan) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = plan->p;
    if (enable) {
        cudaStreamSynchronize(p.stream);
        p.recs.clear();
        p.ev_used = 0;
        p.launches = 0;
        for (int i = 0; i < Plan::kMaxKid; ++i) p.acc_ms[i] = p.acc_bytes[i] = 0.0, p.acc_n[i] = 0;
    }
    p.prof = enable < 0 ? 0 : (enable > 2 ? 2 : enable);
    return BTTB_OK;
}

int bttb_profile_read(bttb_plan plan, int which, bttb_kernel_stats *out) {
    if (!plan || !out) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "plan or out is NULL");
    Plan &p = plan->p;
    cudaError_t e = cudaStreamSynchronize(p.stream);
    if (e != cudaSuccess) return check_cuda(&p, e, "profile sync");
    out->ms = 0.0;
    out->launches = 0;
    out->bytes = 0.0;
    if (which == BTTB_K_ALL) {
        out->launches = p.launches;
        return BTTB_OK;
    }
    for (int kid = 0; kid < Plan::kMaxKid; ++kid) {
        const bool match = kid == which || (which == BTTB_K_BLOCK_PRODUCT && kid >= BTTB_K_BLOCK_PRODUCT_PREC);
        if (!match) continue;
        out->ms += p.acc_ms[kid];
        out->launches += p.acc_n[kid];
        out->bytes += p.acc_bytes[kid];
    }
    for (const Plan::ProfRec &r : p.recs) {
        const bool match = r.kid == which || (which == BTTB_K_BLOCK_PRODUCT && r.kid >= BTTB_K_BLOCK_PRODUCT_PREC);
        if (!match) continue;
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, p.ev_pool[r.ev0], p.ev_pool[r.ev1]);
        if (e != cudaSuccess) return check_cuda(&p, e, "profile event");
        out->ms += ms;
        out->launches += 1;
        out->bytes += r.bytes;
    }
    return BTTB_OK;
}

size_t bttb_plan_workspace_bytes(bttb_plan plan) { return plan ? plan->p.bytes_held : 0; }

int bttb_plan_debug(bttb_plan plan, int what, long long value) {
    if (!plan) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = plan->p;
    switch (what) {
        case BTTB_DEBUG_WAIT_LIMIT_NS:
            if (value < 0 || value > 60000000000ll)
                return set_error(&p, BTTB_ERR_INVALID_ARG, "wait limit must be in [0, 60 s] (0: the default)");
            p.wait_ns = value == 0 ? 2000000000ull : (unsigned long long)value;
            gmres_free(&p);                           // captured cycles hold the old limit
            return BTTB_OK;
        case BTTB_DEBUG_PRODUCT_ROUTE:
            if (value < 0 || value > 4) return set_error(&p, BTTB_ERR_INVALID_ARG, "route must be in [0, 4]");
            p.route_f32 = p.route_df = (int)value;
            gmres_free(&p);                           // captured cycles hold the old route
            return BTTB_OK;
        case BTTB_DEBUG_ROUTE_TAKEN: {
            const int prec = (int)(value >> 8), k = (int)(value & 255);
            if (prec < 0 || prec > BTTB_MV_TC_BF16X3 || k < 1 || k > p.max_rhs)
                return set_error(&p, BTTB_ERR_INVALID_ARG, "value must be (prec << 8) | nrhs, 1 <= nrhs <= max_rhs");
            return product_route(&p, k, prec);
        }
        case BTTB_DEBUG_FUSED_SHAPE: {
            const int prec = (int)((value >> 8) & 255), k = (int)(value & 255), Q = (int)((value >> 16) & 255);
            if ((prec != BTTB_MV_FP64 && prec != BTTB_MV_FP32) || k < 1 || k > 4 || Q > 8)
                return set_error(&p, BTTB_ERR_INVALID_ARG, "value must be (Q << 16) | (prec << 8) | nrhs");
            const int r = ycontract_probe(&p, prec, k, Q);
            return r < 0 ? set_error(&p, BTTB_ERR_INVALID_ARG, "shape does not fit: " + std::to_string(r)) : r;
        }
        case BTTB_DEBUG_FUSED_CLUSTER:
            if (value < 0 || value > 8) return set_error(&p, BTTB_ERR_INVALID_ARG, "cluster size must be in [0, 8]");
            p.yc_force_q = (int)value;
            for (auto &row : p.yc)
                for (auto &y : row) y = YcShape{};
            gmres_free(&p);
            return BTTB_OK;
        case BTTB_DEBUG_WITHHOLD_ARRIVAL:
            if (value < 0 || value > 1000) return set_error(&p, BTTB_ERR_INVALID_ARG, "count must be in [0, 1000]");
            p.withhold = (int)value;
            return BTTB_OK;
        default:
            return set_error(&p, BTTB_ERR_INVALID_ARG, "unknown debug hook");
    }
}

int bttb_plan_destroy(bttb_plan plan) {
    if (!plan) return BTTB_OK;
    plan_release(plan->p);
    delete plan;
    return BTTB_OK;
}

const char *bttb_last_error(bttb_plan) { return g_last_error.c_str(); }

}  // extern "C"
