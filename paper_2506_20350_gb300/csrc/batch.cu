// Batches of independent arrays of uneven sizes (nx, ny, b, number of
// right-hand sides).  Every array has its own plan on its own CUDA stream;
// a batch solve runs the arrays' restarted-GMRES drivers concurrently (one
// host thread per array), so the GPU executes the arrays' captured cycle
// graphs side by side.  An autotuner picks, per distinct (mx, my, b), the form
// of the product and the FFT batch-chunk width by timing products on the
// plan's stream (the same tuner serves single plans through
// bttb_plan_autotune).
#include <algorithm>
#include <map>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "arith.cuh"
#include "internal.h"

struct bttb_batch_s {
    int count = 0;
    std::vector<bttb_plan> plans;
    std::vector<cudaStream_t> streams;
    std::vector<int> nrhs;
};

using namespace bttb;

static int batch_release(bttb_batch b) {
    if (!b) return BTTB_OK;
    for (bttb_plan p : b->plans) bttb_plan_destroy(p);
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    delete b;
    return BTTB_OK;
}

extern "C" {

int bttb_batch_create(bttb_batch *out, int count, const int *nx, const int *ny, const int *b, const int *nrhs,
                      unsigned prec_mask) {
    if (!out) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (count < 1 || count > 4096 || !nx || !ny || !b || !nrhs)
        return set_error(nullptr, BTTB_ERR_INVALID_ARG, "need 1 <= count <= 4096 and size arrays");
    bttb_batch h = new (std::nothrow) bttb_batch_s();
    if (!h) return set_error(nullptr, BTTB_ERR_OOM, "host allocation failed");
    h->count = count;
    h->plans.assign(count, nullptr);
    h->streams.assign(count, nullptr);
    h->nrhs.assign(nrhs, nrhs + count);
    for (int i = 0; i < count; ++i) {
        // Blocking streams: work the caller queued on the legacy default stream (where
        // frameworks usually build inputs) completes before the array's kernels run.
        cudaError_t e = cudaStreamCreateWithFlags(&h->streams[i], cudaStreamDefault);
        if (e != cudaSuccess) {
            batch_release(h);
            return check_cuda(nullptr, e, "batch stream");
        }
        const int rc = bttb_plan_create(&h->plans[i], nx[i], ny[i], b[i], nrhs[i], prec_mask, h->streams[i]);
        if (rc != BTTB_OK) {
            batch_release(h);
            return rc;
        }
        h->plans[i]->p.in_batch = true;
    }
    *out = h;
    return BTTB_OK;
}

int bttb_batch_plan(bttb_batch batch, int index, bttb_plan *out) {
    if (!batch || !out || index < 0 || index >= batch->count)
        return set_error(nullptr, BTTB_ERR_INVALID_ARG, "bad batch, index or out");
    *out = batch->plans[index];
    return BTTB_OK;
}

int bttb_batch_set_generators(bttb_batch batch, int index, const void *gen, bttb_dtype dtype, int gen_is_host) {
    if (!batch || index < 0 || index >= batch->count)
        return set_error(nullptr, BTTB_ERR_INVALID_ARG, "bad batch or index");
    return bttb_set_generators(batch->plans[index], gen, dtype, gen_is_host);
}

// Times `reps` products of `nrhs` columns of precision `prec` on the plan's stream (after one warm-up).
static float time_products(Plan &p, void *x, void *y, int nrhs, int prec, int reps, cudaEvent_t e0, cudaEvent_t e1) {
    const int fmt = prec == PREC_F32 ? FMT_C64 : FMT_C128;
    if (matvec_run(&p, x, fmt, p.n, y, fmt, p.n, nrhs, prec) != BTTB_OK) return 1e30f;
    cudaEventRecord(e0, p.stream);
    for (int r = 0; r < reps; ++r)
        if (matvec_run(&p, x, fmt, p.n, y, fmt, p.n, nrhs, prec) != BTTB_OK) return 1e30f;
    cudaEventRecord(e1, p.stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
}

// Autotuner: for products of `nrhs` columns, times every form of the product that applies to the plan (all
// of them give the strided passes' bits): the strided passes and the fused level-2 kernel, whose x passes
// are strided, with each FFT batch-chunk width in {2, 4, ..., 64}; the fused two-level FFT; the persistent
// kernel; in binary32, and keeps the fastest form and width (a form other than the strided passes only if
// it beats them by 2%); then times those forms of the double-float product (FP64 plans) with that width and
// keeps the fastest the same way.  Returns the width (or a negative status).
static int autotune_plan(Plan &p, int nrhs, int reps) {
    const int widths[6] = {2, 4, 8, 16, 32, 64};
    void *x = nullptr, *y = nullptr;
    const size_t bytes = (size_t)nrhs * p.n * sizeof(double2);
    cudaError_t e = dev_malloc((void **)&x, bytes);
    if (e == cudaSuccess) e = dev_malloc((void **)&y, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, bytes, p.stream);
    if (e != cudaSuccess) {
        cudaFree(x);
        cudaFree(y);
        return check_cuda(&p, e, "autotune buffers");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    int best_w = p.fft_pmax, best_r = ROUTE_PASSES;
    for (int route : {ROUTE_PASSES, ROUTE_FUSED_Y, ROUTE_FUSED_FFT2, ROUTE_PERSISTENT}) {
        p.route_f32 = route;
        if (product_route(&p, nrhs, PREC_F32) != route) continue;          // this form does not apply here
        const bool uses_width = route == ROUTE_PASSES || route == ROUTE_FUSED_Y;
        for (int w : widths) {
            if (!uses_width && w != widths[0]) break;
            p.fft_pmax = w;
            const float ms = time_products(p, x, y, nrhs, PREC_F32, reps, e0, e1);
            // another form than the strided passes has to be faster by 2%, so that timing noise does not
            // flip the choice between forms that tie
            if (ms < best_ms * (route == ROUTE_PASSES || best_r != ROUTE_PASSES ? 1.f : 0.98f)) {
                best_ms = ms;
                best_w = w;
                best_r = route;
            }
        }
    }
    p.fft_pmax = best_w;
    p.route_f32 = best_r;
    if (p.ghat_lo) {                                                     // the double-float product's form
        float best_df = 1e30f;
        int best_rd = ROUTE_AUTO;
        for (int route : {ROUTE_PASSES, ROUTE_FUSED_Y, ROUTE_FUSED_FFT2, ROUTE_PERSISTENT}) {
            p.route_df = route;
            if (product_route(&p, nrhs, PREC_DF64) != route) continue;
            const float ms = time_products(p, x, y, nrhs, PREC_DF64, reps, e0, e1);
            if (ms < best_df * (route == ROUTE_PASSES || best_rd != ROUTE_PASSES ? 1.f : 0.98f)) {
                best_df = ms;
                best_rd = route;
            }
        }
        p.route_df = best_rd;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(y);
    e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(&p, e, "autotune");
    return best_w;
}

int bttb_plan_autotune(bttb_plan plan, int nrhs, int reps, int *chosen_out) {
    if (!plan) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = plan->p;
    if (!p.have_gen || !p.ghat_hi) return set_error(&p, BTTB_ERR_NO_GENERATORS, "autotune needs the binary32 spectrum");
    if (nrhs < 1 || nrhs > p.max_rhs) return set_error(&p, BTTB_ERR_INVALID_ARG, "nrhs out of range [1, max_rhs]");
    const int r = autotune_plan(p, nrhs, reps < 1 ? 1 : reps);
    if (r < 0) return r;
    if (chosen_out) *chosen_out = r;
    gmres_free(&p);                          // captured cycles keep the old launch shapes
    return BTTB_OK;
}

int bttb_batch_autotune(bttb_batch batch, int reps, int *chosen_out) {
    if (!batch) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "batch is NULL");
    if (reps < 1) reps = 1;
    std::map<std::tuple<int, int, int>, std::pair<int, int>> best;   // shape -> (width, tuned plan)
    for (int i = 0; i < batch->count; ++i) {
        Plan &p = batch->plans[i]->p;
        if (!p.have_gen || !p.ghat_hi) continue;
        const auto key = std::make_tuple(p.mx, p.my, p.b);
        if (best.count(key)) continue;
        const int r = autotune_plan(p, 1, reps);
        if (r < 0) return r;
        best[key] = std::make_pair(r, i);
        gmres_free(&p);
    }
    for (int i = 0; i < batch->count; ++i) {
        Plan &p = batch->plans[i]->p;
        const auto it = best.find(std::make_tuple(p.mx, p.my, p.b));
        if (it != best.end()) {
            const Plan &src = batch->plans[it->second.second]->p;
            if (it->second.first != p.fft_pmax || src.route_f32 != p.route_f32 || src.route_df != p.route_df) {
                p.fft_pmax = it->second.first;
                p.route_f32 = src.route_f32;
                p.route_df = src.route_df;
                gmres_free(&p);
            }
        }
        if (chosen_out) chosen_out[i] = p.fft_pmax;
    }
    return BTTB_OK;
}

int bttb_batch_gmres_solve(bttb_batch batch, const void *const *V, void *const *I, const long *ld,
                           const bttb_gmres_opts *opts, bttb_col_result *out_host) {
    if (!batch || !V || !I || !ld || !opts) return set_error(nullptr, BTTB_ERR_INVALID_ARG, "NULL argument");
    const int n = batch->count;
    std::vector<int> rcs(n, BTTB_OK);
    std::vector<std::string> msgs(n);
    std::vector<long> off(n + 1, 0);
    for (int i = 0; i < n; ++i) off[i + 1] = off[i] + batch->nrhs[i];
    int dev = 0;
    cudaGetDevice(&dev);
    // Inputs may come from any stream: let everything already queued finish first.
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return check_cuda(nullptr, e, "batch solve: device synchronise");
    std::vector<std::thread> th;
    th.reserve(n);
    for (int i = 0; i < n; ++i) {
        th.emplace_back([&, i]() {
            cudaSetDevice(dev);
            bttb_gmres_opts o = *opts;
            o.history = nullptr;
            o.history_len = 0;
            rcs[i] = bttb_gmres_solve(batch->plans[i], V[i], I[i], batch->nrhs[i], ld[i], &o,
                                      out_host ? out_host + off[i] : nullptr);
            if (rcs[i] < 0) msgs[i] = bttb_last_error(batch->plans[i]);
        });
    }
    for (auto &t : th) t.join();
    int worst = BTTB_OK;
    for (int i = 0; i < n; ++i) {
        if (rcs[i] < 0 && (worst >= 0 || rcs[i] < worst)) {
            worst = rcs[i];
            set_error(nullptr, rcs[i], "array " + std::to_string(i) + ": " + msgs[i]);
        } else if (worst >= 0 && rcs[i] > worst) {
            worst = rcs[i];
        }
    }
    return worst;
}

int bttb_batch_destroy(bttb_batch batch) { return batch_release(batch); }

}  // extern "C"
