// Host side of the bounds-checked build (check.cuh): the registry of device buffers that kernels may
// access, mirrored into one device-side table, and the report of failed checks.  In the normal build only
// the report entry points exist (they report that the library is not the checked build).
#include <mutex>
#include <vector>

#include "check.cuh"
#include "internal.h"

namespace bttb {

#ifdef BTTB_CHECKED
namespace {
std::mutex &reg_mutex() {
    static std::mutex m;
    return m;
}
std::vector<void (*)(CheckState *)> &reg_units() {
    static std::vector<void (*)(CheckState *)> v;
    return v;
}
CheckState *g_state = nullptr;                 // device table
std::vector<unsigned long long> g_lo, g_hi;    // host mirror
int g_evict = 0;

// The device table, allocated and zeroed once and handed to every translation unit (lock held).
bool state_ready() {
    if (g_state) return true;
    if (cudaMalloc(&g_state, sizeof(CheckState)) != cudaSuccess) {
        g_state = nullptr;
        return false;
    }
    if (cudaMemset(g_state, 0, sizeof(CheckState)) != cudaSuccess) return false;
    for (auto f : reg_units()) f(g_state);
    return true;
}

__global__ void check_probe_kernel(const float4 *past_end, float4 *sink) {
    // one element past the end of a tracked buffer: the check counts a hit and skips the load
    const float4 v = gld(past_end);
    gst(sink, v);
}
}  // namespace

void check_register_unit(void (*set_state)(CheckState *)) {
    std::lock_guard<std::mutex> g(reg_mutex());
    reg_units().push_back(set_state);
    if (g_state) set_state(g_state);
}

void check_track(const void *p, size_t bytes) {
    if (!p || !bytes) return;
    std::lock_guard<std::mutex> g(reg_mutex());
    if (!state_ready()) return;
    const unsigned long long lo = reinterpret_cast<unsigned long long>(p), hi = lo + bytes;
    int slot = -1;
    for (size_t i = 0; i < g_lo.size(); ++i)
        if (g_lo[i] == lo) slot = (int)i;      // an allocation at the same address replaces the old one
    if (slot < 0) {
        if ((int)g_lo.size() < kCheckRegions) {
            slot = (int)g_lo.size();
            g_lo.push_back(0);
            g_hi.push_back(0);
        } else {
            slot = g_evict++ % kCheckRegions;  // the oldest entries make room
        }
    }
    g_lo[slot] = lo;
    g_hi[slot] = hi;
    // the entry first, then the count, so that a kernel reading the table sees only complete entries
    cudaMemcpy(&g_state->lo[slot], &lo, sizeof(lo), cudaMemcpyHostToDevice);
    cudaMemcpy(&g_state->hi[slot], &hi, sizeof(hi), cudaMemcpyHostToDevice);
    const int n = (int)g_lo.size();
    cudaMemcpy(&g_state->nregions, &n, sizeof(n), cudaMemcpyHostToDevice);
}
#endif

}  // namespace bttb

using namespace bttb;

extern "C" int bttb_check_report(unsigned long long *hits, unsigned long long *first_addr) {
    if (hits) *hits = 0;
    if (first_addr) *first_addr = 0;
#ifdef BTTB_CHECKED
    std::lock_guard<std::mutex> g(reg_mutex());
    if (!state_ready()) return set_error(nullptr, BTTB_ERR_CUDA, "bounds-check table");
    cudaError_t e = cudaDeviceSynchronize();
    unsigned long long h = 0, f = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, &g_state->hits, sizeof(h), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&f, &g_state->first, sizeof(f), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return check_cuda(nullptr, e, "bounds-check report");
    if (hits) *hits = h;
    if (first_addr) *first_addr = f;
    return 1;
#else
    return 0;
#endif
}

extern "C" int bttb_check_probe(unsigned long long *hits_added) {
    if (hits_added) *hits_added = 0;
#ifdef BTTB_CHECKED
    float4 *buf = nullptr;
    cudaError_t e = dev_malloc((void **)&buf, 4 * sizeof(float4));
    if (e != cudaSuccess) return check_cuda(nullptr, e, "bounds-check probe buffer");
    unsigned long long h0 = 0, h1 = 0;
    int rc = bttb_check_report(&h0, nullptr);
    if (rc == 1) {
        check_probe_kernel<<<1, 1>>>(buf + 4, buf);
        e = cudaGetLastError();
        rc = e == cudaSuccess ? bttb_check_report(&h1, nullptr) : check_cuda(nullptr, e, "bounds-check probe");
    }
    cudaFree(buf);
    if (rc != 1) return rc;
    if (hits_added) *hits_added = h1 - h0;
    return BTTB_OK;
#else
    return set_error(nullptr, BTTB_ERR_INVALID_ARG, "not the bounds-checked build");
#endif
}
