// Bounds-checked build (compiled with -DBTTB_CHECKED=1 into a separate library): every checked global
// access must lie inside one registered device buffer (the plans' allocations and the caller's device
// buffers of the current calls), every checked shared access inside the CTA's dynamic shared memory (or
// below it, in the static part), and every checked index inside its buffer's length.  A check that fails
// counts a hit, records the first bad address and skips the access, so nothing is read or written out of
// bounds; the host reads the count back with bttb_check_report.  In the normal build every check is the
// constant true and compiles away.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace bttb {

#ifdef BTTB_CHECKED

constexpr int kCheckRegions = 1024;

// Device-side state shared by every translation unit (one allocation; each unit holds a pointer to it).
struct CheckState {
    int nregions;
    int pad;
    unsigned long long hits;                  // failed checks
    unsigned long long first;                 // first bad address (0: none)
    unsigned long long lo[kCheckRegions];     // region i: [lo[i], hi[i])
    unsigned long long hi[kCheckRegions];
};

// Host side (check.cu): every translation unit registers a setter of its state pointer at load time.
void check_register_unit(void (*set_state)(CheckState *));
// Host side: a device buffer that kernels may access (tracked until an allocation at the same address
// replaces it).
void check_track(const void *p, size_t bytes);

// Everything below is local to each translation unit (its own copy of the state pointer).
namespace {
__device__ CheckState *g_chk = nullptr;
void chk_set_state(CheckState *s) { cudaMemcpyToSymbol(g_chk, &s, sizeof(s)); }
struct ChkUnit {
    ChkUnit() { check_register_unit(chk_set_state); }
};
ChkUnit g_chk_unit;

__device__ __noinline__ bool chk_fail(unsigned long long addr) {
    CheckState *s = g_chk;
    if (s) {
        atomicAdd(&s->hits, 1ull);
        atomicCAS(&s->first, 0ull, addr);
    }
    return false;
}

__device__ __noinline__ bool chk_shared(const void *p, size_t bytes);

// A generic pointer: into shared memory (some helpers take either kind), else a tracked global buffer.
__device__ __noinline__ bool chk_global(const void *p, size_t bytes) {
    if (__isShared(p)) return chk_shared(p, bytes);
    const CheckState *s = g_chk;
    if (!s) return true;                      // state not set up: nothing to check against
    const unsigned long long a = reinterpret_cast<unsigned long long>(p), e = a + bytes;
    const int n = s->nregions;
    for (int i = 0; i < n; ++i)
        if (a >= s->lo[i] && e <= s->hi[i]) return true;
    return chk_fail(a);
}

__device__ __noinline__ bool chk_shared(const void *p, size_t bytes) {
    extern __shared__ unsigned char chk_dyn_base[];
    unsigned dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    const unsigned lo = (unsigned)__cvta_generic_to_shared(chk_dyn_base);
    if (a + bytes <= lo) return true;          // static shared memory
    if (a >= lo && a + bytes <= lo + dyn) return true;
    return chk_fail(0x5000000000000000ull | a);
}

// An index into a buffer of n elements (shared-memory buffers of a known length, remote shared memory).
__device__ __forceinline__ bool chk_index(long long i, long long n) {
    return (i >= 0 && i < n) || chk_fail(0x6000000000000000ull | (unsigned long long)(i & 0xffffffffffffll));
}
}  // namespace

#define BTTB_GCHK(p, n) ::bttb::chk_global((p), (n))
#define BTTB_SCHK(p, n) ::bttb::chk_shared((p), (n))
#define BTTB_ICHK(i, n) ::bttb::chk_index((i), (n))

#else

#define BTTB_GCHK(p, n) true
#define BTTB_SCHK(p, n) true
#define BTTB_ICHK(i, n) true
inline void check_track(const void *, size_t) {}

#endif

// The caller's device multi-vector of nrhs columns of n elements (esz bytes each), column stride ld.
inline void check_track_cols(const void *p, long nrhs, long ld, long n, size_t esz) {
    if (p && nrhs > 0) check_track(p, ((size_t)(nrhs - 1) * ld + n) * esz);
}

// cudaMalloc that also tracks the buffer in the bounds-checked build.
inline cudaError_t dev_malloc(void **p, size_t bytes) {
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) check_track(*p, bytes);
    return e;
}

// Checked element load and store through a global pointer (plain accesses in the normal build).
template <class T>
__device__ __forceinline__ T gld(const T *p) {
    return BTTB_GCHK(p, sizeof(T)) ? *p : T{};
}
template <class T>
__device__ __forceinline__ void gst(T *p, const T &v) {
    if (BTTB_GCHK(p, sizeof(T))) *p = v;
}
// Checked load that bypasses L1 (data another CTA of the same launch wrote).
template <class T>
__device__ __forceinline__ T gldcg(const T *p) {
    return BTTB_GCHK(p, sizeof(T)) ? __ldcg(p) : T{};
}
// Checked element load and store through a pointer into this CTA's shared memory.
template <class T>
__device__ __forceinline__ T sld(const T *p) {
    return BTTB_SCHK(p, sizeof(T)) ? *p : T{};
}
template <class T>
__device__ __forceinline__ void sst(T *p, const T &v) {
    if (BTTB_SCHK(p, sizeof(T))) *p = v;
}

}  // namespace bttb
