// Inline-PTX wrappers for the fifth-generation tensor cores (tcgen05: MMA from shared-memory operands into
// tensor memory, TMEM allocation and loads) and the tensor memory accelerator (cp.async.bulk.tensor), as
// the many-column block product uses them.  Operand tiles are K-major with the 128-byte swizzle: an atom
// is 8 rows of 128 bytes (1024-byte aligned), the 16-byte chunk j of row r stored at chunk j ^ (r mod 8).
#pragma once
#include <cstdint>

#include <cuda.h>

#include "ptx.cuh"

namespace bttb {

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading byte offset >> 4 (bits 16-29;
// not used by a K-major 128-byte-swizzled operand whose K block is one atom wide, set to 1), stride byte
// offset >> 4 (bits 32-45: the distance between 8-row groups), the fixed value 0b001 (bits 46-48), base
// offset 0 (atoms 1024-byte aligned), swizzle mode 2 = 128-byte (bits 61-63).
__host__ __device__ constexpr uint64_t tc_smem_desc(uint32_t saddr, uint32_t sbo_bytes) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::tf32 / kind::f16: D in binary32 (bits 4-5 = 1), A and B format (bits 7-9,
// 10-12: 1 = bfloat16, 2 = TF32), no negation, both K-major (bits 15, 16 = 0), N >> 3 (bits 17-22),
// M >> 4 (bits 24-28).
constexpr int kTcFmtBF16 = 1, kTcFmtTF32 = 2;
__host__ __device__ constexpr uint32_t tc_idesc(int fmt, int M, int N) {
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (row, k) of a K-major 128-byte-swizzled tile of `esz`-byte elements, from the
// start of its K block (k < 128 / esz), the block's rows 128 bytes apart.
__host__ __device__ constexpr uint32_t tc_sw128_offset(uint32_t row, uint32_t k, uint32_t esz) {
    return row * 128u + ((((k * esz) >> 4) ^ (row & 7u)) << 4) + ((k * esz) & 15u);
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A * B^T with A (M x K) and B (N x K) K-major in shared memory; accumulate unless accum = 0.
__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
// The mbarrier gets one arrival once every MMA this thread issued before has completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Lanes (taddr's lane + 0..31) x columns (taddr's column + 0..15) of 32-bit words: thread t of the warp
// gets its lane's 16 columns.  A warp may address only the lanes 32 (warp mod 4) .. 32 (warp mod 4) + 31.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Tiled 3-D tensor load into this CTA's shared memory; completion counted in bytes on `bar`.  The innermost
// coordinate c0 times the element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace bttb
