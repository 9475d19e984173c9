// Tensor memory (TMEM) as per-thread storage, through the tcgen05 instructions
// of sm_100-family GPUs (inline PTX).
//
// TMEM is 128 lanes x 512 columns of 32-bit cells per SM.  With the 32x32b
// access shape, thread i of warp w reads and writes lane 32 (w mod 4) + i, so a
// thread sees its own row of cells only: lane-private storage next to the
// register file, with its own data path (it does not use shared-memory
// bandwidth).  The line transforms keep per-thread twiddle factors (which
// depend on the thread's position in the line only, so they are computed once
// per launch) and parked line values there.
//
// Column plan: the warps that share a lane quarter (w, w + 4, w + 8, ...) get
// disjoint column ranges of `cols_per_warp` columns each.
#pragma once

#include <stdint.h>

namespace lsfft {

// One warp allocates `ncols` columns (a power of two, 32..512) and writes the
// base address to shared memory; the block then reads it after a barrier.
__device__ __forceinline__ void tmem_alloc_warp(uint32_t* smem_slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(smem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_warp(uint32_t base, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Address of this warp's first column: lane quarter from the warp index, the
// column range from the warp's rank within its lane quarter.
__device__ __forceinline__ uint32_t tmem_warp_addr(uint32_t base, int warp, int cols_per_warp) {
    return base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * cols_per_warp);
}

// 32 consecutive columns of the thread's lane <-> 32 floats (16 complex values).
__device__ __forceinline__ void tmem_st32(uint32_t ta, const float (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(ta),
        "f"(r[0]), "f"(r[1]), "f"(r[2]), "f"(r[3]), "f"(r[4]), "f"(r[5]), "f"(r[6]), "f"(r[7]), "f"(r[8]),
        "f"(r[9]), "f"(r[10]), "f"(r[11]), "f"(r[12]), "f"(r[13]), "f"(r[14]), "f"(r[15]), "f"(r[16]),
        "f"(r[17]), "f"(r[18]), "f"(r[19]), "f"(r[20]), "f"(r[21]), "f"(r[22]), "f"(r[23]), "f"(r[24]),
        "f"(r[25]), "f"(r[26]), "f"(r[27]), "f"(r[28]), "f"(r[29]), "f"(r[30]), "f"(r[31])
        : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t ta, float (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]),
          "=f"(r[8]), "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15]),
          "=f"(r[16]), "=f"(r[17]), "=f"(r[18]), "=f"(r[19]), "=f"(r[20]), "=f"(r[21]), "=f"(r[22]),
          "=f"(r[23]), "=f"(r[24]), "=f"(r[25]), "=f"(r[26]), "=f"(r[27]), "=f"(r[28]), "=f"(r[29]),
          "=f"(r[30]), "=f"(r[31])
        : "r"(ta)
        : "memory");
}

// 16 consecutive columns -> 16 floats (8 complex values).
__device__ __forceinline__ void tmem_ld16(uint32_t ta, float (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]),
          "=f"(r[8]), "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15])
        : "r"(ta)
        : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t ta, const float (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            ta),
        "f"(r[0]), "f"(r[1]), "f"(r[2]), "f"(r[3]), "f"(r[4]), "f"(r[5]), "f"(r[6]), "f"(r[7]), "f"(r[8]),
        "f"(r[9]), "f"(r[10]), "f"(r[11]), "f"(r[12]), "f"(r[13]), "f"(r[14]), "f"(r[15])
        : "memory");
}

// Park / fetch 16 complex FP32 values (one line's share of a thread).
__device__ __forceinline__ void tmem_park16(uint32_t ta, const float2 (&v)[16]) {
    float r[32];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        r[2 * i] = v[i].x;
        r[2 * i + 1] = v[i].y;
    }
    tmem_st32(ta, r);
}
__device__ __forceinline__ void tmem_fetch16(uint32_t ta, float2 (&v)[16]) {
    float r[32];
    tmem_ld32(ta, r);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = make_float2(r[2 * i], r[2 * i + 1]);
}

}  // namespace lsfft
