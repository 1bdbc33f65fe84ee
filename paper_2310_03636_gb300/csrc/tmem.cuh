// Tensor memory (TMEM) as per-thread table storage.
//
// Each SM of the sm_100 family has 256 KB of tensor memory: 128 lanes x 512 columns of
// 32 bits, allocated per block in power-of-two column counts (32..512) and read or written
// by a warp with tcgen05.ld / tcgen05.st.  In the 32x32b shape thread i of a warp reaches
// lane 32 (w % 4) + i, w the warp's index in the block, and the N consecutive columns the
// instruction names: every thread owns a private row, read without bank conflicts.  The
// path holds no matrix operands there; a kernel whose threads reuse the same table entries
// in every step (their own stage twiddles and kinetic phases) keeps them in that row
// instead of reading them through L1.
//
// Protocol: one warp allocates (the address lands in shared memory) and gives up the
// allocation permit, a fenced block barrier publishes the address, and before the block
// exits every thread has waited for its own accesses and the same warp frees the columns
// behind another fenced barrier.  An allocation that finds too few free columns waits
// for another block on the SM to free its own; every block that holds columns runs to
// completion without waiting for any other block, so such a wait always ends.
#pragma once

#include <stdint.h>

namespace gpe {

// Warp-collective: allocates ncols columns and writes the TMEM address to *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(slot);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Warp-collective: frees the columns of tmem_alloc.
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tmem_fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Address of the calling thread's row at column col: lane 32 (w % 4) + (thread in warp)
// is implied by the warp; the address names the warp's first lane.
__device__ __forceinline__ uint32_t tmem_warp_addr(uint32_t base, int warp, uint32_t col) {
    return base + ((uint32_t)(32 * (warp & 3)) << 16) + col;
}

// Warp-collective: 16 consecutive columns of the thread's row from r[0..15], waiting for
// the store to complete.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16};\n\t"
        "tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

// Warp-collective: 8 consecutive columns of the thread's row into r[0..7] (load and wait).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
}

// Warp-collective: 16 consecutive columns of the thread's row into r[0..15].  The wait for
// the load sits in the same statement, so no register is read before it has arrived.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

}  // namespace gpe
