// Tables of the 4096-point FP32 resident transforms in tensor memory (tmem.cuh).
//
// The resident 1D kernel at N = 4096 and each block of the cluster kernel (slices of
// M = 4096) transform with R = 16 points per thread, 256 threads: two warps on each 32-lane
// quarter of tensor memory.  Every thread keeps in its own row the table entries it reads
// in every step -- the twiddles of the last stage (stage 2: k = t, r = 1..15; 15 x 256
// entries, 61 KB as a table, too large to sit in shared memory beside the field) and the
// kinetic phases of its 16 points for a full step (64 KB as a table) -- instead of reading
// them through L1, which the 108 KB of shared memory per block leave mostly to the field.
// Columns per thread: 4 groups x 16 for the twiddles (group n2 holds r = n2 + 4 n1,
// n1 = 0..3, the inputs of one first-layer DFT of the radix-16 butterfly, as four float4
// table entries) and 4 x 16 for the phases (points 4q .. 4q + 3): 128.  Warps 4..7 use the
// 128 columns after those of warps 0..3: 256 per block, and shared memory allows two blocks
// per SM, so the 512 columns of an SM always suffice.  The entries are the tables' own
// bits and every element goes through the operations of stockham_stage, so the results
// are those of the shared-memory/L1 form bit for bit.
#pragma once

#include "prop_kernels.cuh"
#include "tmem.cuh"

namespace gpe {

constexpr uint32_t kRes1dTmemCols = 256;

template <typename T, int N, int R, int G>
constexpr bool res1d_tmem() { return sizeof(T) == 4 && N == 4096 && R == 16 && G == 1; }

__device__ __forceinline__ float4 u4_to_f4(const uint32_t* r) {
    return make_float4(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]), __uint_as_float(r[3]));
}
__device__ __forceinline__ void f4_to_u4(float4 f, uint32_t* r) {
    r[0] = __float_as_uint(f.x);
    r[1] = __float_as_uint(f.y);
    r[2] = __float_as_uint(f.z);
    r[3] = __float_as_uint(f.w);
}

// Allocates the block's columns (warp 0) and returns the base address to every thread.
__device__ __forceinline__ uint32_t res1d_tmem_open(uint32_t* slot) {
    if (threadIdx.x < 32) tmem_alloc(slot, kRes1dTmemCols);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    return *slot;
}

// Frees them once every thread is done with its row.
__device__ __forceinline__ void res1d_tmem_close(uint32_t base) {
    tmem_fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) {
        tmem_fence_after_sync();
        tmem_dealloc(base, kRes1dTmemCols);
    }
}

// The calling thread's row: lane 32 (w % 4) + (thread in warp), columns from 128 (w / 4).
__device__ __forceinline__ uint32_t res1d_tmem_row(uint32_t base) {
    const int warp = (int)(threadIdx.x / 32);
    return tmem_warp_addr(base, warp, (uint32_t)((warp >> 2) * 128));
}

// Fills thread t's row: stage-2 twiddles of the 4096-point table tws (FftPlan<4096, 16>)
// and the full-step phases ph[ph_stride (t + 256 m) + ph_off], m = 0..15.
__device__ __forceinline__ void res1d_tmem_fill(uint32_t ta, const float4* __restrict__ tws,
                                                const float4* __restrict__ ph, int ph_stride, int ph_off, int t) {
    constexpr int OFF2 = FftPlan<4096, 16>::tw_offset(2);
#pragma unroll 1
    for (int n2 = 0; n2 < 4; ++n2) {
        uint32_t r[16];
#pragma unroll
        for (int n1 = 0; n1 < 4; ++n1) {
            const int rr = n2 + 4 * n1;
            f4_to_u4(rr == 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : tws[OFF2 + (rr - 1) * 256 + t], r + 4 * n1);
        }
        tmem_st16(ta + 16 * n2, r);
    }
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
        uint32_t r[16];
#pragma unroll
        for (int e = 0; e < 4; ++e) f4_to_u4(ph[ph_stride * (t + (4 * q + e) * 256) + ph_off], r + 4 * e);
        tmem_st16(ta + 64 + 16 * q, r);
    }
}

// Last stage (radix 16 on sub-transforms of 256, k = t) with the twiddles from tensor
// memory: each first-layer group is rotated right before its DFT, so only one group's
// four entries are live.
template <int DIR>
__device__ __forceinline__ void last_stage_tmem(float2 (&w)[16], uint32_t ta) {
    constexpr int NS = 256, RS = 16;
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        uint32_t r[16];
        tmem_ld16(ta + 16 * n2, r);
#pragma unroll
        for (int n1 = 0; n1 < 4; ++n1) {
            const int rr = n2 + 4 * n1;
            if (rr == 0) continue;
            const float4 f = u4_to_f4(r + 4 * n1);
            const bool sig = 4 * rr * (NS - 1) > NS * RS;
            w[rr] = sig ? twmul<DIR, true>(w[rr], f) : twmul<DIR, false>(w[rr], f);
        }
        Dft<4, 4, DIR>::run(w + n2);
    }
    Dft<16, 1, DIR>::rest(w);
}

// A 4096-point transform of one pencil: stages 0 and 1 as in fft_pencil (stage 1's
// twiddles from the shared-memory head tws_s of the table), stage 2 from tensor memory.
template <int DIR>
__device__ __forceinline__ void fft4096_tmem(float2 (&v)[1][16], float2* const (&buf)[1], const float4* tws_s,
                                             uint32_t ta, int t) {
    stockham_stage<4096, 16, DIR, 1, 0, Sync::Block>(v, buf, tws_s, t);
    stockham_stage<4096, 16, DIR, 1, 1, Sync::Block>(v, buf, tws_s, t);
    last_stage_tmem<DIR>(v[0], ta);
}

// The full-step kinetic phases of the thread's 16 points, from tensor memory.
__device__ __forceinline__ void phase4096_tmem(float2 (&v)[16], uint32_t ta) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t r[16];
        tmem_ld16(ta + 64 + 16 * q, r);
#pragma unroll
        for (int e = 0; e < 4; ++e) v[4 * q + e] = phmul<-1>(v[4 * q + e], u4_to_f4(r + 4 * e));
    }
}

}  // namespace gpe
