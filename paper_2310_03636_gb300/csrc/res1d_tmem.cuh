// Tables of the resident FP32 transforms in tensor memory (tmem.cuh).
//
// The resident 1D kernel at N = 4096 and 2048, and each block of the cluster kernel (slices
// of M = 4096), transform with R = 16 points per thread: 256 or 128 threads, so one or two
// warps on each 32-lane quarter of tensor memory.  Every thread keeps in its own row the
// table entries it reads in every step -- the twiddles of the last stage (15 x 256 entries,
// 61 KB as a table at 4096; 7 x 256, 28 KB at 2048; too large to share the little L1 that the
// shared-memory field leaves) and the kinetic phases of its 16 points for a full step --
// instead of reading them through L1.  Columns per thread: 64 for the twiddles (grouped by
// the first-layer DFTs of the last stage's butterflies, one float4 table entry each) and
// 4 x 16 for the phases (points 4q .. 4q + 3): 128.  Warps 4..7 use the 128 columns after
// those of warps 0..3.  A block of 4096 holds 256 columns and shared memory allows two per
// SM; a block of 2048 holds 128 and shared memory allows four: the 512 columns of an SM
// suffice for any mix the shared memory admits.  The entries are the tables' own bits and
// every element goes through the operations of stockham_stage, so the results are those of
// the L1 form bit for bit.
#pragma once

#include "prop_kernels.cuh"
#include "tmem.cuh"

namespace gpe {

// Transforms with tables in tensor memory: FP32, R = 16, one thread group, N = 4096 (last
// stage radix 16, one butterfly per thread) or N = 2048 (last stage radix 8, two).
template <typename T, int N, int R, int G>
constexpr bool res1d_tmem() { return sizeof(T) == 4 && R == 16 && G == 1 && (N == 4096 || N == 2048); }

// Columns a block allocates: 128 per thread, the warps beyond the first four on columns of
// their own (4096: 8 warps, 256 columns; 2048: 4 warps, 128 columns, four blocks per SM).
template <int N>
constexpr uint32_t res1d_tmem_cols() { return (uint32_t)((N / 16 / 32 + 3) / 4) * 128u; }

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
__device__ __forceinline__ uint32_t res1d_tmem_open(uint32_t* slot, uint32_t ncols) {
    if (threadIdx.x < 32) tmem_alloc(slot, ncols);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    return *slot;
}

// Frees them once every thread is done with its row.
__device__ __forceinline__ void res1d_tmem_close(uint32_t base, uint32_t ncols) {
    tmem_fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) {
        tmem_fence_after_sync();
        tmem_dealloc(base, ncols);
    }
}

// The calling thread's row: lane 32 (w % 4) + (thread in warp), columns from 128 (w / 4).
__device__ __forceinline__ uint32_t res1d_tmem_row(uint32_t base) {
    const int warp = (int)(threadIdx.x / 32);
    return tmem_warp_addr(base, warp, (uint32_t)((warp >> 2) * 128));
}

// Last stage of FftPlan<N, 16> (sub-transforms of NS = 256, radix RS = N / 256, B = 16 / RS
// butterflies per thread) and the row layout of its twiddles: butterfly u, first-layer
// group n2 of the radix-RS DFT (inputs r = n2 + 4 n1, n1 < R1 = RS / 4) at column
// 64 u / B + 4 R1 n2 + 4 n1, one float4 table entry per twiddle (r = 0 unused).
template <int N>
struct LastStage {
    static constexpr int NS = 256, RS = N / NS, B = 16 / RS, R1 = RS / 4, R2 = 4;
    static constexpr int col(int u, int n2, int n1) { return 64 / B * u + 4 * R1 * n2 + 4 * n1; }
};

// Fills thread t's row: the last stage's twiddles of the table tws (FftPlan<N, 16>) and the
// full-step phases ph[ph_stride (t + TP m) + ph_off], m = 0..15, at columns 64 + 4 m.
template <int N>
__device__ __forceinline__ void res1d_tmem_fill(uint32_t ta, const float4* __restrict__ tws,
                                                const float4* __restrict__ ph, int ph_stride, int ph_off, int t) {
    using L = LastStage<N>;
    constexpr int TP = N / 16;
    constexpr int OFF2 = FftPlan<N, 16>::tw_offset(2);
    uint32_t r[16];
#pragma unroll 1
    for (int h = 0; h < 4; ++h) {   // 16 columns at a time
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = 16 * h + 4 * e;          // column of the entry
            const int u = c / (64 / L::B), rem = c % (64 / L::B);
            const int n2 = rem / (4 * L::R1), n1 = (rem % (4 * L::R1)) / 4;
            const int rr = n2 + 4 * n1;
            const int k = (t + u * TP) & (L::NS - 1);
            f4_to_u4(rr == 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : tws[OFF2 + (rr - 1) * L::NS + k], r + 4 * e);
        }
        tmem_st16(ta + 16 * h, r);
    }
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int e = 0; e < 4; ++e) f4_to_u4(ph[ph_stride * (t + (4 * q + e) * TP) + ph_off], r + 4 * e);
        tmem_st16(ta + 64 + 16 * q, r);
    }
}

// The last stage with the twiddles from tensor memory: each first-layer group is rotated
// right before its DFT, so only one group's entries are live; the same operations per
// element as stockham_stage.
template <int N, int DIR>
__device__ __forceinline__ void last_stage_tmem(float2 (&v)[16], uint32_t ta) {
    using L = LastStage<N>;
#pragma unroll
    for (int u = 0; u < L::B; ++u) {
        float2 w[L::RS];
#pragma unroll
        for (int r = 0; r < L::RS; ++r) w[r] = v[u + r * L::B];
#pragma unroll
        for (int n2 = 0; n2 < L::R2; ++n2) {
            uint32_t q[4 * L::R1];
            if constexpr (L::R1 == 4) tmem_ld16(ta + L::col(u, n2, 0), q);
            else tmem_ld8(ta + L::col(u, n2, 0), q);
#pragma unroll
            for (int n1 = 0; n1 < L::R1; ++n1) {
                const int rr = n2 + 4 * n1;
                if (rr == 0) continue;
                const float4 f = u4_to_f4(q + 4 * n1);
                const bool sig = 4 * rr * (L::NS - 1) > L::NS * L::RS;
                w[rr] = sig ? twmul<DIR, true>(w[rr], f) : twmul<DIR, false>(w[rr], f);
            }
            Dft<L::R1, L::R2, DIR>::run(w + n2);
        }
        Dft<L::RS, 1, DIR>::rest(w);
#pragma unroll
        for (int r = 0; r < L::RS; ++r) v[u + r * L::B] = w[r];
    }
}

// An N-point transform of one pencil: stages 0 and 1 as in fft_pencil (stage 1's twiddles
// from the shared-memory head tws_s of the table), the last stage from tensor memory.
template <int N, int DIR>
__device__ __forceinline__ void fft_tmem(float2 (&v)[1][16], float2* const (&buf)[1], const float4* tws_s,
                                         uint32_t ta, int t) {
    stockham_stage<N, 16, DIR, 1, 0, Sync::Block>(v, buf, tws_s, t);
    stockham_stage<N, 16, DIR, 1, 1, Sync::Block>(v, buf, tws_s, t);
    last_stage_tmem<N, DIR>(v[0], ta);
}

// The full-step kinetic phases of the thread's 16 points, from tensor memory.
__device__ __forceinline__ void phase_tmem(float2 (&v)[16], uint32_t ta) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t r[16];
        tmem_ld16(ta + 64 + 16 * q, r);
#pragma unroll
        for (int e = 0; e < 4; ++e) v[4 * q + e] = phmul<-1>(v[4 * q + e], u4_to_f4(r + 4 * e));
    }
}

}  // namespace gpe
