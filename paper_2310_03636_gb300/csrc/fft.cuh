// Batched pencil FFTs held in registers with shared-memory Stockham exchanges.
//
// A pencil of N = 2^p complex points is owned by TP = N / R threads; thread t holds the
// R points x[t + m TP], m = 0..R-1 (natural order), and after the transform it holds
// X[t + m TP].  Stages are radix R (last one radix N / R^s if R does not divide
// evenly), each computed in registers; between stages the points go through shared
// memory in the Stockham autosort order, so the output needs no bit reversal.  The
// last stage of a forward transform leaves each thread with the very positions the
// first stage of the inverse transform needs, so a momentum-space phase multiply sits
// between them without a shared-memory round trip.
//
// Twiddle factors come from tables computed in FP64.  In FP32 every rotation -- table
// twiddles and the constant rotations inside the radix-8/16 butterflies -- is applied as
// three shears with determinant exactly 1 (common.cuh), so the rounding of the constants
// carries no O(eps) bias in |w| (a bias would repeat identically in every time step and
// accumulate linearly).  Transforms are unnormalised (the 1/N goes into the phase table).
#pragma once

#include "common.cuh"

namespace gpe {

// cos(2 pi e / 16)
__host__ __device__ constexpr double cos16(int e) {
    return (e & 15) == 0 ? 1.0
         : (e & 15) == 1 ? 0.92387953251128675613
         : (e & 15) == 2 ? 0.70710678118654752440
         : (e & 15) == 3 ? 0.38268343236508977173
         : (e & 15) == 4 ? 0.0
         : (e & 15) == 5 ? -0.38268343236508977173
         : (e & 15) == 6 ? -0.70710678118654752440
         : (e & 15) == 7 ? -0.92387953251128675613
         : (e & 15) == 8 ? -1.0
         : (e & 15) == 9 ? -0.92387953251128675613
         : (e & 15) == 10 ? -0.70710678118654752440
         : (e & 15) == 11 ? -0.38268343236508977173
         : (e & 15) == 12 ? 0.0
         : (e & 15) == 13 ? 0.38268343236508977173
         : (e & 15) == 14 ? 0.70710678118654752440
         : 0.92387953251128675613;
}

// a * exp(DIR 2 pi i e / 16), e a compile-time constant after unrolling.  FP32: the
// rotation is reduced by a multiple of pi to at most 3 pi / 8 (the multiple becomes a sign,
// folded into the callers' adds) and applied as three shears with FP64-computed constants.
template <int DIR, typename V>
__device__ __forceinline__ V twc16(V a, int e) {
    using T = decltype(a.x);
    e &= 15;
    if (e == 0) return a;
    if (e == 8) return mk(-a.x, -a.y);
    if (e == 4) return DIR < 0 ? mk(a.y, -a.x) : mk(-a.y, a.x);
    if (e == 12) return DIR < 0 ? mk(-a.y, a.x) : mk(a.y, -a.x);
    if constexpr (sizeof(T) == 4) {
        // angle j pi / 8 with j = DIR e folded into (-8, 8], then into (-4, 4) and a sign
        int j = DIR < 0 ? -e : e;
        if (j > 8) j -= 16;
        if (j <= -8) j += 16;
        bool neg = false;
        if (j > 4) { j -= 8; neg = true; }
        if (j < -4) { j += 8; neg = true; }
        const int aj = j < 0 ? -j : j;
        const double th = aj == 1 ? 0.19891236737965800691      // tan(pi / 16)
                        : aj == 2 ? 0.41421356237309504880      // tan(pi / 8)
                                  : 0.66817863791929891999;     // tan(3 pi / 16)
        const double sn = aj == 1 ? 0.38268343236508977173      // sin(pi / 8)
                        : aj == 2 ? 0.70710678118654752440      // sin(pi / 4)
                                  : 0.92387953251128675613;     // sin(3 pi / 8)
        const float p = (float)(j < 0 ? th : -th), u = (float)(j < 0 ? -sn : sn);
        const float2 r = lift_rot(a, p, u);
        return neg ? mk(-r.x, -r.y) : r;
    }
    const double cr = cos16(e);
    const double ci = DIR * cos16(e + 12);
    if ((e & 1) == 0) {
        const double h = 0.70710678118654752440;
        const T xr = cr > 0 ? a.x : -a.x, yr = cr > 0 ? a.y : -a.y;
        const T xi = ci > 0 ? a.x : -a.x, yi = ci > 0 ? a.y : -a.y;
        return mk(mulc(xr - yi, h), mulc(xi + yr, h));
    }
    return mk(mulc(a.x, cr) - mulc(a.y, ci), mulc(a.x, ci) + mulc(a.y, cr));
}

// In-register DFT of size R on v[0], v[S], ..., v[(R-1) S]; natural order in and out.
template <int R, int S, int DIR> struct Dft;

template <int S, int DIR> struct Dft<1, S, DIR> {
    template <typename V> __device__ __forceinline__ static void run(V*) {}
};

template <int S, int DIR> struct Dft<2, S, DIR> {
    template <typename V> __device__ __forceinline__ static void run(V* v) {
        V a = v[0], b = v[S];
        v[0] = cadd(a, b);
        v[S] = csub(a, b);
    }
};

template <int S, int DIR> struct Dft<4, S, DIR> {
    template <typename V> __device__ __forceinline__ static void run(V* v) {
        V x0 = v[0], x1 = v[S], x2 = v[2 * S], x3 = v[3 * S];
        V a0 = cadd(x0, x2), a1 = csub(x0, x2), a2 = cadd(x1, x3);
        V a3 = twc16<DIR>(csub(x1, x3), 4);
        v[0] = cadd(a0, a2);
        v[2 * S] = csub(a0, a2);
        v[S] = cadd(a1, a3);
        v[3 * S] = csub(a1, a3);
    }
};

// R = R1 * R2: n = R2 n1 + n2, k = k1 + R1 k2.  The first layer is R2 DFTs of size R1 on
// the groups {n2, n2 + R2, ...}; ``rest`` is everything after it, so a caller may rotate
// and transform one group at a time (the same operations on every element).
template <int R, int S, int DIR> struct Dft {
    static constexpr int R1 = (R == 8) ? 2 : 4;
    static constexpr int R2 = R / R1;
    template <typename V> __device__ __forceinline__ static void run(V* v) {
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) Dft<R1, R2 * S, DIR>::run(v + n2 * S);
        rest(v);
    }
    template <typename V> __device__ __forceinline__ static void rest(V* v) {
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1)
#pragma unroll
            for (int n2 = 1; n2 < R2; ++n2)
                v[(R2 * k1 + n2) * S] = twc16<DIR>(v[(R2 * k1 + n2) * S], (16 / R) * n2 * k1);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) Dft<R2, S, DIR>::run(v + R2 * k1 * S);
        V tmp[R];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) tmp[k1 + R1 * k2] = v[(R2 * k1 + k2) * S];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k * S] = tmp[k];
    }
};

// Padded shared-memory index: one spare slot every 16 elements.
__device__ __forceinline__ int spad(int i) { return i + (i >> 4); }

// Shared-memory length per pencil buffer: padded length, rounded so consecutive pencil
// buffers start one 8-byte (float2) / 16-byte (double2) bank slot apart.
template <typename T>
__host__ __device__ constexpr int smem_ld(int n) {
    return ((n + n / 16 + (int)(128 / (2 * sizeof(T))) - 1) / (int)(128 / (2 * sizeof(T)))) *
               (int)(128 / (2 * sizeof(T))) + 1;
}

// Who synchronises a pencil's exchanges: the whole block, one warp (pencils of at most
// 32 threads), or the pencil's own group of threads (a named barrier per group of TP
// consecutive threads, TP a multiple of 32, at most 15 groups per block), so that the
// pencils of one block do not wait for each other.
enum class Sync { Block, Warp, Group };

template <Sync SY, int TP = 0> __device__ __forceinline__ void pencil_sync() {
    if constexpr (SY == Sync::Block) {
        __syncthreads();
    } else if constexpr (SY == Sync::Group) {
        static_assert(TP % 32 == 0 && TP >= 64, "group barriers need whole warps");
        asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / TP)), "r"(TP) : "memory");
    } else {
        __syncwarp(blockDim.x >= 32 ? 0xffffffffu : ((1u << blockDim.x) - 1u));
    }
}

// Stage plan of a length-N transform with R points per thread: stages of radix R, then
// one of radix N / R^s if needed.  Stage s combines sub-transforms of length NS(s).
// Twiddles of stage s (NS > 1) are stored as a block [r = 1..RS-1][k = 0..NS-1] of
// W_{NS RS}^{r k}, so threads with consecutive k read consecutive entries.
template <int N, int R>
struct FftPlan {
    static constexpr int kLogN = ilog2(N), kLogR = ilog2(R);
    static constexpr int kFull = kLogN / kLogR;
    static constexpr int kLast = 1 << (kLogN - kFull * kLogR);
    static constexpr int kStages = kFull + (kLast > 1 ? 1 : 0);
    static constexpr int radix(int s) { return s < kFull ? R : kLast; }
    static constexpr int ns(int s) {
        int v = 1;
        for (int i = 0; i < s; ++i) v *= radix(i);
        return v;
    }
    static constexpr int tw_offset(int s) {
        int off = 0;
        for (int i = 0; i < s; ++i)
            if (ns(i) > 1) off += (radix(i) - 1) * ns(i);
        return off;
    }
    static constexpr int tw_size() { return tw_offset(kStages); }
};

// One Stockham stage S of radix RS on sub-transforms of length NS.  With SPLIT > 0 the
// twiddles of the stages whose entries start at or after SPLIT come from tws_hi (the
// table's tail, e.g. left in global memory) and the others from tws.
template <int N, int R, int DIR, int NC, int S, Sync SY, int SPLIT = 0, typename V, typename TW>
__device__ __forceinline__ void stockham_stage(V (&v)[NC][R], V* const (&buf)[NC],
                                               const TW* __restrict__ tws, int t,
                                               const TW* __restrict__ tws_hi = nullptr) {
    using P = FftPlan<N, R>;
    constexpr int TP = N / R;
    constexpr int RS = P::radix(S);
    constexpr int NS = P::ns(S);
    constexpr bool LAST = (S == P::kStages - 1);
    constexpr int B = R / RS;
    constexpr int OFF = P::tw_offset(S);
#pragma unroll
    for (int u = 0; u < B; ++u) {
        const int j = t + u * TP;
        const int k = j & (NS - 1);
        V w[NC][RS];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int r = 0; r < RS; ++r) w[c][r] = v[c][u + r * B];
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < RS; ++r) {
                TW f;
                if constexpr (SPLIT > 0 && OFF >= SPLIT) f = tws_hi[OFF + (r - 1) * NS + k];
                else f = tws[OFF + (r - 1) * NS + k];
                if constexpr (sizeof(TW) == 8) {
                    // FP32 table of (p, u) pairs only: the sign of the reduced rotation is -1
                    // exactly for angles 2 pi r k / (NS RS) in (pi/2, 3 pi/2)
                    const int x4 = 4 * r * k;
                    const bool neg = x4 > NS * RS && x4 < 3 * NS * RS;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const float2 q = lift_rot(w[c][r], DIR < 0 ? f.x : -f.x, DIR < 0 ? f.y : -f.y);
                        w[c][r] = neg ? make_float2(-q.x, -q.y) : q;
                    }
                } else {
                    // if every twiddle angle 2 pi r k / (NS RS) of this r is within pi/2, the
                    // table's sign is +1 and the scale is skipped (r is a constant once unrolled)
                    const bool sig = 4 * r * (NS - 1) > NS * RS;
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        w[c][r] = sig ? twmul<DIR, true>(w[c][r], f) : twmul<DIR, false>(w[c][r], f);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) Dft<RS, 1, DIR>::run(w[c]);
        if constexpr (LAST) {
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int r = 0; r < RS; ++r) v[c][u + r * B] = w[c][r];
        } else {
            const int base = (j - k) * RS + k;
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int r = 0; r < RS; ++r) buf[c][spad(base + r * NS)] = w[c][r];
        }
    }
    if constexpr (!LAST) {
        pencil_sync<SY, TP>();
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int m = 0; m < R; ++m) v[c][m] = buf[c][spad(t + m * TP)];
        pencil_sync<SY, TP>();
    }
}

template <int N, int R, int DIR, int NC, int S, Sync SY, int SPLIT = 0, typename V, typename TW>
__device__ __forceinline__ void stockham_from(V (&v)[NC][R], V* const (&buf)[NC],
                                              const TW* __restrict__ tws, int t,
                                              const TW* __restrict__ tws_hi = nullptr) {
    if constexpr (S < FftPlan<N, R>::kStages) {
        stockham_stage<N, R, DIR, NC, S, SY, SPLIT>(v, buf, tws, t, tws_hi);
        stockham_from<N, R, DIR, NC, S + 1, SY, SPLIT>(v, buf, tws, t, tws_hi);
    }
}

// Length-N transform of NC pencils at once (one per component), DIR = -1 forward
// (e^{-2 pi i jk/N}), +1 inverse (unnormalised).  Every thread of the sync group must
// call it.  buf[c]: shared buffer of pencil c (smem_ld<T>(N) elements); tws: the stage
// twiddle table of FftPlan<N, R> (usually a shared-memory copy).
template <int N, int R, int DIR, int NC, Sync SY, typename V, typename TW>
__device__ __forceinline__ void fft_pencil(V (&v)[NC][R], V* const (&buf)[NC],
                                           const TW* __restrict__ tws, int t) {
    static_assert((N & (N - 1)) == 0 && N >= R, "N must be a power of two >= R");
    stockham_from<N, R, DIR, NC, 0, SY>(v, buf, tws, t);
}

// The same transform with the stage-twiddle table in two parts: entries [0, SPLIT) from
// tws_lo (a shared-memory copy of the table's head) and the rest from tws_hi (the full
// table, typically in global memory).  SPLIT must be a stage boundary of FftPlan<N, R>.
template <int N, int R, int DIR, int NC, Sync SY, int SPLIT, typename V, typename TW>
__device__ __forceinline__ void fft_pencil_split(V (&v)[NC][R], V* const (&buf)[NC], const TW* __restrict__ tws_lo,
                                                 const TW* __restrict__ tws_hi, int t) {
    static_assert((N & (N - 1)) == 0 && N >= R, "N must be a power of two >= R");
    stockham_from<N, R, DIR, NC, 0, SY, SPLIT>(v, buf, tws_lo, t, tws_hi);
}

// Cooperative copy of a table into shared memory (caller synchronises).
template <typename V>
__device__ __forceinline__ void copy_table(V* dst, const V* __restrict__ src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

}  // namespace gpe
