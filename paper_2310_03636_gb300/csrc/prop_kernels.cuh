// Propagation kernels: the kinetic step as per-axis pencil passes (K is separable,
// exp(-i tau |k|^2/2) = prod_a exp(-i tau k_a^2/2)), the x pass fused with the local
// step (the resident 1D kernels are in res1d.cu and res1d_cluster.cu).
#pragma once

#include "fft.cuh"
#include <type_traits>
#include <cuda.h>

#include "async_copy.cuh"
#include "internal.h"

namespace gpe {

// Shape choices per precision.
template <typename T> struct Tune;
template <> struct Tune<float> {
    static constexpr int kXR = 8;        // points per thread, row pass (3 components live)
    static constexpr int kColR(int n) { return n >= 128 ? 16 : 8; }    // points per thread, column pass
    static constexpr int kColCols(int n) { return n >= 1024 ? 4 : (n >= 512 ? 4 : (n >= 256 ? 8 : 16)); }
    static constexpr int kResR(int n) { return n >= 1024 ? 16 : 8; }
    static constexpr int kRowR(int n) { return n >= 256 ? 16 : 8; }
};
template <> struct Tune<double> {
    static constexpr int kXR = 4;
    static constexpr int kColR(int) { return 8; }
    static constexpr int kColCols(int n) { return n >= 512 ? 4 : 8; }
    static constexpr int kResR(int n) { return n >= 1024 ? 8 : 4; }
    static constexpr int kRowR(int n) { return n >= 256 ? 8 : 4; }
};

template <int R> constexpr int tw_slot() { return R == 4 ? 0 : (R == 8 ? 1 : 2); }

// Offset (in complex elements) of the twiddle block after n data elements, rounded up to
// 16 bytes so the hi/lo float4 entries are aligned.
template <typename T> constexpr int tw_off(int n) { return sizeof(T) == 4 ? ((n + 1) & ~1) : n; }

// Shared-memory length of one column buffer in the column pass: the padded length
// rounded to a whole 128-byte line plus an offset of (128 B / element) / COLS slots, so a
// warp (COLS columns x 32 / COLS pencil threads) touches every bank equally.
template <typename T>
constexpr int smem_ld_cols(int n, int cols) {
    return ((n + n / 16 + (int)(64 / sizeof(T)) - 1) / (int)(64 / sizeof(T))) * (int)(64 / sizeof(T)) +
           ((int)(64 / sizeof(T)) / cols > 0 ? (int)(64 / sizeof(T)) / cols : 1);
}

template <int N, int R> constexpr int rows_per_cta() { return (N / R) >= 256 ? 1 : 256 / (N / R); }

// Rows per block of the x pass for a block of THREADS threads; THREADS = 0 is the default,
// 256 threads except 128 at n = 128 and n = 1024 (measured: 196 vs 207 us at 128^2 x 512,
// 459 vs 474 us at 1024^2 x 16; 256 threads are faster at 256 and 512).  The FP32 tile
// autotuner may pick the other size per shape: every row goes through the same arithmetic
// either way, so the choice changes no result bit.
template <int N, int R, int THREADS = 0> constexpr int xpass_rows() {
    const int threads = THREADS > 0 ? THREADS : ((N == 128 || N == 1024) ? 128 : 256);
    return (N / R) >= threads ? 1 : threads / (N / R);
}

constexpr uint32_t kWaitLimit = 1u << 22;   // mbarrier polls before a wait counts as expired

// Poll limit of a block's first copy wait: the default, or the value a test set
// (wait_first = 1 + limit; 0 keeps the default).  Later waits and the drain after an
// expired wait always take the default.
__host__ __device__ constexpr uint32_t first_wait_limit(uint32_t wait_first) {
    return wait_first == 0 ? kWaitLimit : wait_first - 1;
}

// FFT along x of one row-component held in shared memory (thread t owns positions
// t + m TP), times a phase table, inverse FFT, back into shared memory.  A row of at most
// 32 threads lies within one warp, so its exchanges synchronise the warp only; the rows
// of a block with several larger rows synchronise with a barrier of their own.
// With CPH (FP32) the phases come from a compact table in shared memory: (p, u) of the
// three-shear rotation for modes 0..N/2 (mode k and N - k share an entry) and the common
// factor scale = 1/N, the same numbers phmul takes from the full table, so the same bits.
template <typename T, int N, int R, int RPC = 1, bool CPH = false, typename TW = twel<T>>
__device__ __forceinline__ void kinetic_row(cplx<T>* row, cplx<T>* xbuf, const TW* tws,
                                            const twel<T>* __restrict__ ph, int t, const float2* phc = nullptr,
                                            float scale = 0.0f) {
    using V = cplx<T>;
    constexpr int TP = N / R;
    V v[1][R];
    V* const xb[1] = {xbuf};
#pragma unroll
    for (int m = 0; m < R; ++m) v[0][m] = row[t + m * TP];
    constexpr Sync SY = TP <= 32 ? Sync::Warp : (RPC > 1 ? Sync::Group : Sync::Block);
    fft_pencil<N, R, -1, 1, SY>(v, xb, tws, t);
    if constexpr (CPH && sizeof(T) == 4) {
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const int k = t + m * TP;
            const float2 f = phc[k <= N / 2 ? k : N - k];
            const float2 r = lift_rot(v[0][m], f.x, f.y);
            v[0][m] = make_float2(r.x * scale, r.y * scale);
        }
    } else {
#pragma unroll
        for (int m = 0; m < R; ++m) v[0][m] = phmul<-1>(v[0][m], ph[t + m * TP]);
    }
    fft_pencil<N, R, +1, 1, SY>(v, xb, tws, t);
#pragma unroll
    for (int m = 0; m < R; ++m) row[t + m * TP] = v[0][m];
}

// Row pass over RPC x rows of all three components: bulk copies bring the rows into
// shared memory, then [PRE: Kx(dt/2)] L(dt) per site, Kx(tau) per component, and bulk
// copies write them back.
// Compact phase tables the x pass keeps in shared memory (CPH): one, two with the leading
// half kick.
// Each table takes an even number of entries (whole 16-byte units, for the bulk copy).
template <int N> constexpr int xpass_cph_half() { return (N / 2 + 1 + 1) & ~1; }
template <int N, bool PRE> constexpr int xpass_cph_entries() { return (PRE ? 2 : 1) * xpass_cph_half<N>(); }

template <typename T, int N, int R, bool PRE, int THREADS = 0, bool CPH = false>
__global__ void __launch_bounds__(xpass_rows<N, R, THREADS>() * (N / R))
k_xpass(const PassArgs<T> a) {
    using V = cplx<T>;
    constexpr int TP = N / R;
    constexpr int RPC = xpass_rows<N, R, THREADS>();
    constexpr int LD = smem_ld<T>(N);
    constexpr int TWN = FftPlan<N, R>::tw_size();
    extern __shared__ __align__(128) unsigned char smraw[];
    // CPH (FP32): the stage twiddles as (p, u) pairs, the sign taken from the index
    using TWT = typename std::conditional<CPH, float2, twel<T>>::type;
    V* D = reinterpret_cast<V*>(smraw);                          // [RPC][3][N]
    V* X = D + RPC * 3 * N;                                      // [RPC][LD] exchange
    TWT* tws = reinterpret_cast<TWT*>(X + tw_off<T>(RPC * LD));
    uint64_t* bar = reinterpret_cast<uint64_t*>(tws + ((TWN + 1) & ~1));
    float2* phc = reinterpret_cast<float2*>(bar + 2);   // CPH: [ph][ph_pre] compact tables
    const int lrow = threadIdx.x / TP, t = threadIdx.x % TP;
    const int64_t row0 = (int64_t)blockIdx.x * RPC;
    const int nrows = (int)min((int64_t)RPC, a.total_rows - row0);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        // CPH: the (p, u) stage twiddles and the compact phase tables come with the rows, on
        // the same barrier (bulk copies of whole 16-byte units; the host pads each table)
        constexpr uint32_t CPH_BYTES = CPH ? (uint32_t)(((TWN + 1) & ~1) + xpass_cph_entries<N, PRE>()) * 8u : 0u;
        mbar_expect_tx(bar, (uint32_t)(nrows * 3 * N * sizeof(V)) + CPH_BYTES);
        if constexpr (CPH) {
            bulk_g2s(tws, a.tw2, (uint32_t)(((TWN + 1) & ~1) * 8), bar);
            bulk_g2s(phc, a.phc, (uint32_t)(xpass_cph_half<N>() * 8), bar);
            if constexpr (PRE) bulk_g2s(phc + xpass_cph_half<N>(), a.phc_pre, (uint32_t)(xpass_cph_half<N>() * 8), bar);
        }
        for (int r = 0; r < nrows; ++r) {
            const int64_t g = row0 + r;
            const int traj = (int)(g / a.rows_per_traj);
            const V* src = a.ptrs[traj] + (g - (int64_t)traj * a.rows_per_traj) * N;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                bulk_g2s(D + (r * 3 + c) * N, src + c * a.comp_stride, N * sizeof(V), bar);
        }
    }
    if constexpr (!CPH) copy_table(tws, a.tw[tw_slot<R>()], TWN);
    const bool ok = __syncthreads_and(mbar_wait(bar, 0, first_wait_limit(a.wait_first)));
    if (!ok) {
        if (threadIdx.x == 0) atomicCAS(a.status, 0, (int)GPE_ETIMEOUT);
        mbar_wait(bar, 0, kWaitLimit);
        return;
    }
    V* Dr = D + lrow * 3 * N;
    V* Xr = X + lrow * LD;
    if constexpr (PRE) {
#pragma unroll 1
        for (int c = 0; c < 3; ++c)
            kinetic_row<T, N, R, RPC, CPH, TWT>(Dr + c * N, Xr, tws, a.ph_pre, t, phc + xpass_cph_half<N>(), a.ph_scale);
    }
    if (lrow < nrows) {
        if (a.vpot == nullptr) {
            local_step_sites<T>(Dr, Dr + N, Dr + 2 * N, t, N, TP, a.coef, [](int i) { return i; });
        } else {
            const int64_t g = row0 + lrow;
            const int64_t traj = g / a.rows_per_traj;
            const T* vrow = a.vpot + (g - traj * a.rows_per_traj) * N;
#pragma unroll 2
            for (int m = 0; m < R; ++m) {
                const int i = t + m * TP;
                V p1 = Dr[i], p0 = Dr[N + i], pm = Dr[2 * N + i];
                local_step<true, T>(p1, p0, pm, a.coef, site_pot<T>(vrow, a.comp_stride, i));
                Dr[i] = p1;
                Dr[N + i] = p0;
                Dr[2 * N + i] = pm;
            }
        }
    }
#pragma unroll 1
    for (int c = 0; c < 3; ++c) kinetic_row<T, N, R, RPC, CPH, TWT>(Dr + c * N, Xr, tws, a.ph, t, phc, a.ph_scale);
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int r = 0; r < nrows; ++r) {
            const int64_t g = row0 + r;
            const int traj = (int)(g / a.rows_per_traj);
            V* dst = a.ptrs[traj] + (g - (int64_t)traj * a.rows_per_traj) * N;
#pragma unroll
            for (int c = 0; c < 3; ++c) bulk_s2g(dst + c * a.comp_stride, D + (r * 3 + c) * N, N * sizeof(V));
        }
        bulk_commit();
        bulk_wait_read_all();
    }
}

template <typename T, int N, int R, int THREADS = 0, bool CPH = false, bool PRE = false>
constexpr size_t xpass_smem() {
    return ((size_t)xpass_rows<N, R, THREADS>() * 3 * N + tw_off<T>(xpass_rows<N, R, THREADS>() * smem_ld<T>(N))) *
               sizeof(cplx<T>) +
           (size_t)((FftPlan<N, R>::tw_size() + 1) & ~1) * (CPH ? sizeof(float2) : sizeof(twel<T>)) + 16 +
           (CPH ? (size_t)xpass_cph_entries<N, PRE>() * sizeof(float2) : 0);
}

// Column-pass modes: the kinetic factor (FFT, x ph, iFFT), a forward FFT only, the
// adjoint kinetic factor (FFT, x conj(ph), iFFT), an unnormalised inverse FFT only.
enum ColMode { kColK = 0, kColFwd = 1, kColKConj = 2, kColInv = 3 };

// Column pass: pencils of length N along a strided axis, COLS adjacent x columns per
// block, one component, in mode MODE.  Block index -> (traj, comp, outer, x tile).
template <typename T, int N, int R, int COLS, int MODE>
__global__ void __launch_bounds__(COLS * (N / R))
k_colpass(const PassArgs<T> a) {
    using V = cplx<T>;
    constexpr int TP = N / R;
    constexpr int LD = smem_ld_cols<T>(N, COLS);
    constexpr int TWN = FftPlan<N, R>::tw_size();
    extern __shared__ __align__(128) unsigned char smraw[];
    V* sm = reinterpret_cast<V*>(smraw);
    twel<T>* tws = reinterpret_cast<twel<T>*>(sm + tw_off<T>(COLS * LD));
    copy_table(tws, a.tw[tw_slot<R>()], TWN);
    const int col = threadIdx.x % COLS, t = threadIdx.x / COLS;
    int64_t tile = blockIdx.x;
    const int xt = (int)(tile % a.nx_tiles);
    tile /= a.nx_tiles;
    const int o = (int)(tile % a.n_outer);
    tile /= a.n_outer;
    const int comp = (int)(tile % a.ncomp);
    const int traj = (int)(tile / a.ncomp);
    V* base = a.ptrs[traj] + comp * a.comp_stride + o * a.outer_stride + xt * COLS + col + t * a.stride;
    V* const buf[1] = {sm + col * LD};
    V v[1][R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[0][m] = base[(int64_t)m * TP * a.stride];
    __syncthreads();
    if constexpr (MODE == kColInv) {
        fft_pencil<N, R, +1, 1, Sync::Block>(v, buf, tws, t);
    } else {
        fft_pencil<N, R, -1, 1, Sync::Block>(v, buf, tws, t);
    }
    if constexpr (MODE == kColK || MODE == kColKConj) {
#pragma unroll
        for (int m = 0; m < R; ++m) v[0][m] = phmul<MODE == kColK ? -1 : +1>(v[0][m], a.ph[t + m * TP]);
        fft_pencil<N, R, +1, 1, Sync::Block>(v, buf, tws, t);
    }
#pragma unroll
    for (int m = 0; m < R; ++m) base[(int64_t)m * TP * a.stride] = v[0][m];
}

// Column pass over a contiguous batch, persistent and pipelined: each block walks its
// tiles (COLS adjacent x columns x N pencil points of one component), the TMA engine
// loads tile i+1 while tile i is transformed, and stores each finished tile back through
// the same tensor map.  ZPASS: pencils along z of a 3D map {2 nx, ny, nz 3 ntraj};
// otherwise pencils along y of a 2D map {2 nx, rows}.  FWD_ONLY: forward FFT only.

template <typename T>
struct ColTmaArgs {
    int32_t n_tiles;     // tiles in the whole launch
    int32_t nx_tiles;    // nx / COLS
    int32_t ny;          // ZPASS: points along y (tile -> y, component-trajectory)
    const twel<T>* tw;   // stage twiddles of FftPlan<N, R>
    const twel<T>* ph;   // phase table (unused when FWD_ONLY)
    int* status;
    uint32_t wait_first; // 0 = default poll limit of each block's first wait, else 1 + that limit
};

// Elements of one tile buffer: the tile ([N][COLS], as the TMA engine writes it) and,
// once every thread holds its points, the COLS padded exchange pencils of the transform,
// rounded to whole 128-byte lines so the second buffer is as aligned as the first.
template <typename T, int N, int COLS>
constexpr int colpass_tma_buf() {
    constexpr int E = N * COLS > COLS * smem_ld_cols<T>(N, COLS) ? N * COLS : COLS * smem_ld_cols<T>(N, COLS);
    constexpr int L = 128 / (int)sizeof(cplx<T>);
    return (E + L - 1) / L * L;
}

template <typename T, int N, int COLS>
constexpr size_t colpass_tma_smem() {
    return (size_t)2 * colpass_tma_buf<T, N, COLS>() * sizeof(cplx<T>);
}

template <typename T, int N, int R, int COLS, bool FWD_ONLY, bool ZPASS>
__global__ void __launch_bounds__(COLS * (N / R), (COLS * (N / R)) < 512 ? 512 / (COLS * (N / R)) : 1)
k_colpass_tma(const __grid_constant__ CUtensorMap tmap, const ColTmaArgs<T> a) {
    using V = cplx<T>;
    constexpr int TP = N / R;
    constexpr int LD = smem_ld_cols<T>(N, COLS);
    constexpr int SB = colpass_tma_buf<T, N, COLS>();
    constexpr int TWN = FftPlan<N, R>::tw_size();
    constexpr int BOX = N < 256 ? N : 256;
    constexpr int NBOX = N / BOX;
    constexpr uint32_t TILE_BYTES = (uint32_t)(N * COLS * sizeof(V));
    extern __shared__ __align__(128) unsigned char smraw[];
    V* buf = reinterpret_cast<V*>(smraw);                                   // [2][SB]
    twel<T>* tws = reinterpret_cast<twel<T>*>(buf + 2 * SB);
    uint64_t* bar = reinterpret_cast<uint64_t*>(tws + TWN);
    // the phase table, copied once per (persistent) block: its global loads sat between
    // the two transforms of every tile
    twel<T>* phs = reinterpret_cast<twel<T>*>(bar + 2);
    const int col = threadIdx.x % COLS, t = threadIdx.x / COLS;
    const void* map = &tmap;

    auto coords = [&](int tile, int& c0, int& c1, int& c2) {
        const int xt = tile % a.nx_tiles;
        const int rest = tile / a.nx_tiles;
        c0 = xt * 2 * COLS;
        if constexpr (ZPASS) {
            c1 = rest % a.ny;
            c2 = (rest / a.ny) * N;
        } else {
            c1 = rest * N;
            c2 = 0;
        }
    };
    auto issue_load = [&](int tile, int st) {
        int c0, c1, c2;
        coords(tile, c0, c1, c2);
        V* dst = buf + st * SB;
        mbar_expect_tx(&bar[st], TILE_BYTES);
#pragma unroll
        for (int b = 0; b < NBOX; ++b) {
            if constexpr (ZPASS) tma_load_3d(dst + b * BOX * COLS, map, c0, c1, c2 + b * BOX, &bar[st]);
            else tma_load_2d(dst + b * BOX * COLS, map, c0, c1 + b * BOX, &bar[st]);
        }
    };
    auto issue_store = [&](int tile, int st) {
        int c0, c1, c2;
        coords(tile, c0, c1, c2);
        const V* src = buf + st * SB;
#pragma unroll
        for (int b = 0; b < NBOX; ++b) {
            if constexpr (ZPASS) tma_store_3d(map, c0, c1, c2 + b * BOX, src + b * BOX * COLS);
            else tma_store_2d(map, c0, c1 + b * BOX, src + b * BOX * COLS);
        }
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    __syncthreads();
    const int first = blockIdx.x, stride = gridDim.x;
    if (threadIdx.x == 0) {
        if (first < a.n_tiles) issue_load(first, 0);
        if (first + stride < a.n_tiles) issue_load(first + stride, 1);
    }
    copy_table(tws, a.tw, TWN);
    if constexpr (!FWD_ONLY) copy_table(phs, a.ph, N);
    __syncthreads();
    int it = 0;
    int failed_tile = -1;
    for (int tile = first; tile < a.n_tiles; tile += stride, ++it) {
        const int st = it & 1;
        V* bs = buf + st * SB;
        const uint32_t lim = it == 0 ? first_wait_limit(a.wait_first) : kWaitLimit;
        if (!__syncthreads_and(mbar_wait(&bar[st], (uint32_t)((it >> 1) & 1), lim))) {
            failed_tile = tile;
            break;
        }
        V v[1][R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[0][m] = bs[(t + m * TP) * COLS + col];
        // The transform exchanges through the same buffer (column col at bs + col LD): every
        // thread must hold its points first.  Each exchange ends with a barrier after its
        // reads, so the results can be written back in tile order right after the transform.
        __syncthreads();
        V* const xb[1] = {bs + col * LD};
        fft_pencil<N, R, -1, 1, Sync::Block>(v, xb, tws, t);
        if constexpr (!FWD_ONLY) {
#pragma unroll
            for (int m = 0; m < R; ++m) v[0][m] = phmul<-1>(v[0][m], phs[t + m * TP]);
            fft_pencil<N, R, +1, 1, Sync::Block>(v, xb, tws, t);
        }
#pragma unroll
        for (int m = 0; m < R; ++m) bs[(t + m * TP) * COLS + col] = v[0][m];
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            issue_store(tile, st);
            bulk_commit();
            const int nxt = tile + 2 * stride;
            if (nxt < a.n_tiles) {
                bulk_wait_read_all();
                issue_load(nxt, st);
            }
        }
    }
    if (threadIdx.x == 0) {
        if (failed_tile >= 0) {
            atomicCAS(a.status, 0, (int)GPE_ETIMEOUT);
            // Let the loads still in flight land before the block's shared memory goes away:
            // the one the expired wait was for and, if it was issued, the next tile's (loads
            // run two tiles ahead, so that one exists exactly when the next tile does).
            mbar_wait(&bar[it & 1], (uint32_t)((it >> 1) & 1), kWaitLimit);
            if (failed_tile + stride < a.n_tiles)
                mbar_wait(&bar[(it + 1) & 1], (uint32_t)(((it + 1) >> 1) & 1), kWaitLimit);
        }
        bulk_wait_all();
    }
}

// FFT along x of independent rows (one component per row), in place: DIR = -1 forward,
// +1 unnormalised inverse.
template <typename T, int N, int R, int DIR>
__global__ void __launch_bounds__(rows_per_cta<N, R>() * (N / R))
k_rowfft(cplx<T>* __restrict__ data, int64_t rows, const twel<T>* __restrict__ tw) {
    using V = cplx<T>;
    constexpr int TP = N / R;
    constexpr int RPC = rows_per_cta<N, R>();
    constexpr int LD = smem_ld<T>(N);
    constexpr int TWN = FftPlan<N, R>::tw_size();
    extern __shared__ __align__(128) unsigned char smraw[];
    V* sm = reinterpret_cast<V*>(smraw);
    twel<T>* tws = reinterpret_cast<twel<T>*>(sm + tw_off<T>(RPC * LD));
    copy_table(tws, tw, TWN);
    const int lrow = threadIdx.x / TP, t = threadIdx.x % TP;
    const int64_t grow = (int64_t)blockIdx.x * RPC + lrow;
    const bool valid = grow < rows;
    V* base = data + (valid ? grow : 0) * N + t;
    V* const buf[1] = {sm + lrow * LD};
    V v[1][R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[0][m] = valid ? base[m * TP] : mk((T)0, (T)0);
    __syncthreads();
    fft_pencil<N, R, DIR, 1, Sync::Block>(v, buf, tws, t);
    if (valid) {
#pragma unroll
        for (int m = 0; m < R; ++m) base[m * TP] = v[0][m];
    }
}

// ---------------------------------------------------------------- launch helpers

template <typename K>
inline cudaError_t launch_with_smem(K kernel, int grid, int block, size_t smem, cudaStream_t s,
                                    const void* arg) {
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    void* args[] = {const_cast<void*>(arg)};
    return cudaLaunchKernel((const void*)kernel, dim3(grid), dim3(block), args, smem, s);
}

template <typename T, int N, int THREADS = 0, bool CPH = false>
cudaError_t xpass_n(bool pre, const PassArgs<T>& a, cudaStream_t s) {
    constexpr int R = Tune<T>::kXR;
    constexpr int TP = N / R;
    constexpr int RPC = xpass_rows<N, R, THREADS>();
    const int64_t grid = (a.total_rows + RPC - 1) / RPC;
    if (pre)
        return launch_with_smem(k_xpass<T, N, R, true, THREADS, CPH>, (int)grid, RPC * TP,
                                xpass_smem<T, N, R, THREADS, CPH, true>(), s, &a);
    return launch_with_smem(k_xpass<T, N, R, false, THREADS, CPH>, (int)grid, RPC * TP,
                            xpass_smem<T, N, R, THREADS, CPH, false>(), s, &a);
}

// Block sizes the FP32 x pass is built for (the tuner's candidates); 0 = the default.
constexpr int kXpassThreads[2] = {128, 256};

template <typename T, int N, int MODE>
cudaError_t colpass_n(const PassArgs<T>& a, cudaStream_t s) {
    constexpr int R = Tune<T>::kColR(N);
    constexpr int COLS = Tune<T>::kColCols(N);
    const int64_t grid = (int64_t)a.ntraj * a.ncomp * a.n_outer * a.nx_tiles;
    const size_t smem = (size_t)tw_off<T>(COLS * smem_ld_cols<T>(N, COLS)) * sizeof(cplx<T>) +
                        FftPlan<N, R>::tw_size() * sizeof(twel<T>);
    return launch_with_smem(k_colpass<T, N, R, COLS, MODE>, (int)grid, COLS * (N / R), smem, s, &a);
}

// The persistent column pass is launched with as many blocks as can be resident at once
// (occupancy query, once per kernel): every SM holds the same number of blocks, each walks
// the tiles with the grid stride.  The launch bounds cap a thread at 128 registers (512
// threads per SM); at 512 (FP32, 4 columns) that is 4 blocks per SM with 42 KB of shared
// memory each (3 while the exchange had a buffer of its own).  More blocks than fit would
// run as a second, partial wave.
template <typename T, int N, int COLS, bool FWD_ONLY, bool ZPASS>
cudaError_t colpass_tma_n(const CUtensorMap& map, const ColTmaArgs<T>& a, int sms, cudaStream_t s) {
    constexpr int R = Tune<T>::kColR(N);
    constexpr int THREADS = COLS * (N / R);
    const size_t smem = colpass_tma_smem<T, N, COLS>() + FftPlan<N, R>::tw_size() * sizeof(twel<T>) + 16 +
                        (FWD_ONLY ? 0 : (size_t)N * sizeof(twel<T>));
    auto kern = k_colpass_tma<T, N, R, COLS, FWD_ONLY, ZPASS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    static const int per_sm = [&] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, THREADS, smem) != cudaSuccess) {
            cudaGetLastError();
            b = 1;
        }
        return b > 0 ? b : 1;
    }();
    const int cap = per_sm * sms;
    const int grid = a.n_tiles < cap ? a.n_tiles : cap;
    kern<<<grid, THREADS, smem, s>>>(map, a);
    return cudaGetLastError();
}

template <typename T, int N, int DIR>
cudaError_t rowfft_n(cplx<T>* data, int64_t rows, const twel<T>* const* tw, cudaStream_t s) {
    constexpr int R = Tune<T>::kRowR(N);
    constexpr int TP = N / R;
    constexpr int RPC = rows_per_cta<N, R>();
    const int64_t grid = (rows + RPC - 1) / RPC;
    const size_t smem = (size_t)tw_off<T>(RPC * smem_ld<T>(N)) * sizeof(cplx<T>) + FftPlan<N, R>::tw_size() * sizeof(twel<T>);
    auto kern = k_rowfft<T, N, R, DIR>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<(int)grid, RPC * TP, smem, s>>>(data, rows, tw[tw_slot<R>()]);
    return cudaGetLastError();
}


}  // namespace gpe
