// Resident 1D propagation of long grids on a thread-block cluster.
//
// A trajectory of N = C M points is held by a cluster of C blocks, block c owning the
// contiguous sites [c M, (c+1) M) of all three components in shared memory for all steps.
// The length-N transform splits as one radix-C step across the cluster and length-M
// transforms inside each block (decimation in frequency):
//   X[C k' + r] = FFT_M( y_r )[k'],   y_r[n'] = W_N^{n' r} sum_c x[n' + c M] W_C^{c r},
// so block r gathers x[n' + c M] from every block c through distributed shared memory,
// transforms locally, multiplies by the kinetic phase of k = C k' + r, transforms back,
// and the inverse radix-C step  x[n' + c M] = sum_r W_C^{-c r} W_N^{-n' r} z_r[n']
// gathers z_r from every block r.  The 1/N normalisation is in the phase table.  All
// blocks of a cluster execute the same sequence of cluster barriers.
#include <cooperative_groups.h>

#include "prop_kernels.cuh"
#include "res1d_tmem.cuh"

namespace cg = cooperative_groups;

namespace gpe {

namespace {

// a * W_C^{e} (DIR = -1) or a * W_C^{-e} (DIR = +1) for C in {2, 4, 8}: e counted in C-ths.
template <int C, int DIR, typename V>
__device__ __forceinline__ V twc_rank(V a, int e) {
    return twc16<DIR>(a, (e * (16 / C)) & 15);
}

// Entries of the local transform's stage-twiddle table kept in shared memory (those of
// its first twiddled stage; the rest are read through L1), and the block's shared memory:
// the three component slices and that table head.
template <typename T, int M, int R>
constexpr int res1d_cluster_tw_split() {
    using P = FftPlan<M, R>;
    return P::kStages > 2 ? P::tw_offset(2) : P::tw_size();
}

template <typename T, int M, int R>
constexpr size_t res1d_cluster_smem() {
    return (size_t)tw_off<T>(3 * smem_ld<T>(M)) * sizeof(cplx<T>) +
           (size_t)res1d_cluster_tw_split<T, M, R>() * sizeof(twel<T>);
}

// Blocks per SM the cluster kernel is compiled for: as many as its shared memory allows.
template <typename T, int M, int R>
constexpr int res1d_cluster_blocks() {
    const int b = (227 * 1024) / ((int)res1d_cluster_smem<T, M, R>() + 1024);
    return b < 1 ? 1 : (b > 8 ? 8 : b);
}

// Block ``rank`` keeps its slice [rank M, (rank+1) M) of the three components in shared
// memory (element n of component c at buf[c LD + spad(n)]) for all steps; the kinetic step
// handles one component at a time with its R points per thread in registers, so the kernel
// stays small (the form holding all three components in registers was instruction-fetch
// bound).  Per component: gather the radix-C inputs from every block, barrier (all reads
// done before the slice is overwritten), local transforms and phase, publish z_rank,
// barrier, gather the inverse radix-C step, barrier, store the new slice.  FP32 slices of
// 4096 points keep each thread's last-stage twiddles and full-step phases in tensor memory
// (res1d_tmem.cuh), as the resident kernel does.
template <typename T, int M, int R, int C, bool TMW = true>
__global__ void __launch_bounds__(M / R, res1d_cluster_blocks<T, M, R>())
k_res1d_cluster(const Res1DArgs<T> a, const twel<T>* __restrict__ tw_local, const twel<T>* __restrict__ wn) {
    using V = cplx<T>;
    constexpr int TP = M / R;
    constexpr int N = C * M;
    constexpr int LD = smem_ld<T>(M);
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    extern __shared__ __align__(128) unsigned char smraw[];
    V* buf = reinterpret_cast<V*>(smraw);                                  // [3][LD]
    constexpr int SPLIT = res1d_cluster_tw_split<T, M, R>();
    twel<T>* tws_s = reinterpret_cast<twel<T>*>(buf + tw_off<T>(3 * LD));   // table head
    const int t = threadIdx.x;
    const int traj = blockIdx.x / C;
    V* g = a.ptrs[traj] + rank * M;
    const V* rbuf[C];
#pragma unroll
    for (int c = 0; c < C; ++c) rbuf[c] = cl.map_shared_rank(buf, c);
    constexpr bool TM = TMW && res1d_tmem<T, M, R, 1>();
    __shared__ uint32_t tslot;
    uint32_t tbase = 0, ta = 0;
    if constexpr (TM) {
        tbase = res1d_tmem_open(&tslot, res1d_tmem_cols<M>());
        ta = res1d_tmem_row(tbase);
        res1d_tmem_fill<M>(ta, tw_local, a.ph_full, C, rank, t);
    }
    copy_table(tws_s, tw_local, SPLIT);
#pragma unroll 1
    for (int c = 0; c < 3; ++c)
        for (int i = t; i < M; i += TP) buf[c * LD + spad(i)] = g[c * N + i];

    auto kinetic = [&](const twel<T>* __restrict__ ph, bool ph_tmem) {
        cl.sync();   // every block's slices are final (loads, local step) before they are read
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            V v[1][R];
#pragma unroll
            for (int m = 0; m < R; ++m) {
                const int n = t + m * TP;
                V acc = mk((T)0, (T)0);
#pragma unroll
                for (int src = 0; src < C; ++src) acc = cadd(acc, twc_rank<C, -1>(rbuf[src][c * LD + spad(n)], src * rank));
                v[0][m] = twmul<-1>(acc, wn[rank * M + n]);
            }
            cl.sync();   // all reads of component c done before it is overwritten
            V* const fb[1] = {buf + c * LD};
            if constexpr (TM) {
                fft_tmem<M, -1>(v, fb, tws_s, ta, t);
                if (ph_tmem) {
                    phase_tmem(v[0], ta);
                } else {
#pragma unroll
                    for (int m = 0; m < R; ++m) v[0][m] = phmul<-1>(v[0][m], ph[C * (t + m * TP) + rank]);
                }
                fft_tmem<M, +1>(v, fb, tws_s, ta, t);
            } else {
                fft_pencil_split<M, R, -1, 1, Sync::Block, SPLIT>(v, fb, tws_s, tw_local, t);
#pragma unroll
                for (int m = 0; m < R; ++m) v[0][m] = phmul<-1>(v[0][m], ph[C * (t + m * TP) + rank]);
                fft_pencil_split<M, R, +1, 1, Sync::Block, SPLIT>(v, fb, tws_s, tw_local, t);
            }
#pragma unroll
            for (int m = 0; m < R; ++m) buf[c * LD + spad(t + m * TP)] = v[0][m];
            cl.sync();   // z_rank published
#pragma unroll
            for (int m = 0; m < R; ++m) {
                const int n = t + m * TP;
                V acc = mk((T)0, (T)0);
#pragma unroll
                for (int src = 0; src < C; ++src) {
                    const V z = twmul<+1>(rbuf[src][c * LD + spad(n)], wn[src * M + n]);
                    acc = cadd(acc, twc_rank<C, +1>(z, src * rank));
                }
                v[0][m] = acc;
            }
            cl.sync();   // all reads of z done before the new slice replaces it
#pragma unroll
            for (int m = 0; m < R; ++m) buf[c * LD + spad(t + m * TP)] = v[0][m];
        }
        __syncthreads();
    };

    kinetic(a.ph_half, false);
    LocalCoef<T> coef{a.c0, a.c1, (T)a.q_const, a.dt, a.kind};
    for (int64_t s = 0; s < a.nsteps; ++s) {
        coef.q = (T)q_at(a.t0 + ((double)s + 0.5) * a.dt_d, a.q_const, a.knots, a.n_knots, a.t_end);
        if (a.vpot == nullptr) {
            local_step_sites<T>(buf, buf + LD, buf + 2 * LD, t, M, TP, coef, [](int i) { return spad(i); });
        } else {
#pragma unroll 2
            for (int i = t; i < M; i += TP) {
                const int k = spad(i);
                V p1 = buf[k], p0 = buf[LD + k], pm = buf[2 * LD + k];
                local_step<true, T>(p1, p0, pm, coef, site_pot<T>(a.vpot, N, rank * M + i));
                buf[k] = p1;
                buf[LD + k] = p0;
                buf[2 * LD + k] = pm;
            }
        }
        const bool last = s == a.nsteps - 1;
        kinetic(last ? a.ph_half : a.ph_full, !last);
    }
#pragma unroll 1
    for (int c = 0; c < 3; ++c)
        for (int i = t; i < M; i += TP) g[c * N + i] = buf[c * LD + spad(i)];
    if constexpr (TM) res1d_tmem_close(tbase, res1d_tmem_cols<M>());
}

template <typename T, int M, int R, int C>
cudaError_t res1d_cluster_n(const Res1DArgs<T>& a, const twel<T>* tw_local, const twel<T>* wn, cudaStream_t s) {
    auto kern = k_res1d_cluster<T, M, R, C, true>;
    if constexpr (res1d_tmem<T, M, R, 1>()) {
        if (!tables_in_tmem()) kern = k_res1d_cluster<T, M, R, C, false>;
    }
    const size_t smem = res1d_cluster_smem<T, M, R>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.ntraj * C));
    cfg.blockDim = dim3(M / R);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a, tw_local, wn);
}

}  // namespace

template <> int res1d_cluster_block<float>() { return 4096; }
template <> int res1d_cluster_block<double>() { return 2048; }

template <>
cudaError_t launch_res1d_cluster<float>(int n, const Res1DArgs<float>& a, const twel<float>* tw_local,
                                        const twel<float>* wn, cudaStream_t s) {
    switch (n) {
        case 8192: return res1d_cluster_n<float, 4096, 16, 2>(a, tw_local, wn, s);
        case 16384: return res1d_cluster_n<float, 4096, 16, 4>(a, tw_local, wn, s);
        case 32768: return res1d_cluster_n<float, 4096, 16, 8>(a, tw_local, wn, s);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_res1d_cluster<double>(int n, const Res1DArgs<double>& a, const twel<double>* tw_local,
                                         const twel<double>* wn, cudaStream_t s) {
    switch (n) {
        case 4096: return res1d_cluster_n<double, 2048, 8, 2>(a, tw_local, wn, s);
        case 8192: return res1d_cluster_n<double, 2048, 8, 4>(a, tw_local, wn, s);
        case 16384: return res1d_cluster_n<double, 2048, 8, 8>(a, tw_local, wn, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gpe
