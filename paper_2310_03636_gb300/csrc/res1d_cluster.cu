// Resident 1D propagation of long grids on a thread-block cluster.
//
// A trajectory of N = C M points is held by a cluster of C blocks, block c owning the
// contiguous sites [c M, (c+1) M) of all three components in registers for all steps.
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

namespace cg = cooperative_groups;

namespace gpe {

namespace {

// a * W_C^{e} (DIR = -1) or a * W_C^{-e} (DIR = +1) for C in {2, 4, 8}: e counted in C-ths.
template <int C, int DIR, typename V>
__device__ __forceinline__ V twc_rank(V a, int e) {
    return twc16<DIR>(a, (e * (16 / C)) & 15);
}

template <typename T, int M, int R, int C>
__global__ void __launch_bounds__(M / R)
k_res1d_cluster(const Res1DArgs<T> a, const twel<T>* __restrict__ tw_local, const twel<T>* __restrict__ wn) {
    using V = cplx<T>;
    constexpr int TP = M / R;
    constexpr int N = C * M;
    constexpr int LD = smem_ld<T>(M);
    constexpr int TWN = FftPlan<M, R>::tw_size();
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    extern __shared__ __align__(128) unsigned char smraw[];
    V* buf = reinterpret_cast<V*>(smraw);                                  // [3][LD]
    twel<T>* tws = reinterpret_cast<twel<T>*>(buf + tw_off<T>(3 * LD));
    copy_table(tws, tw_local, TWN);
    const int t = threadIdx.x;
    const int traj = blockIdx.x / C;
    V* base = a.ptrs[traj] + rank * M + t;
    V* const fb[3] = {buf, buf + LD, buf + 2 * LD};
    const V* rbuf[C];
#pragma unroll
    for (int c = 0; c < C; ++c) rbuf[c] = cl.map_shared_rank(buf, c);
    V v[3][R];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < R; ++m) v[c][m] = base[c * N + m * TP];
    __syncthreads();

    auto kinetic = [&](const twel<T>* __restrict__ ph) {
        // publish this block's sites, gather the radix-C inputs of spectrum class ``rank``
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int m = 0; m < R; ++m) buf[c * LD + t + m * TP] = v[c][m];
        cl.sync();
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const int n = t + m * TP;
            const twel<T> w = wn[rank * M + n];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                V acc = mk((T)0, (T)0);
#pragma unroll
                for (int src = 0; src < C; ++src) acc = cadd(acc, twc_rank<C, -1>(rbuf[src][c * LD + n], src * rank));
                v[c][m] = twmul<-1>(acc, w);
            }
        }
        cl.sync();
        fft_pencil<M, R, -1, 3, Sync::Block>(v, fb, tws, t);
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const twel<T> f = ph[C * (t + m * TP) + rank];
#pragma unroll
            for (int c = 0; c < 3; ++c) v[c][m] = phmul<-1>(v[c][m], f);
        }
        fft_pencil<M, R, +1, 3, Sync::Block>(v, fb, tws, t);
        // publish z_rank, gather the inverse radix-C step for this block's sites
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int m = 0; m < R; ++m) buf[c * LD + t + m * TP] = v[c][m];
        cl.sync();
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const int n = t + m * TP;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                V acc = mk((T)0, (T)0);
#pragma unroll
                for (int src = 0; src < C; ++src) {
                    const V z = twmul<+1>(rbuf[src][c * LD + n], wn[src * M + n]);
                    acc = cadd(acc, twc_rank<C, +1>(z, src * rank));
                }
                v[c][m] = acc;
            }
        }
        cl.sync();
    };

    kinetic(a.ph_half);
    LocalCoef<T> coef{a.c0, a.c1, (T)a.q_const, a.dt, a.kind};
    for (int64_t s = 0; s < a.nsteps; ++s) {
        coef.q = (T)q_at(a.t0 + ((double)s + 0.5) * a.dt_d, a.q_const, a.knots, a.n_knots, a.t_end);
        if (a.vpot == nullptr) {
#pragma unroll
            for (int m = 0; m < R; ++m) local_step<T>(v[0][m], v[1][m], v[2][m], coef);
        } else {
#pragma unroll
            for (int m = 0; m < R; ++m)
                local_step<true, T>(v[0][m], v[1][m], v[2][m], coef, site_pot<T>(a.vpot, N, rank * M + t + m * TP));
        }
        kinetic(s == a.nsteps - 1 ? a.ph_half : a.ph_full);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < R; ++m) base[c * N + m * TP] = v[c][m];
}

template <typename T, int M, int R, int C>
cudaError_t res1d_cluster_n(const Res1DArgs<T>& a, const twel<T>* tw_local, const twel<T>* wn, cudaStream_t s) {
    auto kern = k_res1d_cluster<T, M, R, C>;
    const size_t smem = (size_t)tw_off<T>(3 * smem_ld<T>(M)) * sizeof(cplx<T>) + FftPlan<M, R>::tw_size() * sizeof(twel<T>);
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
