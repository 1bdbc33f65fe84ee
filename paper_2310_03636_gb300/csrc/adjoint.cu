// Adjoint of one split step and the late-time spin structure factor loss.
//
// One forward step is psi_{n+1} = K(dt/2) L_n K(dt/2) psi_n (K unitary, q_n at the step
// midpoint).  Its pullback is g_n = K(-dt/2) L_n^T(phi) K(-dt/2) g_{n+1} with
// phi = K(dt/2) psi_n the input of the local step; K's adjoint is K with conjugated
// phases.  L_n^T is the hand-written per-site reverse mode of adjoint.cuh, which also
// yields dL/dq_n, reduced in FP64 in a fixed order and distributed onto the q(t) knots
// with the piecewise-linear interpolation weights of t_n + dt/2.
//
// Loss: L = (1/ntraj) sum_traj sum_{kmin <= |k| <= kmax} S_perp(k) with
// S_perp(k) = dx^d |X(k)|^2 / N, X = unnormalised DFT of F_perp = sqrt2 (psi_1^* psi_0 +
// psi_0^* psi_-1).  Its gradient: g_X = 2 c mask X (c = dx^d / (N ntraj)), g_F = the
// unnormalised inverse DFT of g_X (the DFT's adjoint), then through the bilinear F_perp.
#include <cmath>

#include "adjoint.cuh"
#include "adjoint.h"
#include "prop_kernels.cuh"

namespace gpe {

namespace {

constexpr int kAdjThreads = 256;

template <int NV>
__device__ __forceinline__ void adj_block_sum(double (&v)[NV], double* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) sm[k * 32 + warp] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sm[k * 32 + w];
            v[k] = s;
        }
    }
    __syncthreads();
}

template <typename T> constexpr int adj_r() { return 4; }

// Rows along x of all three components: FFT_x, x ph (or conj(ph)), iFFT_x.
template <typename T, int N, int R, bool CONJ>
__global__ void __launch_bounds__(rows_per_cta<N, R>() * (N / R))
k_xkin(const AdjArgs<T> a, cplx<T>* __restrict__ field) {
    using V = cplx<T>;
    constexpr int TP = N / R;
    constexpr int RPC = rows_per_cta<N, R>();
    constexpr int LD = smem_ld<T>(N);
    constexpr int TWN = FftPlan<N, R>::tw_size();
    extern __shared__ __align__(128) unsigned char smraw[];
    V* sm = reinterpret_cast<V*>(smraw);
    twel<T>* tws = reinterpret_cast<twel<T>*>(sm + tw_off<T>(RPC * 3 * LD));
    copy_table(tws, a.tw[tw_slot<R>()], TWN);
    const int lrow = threadIdx.x / TP, t = threadIdx.x % TP;
    const int64_t grow = (int64_t)blockIdx.x * RPC + lrow;
    const bool valid = grow < a.total_rows;
    const int64_t g = valid ? grow : 0;
    const int64_t traj = g / a.rows_per_traj;
    V* base = field + traj * 3 * a.sites + (g - traj * a.rows_per_traj) * N + t;
    V* const buf[3] = {sm + (lrow * 3 + 0) * LD, sm + (lrow * 3 + 1) * LD, sm + (lrow * 3 + 2) * LD};
    V v[3][R];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < R; ++m) v[c][m] = valid ? base[c * a.sites + m * TP] : mk((T)0, (T)0);
    __syncthreads();
    fft_pencil<N, R, -1, 3, Sync::Block>(v, buf, tws, t);
#pragma unroll
    for (int m = 0; m < R; ++m) {
        const twel<T> f = a.ph[t + m * TP];
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c][m] = phmul<CONJ ? +1 : -1>(v[c][m], f);
    }
    fft_pencil<N, R, +1, 3, Sync::Block>(v, buf, tws, t);
    if (valid) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int m = 0; m < R; ++m) base[c * a.sites + m * TP] = v[c][m];
    }
}

// Adjoint x pass on the cotangent lam, given phi = K(dt/2) psi_n:
//   lam <- Kx(-dt/2) lam;  lam <- L^T(phi) lam (per site);  lam <- Kx(-dt/2) lam,
// with per-block FP64 partial sums of dL/dq.
template <typename T, int N, int R>
__global__ void __launch_bounds__(rows_per_cta<N, R>() * (N / R))
k_xadj(const AdjArgs<T> a, cplx<T>* __restrict__ lam, const cplx<T>* __restrict__ phi, double* __restrict__ part) {
    using V = cplx<T>;
    constexpr int TP = N / R;
    constexpr int RPC = rows_per_cta<N, R>();
    constexpr int LD = smem_ld<T>(N);
    constexpr int TWN = FftPlan<N, R>::tw_size();
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ double red[32];
    V* sm = reinterpret_cast<V*>(smraw);
    twel<T>* tws = reinterpret_cast<twel<T>*>(sm + tw_off<T>(RPC * 3 * LD));
    copy_table(tws, a.tw[tw_slot<R>()], TWN);
    const int lrow = threadIdx.x / TP, t = threadIdx.x % TP;
    const int64_t grow = (int64_t)blockIdx.x * RPC + lrow;
    const bool valid = grow < a.total_rows;
    const int64_t g = valid ? grow : 0;
    const int64_t traj = g / a.rows_per_traj;
    const int64_t site0 = (g - traj * a.rows_per_traj) * N + t;
    const int64_t off = traj * 3 * a.sites + site0;
    V* lbase = lam + off;
    const V* pbase = phi + off;
    V* const buf[3] = {sm + (lrow * 3 + 0) * LD, sm + (lrow * 3 + 1) * LD, sm + (lrow * 3 + 2) * LD};
    V v[3][R];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < R; ++m) v[c][m] = valid ? lbase[c * a.sites + m * TP] : mk((T)0, (T)0);
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            double dq[1] = {0.0};
            if (valid) {
#pragma unroll
                for (int m = 0; m < R; ++m) {
                    const V p[3] = {pbase[m * TP], pbase[a.sites + m * TP], pbase[2 * a.sites + m * TP]};
                    V gg[3] = {v[0][m], v[1][m], v[2][m]};
                    const SitePot<T> vp = a.vpot ? site_pot<T>(a.vpot, a.sites, site0 + m * TP)
                                                 : SitePot<T>{(T)0, (T)0, (T)0};
                    dq[0] += (double)local_step_bwd<T>(p, gg, a.c0, a.c1, a.q, a.dt, vp);
                    v[0][m] = gg[0];
                    v[1][m] = gg[1];
                    v[2][m] = gg[2];
                }
            }
            adj_block_sum<1>(dq, red);
            if (threadIdx.x == 0) part[blockIdx.x] = dq[0];
        }
        fft_pencil<N, R, -1, 3, Sync::Block>(v, buf, tws, t);
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const twel<T> f = a.ph[t + m * TP];
#pragma unroll
            for (int c = 0; c < 3; ++c) v[c][m] = phmul<+1>(v[c][m], f);
        }
        fft_pencil<N, R, +1, 3, Sync::Block>(v, buf, tws, t);
    }
    if (valid) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int m = 0; m < R; ++m) lbase[c * a.sites + m * TP] = v[c][m];
    }
}

// dL/dq_n = sum of the partials (fixed order), spread onto the knots with the linear
// interpolation weights of q(t) at t = (n + 1/2) dt.
__global__ void k_dq_final(const double* __restrict__ part, int nparts, double t_mid, int n_knots, double t_end,
                           double* __restrict__ dLdq) {
    __shared__ double red[32];
    double acc[1] = {0.0};
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc[0] += part[i];
    adj_block_sum<1>(acc, red);
    if (threadIdx.x != 0) return;
    const double tot = acc[0];
    if (n_knots <= 1) {
        dLdq[0] += tot;
        return;
    }
    const double u = t_mid / t_end * (double)(n_knots - 1);
    if (u <= 0.0) {
        dLdq[0] += tot;
    } else if (u >= (double)(n_knots - 1)) {
        dLdq[n_knots - 1] += tot;
    } else {
        const int i = (int)floor(u);
        const double w = u - (double)i;
        dLdq[i] += (1.0 - w) * tot;
        dLdq[i + 1] += w * tot;
    }
}

__global__ void k_fill_ptrs(void** ptrs, char* base, int64_t stride_bytes, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) ptrs[i] = base + i * stride_bytes;
}

// F_perp of every site into W[traj][site].
template <typename T>
__global__ void k_fperp(const cplx<T>* __restrict__ psi, cplx<T>* __restrict__ W, int64_t sites, int64_t total) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t tr = i / sites, s = i - tr * sites;
        const cplx<T>* p = psi + tr * 3 * sites + s;
        const cplx<T> p1 = p[0], p0 = p[sites], pm = p[2 * sites];
        const T r2 = (T)1.41421356237309504880;
        const cplx<T> z = cadd(cmulc(p1, p0), cmulc(p0, pm));
        W[i] = cscale(z, r2);
    }
}

// Masked power of every mode: loss partials, and X <- 2 c mask X (the gradient w.r.t. X).
template <typename T>
__global__ void __launch_bounds__(kAdjThreads)
k_sf_mask(cplx<T>* __restrict__ W, int64_t sites, int64_t total, int nx, int ny, int nz, double dx, double kmin,
          double kmax, double c, double* __restrict__ part) {
    __shared__ double red[32];
    const double two_pi = 6.283185307179586476925286766559;
    double acc[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i % sites;
        const int ix = (int)(s % nx), iy = (int)((s / nx) % ny), iz = (int)(s / ((int64_t)nx * ny));
        const int jx = ix < (nx + 1) / 2 ? ix : ix - nx, jy = iy < (ny + 1) / 2 ? iy : iy - ny,
                  jz = iz < (nz + 1) / 2 ? iz : iz - nz;
        const double kx = two_pi * jx / (nx * dx), ky = two_pi * jy / (ny * dx), kz = two_pi * jz / (nz * dx);
        const double ka = sqrt(kx * kx + ky * ky + kz * kz);
        const bool in = ka >= kmin && ka <= kmax;
        const cplx<T> x = W[i];
        if (in) acc[0] += c * ((double)x.x * x.x + (double)x.y * x.y);
        W[i] = in ? cscale(x, (T)(2.0 * c)) : mk((T)0, (T)0);
    }
    adj_block_sum<1>(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
}

// Seed: lam = pullback of F_perp with g_F in W (sqrt2 factor applied here).
template <typename T>
__global__ void k_sf_seed(const cplx<T>* __restrict__ psi, const cplx<T>* __restrict__ W, cplx<T>* __restrict__ lam,
                          int64_t sites, int64_t total, double scale) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t tr = i / sites, s = i - tr * sites;
        const cplx<T>* p = psi + tr * 3 * sites + s;
        cplx<T>* l = lam + tr * 3 * sites + s;
        const cplx<T> p1 = p[0], p0 = p[sites], pm = p[2 * sites];
        const cplx<T> gz = cscale(W[i], (T)(1.41421356237309504880 * scale));
        const cplx<T> cg = cconj(gz);
        l[0] = cmul(p0, cg);
        l[sites] = cadd(cmul(p1, gz), cmul(pm, cg));
        l[2 * sites] = cmul(p0, gz);
    }
}

__global__ void k_sum_final(const double* __restrict__ part, int nparts, double* __restrict__ out) {
    __shared__ double red[32];
    double acc[1] = {0.0};
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc[0] += part[i];
    adj_block_sum<1>(acc, red);
    if (threadIdx.x == 0) out[0] = acc[0];
}

template <typename T, int N>
cudaError_t xkin_n(const AdjArgs<T>& a, cplx<T>* field, bool conj, cudaStream_t s) {
    constexpr int R = adj_r<T>();
    constexpr int TP = N / R;
    constexpr int RPC = rows_per_cta<N, R>();
    const int64_t grid = (a.total_rows + RPC - 1) / RPC;
    const size_t smem = (size_t)tw_off<T>(RPC * 3 * smem_ld<T>(N)) * sizeof(cplx<T>) + FftPlan<N, R>::tw_size() * sizeof(twel<T>);
    auto kern = conj ? k_xkin<T, N, R, true> : k_xkin<T, N, R, false>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<(int)grid, RPC * TP, smem, s>>>(a, field);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t xadj_n(const AdjArgs<T>& a, cplx<T>* lam, const cplx<T>* phi, double* part, int* nparts, cudaStream_t s) {
    constexpr int R = adj_r<T>();
    constexpr int TP = N / R;
    constexpr int RPC = rows_per_cta<N, R>();
    const int64_t grid = (a.total_rows + RPC - 1) / RPC;
    *nparts = (int)grid;
    const size_t smem = (size_t)tw_off<T>(RPC * 3 * smem_ld<T>(N)) * sizeof(cplx<T>) + FftPlan<N, R>::tw_size() * sizeof(twel<T>);
    auto kern = k_xadj<T, N, R>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<(int)grid, RPC * TP, smem, s>>>(a, lam, phi, part);
    return cudaGetLastError();
}

#define GPE_NSWITCH(CALL)                \
    switch (n) {                         \
        case 64: return CALL(64);        \
        case 128: return CALL(128);      \
        case 256: return CALL(256);      \
        case 512: return CALL(512);      \
        case 1024: return CALL(1024);    \
        default: return cudaErrorInvalidValue; \
    }

}  // namespace

template <typename T>
int64_t adjoint_parts(const Group& g) {
    const int n = g.n[0];
    const int R = adj_r<T>();
    const int tp = n / R;
    const int rpc = tp >= 256 ? 1 : 256 / tp;
    return ((int64_t)g.n[1] * g.n[2] * g.ntraj + rpc - 1) / rpc;
}

template <typename T>
cudaError_t launch_xkin(int n, const AdjArgs<T>& a, cplx<T>* field, bool conj, cudaStream_t s) {
#define GPE_XK(NN) xkin_n<T, NN>(a, field, conj, s)
    GPE_NSWITCH(GPE_XK)
#undef GPE_XK
}

template <typename T>
cudaError_t launch_xadj(int n, const AdjArgs<T>& a, cplx<T>* lam, const cplx<T>* phi, double* part, int* nparts,
                        cudaStream_t s) {
#define GPE_XA(NN) xadj_n<T, NN>(a, lam, phi, part, nparts, s)
    GPE_NSWITCH(GPE_XA)
#undef GPE_XA
}

cudaError_t launch_dq_final(const double* part, int nparts, double t_mid, int n_knots, double t_end, double* dLdq,
                            cudaStream_t s) {
    k_dq_final<<<1, kAdjThreads, 0, s>>>(part, nparts, t_mid, n_knots, t_end, dLdq);
    return cudaGetLastError();
}

cudaError_t launch_fill_ptrs(void** ptrs, void* base, int64_t stride_bytes, int n, cudaStream_t s) {
    k_fill_ptrs<<<(n + 127) / 128, 128, 0, s>>>(ptrs, static_cast<char*>(base), stride_bytes, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fperp(const cplx<T>* psi, cplx<T>* W, int64_t sites, int64_t total, cudaStream_t s) {
    const int64_t grid = std::min<int64_t>((total + 255) / 256, 152 * 16);
    k_fperp<T><<<(int)grid, 256, 0, s>>>(psi, W, sites, total);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sf_mask(cplx<T>* W, int64_t sites, int64_t total, const int n[3], double dx, double kmin, double kmax,
                           double c, double* part, int* nparts, cudaStream_t s) {
    const int grid = (int)std::min<int64_t>((total + kAdjThreads - 1) / kAdjThreads, 152 * 8);
    *nparts = grid;
    k_sf_mask<T><<<grid, kAdjThreads, 0, s>>>(W, sites, total, n[0], n[1], n[2], dx, kmin, kmax, c, part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sf_seed(const cplx<T>* psi, const cplx<T>* W, cplx<T>* lam, int64_t sites, int64_t total,
                           double scale, cudaStream_t s) {
    const int64_t grid = std::min<int64_t>((total + 255) / 256, 152 * 16);
    k_sf_seed<T><<<(int)grid, 256, 0, s>>>(psi, W, lam, sites, total, scale);
    return cudaGetLastError();
}

cudaError_t launch_sum_final(const double* part, int nparts, double* out, cudaStream_t s) {
    k_sum_final<<<1, kAdjThreads, 0, s>>>(part, nparts, out);
    return cudaGetLastError();
}

template int64_t adjoint_parts<float>(const Group&);
template int64_t adjoint_parts<double>(const Group&);
template cudaError_t launch_xkin<float>(int, const AdjArgs<float>&, cplx<float>*, bool, cudaStream_t);
template cudaError_t launch_xkin<double>(int, const AdjArgs<double>&, cplx<double>*, bool, cudaStream_t);
template cudaError_t launch_xadj<float>(int, const AdjArgs<float>&, cplx<float>*, const cplx<float>*, double*, int*,
                                        cudaStream_t);
template cudaError_t launch_xadj<double>(int, const AdjArgs<double>&, cplx<double>*, const cplx<double>*, double*, int*,
                                         cudaStream_t);
template cudaError_t launch_fperp<float>(const cplx<float>*, cplx<float>*, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_fperp<double>(const cplx<double>*, cplx<double>*, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_sf_mask<float>(cplx<float>*, int64_t, int64_t, const int*, double, double, double, double,
                                           double*, int*, cudaStream_t);
template cudaError_t launch_sf_mask<double>(cplx<double>*, int64_t, int64_t, const int*, double, double, double, double,
                                            double*, int*, cudaStream_t);
template cudaError_t launch_sf_seed<float>(const cplx<float>*, const cplx<float>*, cplx<float>*, int64_t, int64_t,
                                           double, cudaStream_t);
template cudaError_t launch_sf_seed<double>(const cplx<double>*, const cplx<double>*, cplx<double>*, int64_t, int64_t,
                                            double, cudaStream_t);

}  // namespace gpe
