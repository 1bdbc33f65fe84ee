// Observables pipeline (sample times only; the fields are read, never written):
//   1. k_obs_prep   real space, per site: copy psi_m and F_perp = sqrt2 (psi_1^* psi_0 +
//                   psi_0^* psi_-1) into a 4-field workspace; FP64 partial sums of N_m,
//                   q (n_1 + n_-1), c0 rho^2 / 2, c1 (F_z^2 + |F_perp|^2) / 2 and, with a
//                   potential, sum_m V_m n_m per site block;
//   2. forward FFTs of the 4 fields along every axis (same pencil FFT as the propagation);
//      1D grids longer than one block's transform (N = C M, the thread-block-cluster
//      sizes) take a four-step transform: k_obs_cross does the length-C DFTs across the C
//      slices of length M and the twiddles W_N^{n k1}, then length-M row FFTs give mode
//      k1 + C k2 at position k1 M + k2; the bin tables and k^2 use that order;
//   3. k_obs_ekin   FP64 partial sums of (k^2/2) |psi_m(k)|^2 per mode block;
//   4. k_obs_bins   per (radial bin, field): sum over trajectories and the bin's modes of
//                   |W|^2 dx^d / N (- 1/2 for the occupations), FP64, into the caller's
//                   accumulator;
//   5. k_obs_final  per trajectory: the partial sums in fixed order into the accumulator.
// Separately, k_obs_winding (1D only, reads the fields directly): the winding number of
// the Larmor angle per trajectory.
// Every reduction has a fixed order (per-thread strided sums, shuffle trees, warp sums
// combined in index order), so results are bitwise reproducible.
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "adjoint.h"
#include "fft.cuh"
#include "obs.h"

namespace gpe {

namespace {

thread_local std::string g_obs_err;

constexpr int kThreads = 256;
constexpr int kSitesPerBlock = 4096;
constexpr int kPartVals = 7;   // real-space partial sums per site block: N_1, N_0, N_-1, E_q, E_c0, E_c1, E_V

gpe_status obs_fail(gpe_status s, const char* what, cudaError_t e) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    g_obs_err = buf;
    return s;
}

// Signed mode number of index i on an axis of n points (n = 1: 0).
__host__ __device__ __forceinline__ int fold(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }

// Fixed-order block sum of NV doubles per thread; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sm /* NV * 32 */) {
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

// Per-site terms are formed in the fields' precision and summed per thread in it (16
// sites per thread), the per-thread partials then reduced in FP64 in a fixed order: for
// FP32 fields the per-site FP64 arithmetic cost far more than the read of the fields, and
// the partials carry the FP32 fields' own relative precision.  FP64 fields stay FP64.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_obs_prep(cplx<T>* const* __restrict__ ptrs, int t0, cplx<T>* __restrict__ W, int64_t sites, double c0,
           double c1, double q, const T* __restrict__ vpot, double* __restrict__ part, int64_t nblk) {
    using V = cplx<T>;
    __shared__ double sm[kPartVals * 32];
    const int tl = blockIdx.y;
    const V* f = ptrs[t0 + tl];
    V* w = W + (int64_t)tl * 4 * sites;
    // n_1, n_0, n_-1, n_1 + n_-1, rho^2, F_z^2 + |F_perp|^2, sum_m V_m n_m
    T pt[kPartVals] = {0, 0, 0, 0, 0, 0, 0};
    const int64_t s0 = (int64_t)blockIdx.x * kSitesPerBlock;
    const T s2 = (T)1.41421356237309504880;
    for (int k = 0; k < kSitesPerBlock / kThreads; ++k) {
        const int64_t i = s0 + k * kThreads + threadIdx.x;
        if (i >= sites) break;
        const V p1 = f[i], p0 = f[sites + i], pm = f[2 * sites + i];
        const T n1 = cabs2(p1), n0 = cabs2(p0), nm = cabs2(pm);
        const T rho = n1 + n0 + nm, fz = n1 - nm;
        // F_perp = sqrt2 (conj(p1) p0 + conj(p0) pm)
        const T fr = s2 * ((p1.x * p0.x + p1.y * p0.y) + (p0.x * pm.x + p0.y * pm.y));
        const T fi = s2 * ((p1.x * p0.y - p1.y * p0.x) + (p0.x * pm.y - p0.y * pm.x));
        pt[0] += n1;
        pt[1] += n0;
        pt[2] += nm;
        pt[3] += n1 + nm;
        pt[4] += rho * rho;
        pt[5] += fz * fz + fr * fr + fi * fi;
        if (vpot) pt[6] += vpot[i] * n1 + vpot[sites + i] * n0 + vpot[2 * sites + i] * nm;
        w[i] = p1;
        w[sites + i] = p0;
        w[2 * sites + i] = pm;
        w[3 * sites + i] = mk(fr, fi);
    }
    double acc[kPartVals];
#pragma unroll
    for (int k = 0; k < kPartVals; ++k) acc[k] = (double)pt[k];
    acc[3] *= q;
    acc[4] *= 0.5 * c0;
    acc[5] *= 0.5 * c1;
    block_sum<kPartVals>(acc, sm);
    if (threadIdx.x == 0) {
        double* o = part + ((int64_t)tl * nblk + blockIdx.x) * kPartVals;
#pragma unroll
        for (int k = 0; k < kPartVals; ++k) o[k] = acc[k];
    }
}

// Kinetic energy partials: sum over a block's modes of (k^2 / 2) |psi_m(k)|^2, mode
// coordinates from shifts (all extents are powers of two), terms in the fields' precision.
// Mode number along x of position i of a transformed row: natural order, or with lm > 0
// the four-step order (position k1 M + k2 holds mode k1 + C k2, M = 2^lm, C = 2^lc).
__host__ __device__ __forceinline__ int64_t x_mode(int64_t i, int lm, int lc) {
    return lm > 0 ? (i >> lm) + ((i & ((1ll << lm) - 1)) << lc) : i;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_obs_ekin(const cplx<T>* __restrict__ W, int64_t sites, int lx, int ly, int nz, double dx,
           double* __restrict__ ekin, int64_t nblk, int lm, int lc) {
    using V = cplx<T>;
    __shared__ double sm[32];
    const int nx = 1 << lx, ny = 1 << ly;
    const int tl = blockIdx.z, c = blockIdx.y;
    const V* w = W + ((int64_t)tl * 4 + c) * sites;
    const double two_pi = 6.283185307179586476925286766559;
    const T gx = (T)(two_pi / (nx * dx)), gy = (T)(two_pi / (ny * dx)), gz = (T)(two_pi / (nz * dx));
    T pt = 0;
    const int64_t s0 = (int64_t)blockIdx.x * kSitesPerBlock;
    for (int k = 0; k < kSitesPerBlock / kThreads; ++k) {
        const int64_t i = s0 + k * kThreads + threadIdx.x;
        if (i >= sites) break;
        const int ix = (int)(x_mode(i & (nx - 1), lm, lc));
        const int iy = (int)((i >> lx) & (ny - 1));
        const int iz = (int)(i >> (lx + ly));
        const T kx = gx * (T)fold(ix, nx), ky = gy * (T)fold(iy, ny), kz = gz * (T)fold(iz, nz);
        const V a = w[i];
        pt += (kx * kx + ky * ky + kz * kz) * cabs2(a);
    }
    double acc[1] = {0.5 * (double)pt};
    block_sum<1>(acc, sm);
    if (threadIdx.x == 0) ekin[((int64_t)tl * 3 + c) * nblk + blockIdx.x] = acc[0];
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_obs_bins(const cplx<T>* __restrict__ W, int64_t sites, int ntl, const int32_t* __restrict__ off,
           const int32_t* __restrict__ modes, double scale, double* __restrict__ acc_spec, int nbins) {
    using V = cplx<T>;
    __shared__ double sm[32];
    const int b = blockIdx.x, qf = blockIdx.y;
    const double sub = (qf < 3) ? 0.5 : 0.0;
    const int beg = off[b], end = off[b + 1];
    double acc[1] = {0.0};
    for (int tl = 0; tl < ntl; ++tl) {
        const V* w = W + ((int64_t)tl * 4 + qf) * sites;
        for (int i = beg + threadIdx.x; i < end; i += kThreads) {
            const V a = w[modes[i]];
            acc[0] += ((double)a.x * a.x + (double)a.y * a.y) * scale - sub;
        }
    }
    block_sum<1>(acc, sm);
    if (threadIdx.x == 0) acc_spec[(int64_t)qf * nbins + b] += acc[0];
}

__global__ void __launch_bounds__(kThreads)
k_obs_final(const double* __restrict__ part, const double* __restrict__ ekin, int64_t nblk, int64_t count,
            const int32_t* __restrict__ ids, int t0, double vol, double inv_sites, double* __restrict__ acc_diag,
            int* status) {
    __shared__ double sm[8 * 32];
    const int tl = blockIdx.x;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t k = threadIdx.x; k < count; k += kThreads) {
        const double* p = part + ((int64_t)tl * nblk + k) * kPartVals;
        acc[0] += p[0];
        acc[1] += p[1];
        acc[2] += p[2];
        acc[4] += p[3];
        acc[5] += p[4];
        acc[6] += p[5];
        acc[7] += p[6];
        acc[3] += ekin[((int64_t)tl * 3 + 0) * nblk + k] + ekin[((int64_t)tl * 3 + 1) * nblk + k] +
                  ekin[((int64_t)tl * 3 + 2) * nblk + k];
    }
    block_sum<8>(acc, sm);
    if (threadIdx.x == 0) {
        double* o = acc_diag + (int64_t)ids[t0 + tl] * 8;
        bool finite = true;
        for (int k = 0; k < 8; ++k) {
            const double v = (k == 3) ? acc[k] * vol * inv_sites : acc[k] * vol;
            finite = finite && isfinite(v);
            o[k] += v;
        }
        if (!finite) atomicCAS(status, 0, (int)GPE_ENONFINITE);
    }
}

// First step of the four-step transform of rows of N = C M points: row element n1 M + n2
// (n1 < C, n2 < M) is replaced by W_N^{n2 k1} sum_{n1} x[n1 M + n2] W_C^{n1 k1} at k1 M + n2,
// so that length-M transforms of the C slices give X[k1 + C k2] at k1 M + k2.  One thread
// per (row, n2); wn[k1 M + n2] = W_N^{n2 k1}.
template <typename T, int C>
__global__ void __launch_bounds__(kThreads)
k_obs_cross(cplx<T>* __restrict__ W, int64_t rows, int M, const twel<T>* __restrict__ wn) {
    using V = cplx<T>;
    const int64_t gid = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (gid >= rows * M) return;
    const int64_t row = gid / M;
    const int n2 = (int)(gid - row * M);
    V* r = W + row * (int64_t)C * M + n2;
    V x[C];
#pragma unroll
    for (int n1 = 0; n1 < C; ++n1) x[n1] = r[(int64_t)n1 * M];
    Dft<C, 1, -1>::run(x);
    r[0] = x[0];
#pragma unroll
    for (int k1 = 1; k1 < C; ++k1) r[(int64_t)k1 * M] = twmul<-1>(x[k1], wn[(int64_t)k1 * M + n2]);
}

template <typename T>
cudaError_t launch_obs_cross(int C, cplx<T>* W, int64_t rows, int M, const twel<T>* wn, cudaStream_t s) {
    const int64_t total = rows * M;
    const unsigned grid = (unsigned)((total + kThreads - 1) / kThreads);
    switch (C) {
        case 2: k_obs_cross<T, 2><<<grid, kThreads, 0, s>>>(W, rows, M, wn); break;
        case 4: k_obs_cross<T, 4><<<grid, kThreads, 0, s>>>(W, rows, M, wn); break;
        case 8: k_obs_cross<T, 8><<<grid, kThreads, 0, s>>>(W, rows, M, wn); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Winding number of the Larmor angle phi_L = arg(F_perp) around a periodic 1D trajectory
// (Sec. 1: Q_w = int dx d_x phi_L), in units of 2 pi: the sum over x of the increments
// arg(F(x)^* F(x+1)) in (-pi, pi], FP64, fixed summation order.  One block per trajectory.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_obs_winding(cplx<T>* const* __restrict__ ptrs, const int32_t* __restrict__ ids, int64_t n,
              double* __restrict__ acc_wind, int* status) {
    using V = cplx<T>;
    __shared__ double sm[32];
    const V* f = ptrs[blockIdx.x];
    auto fperp = [&](int64_t i) {   // conj(p1) p0 + conj(p0) pm (the factor sqrt2 drops out)
        const V p1 = f[i], p0 = f[n + i], pm = f[2 * n + i];
        const double r = ((double)p1.x * p0.x + (double)p1.y * p0.y) + ((double)p0.x * pm.x + (double)p0.y * pm.y);
        const double im = ((double)p1.x * p0.y - (double)p1.y * p0.x) + ((double)p0.x * pm.y - (double)p0.y * pm.x);
        return make_double2(r, im);
    };
    double acc[1] = {0.0};
    for (int64_t i = threadIdx.x; i < n; i += kThreads) {
        const double2 a = fperp(i), b = fperp(i + 1 == n ? 0 : i + 1);
        acc[0] += atan2(a.x * b.y - a.y * b.x, a.x * b.x + a.y * b.y);
    }
    block_sum<1>(acc, sm);
    if (threadIdx.x == 0) {
        const double v = acc[0] / 6.283185307179586476925286766559;
        if (!isfinite(v)) atomicCAS(status, 0, (int)GPE_ENONFINITE);
        acc_wind[ids[blockIdx.x]] += v;
    }
}

template <typename T>
gpe_status run_group(ObsWork& w, const Group& g, const GroupBins& gb, double c0, double c1, double q, double* acc,
                     uint32_t flags, int slot, int* d_status, cudaStream_t s) {
    using V = cplx<T>;
    const int64_t nb4 = 4 * (int64_t)(w.nbins > 0 ? w.nbins : 0);
    const int64_t slot_doubles = nb4 + 9 * w.ntraj_total;
    double* acc_slot = acc + (int64_t)slot * slot_doubles;
    if (flags & GPE_OBS_WINDING) {
        k_obs_winding<T><<<g.ntraj, kThreads, 0, s>>>(reinterpret_cast<V* const*>(g.dptrs), g.d_ids, g.sites,
                                                    acc_slot + nb4 + 8 * w.ntraj_total, d_status);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return obs_fail(GPE_ECUDA, "obs winding", e);
    }
    if (!(flags & (GPE_OBS_SPECTRA | GPE_OBS_DIAG))) return GPE_OK;
    const int64_t nblk = (g.sites + kSitesPerBlock - 1) / kSitesPerBlock;
    const double vol = std::pow(g.dx, g.ndim);
    V* W = reinterpret_cast<V*>(w.d_W);
    for (int t0 = 0; t0 < g.ntraj; t0 += (int)w.chunk) {
        const int nc = (int)std::min<int64_t>(w.chunk, g.ntraj - t0);
        k_obs_prep<T><<<dim3((unsigned)nblk, nc), kThreads, 0, s>>>(
            reinterpret_cast<V* const*>(g.dptrs), t0, W, g.sites, c0, c1, q, reinterpret_cast<const T*>(g.vpot),
            w.d_part, w.nblk);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return obs_fail(GPE_ECUDA, "obs prep", e);
        if (g.cluster > 0) {
            // 1D N = C M: cross step, then length-M row transforms of the C slices
            const int M = g.n[0] / g.cluster;
            const twel<T>* twl[3] = {reinterpret_cast<const twel<T>*>(g.tw_local[0]),
                                     reinterpret_cast<const twel<T>*>(g.tw_local[1]),
                                     reinterpret_cast<const twel<T>*>(g.tw_local[2])};
            e = launch_obs_cross<T>(g.cluster, W, (int64_t)nc * 4, M, reinterpret_cast<const twel<T>*>(g.wn), s);
            if (e == cudaSuccess) e = launch_rowfft<T>(M, W, (int64_t)nc * 4 * g.cluster, twl, s);
        } else {
            const twel<T>* twx[3] = {reinterpret_cast<const twel<T>*>(g.tw[0][0]),
                                     reinterpret_cast<const twel<T>*>(g.tw[0][1]),
                                     reinterpret_cast<const twel<T>*>(g.tw[0][2])};
            e = launch_rowfft<T>(g.n[0], W, (int64_t)nc * 4 * g.n[1] * g.n[2], twx, s);
        }
        if (e != cudaSuccess) return obs_fail(GPE_ECUDA, "obs x fft", e);
        if (g.ndim > 1) {
            // the chunk's 4-field blocks lie back to back at this group's size (as k_obs_prep
            // wrote them and the x transform read them), not at the largest group's
            e = launch_fill_ptrs(w.d_Wptrs, W, (int64_t)4 * g.sites * (int64_t)sizeof(V), nc, s);
            if (e != cudaSuccess) return obs_fail(GPE_ECUDA, "obs workspace pointers", e);
        }
        for (int ax = 1; ax < g.ndim; ++ax) {
            PassArgs<T> a{};
            a.ptrs = reinterpret_cast<V* const*>(w.d_Wptrs);
            a.comp_stride = g.sites;
            a.ntraj = nc;
            a.ncomp = 4;
            a.status = d_status;
            for (int ri = 0; ri < 3; ++ri) a.tw[ri] = reinterpret_cast<const twel<T>*>(g.tw[ax][ri]);
            const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
            if (ax == 1) {
                a.stride = nx;
                a.n_outer = nz;
                a.outer_stride = (int64_t)nx * ny;
            } else {
                a.stride = (int64_t)nx * ny;
                a.n_outer = ny;
                a.outer_stride = nx;
            }
            a.nx_tiles = nx / colpass_cols<T>(g.n[ax]);
            e = launch_colfft<T>(g.n[ax], a, s);
            if (e != cudaSuccess) return obs_fail(GPE_ECUDA, "obs strided fft", e);
        }
        if (flags & GPE_OBS_DIAG) {
            int lx = 0, ly = 0, lm = 0, lc = 0;
            while ((1 << lx) < g.n[0]) ++lx;
            while ((1 << ly) < g.n[1]) ++ly;
            if (g.cluster > 0) {
                while ((1 << lc) < g.cluster) ++lc;
                lm = lx - lc;
            }
            k_obs_ekin<T><<<dim3((unsigned)nblk, 3, nc), kThreads, 0, s>>>(W, g.sites, lx, ly, g.n[2], g.dx,
                                                                          w.d_ekin, w.nblk, lm, lc);
            k_obs_final<<<nc, kThreads, 0, s>>>(w.d_part, w.d_ekin, w.nblk, nblk, g.d_ids, t0, vol, 1.0 / (double)g.sites,
                                                acc_slot + 4 * (int64_t)(w.nbins > 0 ? w.nbins : 0), d_status);
            e = cudaGetLastError();
            if (e != cudaSuccess) return obs_fail(GPE_ECUDA, "obs diagnostics", e);
        }
        if ((flags & GPE_OBS_SPECTRA) && gb.nbins > 0) {
            k_obs_bins<T><<<dim3(gb.nbins, 4), kThreads, 0, s>>>(W, g.sites, nc, gb.d_off, gb.d_modes,
                                                                vol / (double)g.sites, acc_slot + 4 * gb.offset,
                                                                gb.nbins);
            e = cudaGetLastError();
            if (e != cudaSuccess) return obs_fail(GPE_ECUDA, "obs bins", e);
        }
    }
    return GPE_OK;
}

int64_t isqrt_round(int64_t m) {
    // b with (2b - 1)^2 <= 4m < (2b + 1)^2
    int64_t b = (int64_t)std::floor(std::sqrt((double)m) + 0.5);
    while (b > 0 && (2 * b - 1) * (2 * b - 1) > 4 * m) --b;
    while ((2 * b + 1) * (2 * b + 1) <= 4 * m) ++b;
    return b;
}

}  // namespace

const char* obs_last_error() { return g_obs_err.c_str(); }

int64_t obs_launches(const ObsWork& w, const std::vector<Group>& groups, uint32_t flags) {
    int64_t n = 0;
    for (size_t k = 0; k < groups.size(); ++k) {
        const Group& g = groups[k];
        const int64_t chunk = w.ready ? w.chunk : 0;
        int64_t max_traj = 0;
        for (const Group& h : groups) max_traj = std::max<int64_t>(max_traj, h.ntraj);
        const int64_t c = chunk > 0 ? chunk : max_traj;  // before the first call: estimate
        const int64_t nchunks = (g.ntraj + c - 1) / c;
        const bool fields = flags & (GPE_OBS_SPECTRA | GPE_OBS_DIAG);
        const bool spectra = (flags & GPE_OBS_SPECTRA) && k < w.gbins.size() && w.gbins[k].nbins > 0;
        const int64_t per = (fields ? 1 + g.ndim + (g.cluster > 0 ? 1 : 0) + (g.ndim > 1 ? 1 : 0) : 0) +
                            ((flags & GPE_OBS_DIAG) ? 2 : 0) + (spectra ? 1 : 0);
        n += nchunks * per + ((flags & GPE_OBS_WINDING) ? 1 : 0);
    }
    return n;
}

// Bin tables of one group with equal side lengths (radial bins b = round(|j|) of the folded
// mode vector, in the mode order the group's transforms leave), appended to w.counts.
static gpe_status group_bins(ObsWork& w, const Group& g, GroupBins& gb) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    int lm = 0, lc = 0;   // four-step order of 1D cluster groups (see k_obs_cross)
    if (g.cluster > 0) {
        while ((1 << lc) < g.cluster) ++lc;
        while ((1 << lm) < nx / g.cluster) ++lm;
    }
    std::vector<int32_t> bin(g.sites);
    int64_t maxb = 0;
    for (int64_t i = 0; i < g.sites; ++i) {
        const int ix = (int)x_mode(i % nx, lm, lc), iy = (int)((i / nx) % ny), iz = (int)(i / ((int64_t)nx * ny));
        const int64_t jx = fold(ix, nx), jy = fold(iy, ny), jz = fold(iz, nz);
        const int64_t b = isqrt_round(jx * jx + jy * jy + jz * jz);
        bin[i] = (int32_t)b;
        if (b > maxb) maxb = b;
    }
    gb.nbins = (int)(maxb + 1);
    std::vector<int64_t> counts(gb.nbins, 0);
    for (int64_t i = 0; i < g.sites; ++i) counts[bin[i]]++;
    std::vector<int32_t> off(gb.nbins + 1, 0), modes(g.sites);
    for (int b = 0; b < gb.nbins; ++b) off[b + 1] = off[b] + (int32_t)counts[b];
    std::vector<int32_t> fill(off.begin(), off.end() - 1);
    for (int64_t i = 0; i < g.sites; ++i) modes[fill[bin[i]]++] = (int32_t)i;
    cudaError_t e = device_malloc((void**)&gb.d_off, sizeof(int32_t) * (gb.nbins + 1));
    if (e == cudaSuccess) e = device_malloc((void**)&gb.d_modes, sizeof(int32_t) * g.sites);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(gb.d_off);
        gb.d_off = nullptr;
        return obs_fail(GPE_ENOMEM, "bin tables", e);
    }
    e = cudaMemcpy(gb.d_off, off.data(), sizeof(int32_t) * (gb.nbins + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(gb.d_modes, modes.data(), sizeof(int32_t) * g.sites, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return obs_fail(GPE_ECUDA, "copy bin tables", e);
    w.counts.insert(w.counts.end(), counts.begin(), counts.end());
    return GPE_OK;
}

// Bins for every shape group whose side lengths are equal; each group's spectra get a
// block of their own in the accumulator slot, in group order.
gpe_status obs_init(ObsWork& w, const std::vector<Group>& groups, bool f64, int) {
    w.f64 = f64;
    w.ntraj_total = 0;
    for (const Group& g : groups) w.ntraj_total += g.ntraj;
    w.nbins = 0;
    w.counts.clear();
    w.gbins.assign(groups.size(), GroupBins());
    for (size_t k = 0; k < groups.size(); ++k) {
        const Group& g = groups[k];
        bool equal = true;
        for (int a = 1; a < g.ndim; ++a) equal = equal && g.n[a] == g.n[0];
        if (!equal) continue;
        GroupBins& gb = w.gbins[k];
        gb.offset = w.nbins;
        const gpe_status s = group_bins(w, g, gb);
        if (s != GPE_OK) return s;
        w.nbins += gb.nbins;
    }
    return GPE_OK;
}

void obs_free(ObsWork& w) {
    for (GroupBins& gb : w.gbins) {
        cudaFree(gb.d_off);
        cudaFree(gb.d_modes);
    }
    cudaFree(w.d_W);
    cudaFree(w.d_Wptrs);
    cudaFree(w.d_part);
    cudaFree(w.d_ekin);
    w = ObsWork();
}

static gpe_status ensure_workspace(ObsWork& w, const std::vector<Group>& groups) {
    if (w.ready) return GPE_OK;
    const size_t vb = w.f64 ? 16 : 8;
    int64_t max_sites = 0, max_traj = 0;
    for (const Group& g : groups) {
        max_sites = std::max(max_sites, g.sites);
        max_traj = std::max<int64_t>(max_traj, g.ntraj);
    }
    const int64_t per_traj = 4 * max_sites * (int64_t)vb;
    const int64_t budget = (int64_t)1 << 30;
    w.chunk = std::max<int64_t>(1, std::min<int64_t>(max_traj, budget / per_traj));
    w.nblk = (max_sites + kSitesPerBlock - 1) / kSitesPerBlock;
    cudaError_t e = device_malloc(&w.d_W, (size_t)(w.chunk * per_traj));
    if (e == cudaSuccess) e = device_malloc((void**)&w.d_Wptrs, sizeof(void*) * w.chunk);
    if (e == cudaSuccess) e = device_malloc((void**)&w.d_part, sizeof(double) * w.chunk * w.nblk * kPartVals);
    if (e == cudaSuccess) e = device_malloc((void**)&w.d_ekin, sizeof(double) * w.chunk * w.nblk * 3);
    if (e != cudaSuccess) {
        cudaGetLastError();
        // free the part that was allocated: a later call starts over
        cudaFree(w.d_W);
        cudaFree(w.d_Wptrs);
        cudaFree(w.d_part);
        cudaFree(w.d_ekin);
        w.d_W = nullptr;
        w.d_Wptrs = nullptr;
        w.d_part = nullptr;
        w.d_ekin = nullptr;
        return obs_fail(GPE_ENOMEM, "observables workspace", e);
    }
    std::vector<void*> ptrs(w.chunk);
    for (int64_t i = 0; i < w.chunk; ++i) ptrs[i] = (char*)w.d_W + i * per_traj;
    e = cudaMemcpy(w.d_Wptrs, ptrs.data(), sizeof(void*) * w.chunk, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return obs_fail(GPE_ECUDA, "workspace pointers", e);
    w.ready = true;
    return GPE_OK;
}

gpe_status obs_accumulate(ObsWork& w, const std::vector<Group>& groups, bool f64, double c0, double c1, double q,
                          double* acc, uint32_t flags, int slot, int* d_status, cudaStream_t s) {
    const bool fields = flags & (GPE_OBS_SPECTRA | GPE_OBS_DIAG);
    for (const Group& g : groups) {
        if (fields && g.n[0] > 4096 && g.cluster == 0) {
            g_obs_err = "spectra and diagnostics support x extents up to 4096 (longer 1D grids take the cluster path)";
            return GPE_EUNSUPPORTED;
        }
        if ((flags & GPE_OBS_WINDING) && g.ndim != 1) {
            g_obs_err = "the winding number is defined for 1D trajectories only";
            return GPE_EUNSUPPORTED;
        }
    }
    if (fields) {
        gpe_status st = ensure_workspace(w, groups);
        if (st != GPE_OK) return st;
    }
    gpe_status st = GPE_OK;
    for (size_t k = 0; k < groups.size(); ++k) {
        const Group& g = groups[k];
        const GroupBins& gb = w.gbins[k];
        st = f64 ? run_group<double>(w, g, gb, c0, c1, q, acc, flags, slot, d_status, s)
                 : run_group<float>(w, g, gb, c0, c1, q, acc, flags, slot, d_status, s);
        if (st != GPE_OK) return st;
    }
    return GPE_OK;
}

}  // namespace gpe
