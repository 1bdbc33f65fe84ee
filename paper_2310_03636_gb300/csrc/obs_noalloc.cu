// Real-space diagnostics without any device allocation.
//
// Some callers cannot let this library allocate device memory: code that must not
// synchronise the device (cudaMalloc and cudaFree can), a process whose device memory is
// entirely handed out by another allocator, or a health check that inspects a field while
// the device is out of memory.  gpe_diagnostics_noalloc serves them: it computes the
// same real-space sums as the diagnostics part of observables_accumulate (N_1, N_0, N_-1,
// E_q, E_c0, E_c1) for caller-owned fields, with its per-block partial sums kept in a
// fixed scratch array compiled into the library instead of a handle's workspace.
//
// The scratch array is one file-scope __device__ array, so every GPU that loads the
// library holds it (kMaxPartials doubles, 192 KiB) until the process exits.  Its device
// address is looked up once per device on the first call made with that device current
// and kept for the life of the process: after a cudaDeviceReset the module may come back
// at another address, so the entry point must not be used again in that process.
// All calls share the array and it keeps the last call's contents; every slot a call
// reads is written by the same call first, so nothing needs clearing.  Calls that overlap
// on the same GPU (for instance on two streams with no ordering between them) race on
// the array: serialise them.
#include <cmath>
#include <mutex>

#include "gpe.h"
#include "internal.h"

namespace gpe {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaSitesPerBlock = 4096;
constexpr int kNaSums = 6;
constexpr int64_t kMaxPartialBlocks = 4096;                        // trajectories x site blocks
constexpr int64_t kMaxPartials = kMaxPartialBlocks * kNaSums;       // 24576 doubles = 192 KiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kMaxPartials];

std::mutex g_setup_mutex;

gpe_status set_error(gpe_status s, const char* msg) {
    set_last_error(msg);
    return s;
}
double* g_scratch_ptr[kMaxDevices] = {};

template <int NV>
__device__ __forceinline__ void na_block_sum(double (&v)[NV], double* sm) {
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

// Per site block: sums of n_1, n_0, n_-1, q (n_1 + n_-1), c0 rho^2 / 2,
// c1 (F_z^2 + |F_perp|^2) / 2 in FP64, written to scratch[(traj * nblk + block) * 6 ...].
template <typename T>
__global__ void __launch_bounds__(kNaThreads)
k_diag_partials(const cplx<T>* __restrict__ psi, int64_t sites, int64_t nblk, double c0, double c1, double q,
                double* __restrict__ scratch) {
    using V = cplx<T>;
    __shared__ double sm[kNaSums * 32];
    const int tr = blockIdx.y;
    const V* f = psi + (int64_t)tr * 3 * sites;
    double acc[kNaSums] = {0, 0, 0, 0, 0, 0};
    const int64_t s0 = (int64_t)blockIdx.x * kNaSitesPerBlock;
    for (int k = 0; k < kNaSitesPerBlock / kNaThreads; ++k) {
        const int64_t i = s0 + k * kNaThreads + threadIdx.x;
        if (i >= sites) break;
        const V p1 = f[i], p0 = f[sites + i], pm = f[2 * sites + i];
        const double a1r = p1.x, a1i = p1.y, a0r = p0.x, a0i = p0.y, amr = pm.x, ami = pm.y;
        const double n1 = a1r * a1r + a1i * a1i, n0 = a0r * a0r + a0i * a0i, nm = amr * amr + ami * ami;
        const double rho = n1 + n0 + nm, fz = n1 - nm;
        const double s2 = 1.41421356237309504880;
        const double fr = s2 * ((a1r * a0r + a1i * a0i) + (a0r * amr + a0i * ami));
        const double fi = s2 * ((a1r * a0i - a1i * a0r) + (a0r * ami - a0i * amr));
        acc[0] += n1;
        acc[1] += n0;
        acc[2] += nm;
        acc[3] += q * (n1 + nm);
        acc[4] += 0.5 * c0 * rho * rho;
        acc[5] += 0.5 * c1 * (fz * fz + fr * fr + fi * fi);
    }
    na_block_sum<kNaSums>(acc, sm);
    if (threadIdx.x == 0) {
        double* o = scratch + ((int64_t)tr * nblk + blockIdx.x) * kNaSums;
#pragma unroll
        for (int k = 0; k < kNaSums; ++k) o[k] = acc[k];
    }
}

// Per trajectory: the block sums in fixed order, times dx^d, into out[traj * 8 ...] as
// (N_1, N_0, N_-1, 0, E_q, E_c0, E_c1, 0) -- the record layout of observables_accumulate
// with the kinetic energy (slot 3) and the potential energy (slot 7) always zero: this
// entry point takes no potential and does no transform.
__global__ void __launch_bounds__(kNaThreads)
k_diag_final(const double* __restrict__ scratch, int64_t nblk, double vol, double* __restrict__ out) {
    __shared__ double sm[kNaSums * 32];
    const int tr = blockIdx.x;
    double acc[kNaSums] = {0, 0, 0, 0, 0, 0};
    for (int64_t k = threadIdx.x; k < nblk; k += kNaThreads) {
        const double* p = scratch + ((int64_t)tr * nblk + k) * kNaSums;
#pragma unroll
        for (int j = 0; j < kNaSums; ++j) acc[j] += p[j];
    }
    na_block_sum<kNaSums>(acc, sm);
    if (threadIdx.x == 0) {
        double* o = out + (int64_t)tr * 8;
        o[0] = acc[0] * vol;
        o[1] = acc[1] * vol;
        o[2] = acc[2] * vol;
        o[3] = 0.0;
        o[4] = acc[3] * vol;
        o[5] = acc[4] * vol;
        o[6] = acc[5] * vol;
        o[7] = 0.0;
    }
}

}  // namespace
}  // namespace gpe

extern "C" gpe_status gpe_diagnostics_noalloc(const void* psi, int32_t ntraj, int32_t ndim, const int32_t n[3],
                                              double dx, gpe_dtype dtype, double c0, double c1, double q,
                                              double* out, void* stream) {
    using namespace gpe;
    if (!psi || !out || !n) return set_error(GPE_EINVAL, "gpe_diagnostics_noalloc: NULL psi, out or n");
    // An error left pending by earlier, unrelated work is not this call's to report or clear.
    if (cudaPeekAtLastError() != cudaSuccess)
        return set_error(GPE_ECUDA, "gpe_diagnostics_noalloc: a CUDA error from earlier work is pending");
    if (ndim < 1 || ndim > 3 || ntraj <= 0 || !(dx > 0.0))
        return set_error(GPE_EINVAL, "gpe_diagnostics_noalloc: need 1 <= ndim <= 3, ntraj > 0, dx > 0");
    if (dtype != GPE_C64 && dtype != GPE_C128) return set_error(GPE_EINVAL, "gpe_diagnostics_noalloc: bad dtype");
    if (((uintptr_t)psi & 15u) || ((uintptr_t)out & 7u))
        return set_error(GPE_EINVAL, "gpe_diagnostics_noalloc: psi must be 16-byte and out 8-byte aligned");
    // Capacity in sites, checked after every factor so the product cannot overflow
    // (each factor is below 2^31 and the running product stays below 2^24 x 4096).
    constexpr int64_t kMaxSites = kMaxPartialBlocks * kNaSitesPerBlock;
    int64_t sites = 1;
    for (int a = 0; a < 3; ++a) {
        if ((a < ndim && n[a] < 1) || (a >= ndim && n[a] != 1))
            return set_error(GPE_EINVAL, "gpe_diagnostics_noalloc: n[a] >= 1 on used axes, 1 on unused axes");
        sites *= n[a];
        if (sites > kMaxSites)
            return set_error(GPE_EINVAL,
                             "gpe_diagnostics_noalloc: ntraj * ceil(sites / 4096) exceeds the fixed scratch "
                             "capacity of 4096 site blocks");
    }
    const int64_t nblk = (sites + kNaSitesPerBlock - 1) / kNaSitesPerBlock;
    // Sizes beyond the fixed scratch array are rejected: ntraj * ceil(sites / 4096) must
    // not exceed 4096 (e.g. one 256^3 field, or 64 fields of 512^2).
    if ((int64_t)ntraj * nblk > kMaxPartialBlocks)
        return set_error(GPE_EINVAL,
                         "gpe_diagnostics_noalloc: ntraj * ceil(sites / 4096) exceeds the fixed scratch "
                         "capacity of 4096 site blocks");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return set_error(GPE_ECUDA, "gpe_diagnostics_noalloc: no usable current device");
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return set_error(GPE_ECUDA, "gpe_diagnostics_noalloc: cudaGetSymbolAddress of the scratch failed");
            }
            g_scratch_ptr[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const double vol = std::pow(dx, ndim);
    if (dtype == GPE_C64)
        k_diag_partials<float><<<dim3((unsigned)nblk, ntraj), kNaThreads, 0, s>>>(
            static_cast<const float2*>(psi), sites, nblk, c0, c1, q, scratch);
    else
        k_diag_partials<double><<<dim3((unsigned)nblk, ntraj), kNaThreads, 0, s>>>(
            static_cast<const double2*>(psi), sites, nblk, c0, c1, q, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(GPE_ECUDA, cudaGetErrorString(e));
    k_diag_final<<<ntraj, kNaThreads, 0, s>>>(scratch, nblk, vol, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(GPE_ECUDA, cudaGetErrorString(e));
    return GPE_OK;
}
