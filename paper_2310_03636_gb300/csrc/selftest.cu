// Verification hook: the FP32 sin/cos used by the local step next to CUDA's sincosf.
#include "gpe.h"
#include "internal.h"

namespace gpe {

__global__ void k_check_sincos(const float* __restrict__ x, float* __restrict__ out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s, c, sl, cl;
    sincos_t(x[i], &s, &c);
    sincosf(x[i], &sl, &cl);
    out[4 * i + 0] = s;
    out[4 * i + 1] = c;
    out[4 * i + 2] = sl;
    out[4 * i + 3] = cl;
}

}  // namespace gpe

extern "C" gpe_status gpe_check_sincos(const float* x, float* out, int64_t n, void* stream) {
    if (!x || !out || n < 0) return GPE_EINVAL;
    if (n == 0) return GPE_OK;
    gpe::k_check_sincos<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, out, n);
    return cudaGetLastError() == cudaSuccess ? GPE_OK : GPE_ECUDA;
}

// Arithmetic-rate probe for the roofline of the compute-bound passes: every thread runs CH
// independent FMA chains acc <- acc * m + a (m < 1, so the chains stay finite), 16 FMAs
// per chain per loop trip.  KIND 0: FP32 fma; 1: FP32 pairs through the packed two-lane
// fma; 2: FP64 fma.  The sum is stored only if it takes an impossible value, which keeps
// the chains live without a store per thread.
namespace gpe {

template <int KIND>
__global__ void __launch_bounds__(256) k_fma_rate(double* sink, int64_t iters, float mf, float af) {
    constexpr int CH = 8;
    if constexpr (KIND == 0) {
        float acc[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) acc[c] = (float)(threadIdx.x + c) * 1e-3f;
        for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < 16; ++u)
#pragma unroll
                for (int c = 0; c < CH; ++c) acc[c] = fmaf(acc[c], mf, af);
        }
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < CH; ++c) s += acc[c];
        if (s == -12345.0f) sink[0] = s;
    } else if constexpr (KIND == 1) {
        float2 acc[CH / 2];
        const float2 m2 = make_float2(mf, mf), a2 = make_float2(af, af);
#pragma unroll
        for (int c = 0; c < CH / 2; ++c)
            acc[c] = make_float2((float)(threadIdx.x + 2 * c) * 1e-3f, (float)(threadIdx.x + 2 * c + 1) * 1e-3f);
        for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < 16; ++u)
#pragma unroll
                for (int c = 0; c < CH / 2; ++c) acc[c] = __ffma2_rn(acc[c], m2, a2);
        }
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < CH / 2; ++c) s += acc[c].x + acc[c].y;
        if (s == -12345.0f) sink[0] = s;
    } else {
        double acc[CH];
        const double md = mf, ad = af;
#pragma unroll
        for (int c = 0; c < CH; ++c) acc[c] = (double)(threadIdx.x + c) * 1e-3;
        for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < 16; ++u)
#pragma unroll
                for (int c = 0; c < CH; ++c) acc[c] = fma(acc[c], md, ad);
        }
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < CH; ++c) s += acc[c];
        if (s == -12345.0) sink[0] = s;
    }
}

template <int KIND>
cudaError_t fma_rate_run(int64_t iters, double* flops_per_s, cudaStream_t s) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_rate<KIND>, 256, 0);
    if (e != cudaSuccess) return e;
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    double* sink = nullptr;
    e = cudaMallocAsync(&sink, sizeof(double), s);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_rate<KIND><<<grid, 256, 0, s>>>(sink, iters / 8 + 1, 0.999f, 1e-3f);   // warm-up
    cudaEventRecord(e0, s);
    k_fma_rate<KIND><<<grid, 256, 0, s>>>(sink, iters, 0.999f, 1e-3f);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(sink, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    const double flops = (double)grid * 256.0 * (double)iters * 16.0 * 8.0 * 2.0;
    *flops_per_s = ms > 0.0f ? flops / (ms * 1e-3) : 0.0;
    return cudaSuccess;
}

}  // namespace gpe

extern "C" gpe_status gpe_fma_rate(int32_t kind, int64_t iters, double* flops_per_s, void* stream) {
    if (!flops_per_s || iters <= 0 || kind < 0 || kind > 2) return GPE_EINVAL;
    const cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = kind == 0 ? gpe::fma_rate_run<0>(iters, flops_per_s, s)
                  : kind == 1 ? gpe::fma_rate_run<1>(iters, flops_per_s, s)
                              : gpe::fma_rate_run<2>(iters, flops_per_s, s);
    return e == cudaSuccess ? GPE_OK : GPE_ECUDA;
}
