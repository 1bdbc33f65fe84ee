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
