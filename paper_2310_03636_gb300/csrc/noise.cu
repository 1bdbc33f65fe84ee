// Truncated-Wigner initial state: mean spinor (plus an optional mean field) and complex
// Gaussian noise per site and component, Philox4x32-10 integers turned into two FP64
// uniforms and a Box-Muller pair.
#include "internal.h"
#include "philox.cuh"

namespace gpe {

template <typename T>
__global__ void __launch_bounds__(256) k_noise(const NoiseArgs a) {
    using V = cplx<T>;
    const int64_t total = (int64_t)a.ntraj * 3 * a.sites;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t site = i % a.sites;
        const int64_t rest = i / a.sites;
        const int comp = (int)(rest % 3);
        const int tl = (int)(rest / 3);
        const u32x4 w = philox4x32_10(
            u32x4{(uint32_t)(site & 0xFFFFFFFFu), (uint32_t)comp, a.traj_base + (uint32_t)a.traj_ids[tl],
                  (uint32_t)((uint64_t)site >> 32)},
            a.key0, a.key1);
        const uint64_t x1 = ((uint64_t)w.y << 32) | w.x;
        const uint64_t x2 = ((uint64_t)w.w << 32) | w.z;
        const double u1 = ((double)(x1 >> 11) + 1.0) * 0x1.0p-53;   // (0, 1]
        const double u2 = (double)(x2 >> 11) * 0x1.0p-53;           // [0, 1)
        const double r = sqrt(-log(u1)) * a.sigma;
        double s, c;
        sincospi(2.0 * u2, &s, &c);
        double mr = a.mean[2 * comp], mi = a.mean[2 * comp + 1];
        if (a.mean_field) {
            const double2 f = reinterpret_cast<const double2*>(a.mean_field)[comp * a.sites + site];
            mr += f.x;
            mi += f.y;
        }
        V* out = reinterpret_cast<V*>(a.ptrs[tl]);
        out[comp * a.sites + site] = mk((T)(mr + r * c), (T)(mi + r * s));
    }
}

template <typename T>
cudaError_t launch_noise(const NoiseArgs& a, cudaStream_t s) {
    const int64_t total = (int64_t)a.ntraj * 3 * a.sites;
    int64_t grid = (total + 255) / 256;
    if (grid > 152 * 64) grid = 152 * 64;
    if (grid < 1) grid = 1;
    k_noise<T><<<(int)grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_noise<float>(const NoiseArgs&, cudaStream_t);
template cudaError_t launch_noise<double>(const NoiseArgs&, cudaStream_t);

}  // namespace gpe
