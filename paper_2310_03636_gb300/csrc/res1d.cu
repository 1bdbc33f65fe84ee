// Resident 1D kernel instantiations (whole trajectory on chip for all steps).
#include "prop_kernels.cuh"

namespace gpe {

template <> int resident1d_max_n<float>() { return 4096; }
template <> int resident1d_max_n<double>() { return 2048; }

template <>
cudaError_t launch_resident1d<float>(int n, const Res1DArgs<float>& a, cudaStream_t s) {
    switch (n) {
        case 64: return resident1d_n<float, 64>(a, s);
        case 128: return resident1d_n<float, 128>(a, s);
        case 256: return resident1d_n<float, 256>(a, s);
        case 512: return resident1d_n<float, 512>(a, s);
        case 1024: return resident1d_n<float, 1024>(a, s);
        case 2048: return resident1d_n<float, 2048>(a, s);
        case 4096: return resident1d_n<float, 4096>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_resident1d<double>(int n, const Res1DArgs<double>& a, cudaStream_t s) {
    switch (n) {
        case 64: return resident1d_n<double, 64>(a, s);
        case 128: return resident1d_n<double, 128>(a, s);
        case 256: return resident1d_n<double, 256>(a, s);
        case 512: return resident1d_n<double, 512>(a, s);
        case 1024: return resident1d_n<double, 1024>(a, s);
        case 2048: return resident1d_n<double, 2048>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gpe
