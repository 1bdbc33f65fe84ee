// FP32 x pass instantiations for x extents 512, 1024 (split from the other
// passes so the translation units compile in parallel).
#include "prop_kernels.cuh"

namespace gpe {

namespace {

// With compact phase tables (a.phc set) the x pass is built for 128 and 256 threads, and at
// 512 points also for 192 (three rows, four blocks per SM: 24 warps either way, but finer
// blocks interleave their copy and compute phases better; 298 vs 302 us at 512^2 x 64, the
// default there); 0 picks the default.  Without compact tables only the default size.
template <int NN>
static cudaError_t xpass_threads(int threads, bool pre, const PassArgs<float>& a, cudaStream_t s) {
    if (!a.phc || !a.tw2) return threads == 0 ? xpass_n<float, NN>(pre, a, s) : cudaErrorInvalidValue;
    if (threads == 0) threads = NN == 512 ? 192 : xpass_rows<NN, Tune<float>::kXR>() * (NN / Tune<float>::kXR);
    switch (threads) {
        case 128: return xpass_n<float, NN, 128, true>(pre, a, s);
        case 192:
            if constexpr (NN == 512) return xpass_n<float, NN, 192, true>(pre, a, s);
            else return cudaErrorInvalidValue;
        case 256: return xpass_n<float, NN, 256, true>(pre, a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_xpass_f32_large(int n, bool pre, const PassArgs<float>& a, cudaStream_t s, int threads) {
    switch (n) {
        case 512: return xpass_threads<512>(threads, pre, a, s);
        case 1024: return xpass_threads<1024>(threads, pre, a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gpe
