// Row and column pass instantiations for float fields.
#include "prop_kernels.cuh"

namespace gpe {

template <> int xpass_max_n<float>() { return 1024; }
template <> int colpass_max_n<float>() { return 1024; }
template <> int colpass_cols<float>(int n) { return Tune<float>::kColCols(n); }

template <>
cudaError_t launch_xpass<float>(int n, bool pre, const PassArgs<float>& a, cudaStream_t s, int threads) {
    if (n <= 256) return launch_xpass_f32_small(n, pre, a, s, threads);
    return launch_xpass_f32_large(n, pre, a, s, threads);
}

template <>
int xpass_thread_candidates<float>(int n, int* threads) {
    for (int i = 0; i < 2; ++i) threads[i] = kXpassThreads[i];
    if (n != 512) return 2;
    threads[2] = 192;   // three rows per block, built at 512 points only
    return 3;
}

template <>
cudaError_t launch_colpass<float>(int n, const PassArgs<float>& a, cudaStream_t s) {
    switch (n) {
        case 64: return colpass_n<float, 64, kColK>(a, s);
        case 128: return colpass_n<float, 128, kColK>(a, s);
        case 256: return colpass_n<float, 256, kColK>(a, s);
        case 512: return colpass_n<float, 512, kColK>(a, s);
        case 1024: return colpass_n<float, 1024, kColK>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_colfft<float>(int n, const PassArgs<float>& a, cudaStream_t s) {
    switch (n) {
        case 64: return colpass_n<float, 64, kColFwd>(a, s);
        case 128: return colpass_n<float, 128, kColFwd>(a, s);
        case 256: return colpass_n<float, 256, kColFwd>(a, s);
        case 512: return colpass_n<float, 512, kColFwd>(a, s);
        case 1024: return colpass_n<float, 1024, kColFwd>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_colpass_mode<float>(int n, int mode, const PassArgs<float>& a, cudaStream_t s) {
#define GPE_COLMODE(NN)                                              \
    case NN:                                                         \
        switch (mode) {                                              \
            case kColK: return colpass_n<float, NN, kColK>(a, s);         \
            case kColFwd: return colpass_n<float, NN, kColFwd>(a, s);     \
            case kColKConj: return colpass_n<float, NN, kColKConj>(a, s); \
            case kColInv: return colpass_n<float, NN, kColInv>(a, s);     \
            default: return cudaErrorInvalidValue;                   \
        }
    switch (n) {
        GPE_COLMODE(64)
        GPE_COLMODE(128)
        GPE_COLMODE(256)
        GPE_COLMODE(512)
        GPE_COLMODE(1024)
        default: return cudaErrorInvalidValue;
    }
#undef GPE_COLMODE
}

template <>
cudaError_t launch_rowfft<float>(int n, cplx<float>* d, int64_t rows, const twel<float>* const* tw, cudaStream_t s, int dir) {
    if (dir > 0) {
        switch (n) {
            case 64: return rowfft_n<float, 64, 1>(d, rows, tw, s);
            case 128: return rowfft_n<float, 128, 1>(d, rows, tw, s);
            case 256: return rowfft_n<float, 256, 1>(d, rows, tw, s);
            case 512: return rowfft_n<float, 512, 1>(d, rows, tw, s);
            case 1024: return rowfft_n<float, 1024, 1>(d, rows, tw, s);
            case 2048: return rowfft_n<float, 2048, 1>(d, rows, tw, s);
            case 4096: return rowfft_n<float, 4096, 1>(d, rows, tw, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (n) {
        case 64: return rowfft_n<float, 64, -1>(d, rows, tw, s);
        case 128: return rowfft_n<float, 128, -1>(d, rows, tw, s);
        case 256: return rowfft_n<float, 256, -1>(d, rows, tw, s);
        case 512: return rowfft_n<float, 512, -1>(d, rows, tw, s);
        case 1024: return rowfft_n<float, 1024, -1>(d, rows, tw, s);
        case 2048: return rowfft_n<float, 2048, -1>(d, rows, tw, s);
        case 4096: return rowfft_n<float, 4096, -1>(d, rows, tw, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gpe

namespace gpe {


}  // namespace gpe
