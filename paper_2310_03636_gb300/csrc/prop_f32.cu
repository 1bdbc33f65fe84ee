// Row and column pass instantiations for float fields.
#include "prop_kernels.cuh"

namespace gpe {

template <> int xpass_max_n<float>() { return 1024; }
template <> int colpass_max_n<float>() { return 1024; }
template <> int colpass_cols<float>(int n) { return Tune<float>::kColCols(n); }

template <>
cudaError_t launch_xpass<float>(int n, bool pre, const PassArgs<float>& a, cudaStream_t s) {
    switch (n) {
        case 64: return xpass_n<float, 64>(pre, a, s);
        case 128: return xpass_n<float, 128>(pre, a, s);
        case 256: return xpass_n<float, 256>(pre, a, s);
        case 512: return xpass_n<float, 512>(pre, a, s);
        case 1024: return xpass_n<float, 1024>(pre, a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_colpass<float>(int n, const PassArgs<float>& a, cudaStream_t s) {
    switch (n) {
        case 64: return colpass_n<float, 64, false>(a, s);
        case 128: return colpass_n<float, 128, false>(a, s);
        case 256: return colpass_n<float, 256, false>(a, s);
        case 512: return colpass_n<float, 512, false>(a, s);
        case 1024: return colpass_n<float, 1024, false>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_colfft<float>(int n, const PassArgs<float>& a, cudaStream_t s) {
    switch (n) {
        case 64: return colpass_n<float, 64, true>(a, s);
        case 128: return colpass_n<float, 128, true>(a, s);
        case 256: return colpass_n<float, 256, true>(a, s);
        case 512: return colpass_n<float, 512, true>(a, s);
        case 1024: return colpass_n<float, 1024, true>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_rowfft<float>(int n, cplx<float>* d, int64_t rows, const twel<float>* const* tw, cudaStream_t s) {
    switch (n) {
        case 64: return rowfft_n<float, 64>(d, rows, tw, s);
        case 128: return rowfft_n<float, 128>(d, rows, tw, s);
        case 256: return rowfft_n<float, 256>(d, rows, tw, s);
        case 512: return rowfft_n<float, 512>(d, rows, tw, s);
        case 1024: return rowfft_n<float, 1024>(d, rows, tw, s);
        case 2048: return rowfft_n<float, 2048>(d, rows, tw, s);
        case 4096: return rowfft_n<float, 4096>(d, rows, tw, s);
        case 8192: return rowfft_n<float, 8192>(d, rows, tw, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gpe

namespace gpe {

template <>
cudaError_t launch_colpass_tma<float>(int n, int axis, bool fwd_only, const CUtensorMap& map, int n_tiles, int nx_tiles,
                                  int ny, const twel<float>* tws[3], const twel<float>* ph, int* status, cudaStream_t s) {
    ColTmaArgs<float> a{};
    a.n_tiles = n_tiles;
    a.nx_tiles = nx_tiles;
    a.ny = ny;
    a.ph = ph;
    a.status = status;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = n_tiles < 2 * sms ? n_tiles : 2 * sms;
#define GPE_COLTMA(NN)                                                                                     \
    case NN: {                                                                                             \
        a.tw = tws[tw_slot<Tune<float>::kColR(NN)>()];                                                        \
        if (axis == 2) return fwd_only ? colpass_tma_n<float, NN, true, true>(map, a, grid, s)                \
                                       : colpass_tma_n<float, NN, false, true>(map, a, grid, s);              \
        return fwd_only ? colpass_tma_n<float, NN, true, false>(map, a, grid, s)                              \
                        : colpass_tma_n<float, NN, false, false>(map, a, grid, s);                            \
    }
    switch (n) {
        GPE_COLTMA(64)
        GPE_COLTMA(128)
        GPE_COLTMA(256)
        GPE_COLTMA(512)
        GPE_COLTMA(1024)
        default: return cudaErrorInvalidValue;
    }
#undef GPE_COLTMA
}

}  // namespace gpe
