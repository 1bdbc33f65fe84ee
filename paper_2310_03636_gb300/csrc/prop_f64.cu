// Row and column pass instantiations for double fields.
#include "prop_kernels.cuh"

namespace gpe {

template <> int xpass_max_n<double>() { return 1024; }
template <> int xpass_thread_candidates<double>(int, int*) { return 0; }
template <> int colpass_max_n<double>() { return 1024; }
template <> int colpass_cols<double>(int n) { return Tune<double>::kColCols(n); }

template <>
cudaError_t launch_xpass<double>(int n, bool pre, const PassArgs<double>& a, cudaStream_t s, int threads) {
    if (threads != 0) return cudaErrorInvalidValue;   // FP64: the default block size only
    switch (n) {
        case 64: return xpass_n<double, 64>(pre, a, s);
        case 128: return xpass_n<double, 128>(pre, a, s);
        case 256: return xpass_n<double, 256>(pre, a, s);
        case 512: return xpass_n<double, 512>(pre, a, s);
        case 1024: return xpass_n<double, 1024>(pre, a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_colpass<double>(int n, const PassArgs<double>& a, cudaStream_t s) {
    switch (n) {
        case 64: return colpass_n<double, 64, kColK>(a, s);
        case 128: return colpass_n<double, 128, kColK>(a, s);
        case 256: return colpass_n<double, 256, kColK>(a, s);
        case 512: return colpass_n<double, 512, kColK>(a, s);
        case 1024: return colpass_n<double, 1024, kColK>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_colfft<double>(int n, const PassArgs<double>& a, cudaStream_t s) {
    switch (n) {
        case 64: return colpass_n<double, 64, kColFwd>(a, s);
        case 128: return colpass_n<double, 128, kColFwd>(a, s);
        case 256: return colpass_n<double, 256, kColFwd>(a, s);
        case 512: return colpass_n<double, 512, kColFwd>(a, s);
        case 1024: return colpass_n<double, 1024, kColFwd>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_colpass_mode<double>(int n, int mode, const PassArgs<double>& a, cudaStream_t s) {
#define GPE_COLMODE(NN)                                              \
    case NN:                                                         \
        switch (mode) {                                              \
            case kColK: return colpass_n<double, NN, kColK>(a, s);         \
            case kColFwd: return colpass_n<double, NN, kColFwd>(a, s);     \
            case kColKConj: return colpass_n<double, NN, kColKConj>(a, s); \
            case kColInv: return colpass_n<double, NN, kColInv>(a, s);     \
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
cudaError_t launch_rowfft<double>(int n, cplx<double>* d, int64_t rows, const twel<double>* const* tw, cudaStream_t s, int dir) {
    if (dir > 0) {
        switch (n) {
            case 64: return rowfft_n<double, 64, 1>(d, rows, tw, s);
            case 128: return rowfft_n<double, 128, 1>(d, rows, tw, s);
            case 256: return rowfft_n<double, 256, 1>(d, rows, tw, s);
            case 512: return rowfft_n<double, 512, 1>(d, rows, tw, s);
            case 1024: return rowfft_n<double, 1024, 1>(d, rows, tw, s);
            case 2048: return rowfft_n<double, 2048, 1>(d, rows, tw, s);
            case 4096: return rowfft_n<double, 4096, 1>(d, rows, tw, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (n) {
        case 64: return rowfft_n<double, 64, -1>(d, rows, tw, s);
        case 128: return rowfft_n<double, 128, -1>(d, rows, tw, s);
        case 256: return rowfft_n<double, 256, -1>(d, rows, tw, s);
        case 512: return rowfft_n<double, 512, -1>(d, rows, tw, s);
        case 1024: return rowfft_n<double, 1024, -1>(d, rows, tw, s);
        case 2048: return rowfft_n<double, 2048, -1>(d, rows, tw, s);
        case 4096: return rowfft_n<double, 4096, -1>(d, rows, tw, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gpe

namespace gpe {

template <>
int colpass_tma_candidates<double>(int n, int* cols) {
    cols[0] = Tune<double>::kColCols(n);
    return 1;
}

template <>
cudaError_t launch_colpass_tma<double>(int n, int axis, int cols, const CUtensorMap& map, int n_tiles, int nx_tiles,
                                       int ny, const twel<double>* tws[3], const twel<double>* ph, int* status,
                                       cudaStream_t s, uint32_t wait_first) {
    if (cols != Tune<double>::kColCols(n)) return cudaErrorInvalidValue;
    ColTmaArgs<double> a{};
    a.wait_first = wait_first;
    a.n_tiles = n_tiles;
    a.nx_tiles = nx_tiles;
    a.ny = ny;
    a.ph = ph;
    a.status = status;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
#define GPE_COLTMA(NN)                                                                                     \
    case NN: {                                                                                             \
        constexpr int C = Tune<double>::kColCols(NN);                                                      \
        a.tw = tws[tw_slot<Tune<double>::kColR(NN)>()];                                                    \
        if (axis == 2) return colpass_tma_n<double, NN, C, false, true>(map, a, sms, s);                   \
        return colpass_tma_n<double, NN, C, false, false>(map, a, sms, s);                                 \
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
