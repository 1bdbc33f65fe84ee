// FP32 persistent column pass (TMA tiles), instantiated for several tile widths: the
// autotuner of the batch handle times the candidates of each shape and keeps the fastest.
// The width only changes how many adjacent columns a block transforms at once; every
// pencil goes through the same arithmetic, so the results do not depend on it.
#include "prop_kernels.cuh"

namespace gpe {

namespace {

// Candidate tile widths (complex columns per tile) per pencil length: at least one warp
// per block, a box at least 16 bytes wide.
constexpr int kCandSmall[3] = {4, 8, 16};   // n <= 128 (8 or 16 threads per pencil)
constexpr int kCandLarge[3] = {2, 4, 8};    // n >= 256

template <int NN, int C, bool Z>
cudaError_t run(const CUtensorMap& map, const ColTmaArgs<float>& a, int sms, cudaStream_t s) {
    return colpass_tma_n<float, NN, C, false, Z>(map, a, sms, s);
}

template <int NN, bool Z>
cudaError_t by_cols(int cols, const CUtensorMap& map, const ColTmaArgs<float>& a, int sms, cudaStream_t s) {
    if constexpr (NN <= 128) {
        switch (cols) {
            case 4: return run<NN, 4, Z>(map, a, sms, s);
            case 8: return run<NN, 8, Z>(map, a, sms, s);
            case 16: return run<NN, 16, Z>(map, a, sms, s);
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (cols) {
            case 2: return run<NN, 2, Z>(map, a, sms, s);
            case 4: return run<NN, 4, Z>(map, a, sms, s);
            case 8: return run<NN, 8, Z>(map, a, sms, s);
            default: return cudaErrorInvalidValue;
        }
    }
}

}  // namespace

template <>
int colpass_tma_candidates<float>(int n, int* cols) {
    const int* c = n <= 128 ? kCandSmall : kCandLarge;
    for (int i = 0; i < 3; ++i) cols[i] = c[i];
    return 3;
}

template <>
cudaError_t launch_colpass_tma<float>(int n, int axis, int cols, const CUtensorMap& map, int n_tiles, int nx_tiles,
                                      int ny, const twel<float>* tws[3], const twel<float>* ph, int* status,
                                      cudaStream_t s, uint32_t wait_first) {
    ColTmaArgs<float> a{};
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
        a.tw = tws[tw_slot<Tune<float>::kColR(NN)>()];                                                     \
        return axis == 2 ? by_cols<NN, true>(cols, map, a, sms, s) : by_cols<NN, false>(cols, map, a, sms, s); \
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
