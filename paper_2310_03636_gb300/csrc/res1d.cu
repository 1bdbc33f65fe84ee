// Resident 1D kernel: the whole trajectory on chip for all steps.
#include "prop_kernels.cuh"
#include "res1d_tmem.cuh"

namespace gpe {

// Resident 1D: one block per trajectory; the field stays in shared memory for all steps
// (three padded pencil buffers):
//   K(dt/2) [L K(dt)]^(n-1) L K(dt/2).
// Each component's transform holds its R points per thread in registers and exchanges
// through the component's own buffer; the local step is a loop over the sites.  Keeping
// one component in registers at a time, with the site loop not unrolled, keeps the kernel
// small: a form with all three components in registers and every loop unrolled spent
// most of its cycles waiting for instruction fetch at N = 4096 (255 registers, one block
// per SM).  Stage twiddles and phases are read through L1.
//
// For short grids (N / R <= 64 threads per pencil) the block has G = 3 thread groups that
// transform the three components at the same time (group g owns component g), so a lone
// trajectory is not limited by the latency of three transforms in sequence; the local
// step's site loop then runs over all 3 N / R threads.
//
// The stage twiddles of the first twiddled stage (R - 1 rows of R entries: 3.8 KB at
// R = 16) sit in shared memory beside the field, tws_s; the later stages' entries, and the
// phases, are read through L1 (tws), except at N = 4096 and 2048 in FP32, where every thread
// keeps its own last-stage twiddles and full-step phases in tensor memory (res1d_tmem.cuh).
template <typename T, int N, int R>
constexpr int res1d_tw_split() {
    using P = FftPlan<N, R>;
    return P::kStages > 2 ? P::tw_offset(2) : P::tw_size();
}

template <typename T, int N, int R, int G, Sync SY>
__device__ __forceinline__ void kinetic_resident(cplx<T>* const (&buf)[3], const twel<T>* tws_s,
                                                 const twel<T>* __restrict__ tws, const twel<T>* __restrict__ ph,
                                                 int t, int grp) {
    constexpr int SPLIT = res1d_tw_split<T, N, R>();
    using V = cplx<T>;
    constexpr int TP = N / R;
#pragma unroll 1
    for (int c = (G == 3 ? grp : 0); c < 3; c += G) {
        V v[1][R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[0][m] = buf[c][spad(t + m * TP)];
        pencil_sync<SY>();   // every thread has its points before the first exchange overwrites
        V* const b1[1] = {buf[c]};
        fft_pencil_split<N, R, -1, 1, SY, SPLIT>(v, b1, tws_s, tws, t);
#pragma unroll
        for (int m = 0; m < R; ++m) v[0][m] = phmul<-1>(v[0][m], ph[t + m * TP]);
        fft_pencil_split<N, R, +1, 1, SY, SPLIT>(v, b1, tws_s, tws, t);
#pragma unroll
        for (int m = 0; m < R; ++m) buf[c][spad(t + m * TP)] = v[0][m];
    }
    __syncthreads();
}

// kinetic_resident for the tensor-memory variant: the transforms of fft_tmem and, with
// ph_tmem, the phases from tensor memory.
template <int N, int R, Sync SY>
__device__ __forceinline__ void kinetic_resident_tmem(float2* const (&buf)[3], const float4* tws_s,
                                                      const float4* __restrict__ ph, bool ph_tmem, uint32_t ta,
                                                      int t) {
    constexpr int TP = N / R;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        float2 v[1][R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[0][m] = buf[c][spad(t + m * TP)];
        pencil_sync<SY>();
        float2* const b1[1] = {buf[c]};
        fft_tmem<N, -1>(v, b1, tws_s, ta, t);
        if (ph_tmem) {
            phase_tmem(v[0], ta);
        } else {
#pragma unroll
            for (int m = 0; m < R; ++m) v[0][m] = phmul<-1>(v[0][m], ph[t + m * TP]);
        }
        fft_tmem<N, +1>(v, b1, tws_s, ta, t);
#pragma unroll
        for (int m = 0; m < R; ++m) buf[c][spad(t + m * TP)] = v[0][m];
    }
    __syncthreads();
}

// Component groups per block: 3 for short pencils (see kinetic_resident), else 1.
template <typename T, int N>
constexpr int res1d_groups() { return N / Tune<T>::kResR(N) <= 64 ? 3 : 1; }

// Synchronisation inside one component's transform: a warp when the group is a whole warp
// or the entire block fits in one, otherwise the block (all groups run the same stages).
template <int TP, int G>
constexpr Sync res1d_sync() { return (G == 1 ? TP <= 32 : (TP == 32 || G * TP <= 32)) ? Sync::Warp : Sync::Block; }

// Blocks per SM the resident kernel is compiled for: as many as its shared memory allows
// (at most 8), so that the register budget does not cap them further.
template <typename T, int N, int R>
constexpr size_t res1d_smem() {
    return (size_t)tw_off<T>(3 * smem_ld<T>(N)) * sizeof(cplx<T>) + (size_t)res1d_tw_split<T, N, R>() * sizeof(twel<T>);
}

template <typename T, int N, int G>
constexpr int res1d_blocks() {
    const int b = (227 * 1024) / ((int)res1d_smem<T, N, Tune<T>::kResR(N)>() + 1024);
    const int cap = G == 3 ? 4 : 8;
    return b < 1 ? 1 : (b > cap ? cap : b);
}

template <typename T, int N, int R, int G, bool TMW = true>
__global__ void __launch_bounds__(G * (N / R), res1d_blocks<T, N, G>())
k_resident1d(const Res1DArgs<T> a) {
    using V = cplx<T>;
    constexpr int TP = N / R;
    constexpr int NT = G * TP;
    constexpr int LD = smem_ld<T>(N);
    constexpr Sync SY = res1d_sync<TP, G>();
    extern __shared__ __align__(128) unsigned char smraw[];
    V* sm = reinterpret_cast<V*>(smraw);
    const twel<T>* tws = a.tw[tw_slot<R>()];
    twel<T>* tws_s = reinterpret_cast<twel<T>*>(sm + tw_off<T>(3 * LD));
    const int tid = threadIdx.x, grp = tid / TP, t = tid % TP;
    V* g = a.ptrs[blockIdx.x];
    V* const buf[3] = {sm, sm + LD, sm + 2 * LD};
    constexpr bool TM = TMW && res1d_tmem<T, N, R, G>();
    __shared__ uint32_t tslot;
    uint32_t tbase = 0, ta = 0;
    if constexpr (TM) {
        tbase = res1d_tmem_open(&tslot, res1d_tmem_cols<N>());
        ta = res1d_tmem_row(tbase);
        res1d_tmem_fill<N>(ta, tws, a.ph_full, 1, 0, t);
    }
    copy_table(tws_s, tws, res1d_tw_split<T, N, R>());
#pragma unroll 1
    for (int c = 0; c < 3; ++c)
        for (int i = tid; i < N; i += NT) buf[c][spad(i)] = g[c * N + i];
    __syncthreads();
    auto kinetic = [&](const twel<T>* ph, bool ph_full) {
        if constexpr (TM) kinetic_resident_tmem<N, R, SY>(buf, tws_s, ph, ph_full, ta, t);
        else kinetic_resident<T, N, R, G, SY>(buf, tws_s, tws, ph, t, grp);
    };
    kinetic(a.ph_half, false);
    LocalCoef<T> coef{a.c0, a.c1, (T)a.q_const, a.dt, a.kind};
    for (int64_t s = 0; s < a.nsteps; ++s) {
        coef.q = (T)q_at(a.t0 + ((double)s + 0.5) * a.dt_d, a.q_const, a.knots, a.n_knots, a.t_end);
        if (a.vpot == nullptr) {
            local_step_sites<T>(buf[0], buf[1], buf[2], tid, N, NT, coef, [](int i) { return spad(i); });
        } else {
#pragma unroll 2
            for (int i = tid; i < N; i += NT) {
                const int k = spad(i);
                V p1 = buf[0][k], p0 = buf[1][k], pm = buf[2][k];
                local_step<true, T>(p1, p0, pm, coef, site_pot<T>(a.vpot, N, i));
                buf[0][k] = p1;
                buf[1][k] = p0;
                buf[2][k] = pm;
            }
        }
        __syncthreads();
        const bool last = s == a.nsteps - 1;
        kinetic(last ? a.ph_half : a.ph_full, !last);
    }
#pragma unroll 1
    for (int c = 0; c < 3; ++c)
        for (int i = tid; i < N; i += NT) g[c * N + i] = buf[c][spad(i)];
    if constexpr (TM) res1d_tmem_close(tbase, res1d_tmem_cols<N>());
}

template <typename T, int N>
cudaError_t resident1d_n(const Res1DArgs<T>& a, cudaStream_t s) {
    constexpr int R = Tune<T>::kResR(N);
    constexpr int G = res1d_groups<T, N>();
    if constexpr (res1d_tmem<T, N, R, G>()) {
        if (!tables_in_tmem())
            return launch_with_smem(k_resident1d<T, N, R, G, false>, a.ntraj, G * (N / R), res1d_smem<T, N, R>(), s, &a);
    }
    return launch_with_smem(k_resident1d<T, N, R, G>, a.ntraj, G * (N / R), res1d_smem<T, N, R>(), s, &a);
}

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
