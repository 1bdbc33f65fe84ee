// Internal (non-ABI) declarations shared by the kernel translation units and the C-ABI layer.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"
#include "gpe.h"
#include "local_step.cuh"

namespace gpe {

// Arguments of the axis passes.  A "row" pass works on pencils along x (contiguous),
// all three components of a site together; a "column" pass works on pencils along y or
// z (stride ``stride`` elements), one component at a time, COLS adjacent x columns per
// block.
template <typename T>
struct PassArgs {
    cplx<T>* const* ptrs;     // per trajectory of the group: field base pointer
    int64_t comp_stride;      // elements between components (= sites per trajectory)
    int64_t rows_per_traj;    // row pass: ny * nz
    int64_t total_rows;       // row pass: ntraj * rows_per_traj
    int64_t stride;           // column pass: elements between consecutive pencil points
    int64_t outer_stride;     // column pass: elements between consecutive outer indices
    int32_t n_outer;          // column pass: number of outer indices (z for a y pass, y for a z pass)
    int32_t nx_tiles;         // column pass: nx / COLS
    int32_t ntraj;
    int32_t ncomp;            // column pass: fields per trajectory (3, or 4 for spectra work)
    const twel<T>* tw[3];     // stage twiddle tables of the axis for R = 4, 8, 16 points per thread
    const twel<T>* ph_pre;    // row pass with a leading half kinetic step: its phase table
    const twel<T>* ph;        // phase table exp(-i tau k^2 / 2) / N
    LocalCoef<T> coef;        // couplings for the local step (row pass)
    const T* vpot;            // row pass: potential [3][sites] shared by the group, or null
    // FP32 row pass, when every kinetic angle of the x tables lies within +-pi/2: the
    // phase tables as (p, u) of the three-shear rotation for modes 0..N/2 (the table is
    // symmetric in k), the common factor 1/N apart; null otherwise
    const float2* phc;        // for ph
    const float2* phc_pre;    // for ph_pre
    float ph_scale;           // 1/N
    const float2* tw2;        // with phc: the x axis stage twiddles (8 points per thread) as
                              // (p, u) pairs, the sign taken from the index
    int* status;              // device status word (bounded waits that expire)
    uint32_t wait_first;      // row pass: 0 = default limit of the first copy wait, else 1 + its poll limit
};

template <typename T>
struct Res1DArgs {
    cplx<T>* const* ptrs;
    int32_t ntraj;
    const twel<T>* tw[3];     // stage twiddle tables for R = 4, 8, 16
    const twel<T>* ph_full;   // tau = dt
    const twel<T>* ph_half;   // tau = dt / 2
    T c0, c1, dt;
    double dt_d, t0, q_const, t_end;
    const double* knots;      // device, may be null
    int32_t n_knots;
    int64_t nsteps;
    int32_t kind;             // local step: 0 paper scheme, 1 spin rotation
    const T* vpot;            // potential [3][N] shared by the group, or null
};

struct NoiseArgs {
    void* const* ptrs;        // per trajectory field pointer
    const int32_t* traj_ids;  // batch index of each trajectory (Philox counter word 2)
    int32_t ntraj;
    uint32_t traj_base;       // added to the batch index
    int64_t sites;
    uint32_t key0, key1;
    double sigma;             // sqrt(noise_per_mode / dx^d)
    double mean[6];
    const double* mean_field; // [3][sites] (re, im) added to the mean, or null
};

// Trajectories of one shape and spacing, advanced together.
struct Group {
    int ndim = 1;
    int n[3] = {1, 1, 1};
    double dx = 1.0;
    int64_t sites = 0;
    int ntraj = 0;
    std::vector<int> ids;          // batch index of each member
    std::vector<void*> hptrs;      // field pointers (device addresses)
    void** dptrs = nullptr;        // same, on the device
    int32_t* d_ids = nullptr;      // same as ids, on the device
    void* tw[3][3] = {};           // per axis: stage twiddle tables for R = 4, 8, 16
    void* ph_full[3] = {};         // per axis: exp(-i dt k^2/2)/n
    void* ph_half[3] = {};         // per axis: exp(-i dt k^2/4)/n
    void* phc_full = nullptr;      // FP32 x axis: compact (p, u) tables for modes 0..n/2, when
    void* phc_half = nullptr;      //   every angle is within +-pi/2 (else null), and the stage
    void* tw2x = nullptr;          //   twiddles for 8 points per thread as (p, u) pairs
    bool contiguous = false;       // fields back to back from hptrs[0]: tensor-map passes usable
    int cluster = 0;               // 1D on a thread-block cluster: blocks per trajectory (0: off)
    void* tw_local[3] = {};        // cluster 1D: stage twiddles of the per-block length M
    void* wn = nullptr;            // cluster 1D: W_N^{n r}, r < cluster, n < M
    CUtensorMap map_y{};           // 2D map {2 nx, ntraj 3 nz ny} of the batch (ndim >= 2)
    CUtensorMap map_z{};           // 3D map {2 nx, ny, nz 3 ntraj} (ndim == 3)
    int cols[3] = {0, 0, 0};       // column-pass tile width per axis (1: y, 2: z)
    int xthreads = 0;              // x-pass block size (0: the default)
    bool xfixed = false;           // x-pass block size set by the caller (the autotuner leaves it)
    bool tuned = false;            // tile widths chosen by timing
    bool fixed = false;            // tile widths set by the caller (the autotuner skips the group)
    const void* vpot = nullptr;    // caller's potential [3][sites] (real, the batch's precision), or null
    const double* mean_field = nullptr;   // caller's initial mean field [3][sites] complex FP64, or null
};

// Sets the message gpe_last_error() returns on this thread.
void set_last_error(const char* msg);

// Every device allocation of the library goes through here, so that a test hook
// (gpe_debug_fail_alloc) can make one fail as if the device were out of memory.
cudaError_t device_malloc(void** p, size_t bytes);

// Whether kernels built for it may keep per-thread tables in tensor memory (the test hook
// gpe_debug_table_memory; on by default).
bool tables_in_tmem();

template <typename T> int xpass_max_n();
template <typename T> int colpass_max_n();
template <typename T> int resident1d_max_n();

// threads: block size of the x pass (0: the default; FP32 also one of
// xpass_thread_candidates).
template <typename T>
cudaError_t launch_xpass(int n, bool pre, const PassArgs<T>& a, cudaStream_t s, int threads = 0);
template <typename T>
int xpass_thread_candidates(int n, int* threads);
// The FP32 x pass for x extents up to 256 and from 512 (two translation units).
cudaError_t launch_xpass_f32_small(int n, bool pre, const PassArgs<float>& a, cudaStream_t s, int threads);
cudaError_t launch_xpass_f32_large(int n, bool pre, const PassArgs<float>& a, cudaStream_t s, int threads);
template <typename T>
cudaError_t launch_colpass(int n, const PassArgs<T>& a, cudaStream_t s);
// Column pass in a given mode: 0 kinetic factor, 1 forward FFT only, 2 adjoint kinetic
// factor (conjugate phases), 3 unnormalised inverse FFT only.
template <typename T>
cudaError_t launch_colpass_mode(int n, int mode, const PassArgs<T>& a, cudaStream_t s);
// Forward transform only (no phase, no inverse): used on spectra workspaces.
template <typename T>
cudaError_t launch_colfft(int n, const PassArgs<T>& a, cudaStream_t s);
// Row FFTs along x, dir = -1 forward, +1 unnormalised inverse.
template <typename T>
cudaError_t launch_rowfft(int n, cplx<T>* data, int64_t rows, const twel<T>* const* tw, cudaStream_t s, int dir = -1);
template <typename T>
int colpass_cols(int n);
// Persistent TMA column pass over a contiguous group: axis 1 (y) or 2 (z), tiles ``cols``
// complex columns wide (one of colpass_tma_candidates; the map's box must match).
template <typename T>
cudaError_t launch_colpass_tma(int n, int axis, int cols, const CUtensorMap& map, int n_tiles, int nx_tiles,
                               int ny, const twel<T>* tw4_8_16[3], const twel<T>* ph, int* status, cudaStream_t s,
                               uint32_t wait_first = 0);
// Tile widths the column pass is built for at pencil length n (written to cols[0..]).
template <typename T>
int colpass_tma_candidates(int n, int* cols);
// Tensor maps for the column passes of a group's shape over ntraj fields stored back to
// back from base (elements of ``elem_bytes`` per real), boxes cols_y / cols_z wide.
bool encode_maps(CUtensorMap* map_y, CUtensorMap* map_z, const Group& g, void* base, int ntraj, int elem_bytes,
                 int cols_y, int cols_z);
// Encodes the group's own maps with its current tile widths.
bool encode_group_maps(Group& g, int elem_bytes);
template <typename T>
cudaError_t launch_resident1d(int n, const Res1DArgs<T>& a, cudaStream_t s);
template <typename T>
cudaError_t launch_noise(const NoiseArgs& a, cudaStream_t s);
// Points per block of the cluster-resident 1D kernel, and its launcher (N = C M).
template <typename T> int res1d_cluster_block();
template <typename T>
cudaError_t launch_res1d_cluster(int n, const Res1DArgs<T>& a, const twel<T>* tw_local, const twel<T>* wn,
                                 cudaStream_t s);

}  // namespace gpe
