// Internal declarations of the adjoint and loss kernels (adjoint.cu).
#pragma once

#include "internal.h"

namespace gpe {

template <typename T>
struct AdjArgs {
    int64_t sites;            // sites per trajectory (fields are [traj][3][sites], contiguous)
    int64_t rows_per_traj;    // ny * nz
    int64_t total_rows;       // ntraj * rows_per_traj
    const twel<T>* tw[3];     // x-axis stage twiddles for R = 4, 8, 16
    const twel<T>* ph;        // x-axis phase table exp(-i dt k^2 / 4) / nx
    T c0, c1, q, dt;
    const T* vpot;            // potential [3][sites] shared by the trajectories, or null
};

template <typename T> int64_t adjoint_parts(const Group& g);
template <typename T>
cudaError_t launch_xkin(int n, const AdjArgs<T>& a, cplx<T>* field, bool conj, cudaStream_t s);
template <typename T>
cudaError_t launch_xadj(int n, const AdjArgs<T>& a, cplx<T>* lam, const cplx<T>* phi, double* part, int* nparts,
                        cudaStream_t s);
cudaError_t launch_dq_final(const double* part, int nparts, double t_mid, int n_knots, double t_end, double* dLdq,
                            cudaStream_t s);
cudaError_t launch_fill_ptrs(void** ptrs, void* base, int64_t stride_bytes, int n, cudaStream_t s);
template <typename T>
cudaError_t launch_fperp(const cplx<T>* psi, cplx<T>* W, int64_t sites, int64_t total, cudaStream_t s);
template <typename T>
cudaError_t launch_sf_mask(cplx<T>* W, int64_t sites, int64_t total, const int n[3], double dx, double kmin, double kmax,
                           double c, double* part, int* nparts, cudaStream_t s);
template <typename T>
cudaError_t launch_sf_seed(const cplx<T>* psi, const cplx<T>* W, cplx<T>* lam, int64_t sites, int64_t total,
                           double scale, cudaStream_t s);
cudaError_t launch_sum_final(const double* part, int nparts, double* out, cudaStream_t s);

}  // namespace gpe
