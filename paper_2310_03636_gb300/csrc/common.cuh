// Complex helpers and shared device utilities for the spin-1 GPE kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gpe {

template <typename T> struct cplx_sel;
template <> struct cplx_sel<float> { using type = float2; };
template <> struct cplx_sel<double> { using type = double2; };
template <typename T> using cplx = typename cplx_sel<T>::type;

// Table entry for twiddles and phase factors: FP32 tables carry each constant as a
// hi + lo pair (hi = fl(c), lo = fl(c - hi)), so the rounding of the constant itself,
// which would repeat identically in every step, drops to O(eps^2); FP64 tables hold c.
template <typename T> struct tw_sel;
template <> struct tw_sel<float> { using type = float4; };
template <> struct tw_sel<double> { using type = double2; };
template <typename T> using twel = typename tw_sel<T>::type;

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cconj(V a) { return mk(a.x, -a.y); }
// a * b
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
    return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename V, typename T> __device__ __forceinline__ V cscale(V a, T s) { return mk(a.x * s, a.y * s); }
// -i * a
template <typename V> __device__ __forceinline__ V cmul_mi(V a) { return mk(a.y, -a.x); }
template <typename V> __device__ __forceinline__ auto cabs2(V a) { return a.x * a.x + a.y * a.y; }

// w * f (DIR < 0) or w * conj(f) (DIR > 0) with f a table entry.
template <int DIR>
__device__ __forceinline__ float2 twmul(float2 w, float4 f) {
    const float fy = DIR < 0 ? f.y : -f.y, ly = DIR < 0 ? f.w : -f.w;
    const float sr = fmaf(w.x, f.z, -w.y * ly);
    const float si = fmaf(w.x, ly, w.y * f.z);
    return mk(fmaf(w.x, f.x, fmaf(-w.y, fy, sr)), fmaf(w.x, fy, fmaf(w.y, f.x, si)));
}
template <int DIR>
__device__ __forceinline__ double2 twmul(double2 w, double2 f) {
    const double fy = DIR < 0 ? f.y : -f.y;
    return mk(w.x * f.x - w.y * fy, w.x * fy + w.y * f.x);
}
// x * c for a compile-time constant c given in double: FP32 uses c_hi + c_lo.
__device__ __forceinline__ float mulc(float x, double c) {
    const float hi = (float)c;
    const float lo = (float)(c - (double)hi);
    return fmaf(x, lo, x * hi);
}
__device__ __forceinline__ double mulc(double x, double c) { return x * c; }

__device__ __forceinline__ void sincos_t(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_t(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_t(double x) { return sqrt(x); }

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

// q(t): piecewise linear through knots at t_j = j t_end / (K - 1), clamped (FP64).
__device__ __forceinline__ double q_at(double t, double q_const, const double* knots, int K,
                                       double t_end) {
    if (K <= 0) return q_const;
    if (K == 1) return knots[0];
    double u = t / t_end * (double)(K - 1);
    if (u <= 0.0) return knots[0];
    if (u >= (double)(K - 1)) return knots[K - 1];
    int i = (int)floor(u);
    double w = u - (double)i;
    return knots[i] * (1.0 - w) + knots[i + 1] * w;
}

}  // namespace gpe
