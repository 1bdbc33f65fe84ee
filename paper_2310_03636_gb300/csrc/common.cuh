// Complex helpers and shared device utilities for the spin-1 GPE kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gpe {

template <typename T> struct cplx_sel;
template <> struct cplx_sel<float> { using type = float2; };
template <> struct cplx_sel<double> { using type = double2; };
template <typename T> using cplx = typename cplx_sel<T>::type;

// Table entry for twiddles and phase factors c = m e^{i phi} (m = 1 for twiddles, 1/N for
// the kinetic phases).  FP64 tables hold c.  FP32 tables hold the rotation in three-shear
// ("lifting") form: phi is reduced by a multiple j of pi to phi' in [-pi/2, pi/2], and the
// entry is (p, u, s, 0) with p = -tan(phi'/2), u = sin(phi'), s = (-1)^j m, each computed in
// FP64 and rounded once.  The rotation is applied as x += p y; y += u x; x += p y (three
// fmas) and scaled by s.  The three shears have determinant exactly 1 whatever the rounding
// of p and u, so the map preserves area: its mean gain in |w|^2 over the phase of w is
// 1 + O(eps^2), whereas an FP32 pair (fl(cos), fl(sin)) scales |w|^2 by a fixed
// 1 + O(eps) that repeats in every step and accumulates.  The angle error is relative
// (O(eps phi)), so small kinetic phases stay exact to FP32 precision.
template <typename T> struct tw_sel;
template <> struct tw_sel<float> { using type = float4; };
template <> struct tw_sel<double> { using type = double2; };
template <typename T> using twel = typename tw_sel<T>::type;

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk(a.x - b.x, a.y - b.y); }
// FP32 complex add / subtract as one packed two-lane instruction (sm_100 family).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
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

// w e^{i phi} by three shears (p = -tan(phi/2), u = sin(phi), |phi| <= pi/2).
__device__ __forceinline__ float2 lift_rot(float2 w, float p, float u) {
    const float x1 = fmaf(p, w.y, w.x);
    const float y1 = fmaf(u, x1, w.y);
    return make_float2(fmaf(p, y1, x1), y1);
}

// w * f (DIR < 0) or w * conj(f) (DIR > 0) with f a table entry.  SIG = false skips the
// factor s where the caller knows every entry it reads has s = +1 (angles within +-pi/2,
// unit modulus).
template <int DIR, bool SIG = true>
__device__ __forceinline__ float2 twmul(float2 w, float4 f) {
    const float2 r = lift_rot(w, DIR < 0 ? f.x : -f.x, DIR < 0 ? f.y : -f.y);
    if constexpr (SIG) return make_float2(r.x * f.z, r.y * f.z);
    return r;
}
template <int DIR, bool SIG = true>
__device__ __forceinline__ double2 twmul(double2 w, double2 f) {
    const double fy = DIR < 0 ? f.y : -f.y;
    return mk(w.x * f.x - w.y * fy, w.x * fy + w.y * f.x);
}

// The same product for a kinetic phase-table entry (scale 1/N included).
template <int DIR>
__device__ __forceinline__ float2 phmul(float2 w, float4 f) {
    return twmul<DIR, true>(w, f);
}
template <int DIR>
__device__ __forceinline__ double2 phmul(double2 w, double2 f) {
    return twmul<DIR>(w, f);
}
// x * c for a compile-time constant c given in double: FP32 uses c_hi + c_lo, with the
// small product x c_lo added inside the fma that forms the exact x c_hi, so the result is
// x c rounded once.  (Rounding x c_hi first and adding x c_lo afterwards would lose the
// correction, which is below half an ulp: every product would then carry the constant's
// own rounding error, the same sign in every transform, and the norm would drift.)
__device__ __forceinline__ float mulc(float x, double c) {
    const float hi = (float)c;
    const float lo = (float)(c - (double)hi);
    return fmaf(x, hi, x * lo);
}
__device__ __forceinline__ double mulc(double x, double c) { return x * c; }

static __device__ __noinline__ void sincos_lib(float x, float* s, float* c) { sincosf(x, s, c); }

// sin and cos in FP32 without a slow path: Cody-Waite reduction x = r + q pi/2 with
// pi/2 split into fl(pi/2) and its remainder, then Taylor polynomials of sin (to r^9)
// and cos (to r^10) on |r| <= pi/4 (truncation below 3e-9 relative).  |x| > 1e4 goes
// to the library routine.
__device__ __forceinline__ void sincos_t(float x, float* s, float* c) {
    if (fabsf(x) > 1.0e4f) {
        sincos_lib(x, s, c);
        return;
    }
    const float q = rintf(x * 0.636619772367581343f);
    float r = fmaf(q, -1.57079637050628662109375f, x);
    r = fmaf(q, 4.37113900018624283e-8f, r);
    const float r2 = r * r;
    float ps = fmaf(r2, 2.75573192239858907e-6f, -1.98412698412698413e-4f);
    ps = fmaf(ps, r2, 8.33333333333333333e-3f);
    ps = fmaf(ps, r2, -1.66666666666666667e-1f);
    const float sn = fmaf(ps * r2, r, r);
    float pc = fmaf(r2, -2.75573192239858907e-7f, 2.48015873015873016e-5f);
    pc = fmaf(pc, r2, -1.38888888888888889e-3f);
    pc = fmaf(pc, r2, 4.16666666666666667e-2f);
    pc = fmaf(pc, r2, -0.5f);
    const float cs = fmaf(pc, r2, 1.0f);
    const int iq = (int)q;
    float so = (iq & 1) ? cs : sn;
    float co = (iq & 1) ? sn : cs;
    if (iq & 2) so = -so;
    if ((iq + 1) & 2) co = -co;
    *s = so;
    *c = co;
}
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
