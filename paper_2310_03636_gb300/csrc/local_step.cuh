// Per-site nonlinear part of the split step: L(dt) = D(dt/2) O(dt) D(dt/2).
//
// D (diagonal step of Sec. 2.2): psi_m <- psi_m exp(-i (V_m + f_m) tau) with the
// external potential V_m(x) (zero unless the caller sets one) and the diagonal
// entries of the operator of Eq. (GPE):
//   f_1  = q + (c0 + c1) rho - 2 c1 |psi_-1|^2
//   f_0  =     (c0 + c1) rho -   c1 |psi_0|^2        (q - c1 q / c1 = 0)
//   f_-1 = q + (c0 + c1) rho - 2 c1 |psi_1|^2
// evaluated on the field D acts on (D leaves every density unchanged, so it is exact).
//
// O (off-diagonal step of Sec. 2.2): with S = [[0, a, 0], [a*, 0, b], [0, b*, 0]],
// a = psi_-1^* psi_0, b = psi_0^* psi_1, the predictor psi~ = psi - i c1 dt S psi, and
// the averages A = (a + a~)/2, B = (b + b~)/2, the printed 3x3 matrix equals
//   U = exp(-i c1 dt S_AB) = 1 - i (sin th / lambda) S_AB + ((cos th - 1) / lambda^2) S_AB^2,
// th = lambda c1 dt, lambda^2 = |A|^2 + |B|^2 (S_AB^3 = lambda^2 S_AB).  The kernel
// applies it as psi - i eps s1 S psi - eps^2 s2 S (S psi) with eps = c1 dt,
// s1 = sin(th)/th and s2 = (1 - cos th)/th^2 = sinc^2(th/2)/2, both from one sincos of
// th/2, which is finite and accurate down to lambda = 0 (where U = 1).  The paper's
// form divides by lambda^2; this one does not, and is algebraically identical.
#pragma once

#include "common.cuh"

namespace gpe {

template <typename T>
struct LocalCoef {
    T c0, c1, q, dt;
    int kind;   // 0: the paper's D O D step, 1: exact spin rotation (see local_step_rot)
};

// External potential at one site: V_1, V_0, V_-1.
template <typename T>
struct SitePot {
    T v1, v0, vm;
};

template <typename T, typename V>
__device__ __forceinline__ void diag_phase(V& p1, V& p0, V& pm, T c0, T c1, T q, T tau, SitePot<T> vp) {
    const T n1 = cabs2(p1), n0 = cabs2(p0), nm = cabs2(pm);
    const T g = (c0 + c1) * (n1 + n0 + nm);
    const T th1 = (vp.v1 + q + g - (T)2 * c1 * nm) * tau;
    const T th0 = (vp.v0 + g - c1 * n0) * tau;
    const T thm = (vp.vm + q + g - (T)2 * c1 * n1) * tau;
    T s, c;
    sincos_t(th1, &s, &c);
    p1 = mk(p1.x * c + p1.y * s, p1.y * c - p1.x * s);
    sincos_t(th0, &s, &c);
    p0 = mk(p0.x * c + p0.y * s, p0.y * c - p0.x * s);
    sincos_t(thm, &s, &c);
    pm = mk(pm.x * c + pm.y * s, pm.y * c - pm.x * s);
}

template <typename T, typename V>
__device__ __forceinline__ void offdiag_mix(V& p1, V& p0, V& pm, T c1, T dt) {
    const T eps = c1 * dt;
    const V a = cmulc(pm, p0);   // psi_-1^* psi_0
    const V b = cmulc(p0, p1);   // psi_0^* psi_1
    // predictor psi~ = psi - i eps S psi
    const V s1 = cmul(a, p0);
    const V s0 = cadd(cmulc(a, p1), cmul(b, pm));
    const V sm = cmulc(b, p0);
    const V t1 = csub(p1, cscale(mk(-s1.y, s1.x), eps));
    const V t0 = csub(p0, cscale(mk(-s0.y, s0.x), eps));
    const V tm = csub(pm, cscale(mk(-sm.y, sm.x), eps));
    const V A = cscale(cadd(a, cmulc(tm, t0)), (T)0.5);
    const V B = cscale(cadd(b, cmulc(t0, t1)), (T)0.5);
    const T lam = sqrt_t(cabs2(A) + cabs2(B));
    const T x = (T)0.5 * lam * eps;   // th / 2
    T sx, cx;
    sincos_t(x, &sx, &cx);
    const T r = (x != (T)0) ? sx / x : (T)1;   // sinc(th/2)
    const T e1 = eps * r * cx;                 // eps sin(th)/th
    const T e2 = (T)0.5 * eps * eps * r * r;   // eps^2 (1 - cos th)/th^2
    // S_AB psi and S_AB^2 psi
    const V u1 = cmul(A, p0);
    const V u0 = cadd(cmulc(A, p1), cmul(B, pm));
    const V um = cmulc(B, p0);
    const V w1 = cmul(A, u0);
    const V w0 = cadd(cmulc(A, u1), cmul(B, um));
    const V wm = cmulc(B, u0);
    // psi + (-i e1 u - e2 w): the change is formed first and added once (see local_step_fast)
    p1 = mk(p1.x + (e1 * u1.y - e2 * w1.x), p1.y - (e1 * u1.x + e2 * w1.y));
    p0 = mk(p0.x + (e1 * u0.y - e2 * w0.x), p0.y - (e1 * u0.x + e2 * w0.y));
    pm = mk(pm.x + (e1 * um.y - e2 * wm.x), pm.y - (e1 * um.x + e2 * wm.y));
}

// sin x and cos x - 1: Taylor polynomials for |x| <= 1/2 (truncation below 2e-11), so
// cos x - 1 keeps its relative accuracy for small x; otherwise the range-reduced routine.
__device__ __forceinline__ void sincosm1(float x, float* s, float* cm1) {
    if (fabsf(x) > 0.5f) {
        float c;
        sincos_t(x, s, &c);
        *cm1 = c - 1.0f;
        return;
    }
    const float x2 = x * x;
    float ps = fmaf(x2, 2.75573192239858907e-6f, -1.98412698412698413e-4f);
    ps = fmaf(ps, x2, 8.33333333333333333e-3f);
    ps = fmaf(ps, x2, -1.66666666666666667e-1f);
    *s = fmaf(ps * x2, x, x);
    float pc = fmaf(x2, -2.75573192239858907e-7f, 2.48015873015873016e-5f);
    pc = fmaf(pc, x2, -1.38888888888888889e-3f);
    pc = fmaf(pc, x2, 4.16666666666666667e-2f);
    pc = fmaf(pc, x2, -0.5f);
    *cm1 = pc * x2;
}
__device__ __forceinline__ void sincosm1(double x, double* s, double* cm1) {
    double c;
    sincos(x, s, &c);
    *cm1 = c - 1.0;
}

// p e^{-i ang}, written p + [p (cos ang - 1) - i p sin ang] so that the rotation changes
// |p| only through the rounding of that final sum (unbiased).  The direct form
// p cos + ... is biased in FP32: near 1, fl(cos) carries a relative error of up to
// 2^-25 that is the same for every site and step when the angle barely varies (a
// constant q dt/2, or angles below 2.4e-4, where fl(cos) = 1 while sin != 0), and
// |p|^2 then drifts by up to ~1e-7 per step.
template <typename T, typename V>
__device__ __forceinline__ V rot_minus(V p, T ang) {
    T s, cm1;
    sincosm1(ang, &s, &cm1);
    return mk(p.x + (p.x * cm1 + p.y * s), p.y + (p.y * cm1 - p.x * s));
}

// FP32 local step, same operator as D(dt/2) O(dt) D(dt/2) but arranged for fewer
// transcendental evaluations:
//  * a common phase of all three components commutes with O (a and b are invariant),
//    so each D applies the m = +-1 phases relative to m = 0 and the two m = 0 phases
//    are applied once at the end;
//  * the O coefficients sin(th)/th and (1 - cos th)/th^2 are even in th, so they are
//    power series in u = th^2 = lambda^2 (c1 dt)^2 (no square root or division):
//    sum (-u)^k / (2k+1)! and sum (-u)^k / (2k+2)! to k = 4 for u <= 1/4 (truncation
//    below 3e-11), the trigonometric form otherwise.
// With HAS_V the potential enters the same angles: V_0 in the common phase, V_+-1 - V_0
// in the relative ones.
template <bool HAS_V>
__device__ __forceinline__ void local_step_fast(float2& p1, float2& p0, float2& pm, const LocalCoef<float>& k,
                                                SitePot<float> vp) {
    const float h = 0.5f * k.dt;
    const float c0 = k.c0, c1 = k.c1, q = k.q;
    const float q1 = HAS_V ? q + (vp.v1 - vp.v0) : q;
    const float qm = HAS_V ? q + (vp.vm - vp.v0) : q;
    // D(dt/2), relative to m = 0
    float n1 = cabs2(p1), n0 = cabs2(p0), nm = cabs2(pm);
    const float g0 = HAS_V ? ((c0 + c1) * (n1 + n0 + nm) - c1 * n0 + vp.v0) * h
                           : ((c0 + c1) * (n1 + n0 + nm) - c1 * n0) * h;
    p1 = rot_minus(p1, (q1 - 2.0f * c1 * nm + c1 * n0) * h);
    pm = rot_minus(pm, (qm - 2.0f * c1 * n1 + c1 * n0) * h);
    // O(dt)
    const float eps = c1 * k.dt;
    const float2 a = cmulc(pm, p0);
    const float2 b = cmulc(p0, p1);
    const float2 s1 = cmul(a, p0);
    const float2 s0 = cadd(cmulc(a, p1), cmul(b, pm));
    const float2 sm = cmulc(b, p0);
    const float2 t1 = make_float2(fmaf(eps, s1.y, p1.x), fmaf(-eps, s1.x, p1.y));
    const float2 t0 = make_float2(fmaf(eps, s0.y, p0.x), fmaf(-eps, s0.x, p0.y));
    const float2 tm = make_float2(fmaf(eps, sm.y, pm.x), fmaf(-eps, sm.x, pm.y));
    const float2 A = cscale(cadd(a, cmulc(tm, t0)), 0.5f);
    const float2 B = cscale(cadd(b, cmulc(t0, t1)), 0.5f);
    const float u = (cabs2(A) + cabs2(B)) * (eps * eps);
    float f1, f2;
    if (u <= 0.25f) {
        f1 = fmaf(u, 2.75573192239858907e-6f, -1.98412698412698413e-4f);
        f1 = fmaf(f1, u, 8.33333333333333333e-3f);
        f1 = fmaf(f1, u, -1.66666666666666667e-1f);
        f1 = fmaf(f1, u, 1.0f);
        f2 = fmaf(u, 2.75573192239858907e-7f, -2.48015873015873016e-5f);
        f2 = fmaf(f2, u, 1.38888888888888889e-3f);
        f2 = fmaf(f2, u, -4.16666666666666667e-2f);
        f2 = fmaf(f2, u, 0.5f);
    } else {
        const float x = 0.5f * sqrtf(u);
        float sx, cx;
        sincos_t(x, &sx, &cx);
        const float r = sx / x;
        f1 = r * cx;
        f2 = 0.5f * r * r;
    }
    const float e1 = eps * f1, e2 = eps * eps * f2;
    const float2 u1 = cmul(A, p0);
    const float2 u0 = cadd(cmulc(A, p1), cmul(B, pm));
    const float2 um = cmulc(B, p0);
    const float2 w1 = cmul(A, u0);
    const float2 w0 = cadd(cmulc(A, u1), cmul(B, um));
    const float2 wm = cmulc(B, u0);
    // psi + (-i e1 u - e2 w), the change formed first and added with one rounding.  Adding
    // -i e1 u and -e2 w to psi one after the other loses the second-order term wherever it
    // is below half an ulp of psi (psi_0 while the spin modes are still small): the
    // first-order transfer into psi_+-1 then goes uncompensated and |psi|^2 grows.
    p1 = make_float2(p1.x + (e1 * u1.y - e2 * w1.x), p1.y - (e1 * u1.x + e2 * w1.y));
    p0 = make_float2(p0.x + (e1 * u0.y - e2 * w0.x), p0.y - (e1 * u0.x + e2 * w0.y));
    pm = make_float2(pm.x + (e1 * um.y - e2 * wm.x), pm.y - (e1 * um.x + e2 * wm.y));
    // D(dt/2) with the deferred m = 0 phases of both halves
    n1 = cabs2(p1);
    n0 = cabs2(p0);
    nm = cabs2(pm);
    const float gg = HAS_V ? g0 + ((c0 + c1) * (n1 + n0 + nm) - c1 * n0 + vp.v0) * h
                           : g0 + ((c0 + c1) * (n1 + n0 + nm) - c1 * n0) * h;
    p1 = rot_minus(p1, gg + (q1 - 2.0f * c1 * nm + c1 * n0) * h);
    pm = rot_minus(pm, gg + (qm - 2.0f * c1 * n1 + c1 * n0) * h);
    p0 = rot_minus(p0, gg);
}

// Alternative local step with the same operator split differently: the interaction part
// of Eq. (GPE) is c0 rho + c1 F.f + q f_z^2 (f: spin-1 matrices, F = psi^+ f psi).  The
// flow of c0 rho + c1 F.f keeps rho and F fixed, so it is exactly
// exp(-i c0 rho tau) exp(-i c1 tau F.f); for spin 1, with th = c1 tau |F|,
//   exp(-i c1 tau F.f) = 1 - i c1 tau s1(th) F.f - (c1 tau)^2 s2(th) (F.f)^2,
// s1 = sin(th)/th, s2 = (1 - cos th)/th^2 as power series in th^2 (no division).  The
// q f_z^2 phase is split symmetrically around it: Q(dt/2) R(dt) Q(dt/2).  F_z is kept
// exactly by every factor.  A potential V_m is diagonal like q f_z^2 and joins Q.
template <bool HAS_V, typename T, typename V>
__device__ __forceinline__ void local_step_rot(V& p1, V& p0, V& pm, const LocalCoef<T>& k, SitePot<T> vp) {
    const T h = (T)0.5 * k.dt;
    const T v1 = HAS_V ? vp.v1 : (T)0, v0 = HAS_V ? vp.v0 : (T)0, vm = HAS_V ? vp.vm : (T)0;
    p1 = rot_minus(p1, (k.q + v1) * h);
    pm = rot_minus(pm, (k.q + vm) * h);
    if (HAS_V) p0 = rot_minus(p0, v0 * h);
    const T n1 = cabs2(p1), n0 = cabs2(p0), nm = cabs2(pm);
    const T rho = n1 + n0 + nm, fz = n1 - nm;
    const V A = cadd(cmulc(p1, p0), cmulc(p0, pm));   // F_+ / sqrt2
    const T eps = k.c1 * k.dt;
    const T u = eps * eps * (fz * fz + (T)2 * cabs2(A));
    T s1, s2;
    if (u <= (T)0.25) {
        s1 = (T)2.75573192239858907e-6;
        s1 = s1 * u + (T)(-1.98412698412698413e-4);
        s1 = s1 * u + (T)8.33333333333333333e-3;
        s1 = s1 * u + (T)(-1.66666666666666667e-1);
        s1 = s1 * u + (T)1;
        s2 = (T)2.75573192239858907e-7;
        s2 = s2 * u + (T)(-2.48015873015873016e-5);
        s2 = s2 * u + (T)1.38888888888888889e-3;
        s2 = s2 * u + (T)(-4.16666666666666667e-2);
        s2 = s2 * u + (T)0.5;
    }
    if (u > (T)0.25 || (sizeof(T) == 8 && u > (T)1e-6)) {
        // trigonometric form from the half angle: sin th = 2 sh ch, 1 - cos th = 2 sh^2
        const T th = sqrt_t(u);
        T sh, ch;
        sincos_t((T)0.5 * th, &sh, &ch);
        s1 = (T)2 * sh * ch / th;
        s2 = (T)2 * sh * sh / u;
    }
    const T e1 = eps * s1, e2 = eps * eps * s2;
    // g = (F.f) p, w = (F.f) g with F.f = [[fz, A*, 0], [A, 0, A*], [0, A, -fz]]
    const V g1 = cadd(cscale(p1, fz), cmulc(A, p0));
    const V g0 = cadd(cmul(A, p1), cmulc(A, pm));
    const V gm = csub(cmul(A, p0), cscale(pm, fz));
    const V w1 = cadd(cscale(g1, fz), cmulc(A, g0));
    const V w0 = cadd(cmul(A, g1), cmulc(A, gm));
    const V wm = csub(cmul(A, g0), cscale(gm, fz));
    V r1 = mk(p1.x + (e1 * g1.y - e2 * w1.x), p1.y - (e1 * g1.x + e2 * w1.y));
    V r0 = mk(p0.x + (e1 * g0.y - e2 * w0.x), p0.y - (e1 * g0.x + e2 * w0.y));
    V rm = mk(pm.x + (e1 * gm.y - e2 * wm.x), pm.y - (e1 * gm.x + e2 * wm.y));
    // c0 phase on all three and the second half of Q, one angle per component
    const T a0 = k.c0 * rho * k.dt;
    p1 = rot_minus(r1, a0 + (k.q + v1) * h);
    p0 = rot_minus(r0, a0 + v0 * h);
    pm = rot_minus(rm, a0 + (k.q + vm) * h);
}

// The local step at one site; HAS_V adds the potential vp (otherwise ignored).
template <bool HAS_V, typename T, typename V>
__device__ __forceinline__ void local_step(V& p1, V& p0, V& pm, const LocalCoef<T>& k, SitePot<T> vp) {
    if (k.kind == 1) {
        local_step_rot<HAS_V, T>(p1, p0, pm, k, vp);
        return;
    }
    if constexpr (sizeof(T) == 4) {
        local_step_fast<HAS_V>(p1, p0, pm, k, vp);
    } else {
        const T h = (T)0.5 * k.dt;
        const SitePot<T> v = HAS_V ? vp : SitePot<T>{(T)0, (T)0, (T)0};
        diag_phase<T>(p1, p0, pm, k.c0, k.c1, k.q, h, v);
        offdiag_mix<T>(p1, p0, pm, k.c1, k.dt);
        diag_phase<T>(p1, p0, pm, k.c0, k.c1, k.q, h, v);
    }
}

template <typename T, typename V>
__device__ __forceinline__ void local_step(V& p1, V& p0, V& pm, const LocalCoef<T>& k) {
    local_step<false, T>(p1, p0, pm, k, SitePot<T>{(T)0, (T)0, (T)0});
}

// Potential of site i from a [3][sites] array (comp_stride = sites), or zero.
template <typename T>
__device__ __forceinline__ SitePot<T> site_pot(const T* __restrict__ vpot, int64_t comp_stride, int64_t i) {
    return SitePot<T>{__ldg(vpot + i), __ldg(vpot + comp_stride + i), __ldg(vpot + 2 * comp_stride + i)};
}

}  // namespace gpe
