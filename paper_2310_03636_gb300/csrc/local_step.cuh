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

// sin x and cos x - 1: Taylor polynomials for |x| <= 1/2 (sin to x^7, cos - 1 to x^8:
// truncation at most 1.1e-8 and 2.2e-9 relative at |x| = 1/2, far less for the small angles
// of a time step), so cos x - 1 keeps its relative accuracy for small x; otherwise the
// range-reduced routine.  In the rotation form of rot_minus an error d in either term
// changes |p| only at second order in x (|1 + (c - 1) - i s|^2 - 1 = O(x^2 d)) and the angle
// by x d.
__device__ __forceinline__ void sincosm1(float x, float* s, float* cm1) {
    if (fabsf(x) > 0.5f) {
        float c;
        sincos_t(x, s, &c);
        *cm1 = c - 1.0f;
        return;
    }
    const float x2 = x * x;
    float ps = fmaf(x2, -1.98412698412698413e-4f, 8.33333333333333333e-3f);
    ps = fmaf(ps, x2, -1.66666666666666667e-1f);
    *s = fmaf(ps * x2, x, x);
    float pc = fmaf(x2, 2.48015873015873016e-5f, -1.38888888888888889e-3f);
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
    return mk(p.x + fma(p.x, cm1, p.y * s), p.y + fma(p.y, cm1, (-p.x) * s));
}

// FP32 local step, same operator as D(dt/2) O(dt) D(dt/2) but arranged for fewer
// operations:
//  * a common phase of all three components commutes with O (a and b are invariant),
//    so each D applies the m = +-1 phases relative to m = 0 and the two m = 0 phases
//    are applied once at the end;
//  * h = dt/2 is folded into the angle coefficients;
//  * O is applied with 2A = a + a~ and 2B = b + b~ (the averages without their factor
//    1/2, which goes into the coefficients as exact powers of two);
//  * the O coefficients sin(th)/th and (1 - cos th)/th^2 are even in th, so they are
//    power series in u = th^2 = |A|^2 + |B|^2 (c1 dt)^2 (no square root or division):
//    sum (-u)^k / (2k+1)! and sum (-u)^k / (2k+2)! to k = 3 for u <= 1/4 (truncation
//    below 1.1e-8 relative), the trigonometric form otherwise.
// Products are written as explicit fmas so that local_step_pair, the same step for two
// sites in the two lanes of the packed FP32 instructions, gives the same bits per lane.
// With HAS_V the potential enters the same angles: V_0 in the common phase, V_+-1 - V_0
// in the relative ones.
__device__ __forceinline__ float abs2f(float2 z) { return fmaf(z.x, z.x, z.y * z.y); }
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {   // a b
    return make_float2(fmaf(a.x, b.x, (-a.y) * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulcf(float2 a, float2 b) {  // conj(a) b
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, (-a.y) * b.x));
}
__device__ __forceinline__ float2 caddf(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

// The O coefficients f1 = sin(th)/th, f2 = (1 - cos th)/th^2 from u = th^2.
__device__ __forceinline__ void o_coef(float u, float* f1, float* f2) {
    if (u <= 0.25f) {
        float g1 = fmaf(u, -1.98412698412698413e-4f, 8.33333333333333333e-3f);
        g1 = fmaf(g1, u, -1.66666666666666667e-1f);
        *f1 = fmaf(g1, u, 1.0f);
        float g2 = fmaf(u, -2.48015873015873016e-5f, 1.38888888888888889e-3f);
        g2 = fmaf(g2, u, -4.16666666666666667e-2f);
        *f2 = fmaf(g2, u, 0.5f);
        return;
    }
    const float x = 0.5f * sqrtf(u);
    float sx, cx;
    sincos_t(x, &sx, &cx);
    const float r = sx / x;
    *f1 = r * cx;
    *f2 = 0.5f * r * r;
}

template <bool HAS_V>
__device__ __forceinline__ void local_step_fast(float2& p1, float2& p0, float2& pm, const LocalCoef<float>& k,
                                                SitePot<float> vp) {
    const float h = 0.5f * k.dt;
    const float c1h = k.c1 * h, mc1h = -k.c1 * h, m2c1h = -2.0f * k.c1 * h, cch = (k.c0 + k.c1) * h;
    const float q1h = HAS_V ? (k.q + (vp.v1 - vp.v0)) * h : k.q * h;
    const float qmh = HAS_V ? (k.q + (vp.vm - vp.v0)) * h : k.q * h;
    // D(dt/2), relative to m = 0
    float n1 = abs2f(p1), n0 = abs2f(p0), nm = abs2f(pm);
    float g0 = fmaf(cch, (n1 + n0) + nm, mc1h * n0);
    if (HAS_V) g0 += vp.v0 * h;
    p1 = rot_minus(p1, fmaf(c1h, n0, fmaf(m2c1h, nm, q1h)));
    pm = rot_minus(pm, fmaf(c1h, n0, fmaf(m2c1h, n1, qmh)));
    // O(dt) with the predictor psi~ = psi - i eps S psi
    const float eps = k.c1 * k.dt, he = 0.5f * eps;
    const float2 a = cmulcf(pm, p0);   // psi_-1^* psi_0
    const float2 b = cmulcf(p0, p1);   // psi_0^* psi_1
    const float2 s1 = cmulf(a, p0);
    const float2 s0 = caddf(cmulcf(a, p1), cmulf(b, pm));
    const float2 sm = cmulcf(b, p0);
    const float2 t1 = make_float2(fmaf(eps, s1.y, p1.x), fmaf(-eps, s1.x, p1.y));
    const float2 t0 = make_float2(fmaf(eps, s0.y, p0.x), fmaf(-eps, s0.x, p0.y));
    const float2 tm = make_float2(fmaf(eps, sm.y, pm.x), fmaf(-eps, sm.x, pm.y));
    const float2 A2 = caddf(a, cmulcf(tm, t0));   // 2 A
    const float2 B2 = caddf(b, cmulcf(t0, t1));   // 2 B
    float f1, f2;
    o_coef((abs2f(A2) + abs2f(B2)) * (he * he), &f1, &f2);
    const float e1 = he * f1, e2 = (he * he) * f2;   // eps f1 and eps^2 f2 against 2A, 2B
    const float2 u1 = cmulf(A2, p0);
    const float2 u0 = caddf(cmulcf(A2, p1), cmulf(B2, pm));
    const float2 um = cmulcf(B2, p0);
    const float2 w1 = cmulf(A2, u0);
    const float2 w0 = caddf(cmulcf(A2, u1), cmulf(B2, um));
    const float2 wm = cmulcf(B2, u0);
    // psi + (-i e1 u - e2 w), the change formed first and added with one rounding.  Adding
    // -i e1 u and -e2 w to psi one after the other loses the second-order term wherever it
    // is below half an ulp of psi (psi_0 while the spin modes are still small): the
    // first-order transfer into psi_+-1 then goes uncompensated and |psi|^2 grows.
    p1 = make_float2(p1.x + fmaf(e1, u1.y, (-e2) * w1.x), p1.y - fmaf(e1, u1.x, e2 * w1.y));
    p0 = make_float2(p0.x + fmaf(e1, u0.y, (-e2) * w0.x), p0.y - fmaf(e1, u0.x, e2 * w0.y));
    pm = make_float2(pm.x + fmaf(e1, um.y, (-e2) * wm.x), pm.y - fmaf(e1, um.x, e2 * wm.y));
    // D(dt/2) with the deferred m = 0 phases of both halves
    n1 = abs2f(p1);
    n0 = abs2f(p0);
    nm = abs2f(pm);
    float gg = fmaf(cch, (n1 + n0) + nm, mc1h * n0);
    if (HAS_V) gg += vp.v0 * h;
    gg = g0 + gg;
    p1 = rot_minus(p1, gg + fmaf(c1h, n0, fmaf(m2c1h, nm, q1h)));
    pm = rot_minus(pm, gg + fmaf(c1h, n0, fmaf(m2c1h, n1, qmh)));
    p0 = rot_minus(p0, gg);
}

// ---- two sites at once (packed FP32: lane x is site A, lane y site B)

// Two complex numbers, one per lane.
struct cpair {
    float2 re, im;
};

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 abs2p(const cpair& z) { return fma2(z.re, z.re, mul2(z.im, z.im)); }
__device__ __forceinline__ cpair cmulp(const cpair& a, const cpair& b) {
    return {fma2(a.re, b.re, mul2(neg2(a.im), b.im)), fma2(a.re, b.im, mul2(a.im, b.re))};
}
__device__ __forceinline__ cpair cmulcp(const cpair& a, const cpair& b) {
    return {fma2(a.re, b.re, mul2(a.im, b.im)), fma2(a.re, b.im, mul2(neg2(a.im), b.re))};
}
__device__ __forceinline__ cpair caddp(const cpair& a, const cpair& b) { return {add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ cpair pack_pair(float2 a, float2 b) { return {make_float2(a.x, b.x), make_float2(a.y, b.y)}; }
__device__ __forceinline__ float2 lane_x(const cpair& z) { return make_float2(z.re.x, z.im.x); }
__device__ __forceinline__ float2 lane_y(const cpair& z) { return make_float2(z.re.y, z.im.y); }

// rot_minus on both lanes: the polynomials of sincosm1 when both |x| <= 1/2, otherwise
// sincosm1 lane by lane.
__device__ __forceinline__ cpair rot_minus_pair(const cpair& p, float2 x) {
    float2 s, cm1;
    if (fabsf(x.x) > 0.5f || fabsf(x.y) > 0.5f) {
        sincosm1(x.x, &s.x, &cm1.x);
        sincosm1(x.y, &s.y, &cm1.y);
    } else {
        const float2 x2 = mul2(x, x);
        float2 ps = fma2(x2, bc2(-1.98412698412698413e-4f), bc2(8.33333333333333333e-3f));
        ps = fma2(ps, x2, bc2(-1.66666666666666667e-1f));
        s = fma2(mul2(ps, x2), x, x);
        float2 pc = fma2(x2, bc2(2.48015873015873016e-5f), bc2(-1.38888888888888889e-3f));
        pc = fma2(pc, x2, bc2(4.16666666666666667e-2f));
        pc = fma2(pc, x2, bc2(-0.5f));
        cm1 = mul2(pc, x2);
    }
    return {add2(p.re, fma2(p.re, cm1, mul2(p.im, s))), add2(p.im, fma2(p.im, cm1, mul2(neg2(p.re), s)))};
}

// local_step_fast<false> for two sites: the same operations in the same order, each
// instruction covering both sites, so the per-lane results are those of the scalar step
// and the step costs about half the issue slots.
__device__ __forceinline__ void local_step_pair(cpair& p1, cpair& p0, cpair& pm, const LocalCoef<float>& k) {
    const float h = 0.5f * k.dt;
    const float2 C1H = bc2(k.c1 * h), mC1H = bc2(-k.c1 * h), m2C1H = bc2(-2.0f * k.c1 * h), QH = bc2(k.q * h),
                 CCH = bc2((k.c0 + k.c1) * h);
    float2 n1 = abs2p(p1), n0 = abs2p(p0), nm = abs2p(pm);
    const float2 g0 = fma2(CCH, add2(add2(n1, n0), nm), mul2(mC1H, n0));
    p1 = rot_minus_pair(p1, fma2(C1H, n0, fma2(m2C1H, nm, QH)));
    pm = rot_minus_pair(pm, fma2(C1H, n0, fma2(m2C1H, n1, QH)));
    const float eps = k.c1 * k.dt, he = 0.5f * eps;
    const float2 E = bc2(eps), mE = bc2(-eps);
    const cpair a = cmulcp(pm, p0);
    const cpair b = cmulcp(p0, p1);
    const cpair s1 = cmulp(a, p0);
    const cpair s0 = caddp(cmulcp(a, p1), cmulp(b, pm));
    const cpair sm = cmulcp(b, p0);
    const cpair t1 = {fma2(E, s1.im, p1.re), fma2(mE, s1.re, p1.im)};
    const cpair t0 = {fma2(E, s0.im, p0.re), fma2(mE, s0.re, p0.im)};
    const cpair tm = {fma2(E, sm.im, pm.re), fma2(mE, sm.re, pm.im)};
    const cpair A2 = caddp(a, cmulcp(tm, t0));
    const cpair B2 = caddp(b, cmulcp(t0, t1));
    const float2 u = mul2(add2(abs2p(A2), abs2p(B2)), bc2(he * he));
    float2 f1, f2;
    if (u.x <= 0.25f && u.y <= 0.25f) {
        f1 = fma2(u, bc2(-1.98412698412698413e-4f), bc2(8.33333333333333333e-3f));
        f1 = fma2(f1, u, bc2(-1.66666666666666667e-1f));
        f1 = fma2(f1, u, bc2(1.0f));
        f2 = fma2(u, bc2(-2.48015873015873016e-5f), bc2(1.38888888888888889e-3f));
        f2 = fma2(f2, u, bc2(-4.16666666666666667e-2f));
        f2 = fma2(f2, u, bc2(0.5f));
    } else {
        o_coef(u.x, &f1.x, &f2.x);
        o_coef(u.y, &f1.y, &f2.y);
    }
    const float2 e1 = mul2(bc2(he), f1), e2 = mul2(bc2(he * he), f2);
    const cpair u1 = cmulp(A2, p0);
    const cpair u0 = caddp(cmulcp(A2, p1), cmulp(B2, pm));
    const cpair um = cmulcp(B2, p0);
    const cpair w1 = cmulp(A2, u0);
    const cpair w0 = caddp(cmulcp(A2, u1), cmulp(B2, um));
    const cpair wm = cmulcp(B2, u0);
    p1 = {add2(p1.re, fma2(e1, u1.im, mul2(neg2(e2), w1.re))), sub2(p1.im, fma2(e1, u1.re, mul2(e2, w1.im)))};
    p0 = {add2(p0.re, fma2(e1, u0.im, mul2(neg2(e2), w0.re))), sub2(p0.im, fma2(e1, u0.re, mul2(e2, w0.im)))};
    pm = {add2(pm.re, fma2(e1, um.im, mul2(neg2(e2), wm.re))), sub2(pm.im, fma2(e1, um.re, mul2(e2, wm.im)))};
    n1 = abs2p(p1);
    n0 = abs2p(p0);
    nm = abs2p(pm);
    const float2 gg = add2(g0, fma2(CCH, add2(add2(n1, n0), nm), mul2(mC1H, n0)));
    p1 = rot_minus_pair(p1, add2(gg, fma2(C1H, n0, fma2(m2C1H, nm, QH))));
    pm = rot_minus_pair(pm, add2(gg, fma2(C1H, n0, fma2(m2C1H, n1, QH))));
    p0 = rot_minus_pair(p0, gg);
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

// The local step (no potential) over the sites i0, i0 + stride, ... below n of three
// component arrays (site i of component c at bc[idx(i)]): the FP32 paper scheme two sites
// at a time in packed instructions, any site left over (and every other case) one at a
// time.
template <typename T, typename V, typename IDX>
__device__ __forceinline__ void local_step_sites(V* b0, V* b1, V* b2, int i0, int n, int stride,
                                                 const LocalCoef<T>& k, IDX idx) {
    int i = i0;
    if constexpr (sizeof(T) == 4) {
        if (k.kind == 0) {
#pragma unroll 1
            for (; i + stride < n; i += 2 * stride) {
                const int ka = idx(i), kb = idx(i + stride);
                cpair p1 = pack_pair(b0[ka], b0[kb]), p0 = pack_pair(b1[ka], b1[kb]), pm = pack_pair(b2[ka], b2[kb]);
                local_step_pair(p1, p0, pm, k);
                b0[ka] = lane_x(p1);
                b0[kb] = lane_y(p1);
                b1[ka] = lane_x(p0);
                b1[kb] = lane_y(p0);
                b2[ka] = lane_x(pm);
                b2[kb] = lane_y(pm);
            }
        }
    }
#pragma unroll 2
    for (; i < n; i += stride) {
        const int kk = idx(i);
        V p1 = b0[kk], p0 = b1[kk], pm = b2[kk];
        local_step<T>(p1, p0, pm, k);
        b0[kk] = p1;
        b1[kk] = p0;
        b2[kk] = pm;
    }
}

// Potential of site i from a [3][sites] array (comp_stride = sites), or zero.
template <typename T>
__device__ __forceinline__ SitePot<T> site_pot(const T* __restrict__ vpot, int64_t comp_stride, int64_t i) {
    return SitePot<T>{__ldg(vpot + i), __ldg(vpot + comp_stride + i), __ldg(vpot + 2 * comp_stride + i)};
}

}  // namespace gpe
