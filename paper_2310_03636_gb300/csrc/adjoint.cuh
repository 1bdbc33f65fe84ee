// Hand-written reverse-mode (vector-Jacobian) of the local step L = D(dt/2) O(dt) D(dt/2).
//
// Convention: for a real loss, the gradient of a complex variable z is
// g_z = dL/dRe z + i dL/dIm z (the convention of torch autograd).  For z' = F(z) with
// dz' = A dz + B dz*, the pullback is g_z = A^H g_z' + B^T conj(g_z').  Rules used:
//   z = x y        : g_x += conj(y) g_z,  g_y += conj(x) g_z
//   z = conj(x) y  : g_x += y conj(g_z),  g_y += x g_z
//   r = |z|^2 real : g_z += 2 g_r z
//   z = c(s) x, c real function of s: g_x += c g_z, g_s += Re(conj(x) g_z) dc/ds
// The forward intermediates are recomputed from the step's input state.
#pragma once

#include "common.cuh"
#include "local_step.cuh"

namespace gpe {

// acc += conj(x) * y  (complex)
template <typename V> __device__ __forceinline__ void acc_cmulc(V& acc, V x, V y) { acc = cadd(acc, cmulc(x, y)); }
template <typename V> __device__ __forceinline__ void acc_cmul(V& acc, V x, V y) { acc = cadd(acc, cmul(x, y)); }
// x * conj(y)
template <typename V> __device__ __forceinline__ V cmul_cy(V x, V y) { return mk(x.x * y.x + x.y * y.y, x.y * y.x - x.x * y.y); }
// Re(conj(x) y)
template <typename V> __device__ __forceinline__ auto re_cxy(V x, V y) { return x.x * y.x + x.y * y.y; }
// Im(conj(x) y)
template <typename V> __device__ __forceinline__ auto im_cxy(V x, V y) { return x.x * y.y - x.y * y.x; }

// Diagonal step D(tau) forward: p <- p e^{-i theta(p)}; returns the phases.  The
// potential vp adds a field-independent part to theta.
template <typename T, typename V>
__device__ __forceinline__ void diag_fwd(V (&p)[3], T (&th)[3], T c0, T c1, T q, T tau, SitePot<T> vp) {
    const T n1 = cabs2(p[0]), n0 = cabs2(p[1]), nm = cabs2(p[2]);
    const T g = (c0 + c1) * (n1 + n0 + nm);
    th[0] = (vp.v1 + q + g - (T)2 * c1 * nm) * tau;
    th[1] = (vp.v0 + g - c1 * n0) * tau;
    th[2] = (vp.vm + q + g - (T)2 * c1 * n1) * tau;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        T s, c;
        sincos_t(th[m], &s, &c);
        p[m] = mk(p[m].x * c + p[m].y * s, p[m].y * c - p[m].x * s);
    }
}

// Pullback of D(tau) at input p (before the phase) with output p' = p e^{-i theta}.
// g: in = gradient w.r.t. p', out = gradient w.r.t. p.  Returns dL/dq contribution.
template <typename T, typename V>
__device__ __forceinline__ T diag_bwd(const V (&p)[3], V (&g)[3], T c0, T c1, T q, T tau, SitePot<T> vp) {
    const T n1 = cabs2(p[0]), n0 = cabs2(p[1]), nm = cabs2(p[2]);
    const T G = c0 + c1;
    const T g0 = G * (n1 + n0 + nm);
    const T th[3] = {(vp.v1 + q + g0 - (T)2 * c1 * nm) * tau, (vp.v0 + g0 - c1 * n0) * tau,
                     (vp.vm + q + g0 - (T)2 * c1 * n1) * tau};
    T w[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        T s, c;
        sincos_t(th[m], &s, &c);
        const V po = mk(p[m].x * c + p[m].y * s, p[m].y * c - p[m].x * s);   // p'
        w[m] = im_cxy(g[m], po);                                            // Im(conj(g') p')
        g[m] = mk(g[m].x * c - g[m].y * s, g[m].y * c + g[m].x * s);        // g' e^{+i theta}
    }
    // s_k = tau sum_m w_m d f_m / d n_k
    const T sw = w[0] + w[1] + w[2];
    const T s1 = tau * (G * sw - (T)2 * c1 * w[2]);
    const T s0 = tau * (G * sw - c1 * w[1]);
    const T sm = tau * (G * sw - (T)2 * c1 * w[0]);
    g[0] = cadd(g[0], cscale(p[0], (T)2 * s1));
    g[1] = cadd(g[1], cscale(p[1], (T)2 * s0));
    g[2] = cadd(g[2], cscale(p[2], (T)2 * sm));
    return tau * (w[0] + w[2]);
}

// f1(u) = sin(th)/th, f2(u) = (1 - cos th)/th^2 with u = th^2, and their u-derivatives.
template <typename T>
__device__ __forceinline__ void sinc_coeffs(T u, T& f1, T& f2, T& d1, T& d2) {
    if (u <= (T)0.0625) {
        // series: f1 = sum (-u)^k/(2k+1)!, f2 = sum (-u)^k/(2k+2)!, k <= 6
        const T c1[7] = {(T)1, (T)(-1.0 / 6), (T)(1.0 / 120), (T)(-1.0 / 5040), (T)(1.0 / 362880),
                         (T)(-1.0 / 39916800), (T)(1.0 / 6227020800.0)};
        const T c2[7] = {(T)0.5, (T)(-1.0 / 24), (T)(1.0 / 720), (T)(-1.0 / 40320), (T)(1.0 / 3628800),
                         (T)(-1.0 / 479001600), (T)(1.0 / 87178291200.0)};
        f1 = c1[6];
        f2 = c2[6];
        d1 = (T)6 * c1[6];
        d2 = (T)6 * c2[6];
#pragma unroll
        for (int k = 5; k >= 0; --k) {
            f1 = f1 * u + c1[k];
            f2 = f2 * u + c2[k];
            if (k >= 1) {
                d1 = d1 * u + (T)k * c1[k];
                d2 = d2 * u + (T)k * c2[k];
            }
        }
    } else {
        const T th = sqrt_t(u);
        T s, c;
        sincos_t(th, &s, &c);
        f1 = s / th;
        f2 = ((T)1 - c) / u;
        d1 = (c - f1) / ((T)2 * u);
        d2 = ((T)0.5 * f1 - f2) / u;
    }
}

// Pullback of O(dt) (predictor-averaged spin-mixing matrix) at input r.
// g: in = gradient w.r.t. O(r), out = gradient w.r.t. r.
template <typename T, typename V>
__device__ __forceinline__ void offdiag_bwd(const V (&r)[3], V (&g)[3], T c1, T dt) {
    const T eps = c1 * dt;
    const V zero = mk((T)0, (T)0);
    // forward recomputation
    const V al = cmulc(r[2], r[1]);   // conj(r-1) r0
    const V be = cmulc(r[1], r[0]);   // conj(r0) r1
    const V s1 = cmul(al, r[1]);
    const V s0 = cadd(cmulc(al, r[0]), cmul(be, r[2]));
    const V sm = cmulc(be, r[1]);
    const V t1 = mk(r[0].x + eps * s1.y, r[0].y - eps * s1.x);   // r - i eps s
    const V t0 = mk(r[1].x + eps * s0.y, r[1].y - eps * s0.x);
    const V tm = mk(r[2].x + eps * sm.y, r[2].y - eps * sm.x);
    const V alt = cmulc(tm, t0);
    const V bet = cmulc(t0, t1);
    const V A = cscale(cadd(al, alt), (T)0.5);
    const V B = cscale(cadd(be, bet), (T)0.5);
    const T u = eps * eps * (cabs2(A) + cabs2(B));
    T f1, f2, d1, d2;
    sinc_coeffs<T>(u, f1, f2, d1, d2);
    const T e1 = eps * f1, e2 = eps * eps * f2;
    const V v1 = cmul(A, r[1]);
    const V v0 = cadd(cmulc(A, r[0]), cmul(B, r[2]));
    const V vm = cmulc(B, r[1]);
    const V w1 = cmul(A, v0);
    const V w0 = cadd(cmulc(A, v1), cmul(B, vm));
    const V wm = cmulc(B, v0);
    // backward: o = r - i e1 v - e2 w
    const V go1 = g[0], go0 = g[1], gom = g[2];
    V gr1 = go1, gr0 = go0, grm = gom;
    const V gv1 = cscale(mk(-go1.y, go1.x), e1);   // i e1 g
    const V gv0_a = cscale(mk(-go0.y, go0.x), e1);
    const V gvm_a = cscale(mk(-gom.y, gom.x), e1);
    // g_e1 = sum Re(conj(-i v) g) = sum Im(conj(v) g)... Re(i conj(v) g) = -Im(conj(v) g)
    const T ge1 = -(im_cxy(v1, go1) + im_cxy(v0, go0) + im_cxy(vm, gom));
    const T ge2 = -(re_cxy(w1, go1) + re_cxy(w0, go0) + re_cxy(wm, gom));
    const V gw1 = cscale(go1, -e2), gw0 = cscale(go0, -e2), gwm = cscale(gom, -e2);
    V gA = zero, gB = zero;
    V gv1t = gv1, gv0 = gv0_a, gvm = gvm_a;
    // w1 = A v0
    acc_cmulc(gA, v0, gw1);
    acc_cmulc(gv0, A, gw1);
    // w0 = conj(A) v1 + B vm
    acc_cmul(gv1t, A, gw0);
    gA = cadd(gA, cmul_cy(v1, gw0));
    acc_cmulc(gB, vm, gw0);
    acc_cmulc(gvm, B, gw0);
    // wm = conj(B) v0
    acc_cmul(gv0, B, gwm);
    gB = cadd(gB, cmul_cy(v0, gwm));
    // v1 = A r0 ; v0 = conj(A) r1 + B rm ; vm = conj(B) r0
    acc_cmulc(gA, r[1], gv1t);
    acc_cmulc(gr0, A, gv1t);
    acc_cmul(gr1, A, gv0);
    gA = cadd(gA, cmul_cy(r[0], gv0));
    acc_cmulc(gB, r[2], gv0);
    acc_cmulc(grm, B, gv0);
    acc_cmul(gr0, B, gvm);
    gB = cadd(gB, cmul_cy(r[1], gvm));
    // e1 = eps f1(u), e2 = eps^2 f2(u), u = eps^2 (|A|^2 + |B|^2)
    const T gu = ge1 * eps * d1 + ge2 * eps * eps * d2;
    gA = cadd(gA, cscale(A, (T)2 * gu * eps * eps));
    gB = cadd(gB, cscale(B, (T)2 * gu * eps * eps));
    // A = (al + alt)/2, B = (be + bet)/2
    const V gal_h = cscale(gA, (T)0.5), gbe_h = cscale(gB, (T)0.5);
    V gal = gal_h, gbe = gbe_h;
    // alt = conj(tm) t0 ; bet = conj(t0) t1
    V gt1 = zero, gt0 = zero, gtm = zero;
    acc_cmul(gt0, tm, gal_h);
    gtm = cadd(gtm, cmul_cy(t0, gal_h));
    acc_cmul(gt1, t0, gbe_h);
    gt0 = cadd(gt0, cmul_cy(t1, gbe_h));
    // t = r - i eps s
    gr1 = cadd(gr1, gt1);
    gr0 = cadd(gr0, gt0);
    grm = cadd(grm, gtm);
    const V gs1 = cscale(mk(-gt1.y, gt1.x), eps);
    const V gs0 = cscale(mk(-gt0.y, gt0.x), eps);
    const V gsm = cscale(mk(-gtm.y, gtm.x), eps);
    // s1 = al r0 ; s0 = conj(al) r1 + be rm ; sm = conj(be) r0
    acc_cmulc(gal, r[1], gs1);
    acc_cmulc(gr0, al, gs1);
    acc_cmul(gr1, al, gs0);
    gal = cadd(gal, cmul_cy(r[0], gs0));
    acc_cmulc(gbe, r[2], gs0);
    acc_cmulc(grm, be, gs0);
    acc_cmul(gr0, be, gsm);
    gbe = cadd(gbe, cmul_cy(r[1], gsm));
    // al = conj(rm) r0 ; be = conj(r0) r1
    acc_cmul(gr0, r[2], gal);
    grm = cadd(grm, cmul_cy(r[1], gal));
    acc_cmul(gr1, r[1], gbe);
    gr0 = cadd(gr0, cmul_cy(r[0], gbe));
    g[0] = gr1;
    g[1] = gr0;
    g[2] = grm;
}

// Forward O(dt) (same formula as the pullback's recomputation), used to rebuild the
// input of the second D.
template <typename T, typename V>
__device__ __forceinline__ void offdiag_fwd(V (&r)[3], T c1, T dt) {
    const T eps = c1 * dt;
    const V al = cmulc(r[2], r[1]);
    const V be = cmulc(r[1], r[0]);
    const V s1 = cmul(al, r[1]);
    const V s0 = cadd(cmulc(al, r[0]), cmul(be, r[2]));
    const V sm = cmulc(be, r[1]);
    const V t1 = mk(r[0].x + eps * s1.y, r[0].y - eps * s1.x);
    const V t0 = mk(r[1].x + eps * s0.y, r[1].y - eps * s0.x);
    const V tm = mk(r[2].x + eps * sm.y, r[2].y - eps * sm.x);
    const V A = cscale(cadd(al, cmulc(tm, t0)), (T)0.5);
    const V B = cscale(cadd(be, cmulc(t0, t1)), (T)0.5);
    const T u = eps * eps * (cabs2(A) + cabs2(B));
    T f1, f2, d1, d2;
    sinc_coeffs<T>(u, f1, f2, d1, d2);
    const T e1 = eps * f1, e2 = eps * eps * f2;
    const V v1 = cmul(A, r[1]);
    const V v0 = cadd(cmulc(A, r[0]), cmul(B, r[2]));
    const V vm = cmulc(B, r[1]);
    const V w1 = cmul(A, v0);
    const V w0 = cadd(cmulc(A, v1), cmul(B, vm));
    const V wm = cmulc(B, v0);
    r[0] = mk(r[0].x + (e1 * v1.y - e2 * w1.x), r[0].y - (e1 * v1.x + e2 * w1.y));
    r[1] = mk(r[1].x + (e1 * v0.y - e2 * w0.x), r[1].y - (e1 * v0.x + e2 * w0.y));
    r[2] = mk(r[2].x + (e1 * vm.y - e2 * wm.x), r[2].y - (e1 * vm.x + e2 * wm.y));
}

// Pullback of the whole local step at input p (= the state after the leading half
// kinetic step).  g: in = gradient w.r.t. L(p), out = gradient w.r.t. p.  Returns dL/dq.
template <typename T, typename V>
__device__ __forceinline__ T local_step_bwd(const V (&p)[3], V (&g)[3], T c0, T c1, T q, T dt, SitePot<T> vp) {
    const T h = (T)0.5 * dt;
    V r[3] = {p[0], p[1], p[2]};
    T th[3];
    diag_fwd<T>(r, th, c0, c1, q, h, vp);   // r = D(h) p
    V o[3] = {r[0], r[1], r[2]};
    offdiag_fwd<T>(o, c1, dt);              // o = O r
    T dq = diag_bwd<T>(o, g, c0, c1, q, h, vp);
    offdiag_bwd<T>(r, g, c1, dt);
    dq += diag_bwd<T>(p, g, c0, c1, q, h, vp);
    return dq;
}

}  // namespace gpe
