// Device-side Kalman step for one track candidate per CUDA lane (sm_103a).
//
// Propagation to a barrel cylinder or endcap disk in a uniform solenoid field with its
// 6x6 Jacobian, covariance transport J C J^T, multiple scattering and mean energy loss
// (a4-a7), the eta-phi window (a8), the 3D chi2 (a9) and the Joseph-form gain/update
// (a11); the step from a layer's surface to the plane of a flat (or tilted) module
// (Sec. 3.1 module position and normal) for the hits measured on modules.  The paper (Sec. 3.1) names propagation, hit selection and the Kalman filter
// calculations as the per-layer work; the formulas are the textbook ones it cites.
//
// Every function is a template on the scalar type F: float is the bulk path, double the
// seed fit (whose diffuse prior makes it ill-conditioned) and the plain all-FP64 path.
//
// FP32 precision measures:
//  - the track position is an unevaluated sum hi + lo of two floats: positions reach
//    |z| = 275 cm where one FP32 ulp is 15 nm, comparable to the 1e-3 chi2 tolerance on
//    30 um hits; the crossing equation is written relative to the current position, the
//    crossing point is polished onto the cylinder with an exactly evaluated gap, and the
//    helix step uses the chord form with an unrounded mid-angle;
//  - the predicted covariance is kept in surface coordinates (exactly zero along the
//    surface normal) and the chi2 and the update run in the local measurement frame.
#pragma once

#include <cuda_runtime.h>

#include "dual.cuh"
#include "trig.cuh"
#include <math.h>
#include <stdint.h>

#include "mkgb.h"

namespace mk {

constexpr float kCLight = 0.00299792458f;   // curvature [1/cm] per (T / GeV)
constexpr float kPi = 3.14159265358979f;
constexpr float kTwoPi = 6.28318530717959f;

// Physical constants in the scalar type of F (dual numbers take the constants of their value type).
template <class F> struct Phys {
    using S = typename ScalarOf<F>::type;
    static constexpr S mpi = S(0.13957039);       // pion mass, GeV
    static constexpr S me = S(0.51099895e-3);     // electron mass, GeV
    static constexpr S K = S(0.307075);           // MeV cm^2/mol
    static constexpr S ZA = S(0.49848);           // silicon Z/A
    static constexpr S rho = S(2.329);            // g/cm^3
    static constexpr S X0 = S(9.37);              // cm
    static constexpr S I = S(173.0e-9);           // GeV
    static constexpr S inc_cap = S(10.0);
    static constexpr S pi = S(3.14159265358979323846);
    static constexpr S two_pi = S(6.28318530717959647692);
    static constexpr S two_pi_lo = S(6.28318530717959647692 - double(S(6.28318530717959647692)));   // 2 pi - two_pi
};

struct DevLayer {
    int kind;
    float pos, lo, hi, xx0;
    float sig[3];
    int n_eta, n_phi;
    float eta_lo, eta_scale;   // bin = floor((eta - eta_lo) * eta_scale)
    int bin_base;              // first bin of this layer inside an event's bin block
    int modular;               // 1: the layer is built from flat modules (its hits lie on module planes)
};

// 16-byte aligned so that kernels copy it into shared memory as whole int4 words.
struct alignas(16) DevGeom {
    int n_layers, n_regions, bins_per_event, max_plan;
    float bz, cB, barrel_eta_max, pad;
    DevLayer layers[MKGB_MAX_LAYERS];
    int plan_off[MKGB_MAX_REGIONS + 1];
    int plan[MKGB_MAX_REGIONS * MKGB_MAX_PLAN];
    // module planes (Sec. 3.1): per module (cx, cy, cz, layer) and (nx, ny, nz, 0); nullptr: none
    const float4* mods;
    int n_mods;
};
static_assert(sizeof(DevGeom) % 16 == 0, "DevGeom is copied as int4 words");

struct DevParams {
    float chi2_cut;
    int max_cands, max_holes, material;
    float nsig, deta_min, deta_max, dphi_min, dphi_max;
    float score_hit, score_hole, barrel_eta_max;
    int precision;      // MKGB_FP32: FP32 Kalman steps (mixed-precision seed fit); MKGB_FP64: every step in FP64
    float kappa_fp64;   // fit: tracks with an update whose S condition estimate exceeds this are refit in FP64
    float fit_outlier_chi2;   // fits: a listed hit with a predicted chi2 above this is not used (0: off)
    float score_overlap;      // search: score of a picked-up overlap hit (Sec. 2.2)
};

// Packed lower-triangle index of a symmetric matrix (i, j >= 0).
__host__ __device__ constexpr int ix(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

template <class F> struct StateT {
    F xh, yh, zh;   // position, high part
    F xl, yl, zl;   // position, low part (|lo| <= ulp(hi)/2)
    F k, phi, th;   // q/pT, direction phi, polar angle
    // theta's and phi's low parts (theta = th + tl, phi = phi + pl): an FP32 angle near pi has
    // an ulp of 2.4e-7 rad, which moves a steep track's z by s / sin^2(theta) x 1.2e-7 (~1 um
    // over 10 cm at eta 2.7) and every predicted transverse position by s x 1.2e-7, enough to
    // shift the fitted curvature of a 40 GeV track by 1e-4
    F tl = F(0), pl = F(0);
    F c[21];        // covariance of (x, y, z, k, phi, theta), packed
};

// Predicted state at a layer surface; covariance of (u1, u2, k, phi, theta) where (u1, u2)
// are coordinates along the surface frame axes e1, e2 (see frame_of).
template <class F> struct PredT {
    F xh, yh, zh, xl, yl, zl, k, phi, th;
    F tl = F(0), pl = F(0);   // theta's and phi's low parts, as StateT
    F c[15];
};

using State = StateT<float>;
using Pred = PredT<float>;

// ----------------------------------------------------------------- scalar helpers

__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
// FP32: reduction by pi/2 and Taylor series (trig.cuh), no large-argument path
__device__ __forceinline__ void sin_cos(float x, float* s, float* c) { sin_cos_cw(x, s, c); }
__device__ __forceinline__ void sin_cos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
// Correctly rounded division where it sets the trajectory (path length, chord, dz/ds): kernels
// built with approximate FP32 division keep these at 0.5 ulp.
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return a / b; }
// Logarithm inside the material terms (Highland's log correction, Bethe-Bloch's log term): an
// absolute error of ~1e-6 there moves theta0 and dE/dx by ~1e-7 relative, so FP32 takes the
// hardware logarithm (__logf, at most 3 ulp off outside [0.5, 2]).
__device__ __forceinline__ float log_mat(float x) { return __logf(x); }
__device__ __forceinline__ double log_mat(double x) { return log(x); }

// The same helpers on dual numbers (derivative of the fit): values through the scalar helper,
// derivatives by the chain rule.
template <class T, int K> __device__ __forceinline__ Dual<T, K> add_rn(const Dual<T, K>& a, const Dual<T, K>& b) {
    Dual<T, K> r = a + b;
    r.v = add_rn(a.v, b.v);
    return r;
}
template <class T, int K> __device__ __forceinline__ Dual<T, K> sub_rn(const Dual<T, K>& a, const Dual<T, K>& b) {
    Dual<T, K> r = a - b;
    r.v = sub_rn(a.v, b.v);
    return r;
}
template <class T, int K> __device__ __forceinline__ Dual<T, K> mul_rn(const Dual<T, K>& a, const Dual<T, K>& b) {
    Dual<T, K> r = a * b;
    r.v = mul_rn(a.v, b.v);
    return r;
}
template <class T, int K>
__device__ __forceinline__ Dual<T, K> fma_rn(const Dual<T, K>& a, const Dual<T, K>& b, const Dual<T, K>& c) {
    Dual<T, K> r = fma(a, b, c);
    r.v = fma_rn(a.v, b.v, c.v);
    return r;
}
template <class T, int K> __device__ __forceinline__ void sin_cos(const Dual<T, K>& x, Dual<T, K>* s, Dual<T, K>* c) {
    T sv, cv;
    sin_cos(x.v, &sv, &cv);
    *s = x.chain(sv, cv);
    *c = x.chain(cv, -sv);
}
template <class T, int K> __device__ __forceinline__ Dual<T, K> div_rn(const Dual<T, K>& a, const Dual<T, K>& b) {
    Dual<T, K> r = a / b;
    r.v = div_rn(a.v, b.v);
    return r;
}
template <class T, int K> __device__ __forceinline__ Dual<T, K> rsq(const Dual<T, K>& x) {
    const T r = rsq(x.v);
    return x.chain(r, T(-0.5) * r * r * r);
}
template <class T, int K> __device__ __forceinline__ Dual<T, K> log_mat(const Dual<T, K>& x) {
    return x.chain(log_mat(x.v), T(1) / x.v);
}

// FP32 arithmetic (float, or dual numbers over float): looser iteration tolerances
template <class F> __host__ __device__ constexpr bool is_fp32() { return sizeof(typename ScalarOf<F>::type) == 4; }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

template <class F> __device__ __forceinline__ void two_sum(F a, F b, F& s, F& e) {
    s = add_rn(a, b);
    const F bb = sub_rn(s, a);
    e = add_rn(sub_rn(a, sub_rn(s, bb)), sub_rn(b, bb));
}

// (hi, lo) += d, renormalised.
template <class F> __device__ __forceinline__ void add_ff(F& hi, F& lo, F d) {
    F s, e;
    two_sum(hi, d, s, e);
    e = add_rn(e, lo);
    hi = add_rn(s, e);
    lo = sub_rn(e, sub_rn(hi, s));
}

// R^2 - (x^2 + y^2) for x = xh + xl, y = yh + yl, with the squares split exactly by FMA.
template <class F> __device__ __forceinline__ F r2_gap(F R, F xh, F xl, F yh, F yl) {
    const F pR = mul_rn(R, R), eR = fma_rn(R, R, -pR);
    const F p1 = mul_rn(xh, xh), e1 = fma_rn(xh, xh, -p1);
    const F p2 = mul_rn(yh, yh), e2 = fma_rn(yh, yh, -p2);
    F s1, t1, s2, t2;
    two_sum(pR, -p1, s1, t1);
    two_sum(s1, -p2, s2, t2);
    F tail = add_rn(add_rn(t1, t2), sub_rn(sub_rn(eR, e1), e2));
    tail = sub_rn(tail, F(2) * (xh * xl + yh * yl));
    return add_rn(s2, tail);
}

// phi = hi + lo (float-float) into (-pi, pi]: whole turns of 2 pi taken off as the two-word
// constant two_pi + two_pi_lo, so that the wrap adds no rounding of 2 pi to phi.
template <class F> __device__ __forceinline__ void wrap_pi_ff(F& hi, F& lo) {
    const F n = rint(hi * (F(1) / Phys<F>::two_pi));
    if (n != F(0)) {
        add_ff(hi, lo, -n * Phys<F>::two_pi);
        add_ff(hi, lo, -n * Phys<F>::two_pi_lo);
    }
    if (hi <= -Phys<F>::pi) {
        add_ff(hi, lo, F(Phys<F>::two_pi));
        add_ff(hi, lo, F(Phys<F>::two_pi_lo));
    }
    if (hi > Phys<F>::pi) {
        add_ff(hi, lo, F(-Phys<F>::two_pi));
        add_ff(hi, lo, F(-Phys<F>::two_pi_lo));
    }
}

template <class F> __device__ __forceinline__ F wrap_pi(F a) {
    // into (-pi, pi]
    a = a - Phys<F>::two_pi * rint(a * (F(1) / Phys<F>::two_pi));
    if (a <= -Phys<F>::pi) a += Phys<F>::two_pi;
    if (a > Phys<F>::pi) a -= Phys<F>::two_pi;
    return a;
}

// sin(a)/a and (1 - cos a)/a.
template <class F> __device__ __forceinline__ void s1c1(F a, F& S1, F& C1) {
    if (fabs(a) < F(1e-4)) {
        S1 = F(1) - a * a * (F(1) / F(6));
        C1 = a * (F(0.5) - a * a * (F(1) / F(24)));
    } else {
        F sh, ch;
        sin_cos(F(0.5) * a, &sh, &ch);
        const F inv = F(1) / a;
        S1 = F(2) * sh * ch * inv;
        C1 = F(2) * sh * sh * inv;
    }
}

// Derivatives of S1 and C1 with respect to a (power series for small |a|).
template <class F> __device__ __forceinline__ void s1c1_deriv(F a, F S1, F C1, F& dS1, F& dC1) {
    const F lim = is_fp32<F>() ? F(0.3) : F(0.05);
    if (fabs(a) < lim) {
        const F a2 = a * a;
        dS1 = a * (F(-1) / F(3) + a2 * (F(1) / F(30) + a2 * (F(-1) / F(840) + a2 * (F(1) / F(45360) - a2 * (F(1) / F(3991680))))));
        dC1 = F(0.5) + a2 * (F(-1) / F(8) + a2 * (F(1) / F(144) + a2 * (F(-1) / F(5760) + a2 * (F(1) / F(403200)))));
    } else {
        const F inv = F(1) / a;
        const F sa = S1 * a, ca = F(1) - C1 * a;   // sin(a), cos(a)
        dS1 = (ca - S1) * inv;
        dC1 = (sa - C1) * inv;
    }
}

// ----------------------------------------------------------------- surface frame
//
// Orthonormal frame of a predicted state on its surface: n the surface normal, e1 the
// direction of the track projected onto the surface, e2 = n x e1 (in the surface).  Aligning
// e1 with the track keeps the large along-track spread of a grazing crossing in the u1
// variance alone: the u2 row of the Jacobian has no path-length term, so no covariance entry
// is a difference of large FP32 numbers.  Barrel n = (x, y, 0)/r, disk n = z-hat.

template <class F> struct FrameT {
    F n[3], e1[3], e2[3];
};

template <class F> __device__ __forceinline__ FrameT<F> frame_of(int kind, F x, F y, F sphi, F cphi, F st, F ct) {
    FrameT<F> f;
    if (kind == MKGB_DISK) {
        f.n[0] = F(0); f.n[1] = F(0); f.n[2] = F(1);
        f.e1[0] = cphi; f.e1[1] = sphi; f.e1[2] = F(0);
        f.e2[0] = -sphi; f.e2[1] = cphi; f.e2[2] = F(0);
    } else {
        const F ir = rsq(x * x + y * y);
        const F c = x * ir, s = y * ir;
        // projection of the direction onto (t-hat = (-s, c, 0), z-hat)
        F a = st * (c * sphi - s * cphi), b = ct;
        const F nrm2 = a * a + b * b;
        if (nrm2 > F(1e-12)) {
            const F inv = rsq(nrm2);
            a *= inv;
            b *= inv;
        } else {
            a = F(1);
            b = F(0);
        }
        f.n[0] = c; f.n[1] = s; f.n[2] = F(0);
        f.e1[0] = -a * s; f.e1[1] = a * c; f.e1[2] = b;
        f.e2[0] = b * s; f.e2[1] = -b * c; f.e2[2] = a;
    }
    return f;
}

template <class F> __device__ __forceinline__ FrameT<F> frame_of(int kind, const PredT<F>& q) {
    F sp, cp, st, ct;
    sin_cos(q.phi, &sp, &cp);
    sin_cos(q.th, &st, &ct);
    return frame_of(kind, q.xh, q.yh, sp, cp, st, ct);
}

template <class F> __device__ __forceinline__ F dot3(const F a[3], const F b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// global 3-vector -> local (n, e1, e2) components
template <class F> __device__ __forceinline__ void to_local3(const FrameT<F>& f, const F g[3], F l[3]) {
    l[0] = dot3(f.n, g);
    l[1] = dot3(f.e1, g);
    l[2] = dot3(f.e2, g);
}

// surface displacement (d1 along e1, d2 along e2) -> global
template <class F> __device__ __forceinline__ void surface_to_global(const FrameT<F>& f, F d1, F d2, F g[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) g[i] = d1 * f.e1[i] + d2 * f.e2[i];
}

// packed 3x3 symmetric (xx, yx, yy, zx, zy, zz) global -> local frame (n, e1, e2)
template <class F> __device__ __forceinline__ void to_local_sym3(const FrameT<F>& f, const F v[6], F w[6]) {
    const F M[3][3] = {{v[0], v[1], v[3]}, {v[1], v[2], v[4]}, {v[3], v[4], v[5]}};
    const F* R[3] = {f.n, f.e1, f.e2};
    F MR[3][3];   // M R[b]
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int i = 0; i < 3; ++i) MR[b][i] = M[i][0] * R[b][0] + M[i][1] * R[b][1] + M[i][2] * R[b][2];
#pragma unroll
    for (int a2 = 0; a2 < 3; ++a2)
#pragma unroll
        for (int b = 0; b <= a2; ++b) w[ix(a2, b)] = dot3(R[a2], MR[b]);
}

// Surface-frame covariance (15) -> global state covariance (21).
template <class F> __device__ __forceinline__ void embed_cov(const FrameT<F>& f, const F q[15], F c[21]) {
    const F cuu[2][2] = {{q[0], q[1]}, {q[1], q[2]}};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const F m0 = f.e1[i] * cuu[0][0] + f.e2[i] * cuu[1][0];
        const F m1 = f.e1[i] * cuu[0][1] + f.e2[i] * cuu[1][1];
#pragma unroll
        for (int j = 0; j <= i; ++j) c[ix(i, j)] = m0 * f.e1[j] + m1 * f.e2[j];
#pragma unroll
        for (int o = 0; o < 3; ++o) c[ix(3 + o, i)] = f.e1[i] * q[ix(2 + o, 0)] + f.e2[i] * q[ix(2 + o, 1)];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) c[ix(3 + a, 3 + b)] = q[ix(2 + a, 2 + b)];
}

// Global-frame state on a surface -> predicted state in the surface frame f (the inverse of
// embed_cov): positions and angles copied, the covariance projected onto (u1, u2) along e1, e2;
// any variance along the surface normal (zero for a state on the surface) is dropped.
template <class F> __device__ __forceinline__ void state_to_pred(const FrameT<F>& f, const StateT<F>& t, PredT<F>& q) {
    q.xh = t.xh; q.yh = t.yh; q.zh = t.zh; q.xl = t.xl; q.yl = t.yl; q.zl = t.zl;
    q.k = t.k; q.phi = t.phi; q.pl = t.pl; q.th = t.th; q.tl = t.tl;
    const F* e[2] = {f.e1, f.e2};
    F Ce[2][3];   // C_pos e_a
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i)
            Ce[a][i] = t.c[ix(i, 0)] * e[a][0] + t.c[ix(i, 1)] * e[a][1] + t.c[ix(i, 2)] * e[a][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) q.c[ix(a, b)] = dot3(e[a], Ce[b]);
#pragma unroll
    for (int o = 0; o < 3; ++o)
#pragma unroll
        for (int a = 0; a < 2; ++a)
            q.c[ix(2 + o, a)] = t.c[ix(3 + o, 0)] * e[a][0] + t.c[ix(3 + o, 1)] * e[a][1] + t.c[ix(3 + o, 2)] * e[a][2];
#pragma unroll
    for (int o = 0; o < 3; ++o)
#pragma unroll
        for (int r = 0; r <= o; ++r) q.c[ix(2 + o, 2 + r)] = t.c[ix(3 + o, 3 + r)];
}

template <class F> __device__ __forceinline__ void pred_to_state(int kind, const PredT<F>& q, StateT<F>& t) {
    t.xh = q.xh; t.yh = q.yh; t.zh = q.zh; t.xl = q.xl; t.yl = q.yl; t.zl = q.zl;
    t.k = q.k; t.phi = q.phi; t.th = q.th; t.tl = q.tl; t.pl = q.pl;
    embed_cov(frame_of(kind, q), q.c, t.c);
}

// ----------------------------------------------------------------- propagation (a4-a7)

// Material of layer L at the predicted state (Sec. 3.1 material; a7): the Highland variance
// th02 of the scattering angle, kc = k cot(theta), and the factor a = p / p' of the mean energy
// loss (gain: the energy is added instead, for the backward fit).  Returns 1 (material applied),
// 0 (no material: zero thickness or k = 0) or -1 (the particle stops).  Computed in the
// trajectory precision F.
template <class F>
__device__ __forceinline__ int material_terms(const DevLayer& L, F xh, F yh, F k, F st, F ct, F sfp, F cfp,
                                              F& th02, F& kc, F& a, const F* xscale = nullptr,
                                              bool gain = false) {
    using P = Phys<F>;
    F cosi;
    if (L.kind == MKGB_BARREL) {
        const F ir = rsq(xh * xh + yh * yh);
        cosi = fabs((xh * cfp + yh * sfp) * st * ir);
    } else {
        cosi = fabs(ct);
    }
    const F fac = (cosi * P::inc_cap > F(1)) ? F(1) / cosi : P::inc_cap;
    F tt = F(L.xx0) * fac;
    if (xscale) tt = tt * *xscale;   // thickness scale (derivative of the fit)
    if (!(tt > F(0)) || k == F(0)) return 0;
    const F pm = F(1) / (fabs(k) * st);
    const F e2 = pm * pm + P::mpi * P::mpi;
    const F beta2 = pm * pm / e2;
    const F beta = sqrt(beta2);
    const F th0 = F(0.0136) / (beta * pm) * sqrt(tt) * (F(1) + F(0.038) * log_mat(tt / beta2));
    th02 = th0 * th0;
    kc = k * (ct / st);
    // PDG Bethe-Bloch mean energy loss in silicon (no density effect)
    const F e = sqrt(e2);
    const F bg2 = pm * pm * (F(1) / (P::mpi * P::mpi));
    const F gam = e * (F(1) / P::mpi);
    const F rme = P::me / P::mpi;
    const F tmax = F(2) * P::me * bg2 / (F(1) + F(2) * gam * rme + rme * rme);
    const F dedx = P::K * P::ZA / beta2 * (F(0.5) * log_mat(F(2) * P::me * bg2 * tmax / (P::I * P::I)) - beta2);
    const F de = dedx * P::rho * (tt * P::X0) * F(1e-3);
    const F en = gain ? e + de : e - de;   // gain: the backward fit adds the loss back
    if (!(en > P::mpi)) return -1;
    a = pm / sqrt((en - P::mpi) * (en + P::mpi));
    return 1;
}

// Adds the Highland Q to the (k, phi, theta) block of the surface-frame covariance qc and scales
// row/column k by a (material_terms' outputs; the terms are formed in F, added in G).
template <class F, class G>
__device__ __forceinline__ void material_cov(G qc[15], F th02, F kc, F st, F a) {
    qc[ix(3, 3)] += G(th02 / (st * st));
    qc[ix(4, 4)] += G(th02);
    qc[ix(2, 2)] += G(kc * kc * th02);
    qc[ix(4, 2)] -= G(kc * th02);
    const G ag = G(a);
    qc[ix(2, 0)] *= ag; qc[ix(2, 1)] *= ag; qc[ix(3, 2)] *= ag; qc[ix(4, 2)] *= ag;
    qc[ix(2, 2)] *= G(a * a);
}

// Propagates t to layer L.  Returns 1 (crossed; q holds the predicted state with material),
// 0 (not crossed) or -1 (particle stopped in the material).  newton_it counts iterations.
// dir (optional) gets sin(phi'), cos(phi'), sin(theta), cos(theta) at the crossing.
// The trajectory, its Jacobian and the material terms are computed in F; the covariance cin (21,
// global frame) is transported into qc (15, surface frame) in G.  q.c is not touched.
// BACKWARD (the backward fit, Sec. 2.2): the crossing behind the state, at a negative path length
// s, as the trajectory is traversed backwards from an outer layer: barrel from outside the
// cylinder, the radius falling as s decreases, no further back than the point of smallest
// radius of the current turn; disk behind the state, no further back than that point; the
// material then adds the mean energy loss back (the state describes the segment on the inner
// side of the layer).  The parametrisation, the frame and the Jacobian are those of the forward
// step with s < 0.
// Options: xscale scales the layer's thickness; s_guess starts the barrel Newton iteration at a
// path length solved in a lower precision (the FP64 steps then need one or two iterations);
// s_out returns the path length; mat_fp32 computes the material terms (Highland angle, energy-
// loss factor: small corrections, ~1e-7 relative in FP32) in FP32 for an FP64 step.
template <class F, class G, bool BACKWARD = false>
__device__ __forceinline__ int propagate_core(const DevLayer& L, float cBf, int material, const StateT<F>& t,
                                              const G cin[21], PredT<F>& q, G qc[15], int& newton_it,
                                              F* dir = nullptr, const F* xscale = nullptr,
                                              const F* s_guess = nullptr, F* s_out = nullptr,
                                              bool mat_fp32 = false) {
    using P = Phys<F>;
    const F cB = F(cBf);
    F sf, cf, st, ct;
    sin_cos(t.phi, &sf, &cf);
    sin_cos(t.th, &st, &ct);
    {   // phi + pl, theta + tl: first order in the low parts (below 1.2e-7; second order < 1e-14)
        const F s0 = st, f0 = sf;
        st = fma(ct, t.tl, st);
        ct = fma(-s0, t.tl, ct);
        sf = fma(cf, t.pl, sf);
        cf = fma(-f0, t.pl, cf);
    }
    const F om = -cB * t.k;
    const F ux = t.xh + t.xl, uy = t.yh + t.yl;
    const F Rl = F(L.pos), zd = F(L.pos);
    F s, S1, C1, dx, dy;
    if (L.kind == MKGB_BARREL) {
        const F c0 = r2_gap(Rl, t.xh, t.xl, t.yh, t.yl);   // R^2 - |u|^2
        if (BACKWARD ? !(c0 < F(0)) : !(c0 > F(0))) return 0;
        F lo = F(0), hi = F(3.0e38);
        // refinement of a crossing solved in a lower precision (s_guess within ~1e-6 of the
        // root, reach and turn checked there): the root lies inside (0, 2 s_guess), and Newton
        // from s_guess stops once its step is below 1e-5 of s (the error after that step is of
        // order the step squared, ~1e-12 of s)
        const bool refine = s_guess && *s_guess > F(0);
        if (refine) {
            s = *s_guess;
            hi = F(2) * s;
        } else if constexpr (BACKWARD) {
            // from outside, moving outward at s = 0: backwards the radius falls to its minimum
            // at the point of smallest radius behind the state; on that stretch g(s) = |u + d|^2
            // - R^2 rises with s through the root, so Newton runs as forward on the bracket
            // [-s_near, 0] from the straight-line root c0 / (b + sqrt(b^2 + c0)) < 0
            const F b = ux * cf + uy * sf;
            if (!(b > F(0))) return 0;
            const F disc = b * b + c0;
            lo = F(-3.0e38);
            hi = F(0);
            if (fabs(om) > F(1e-12)) {
                const F inv = F(1) / om;
                const F cx = ux - sf * inv, cy = uy + cf * inv;
                const F rho = fabs(inv);
                if (fabs(sqrt(cx * cx + cy * cy) - rho) > Rl) return 0;   // never comes down to R
                const F sg = om > F(0) ? F(1) : F(-1);
                F back = (t.phi - atan2(sg * cx, -sg * cy) - P::pi) * sg;   // turn since that point
                back -= P::two_pi * floor(back * (F(1) / P::two_pi));
                lo = -back * rho;
            } else if (!(disc >= F(0))) {
                return 0;
            }
            const F s0 = c0 / (b + sqrt(fmax(disc, F(0))));
            s = (s0 > lo && s0 < hi) ? s0 : F(0.5) * (lo + hi);
        } else {
            const F b = ux * cf + uy * sf;
            const F sq = sqrt(b * b + c0);
            const F s0 = (b > F(0)) ? c0 / (b + sq) : sq - b;
            if (fabs(om) > F(1e-12)) {
                const F inv = F(1) / om;
                const F cx = ux - sf * inv, cy = uy + cf * inv;
                const F rho = fabs(inv);
                const F reach = sqrt(cx * cx + cy * cy) + rho - Rl;
                if (reach < F(0)) return 0;
                const F sg = om > F(0) ? F(1) : F(-1);
                F turn = (atan2(sg * cx, -sg * cy) - t.phi) * sg;
                turn -= P::two_pi * floor(turn * (F(1) / P::two_pi));
                hi = turn * rho;
            }
            s = (s0 > lo && s0 < hi) ? s0 : F(0.5) * (lo + hi);
        }
        const F tol = is_fp32<F>() ? F(1e-6) : refine ? F(1e-5) : F(1e-13);
        for (int it = 0; it < 60; ++it) {
            ++newton_it;
            const F a = om * s;
            // one sine/cosine of the half angle per iterate: S1, C1 and the direction at s follow
            F sh, ch;
            sin_cos(F(0.5) * a, &sh, &ch);
            const F sa = F(2) * sh * ch, oc = F(2) * sh * sh;   // sin(a), 1 - cos(a)
            if (fabs(a) < F(1e-4)) {
                S1 = F(1) - a * a * (F(1) / F(6));
                C1 = a * (F(0.5) - a * a * (F(1) / F(24)));
            } else {
                S1 = sa / a;
                C1 = oc / a;
            }
            dx = s * (cf * S1 - sf * C1);
            dy = s * (sf * S1 + cf * C1);
            // g(s) = |u + d|^2 - R^2 = 2 u.d + |d|^2 - c0 (terms of size |u||d|, not R^2)
            const F g = F(2) * (ux * dx + uy * dy) + (dx * dx + dy * dy) - c0;
            if (g == F(0)) break;
            if (g < F(0)) lo = s; else hi = s;
            const F cpn = cf * (F(1) - oc) - sf * sa, spn = sf * (F(1) - oc) + cf * sa;   // direction at s
            const F dg = F(2) * ((ux + dx) * cpn + (uy + dy) * spn);
            F sn = (dg > F(0)) ? s - g / dg : F(0.5) * (lo + hi);
            if (!(sn >= lo && sn <= hi)) sn = F(0.5) * (lo + hi);
            const F ds = sn - s;
            s = sn;
            if (fabs(ds) <= tol * fabs(s)) break;
        }
    } else {
        if (fabs(ct) < F(1e-7)) return 0;
        const F dzp = sub_rn(sub_rn(zd, t.zh), t.zl);
        s = div_rn(dzp * st, ct);
        if (BACKWARD ? !(s < F(0)) : !(s > F(0))) return 0;
        // loopers are followed on the outgoing part of their current turn only: the disk must be
        // reached before the next point of largest radius (and moving outward, checked below);
        // backwards, no further back than the point of smallest radius
        if (fabs(om) > F(1e-12)) {
            const F inv = F(1) / om;
            const F cx = ux - sf * inv, cy = uy + cf * inv;
            const F sg = om > F(0) ? F(1) : F(-1);
            const F psi_far = atan2(sg * cx, -sg * cy);
            F turn = BACKWARD ? (t.phi - psi_far - P::pi) * sg : (psi_far - t.phi) * sg;
            turn -= P::two_pi * floor(turn * (F(1) / P::two_pi));
            if (fabs(s) > turn * fabs(inv)) return 0;
        }
    }
    const F a = om * s;
    F sh, ch;
    sin_cos(F(0.5) * a, &sh, &ch);
    const F sa = F(2) * sh * ch, ca = fma(F(-2) * sh, sh, F(1));   // sin(a), cos(a)
    if (fabs(a) < F(1e-4)) {
        S1 = F(1) - a * a * (F(1) / F(6));
        C1 = a * (F(0.5) - a * a * (F(1) / F(24)));
    } else {
        S1 = sa / a;
        C1 = F(2) * sh * sh / a;
    }
    {
        // chord form: d = s sinc(a/2) (cos psi, sin psi) with psi = phi + a/2; sin and cos of psi
        // by the angle-addition formulas, so psi is never rounded
        const F sp = fma(sf, ch, cf * sh), cp = fma(cf, ch, -sf * sh);
        const F h = F(0.5) * a;
        F sinc;
        if (fabs(h) < F(0.05)) {
            const F h2 = h * h;
            sinc = F(1) + h2 * (F(-1) / F(6) + h2 * (F(1) / F(120) + h2 * (F(-1) / F(5040) + h2 * (F(1) / F(362880)))));
        } else {
            sinc = div_rn(sh, h);
        }
        const F chord = s * sinc;
        dx = chord * cp;
        dy = chord * sp;
    }
    const F cot = div_rn(ct, st);
    const F dz = (L.kind == MKGB_BARREL) ? s * cot : sub_rn(sub_rn(zd, t.zh), t.zl);
    F xh = t.xh, xl = t.xl, yh = t.yh, yl = t.yl, zh = t.zh, zl = t.zl;
    add_ff(xh, xl, dx);
    add_ff(yh, yl, dy);
    add_ff(zh, zl, dz);
    const F sfp = fma(sf, ca, cf * sa), cfp = fma(cf, ca, -sf * sa);   // direction at the crossing
    if (L.kind == MKGB_BARREL) {
        // polish: the Newton iterate carries ~1e-6 relative error (FP32 tolerance), i.e.
        // the point may sit ~1e-5 cm off the cylinder along the normal, where the hit error is
        // 30 um; the gap R^2 - r'^2 of the compensated position is exact to ~eps^2, so one
        // more Newton step along the track puts the predicted point on the surface
        const F gap = r2_gap(Rl, xh, xl, yh, yl);
        const F dsp = div_rn(gap, F(2) * (xh * cfp + yh * sfp));
        add_ff(xh, xl, dsp * cfp);
        add_ff(yh, yl, dsp * sfp);
        add_ff(zh, zl, dsp * cot);
        if (!(zh >= F(L.lo) && zh <= F(L.hi))) return 0;
    } else {
        const F r = sqrt(xh * xh + yh * yh);
        if (!(r >= F(L.lo) && r <= F(L.hi))) return 0;
    }
    if (L.kind == MKGB_DISK && xh * cfp + yh * sfp < F(0)) return 0;   // moving inward: past the apex

    // ---- Jacobian rows x, y, z, phi: J = A + (df/ds)(ds/dp); rows k, theta are identity
    F dS1, dC1;
    s1c1_deriv(a, S1, C1, dS1, dC1);
    const F A03 = -cB * s * s * (cf * dS1 - sf * dC1);
    const F A13 = -cB * s * s * (sf * dS1 + cf * dC1);
    const F A04 = -dy, A14 = dx;
    const F A25 = -s / (st * st);
    const F A43 = -cB * s;
    F ds[6];
    if (L.kind == MKGB_BARREL) {
        const F ig = F(-1) / (xh * cfp + yh * sfp);
        ds[0] = xh * ig; ds[1] = yh * ig; ds[2] = F(0);
        ds[3] = (xh * A03 + yh * A13) * ig;
        ds[4] = (xh * A04 + yh * A14) * ig;
        ds[5] = F(0);
    } else {
        const F ig = F(-1) / cot;
        ds[0] = F(0); ds[1] = F(0); ds[2] = ig;
        ds[3] = F(0); ds[4] = F(0); ds[5] = A25 * ig;
    }
    // Rows of the fixed-s Jacobian for x, y, z (identity + A terms), projected on e1 and e2.
    // df/ds along the position is the track direction / sin(theta), whose surface projection
    // lies along e1: the path-length term enters u1 only (e2 . df/ds = 0 by construction).
    const FrameT<F> fr = frame_of(L.kind, xh, yh, sfp, cfp, st, ct);
    const F Apos[3][6] = {{F(1), F(0), F(0), A03, A04, F(0)},
                          {F(0), F(1), F(0), A13, A14, F(0)},
                          {F(0), F(0), F(1), F(0), F(0), A25}};
    const F fpos[3] = {cfp, sfp, cot};
    const F f1 = dot3(fr.e1, fpos);
    F J[3][6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const F a1 = fr.e1[0] * Apos[0][j] + fr.e1[1] * Apos[1][j] + fr.e1[2] * Apos[2][j];
        const F a2 = fr.e2[0] * Apos[0][j] + fr.e2[1] * Apos[1][j] + fr.e2[2] * Apos[2][j];
        J[0][j] = fma(f1, ds[j], a1);
        J[1][j] = a2;
        J[2][j] = om * ds[j];
    }
    J[2][3] += A43; J[2][4] += F(1);

    // ---- transport into the surface frame: rows (u1, u2, phi) dense, (k, theta) identity
    constexpr int D[3] = {0, 1, 3};   // local indices of the dense rows
    G T[3][6];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            G acc = G(0);
#pragma unroll
            for (int l = 0; l < 6; ++l) acc = fma(G(J[r][l]), cin[ix(l, j)], acc);
            T[r][j] = acc;
        }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int p = 0; p <= r; ++p) {
            G acc = G(0);
#pragma unroll
            for (int l = 0; l < 6; ++l) acc = fma(T[r][l], G(J[p][l]), acc);
            qc[ix(D[r], D[p])] = acc;
        }
        qc[ix(D[r], 2)] = T[r][3];
        qc[ix(4, D[r])] = T[r][5];
    }
    qc[ix(2, 2)] = cin[ix(3, 3)];
    qc[ix(4, 2)] = cin[ix(5, 3)];
    qc[ix(4, 4)] = cin[ix(5, 5)];
    q.xh = xh; q.xl = xl; q.yh = yh; q.yl = yl; q.zh = zh; q.zl = zl;
    q.k = t.k;
    q.phi = t.phi;
    q.pl = t.pl;
    add_ff(q.phi, q.pl, a);
    wrap_pi_ff(q.phi, q.pl);
    q.th = t.th;
    q.tl = t.tl;
    if (dir) {
        dir[0] = sfp; dir[1] = cfp; dir[2] = st; dir[3] = ct;
    }
    if (material) {
        F th02, kc, ea;
        int mr;
        if (mat_fp32) {
            float th02f = 0.0f, kcf = 0.0f, eaf = 1.0f;
            mr = material_terms<float>(L, float(q.xh), float(q.yh), float(q.k), float(st), float(ct),
                                       float(sfp), float(cfp), th02f, kcf, eaf, nullptr, BACKWARD);
            th02 = F(th02f); kc = F(kcf); ea = F(eaf);
        } else {
            mr = material_terms(L, q.xh, q.yh, q.k, st, ct, sfp, cfp, th02, kc, ea, xscale, BACKWARD);
        }
        if (mr < 0) return -1;
        if (mr > 0) {
            material_cov(qc, th02, kc, st, ea);
            q.k = q.k * ea;
        }
    }
    if (s_out) *s_out = s;
    return 1;
}

template <class F>
__device__ __forceinline__ int propagate(const DevLayer& L, float cBf, int material, const StateT<F>& t, PredT<F>& q,
                                         int& newton_it, F* dir = nullptr) {
    return propagate_core<F, F>(L, cBf, material, t, t.c, q, q.c, newton_it, dir);
}

// The propagation of the FP64 steps that serve the FP32 path (seed fits, refits of ill-conditioned
// fits) when fast: the crossing is solved in FP32 first and refined by FP64 Newton iterations
// from there (one or two instead of ~5), and the material terms are FP32.  The plain all-FP64
// path takes fast = false.
template <class F>
__device__ __forceinline__ int propagate_refined(const DevLayer& L, float cBf, int material, const StateT<F>& t,
                                                 PredT<F>& q, int& newton_it, bool fast, F* dir = nullptr);

// ----------------------------------------------------------------- module planes (Sec. 3.1)
//
// A Phase-2 module is flat (and tilted in the outer rings of the barrel): a hit on a module is
// measured on the plane through the module's position c with unit normal n.  The search and the
// fit take the state on the layer's reference surface (cylinder or disk: window, material,
// binning) and move it along the helix to the hit's module plane before its chi2 and update.
// The step is a few millimetres, in either direction, and crosses no material.

constexpr float kPlaneMaxPath = 10.0f;   // cm: longest |s| accepted for the step to a module
constexpr float kPlaneMinCos = 1e-3f;    // smallest |n . dx/ds| (per transverse path) accepted

// Frame of a state on a plane with unit normal n: e1 the direction projected onto the plane,
// e2 = n x e1 (for n = r-hat this is the barrel frame of frame_of).
template <class F> __device__ __forceinline__ FrameT<F> plane_frame(const F n[3], F sfp, F cfp, F st, F ct) {
    FrameT<F> f;
    const F d[3] = {st * cfp, st * sfp, ct};
    const F dn = dot3(n, d);
    F e[3] = {d[0] - dn * n[0], d[1] - dn * n[1], d[2] - dn * n[2]};
    F nrm2 = dot3(e, e);
    if (!(nrm2 > F(1e-12))) {   // moving along the normal: any axis of the plane
        const F a[3] = {fabs(n[2]) < F(0.9) ? F(0) : F(1), F(0), fabs(n[2]) < F(0.9) ? F(1) : F(0)};
        const F an = dot3(a, n);
        e[0] = a[0] - an * n[0]; e[1] = a[1] - an * n[1]; e[2] = a[2] - an * n[2];
        nrm2 = dot3(e, e);
    }
    const F inv = rsq(nrm2);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        f.n[i] = n[i];
        f.e1[i] = e[i] * inv;
    }
    f.e2[0] = n[1] * f.e1[2] - n[2] * f.e1[1];
    f.e2[1] = n[2] * f.e1[0] - n[0] * f.e1[2];
    f.e2[2] = n[0] * f.e1[1] - n[1] * f.e1[0];
    return f;
}

// Moves t (global frame, on or near a surface) to the plane through cm.xyz with normal nm.xyz:
// the crossing nearest to t (Newton on g(s) = n.(u + d(s) - c) from the tangent-line root,
// written relative to the current position; the crossing point polished onto the plane with the
// compensated gap), the Jacobian of the plane map and the covariance transported into the plane
// frame fr (q.c, 15).  Returns 1, or 0 if Newton fails, |s| > kPlaneMaxPath or the crossing is
// grazing (|n . dx/ds| < kPlaneMinCos).  newton_it counts iterations.
template <class F>
__device__ __forceinline__ int propagate_plane(const StateT<F>& t, const float4 cm, const float4 nm, float cBf,
                                               PredT<F>& q, FrameT<F>& fr, int& newton_it) {
    const F cB = F(cBf);
    const F n[3] = {F(nm.x), F(nm.y), F(nm.z)};
    F sf, cf, st, ct;
    sin_cos(t.phi, &sf, &cf);
    sin_cos(t.th, &st, &ct);
    {
        const F s0 = st, f0 = sf;
        st = fma(ct, t.tl, st);
        ct = fma(-s0, t.tl, ct);
        sf = fma(cf, t.pl, sf);
        cf = fma(-f0, t.pl, cf);
    }
    const F om = -cB * t.k;
    const F cot = div_rn(ct, st);
    // n.(c - u) with the compensated position: terms of the size of the distance, not of |c|
    const F g0 = n[0] * sub_rn(sub_rn(F(cm.x), t.xh), t.xl) + n[1] * sub_rn(sub_rn(F(cm.y), t.yh), t.yl) +
                 n[2] * sub_rn(sub_rn(F(cm.z), t.zh), t.zl);
    const F dg0 = n[0] * cf + n[1] * sf + n[2] * cot;
    if (dg0 == F(0)) return 0;
    F s = g0 / dg0;
    const F tol = is_fp32<F>() ? F(1e-6) : F(1e-13);
    bool conv = false;
    for (int it = 0; it < 20 && !conv; ++it) {
        ++newton_it;
        const F a = om * s;
        F sh, ch;
        sin_cos(F(0.5) * a, &sh, &ch);
        const F sa = F(2) * sh * ch, oc = F(2) * sh * sh;
        F S1, C1;
        if (fabs(a) < F(1e-4)) {
            S1 = F(1) - a * a * (F(1) / F(6));
            C1 = a * (F(0.5) - a * a * (F(1) / F(24)));
        } else {
            S1 = sa / a;
            C1 = oc / a;
        }
        const F dx = s * (cf * S1 - sf * C1), dy = s * (sf * S1 + cf * C1);
        const F g = n[0] * dx + n[1] * dy + n[2] * (s * cot) - g0;
        const F cpn = cf * (F(1) - oc) - sf * sa, spn = sf * (F(1) - oc) + cf * sa;
        const F dg = n[0] * cpn + n[1] * spn + n[2] * cot;
        if (dg == F(0)) return 0;
        const F ds = -g / dg;
        s += ds;
        conv = fabs(ds) <= tol * (F(1) + fabs(s));
    }
    if (!conv || !(fabs(s) <= F(2 * kPlaneMaxPath))) return 0;
    const F a = om * s;
    F sh, ch;
    sin_cos(F(0.5) * a, &sh, &ch);
    const F sa = F(2) * sh * ch, ca = fma(F(-2) * sh, sh, F(1));
    F S1, C1;
    if (fabs(a) < F(1e-4)) {
        S1 = F(1) - a * a * (F(1) / F(6));
        C1 = a * (F(0.5) - a * a * (F(1) / F(24)));
    } else {
        S1 = sa / a;
        C1 = F(2) * sh * sh / a;
    }
    F dx, dy;
    {
        const F sp = fma(sf, ch, cf * sh), cp = fma(cf, ch, -sf * sh);
        const F h = F(0.5) * a;
        F sinc;
        if (fabs(h) < F(0.05)) {
            const F h2 = h * h;
            sinc = F(1) + h2 * (F(-1) / F(6) + h2 * (F(1) / F(120) + h2 * (F(-1) / F(5040) + h2 * (F(1) / F(362880)))));
        } else {
            sinc = div_rn(sh, h);
        }
        const F chord = s * sinc;
        dx = chord * cp;
        dy = chord * sp;
    }
    F xh = t.xh, xl = t.xl, yh = t.yh, yl = t.yl, zh = t.zh, zl = t.zl;
    add_ff(xh, xl, dx);
    add_ff(yh, yl, dy);
    add_ff(zh, zl, s * cot);
    const F sfp = fma(sf, ca, cf * sa), cfp = fma(cf, ca, -sf * sa);
    const F den = n[0] * cfp + n[1] * sfp + n[2] * cot;   // n . dx/ds at the crossing
    {   // polish onto the plane along the track with the compensated gap
        const F gap = n[0] * sub_rn(sub_rn(F(cm.x), xh), xl) + n[1] * sub_rn(sub_rn(F(cm.y), yh), yl) +
                      n[2] * sub_rn(sub_rn(F(cm.z), zh), zl);
        const F dsp = div_rn(gap, den);
        add_ff(xh, xl, dsp * cfp);
        add_ff(yh, yl, dsp * sfp);
        add_ff(zh, zl, dsp * cot);
    }
    if (!(fabs(s) <= F(kPlaneMaxPath)) || !(fabs(den) >= F(kPlaneMinCos))) return 0;

    // ---- Jacobian: J = A + (df/ds)(ds/dp), ds/dp = -(n . A_pos) / (n . df/ds); rows k, theta identity
    F dS1, dC1;
    s1c1_deriv(a, S1, C1, dS1, dC1);
    const F A03 = -cB * s * s * (cf * dS1 - sf * dC1);
    const F A13 = -cB * s * s * (sf * dS1 + cf * dC1);
    const F A04 = -dy, A14 = dx;
    const F A25 = -s / (st * st);
    const F A43 = -cB * s;
    const F ig = F(-1) / den;
    F ds[6];
    ds[0] = n[0] * ig; ds[1] = n[1] * ig; ds[2] = n[2] * ig;
    ds[3] = (n[0] * A03 + n[1] * A13) * ig;
    ds[4] = (n[0] * A04 + n[1] * A14) * ig;
    ds[5] = n[2] * A25 * ig;
    fr = plane_frame(n, sfp, cfp, st, ct);
    const F Apos[3][6] = {{F(1), F(0), F(0), A03, A04, F(0)},
                          {F(0), F(1), F(0), A13, A14, F(0)},
                          {F(0), F(0), F(1), F(0), F(0), A25}};
    const F fpos[3] = {cfp, sfp, cot};
    const F f1 = dot3(fr.e1, fpos);
    F J[3][6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const F a1 = fr.e1[0] * Apos[0][j] + fr.e1[1] * Apos[1][j] + fr.e1[2] * Apos[2][j];
        const F a2 = fr.e2[0] * Apos[0][j] + fr.e2[1] * Apos[1][j] + fr.e2[2] * Apos[2][j];
        J[0][j] = fma(f1, ds[j], a1);
        J[1][j] = a2;   // e2 . df/ds = 0: the direction projects onto e1
        J[2][j] = om * ds[j];
    }
    J[2][3] += A43; J[2][4] += F(1);
    constexpr int D[3] = {0, 1, 3};
    F T[3][6];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            F acc = F(0);
#pragma unroll
            for (int l = 0; l < 6; ++l) acc = fma(J[r][l], t.c[ix(l, j)], acc);
            T[r][j] = acc;
        }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int p = 0; p <= r; ++p) {
            F acc = F(0);
#pragma unroll
            for (int l = 0; l < 6; ++l) acc = fma(T[r][l], J[p][l], acc);
            q.c[ix(D[r], D[p])] = acc;
        }
        q.c[ix(D[r], 2)] = T[r][3];
        q.c[ix(4, D[r])] = T[r][5];
    }
    q.c[ix(2, 2)] = t.c[ix(3, 3)];
    q.c[ix(4, 2)] = t.c[ix(5, 3)];
    q.c[ix(4, 4)] = t.c[ix(5, 5)];
    q.xh = xh; q.xl = xl; q.yh = yh; q.yl = yl; q.zh = zh; q.zl = zl;
    q.k = t.k;
    q.phi = t.phi;
    q.pl = t.pl;
    add_ff(q.phi, q.pl, a);
    wrap_pi_ff(q.phi, q.pl);
    q.th = t.th;
    q.tl = t.tl;
    return 1;
}

// The prediction q on a layer's reference surface (kind) moved to module mod's plane (table mods:
// two float4 per module): qp and its frame fp.
template <class F>
__device__ __forceinline__ int to_module_plane(int kind, const PredT<F>& q, const float4* __restrict__ mods, int mod,
                                               float cBf, PredT<F>& qp, FrameT<F>& fp) {
    StateT<F> t;
    pred_to_state(kind, q, t);
    int it = 0;
    return propagate_plane(t, __ldg(mods + 2 * mod), __ldg(mods + 2 * mod + 1), cBf, qp, fp, it);
}

// The chi2 of a module hit (m, v) on its module's plane, for the search's window loop: from the
// prediction q on the layer's reference surface, in its surface frame fr, with the direction
// dir = (sin phi', cos phi', sin theta, cos theta) at the crossing (as propagate returns it).  The
// plane crossing as propagate_plane finds it, but only the two rows of the Jacobian that the
// position covariance on the plane needs, contracted with the surface-frame covariance directly
// (the 21-term global covariance is never formed).  False if the plane is not reached or S is
// not positive definite.  The module-hit steps are not inlined, so that the search and fit
// kernels keep their register allocation for the layers without modules.
template <class F>
__device__ __noinline__ bool module_chi2_dir(const PredT<F>& q, const FrameT<F>& fr, const F dir[4],
                                             const float4* __restrict__ mods, int mod, float cBf, const F m[3],
                                             const F v[6], F& x2) {
    const float4 cm = __ldg(mods + 2 * mod), nm = __ldg(mods + 2 * mod + 1);
    const F n[3] = {F(nm.x), F(nm.y), F(nm.z)};
    const F cB = F(cBf);
    const F sf = dir[0], cf = dir[1], st = dir[2], ct = dir[3];
    const F om = -cB * q.k;
    const F cot = div_rn(ct, st);
    const F g0 = n[0] * sub_rn(sub_rn(F(cm.x), q.xh), q.xl) + n[1] * sub_rn(sub_rn(F(cm.y), q.yh), q.yl) +
                 n[2] * sub_rn(sub_rn(F(cm.z), q.zh), q.zl);
    const F dg0 = n[0] * cf + n[1] * sf + n[2] * cot;
    if (dg0 == F(0)) return false;
    F s = g0 / dg0;
    const F tol = is_fp32<F>() ? F(1e-6) : F(1e-13);
    bool conv = false;
    for (int it = 0; it < 20 && !conv; ++it) {
        const F a = om * s;
        F sh, ch;
        sin_cos(F(0.5) * a, &sh, &ch);
        const F sa = F(2) * sh * ch, oc = F(2) * sh * sh;
        F S1, C1;
        if (fabs(a) < F(1e-4)) {
            S1 = F(1) - a * a * (F(1) / F(6));
            C1 = a * (F(0.5) - a * a * (F(1) / F(24)));
        } else {
            S1 = sa / a;
            C1 = oc / a;
        }
        const F dx = s * (cf * S1 - sf * C1), dy = s * (sf * S1 + cf * C1);
        const F g = n[0] * dx + n[1] * dy + n[2] * (s * cot) - g0;
        const F cpn = cf * (F(1) - oc) - sf * sa, spn = sf * (F(1) - oc) + cf * sa;
        const F dg = n[0] * cpn + n[1] * spn + n[2] * cot;
        if (dg == F(0)) return false;
        const F ds = -g / dg;
        s += ds;
        conv = fabs(ds) <= tol * (F(1) + fabs(s));
    }
    if (!conv || !(fabs(s) <= F(2 * kPlaneMaxPath))) return false;
    const F a = om * s;
    F sh, ch;
    sin_cos(F(0.5) * a, &sh, &ch);
    const F sa = F(2) * sh * ch, ca = fma(F(-2) * sh, sh, F(1));
    F S1, C1;
    if (fabs(a) < F(1e-4)) {
        S1 = F(1) - a * a * (F(1) / F(6));
        C1 = a * (F(0.5) - a * a * (F(1) / F(24)));
    } else {
        S1 = sa / a;
        C1 = F(2) * sh * sh / a;
    }
    F dx, dy;
    {
        const F sp = fma(sf, ch, cf * sh), cp = fma(cf, ch, -sf * sh);
        const F h = F(0.5) * a;
        F sinc;
        if (fabs(h) < F(0.05)) {
            const F h2 = h * h;
            sinc = F(1) + h2 * (F(-1) / F(6) + h2 * (F(1) / F(120) + h2 * (F(-1) / F(5040) + h2 * (F(1) / F(362880)))));
        } else {
            sinc = div_rn(sh, h);
        }
        const F chord = s * sinc;
        dx = chord * cp;
        dy = chord * sp;
    }
    PredT<F> qp;
    qp.xh = q.xh; qp.xl = q.xl; qp.yh = q.yh; qp.yl = q.yl; qp.zh = q.zh; qp.zl = q.zl;
    add_ff(qp.xh, qp.xl, dx);
    add_ff(qp.yh, qp.yl, dy);
    add_ff(qp.zh, qp.zl, s * cot);
    const F sfp = fma(sf, ca, cf * sa), cfp = fma(cf, ca, -sf * sa);
    const F den = n[0] * cfp + n[1] * sfp + n[2] * cot;
    {
        const F gap = n[0] * sub_rn(sub_rn(F(cm.x), qp.xh), qp.xl) + n[1] * sub_rn(sub_rn(F(cm.y), qp.yh), qp.yl) +
                      n[2] * sub_rn(sub_rn(F(cm.z), qp.zh), qp.zl);
        const F dsp = div_rn(gap, den);
        add_ff(qp.xh, qp.xl, dsp * cfp);
        add_ff(qp.yh, qp.yl, dsp * sfp);
        add_ff(qp.zh, qp.zl, dsp * cot);
    }
    if (!(fabs(s) <= F(kPlaneMaxPath)) || !(fabs(den) >= F(kPlaneMinCos))) return false;
    // rows u1, u2 of the plane map's Jacobian in the global parameters (as propagate_plane) ...
    F dS1, dC1;
    s1c1_deriv(a, S1, C1, dS1, dC1);
    const F A03 = -cB * s * s * (cf * dS1 - sf * dC1);
    const F A13 = -cB * s * s * (sf * dS1 + cf * dC1);
    const F A04 = -dy, A14 = dx;
    const F A25 = -s / (st * st);
    const F ig = F(-1) / den;
    F ds[6];
    ds[0] = n[0] * ig; ds[1] = n[1] * ig; ds[2] = n[2] * ig;
    ds[3] = (n[0] * A03 + n[1] * A13) * ig;
    ds[4] = (n[0] * A04 + n[1] * A14) * ig;
    ds[5] = n[2] * A25 * ig;
    const FrameT<F> fp = plane_frame(n, sfp, cfp, st, ct);
    const F Apos[3][6] = {{F(1), F(0), F(0), A03, A04, F(0)},
                          {F(0), F(1), F(0), A13, A14, F(0)},
                          {F(0), F(0), F(1), F(0), F(0), A25}};
    const F fpos[3] = {cfp, sfp, cot};
    const F f1 = dot3(fp.e1, fpos);
    F J[2][6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const F a1 = fp.e1[0] * Apos[0][j] + fp.e1[1] * Apos[1][j] + fp.e1[2] * Apos[2][j];
        const F a2 = fp.e2[0] * Apos[0][j] + fp.e2[1] * Apos[1][j] + fp.e2[2] * Apos[2][j];
        J[0][j] = fma(f1, ds[j], a1);
        J[1][j] = a2;
    }
    // ... times the map from the reference surface's parameters (u1, u2, k, phi, theta) to the
    // global ones (position columns e1, e2 of fr; the angles and k one to one)
    F Js[2][5];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        Js[r][0] = J[r][0] * fr.e1[0] + J[r][1] * fr.e1[1] + J[r][2] * fr.e1[2];
        Js[r][1] = J[r][0] * fr.e2[0] + J[r][1] * fr.e2[1] + J[r][2] * fr.e2[2];
        Js[r][2] = J[r][3];
        Js[r][3] = J[r][4];
        Js[r][4] = J[r][5];
    }
    F T[2][5];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            F acc = F(0);
#pragma unroll
            for (int l = 0; l < 5; ++l) acc = fma(Js[r][l], q.c[ix(l, j)], acc);
            T[r][j] = acc;
        }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int p = 0; p <= r; ++p) {
            F acc = F(0);
#pragma unroll
            for (int l = 0; l < 5; ++l) acc = fma(T[r][l], Js[p][l], acc);
            qp.c[ix(r, p)] = acc;
        }
    return chi2_hit(fp, qp, m[0], m[1], m[2], v, x2);
}

// Update with a module hit on its module's plane.  Returns 0 (out updated), 1 (plane not reached),
// 2 (the update failed) or, with outlier_cut > 0 and a predicted chi2 above it, 3 (out untouched).
// x2 gets the predicted chi2, kappa the condition estimate of S.
template <class F>
__device__ __forceinline__ int plane_update_core(const FrameT<F>& fp, const PredT<F>& qp, const F m[3], const F v[6],
                                                 float outlier_cut, StateT<F>& out, F& x2, float& kappa) {
    if (!chi2_hit(fp, qp, m[0], m[1], m[2], v, x2)) return 2;
    if (outlier_cut > 0.0f && x2 > F(outlier_cut)) return 3;
    return kalman_update_f(fp, qp, m[0], m[1], m[2], v, out, &kappa) ? 0 : 2;
}

template <class F>
__device__ __noinline__ int module_update(int kind, const PredT<F>& q, const float4* __restrict__ mods, int mod,
                                          float cBf, const F m[3], const F v[6], float outlier_cut, StateT<F>& out,
                                          F& x2, float& kappa) {
    PredT<F> qp;
    FrameT<F> fp;
    if (!to_module_plane(kind, q, mods, mod, cBf, qp, fp)) return 1;
    return plane_update_core(fp, qp, m, v, outlier_cut, out, x2, kappa);
}

// The same for a global-frame state t that already lies on module mod's plane (the start state
// of the backward fit): its covariance is taken in the plane's frame (the variance along the
// normal dropped), then chi2 and update.  Return codes as module_update without 1; with 3 (an
// outlier) out gets t taken on the plane.
template <class F>
__device__ __noinline__ int module_update_on_plane(const StateT<F>& t, const float4* __restrict__ mods, int mod,
                                                   const F m[3], const F v[6], float outlier_cut, StateT<F>& out,
                                                   F& x2, float& kappa) {
    const float4 nm = __ldg(mods + 2 * mod + 1);
    const F n[3] = {F(nm.x), F(nm.y), F(nm.z)};
    F sf, cf, st, ct;
    sin_cos(t.phi, &sf, &cf);
    sin_cos(t.th, &st, &ct);
    const FrameT<F> fp = plane_frame(n, sf, cf, st, ct);
    PredT<F> qp;
    state_to_pred(fp, t, qp);
    const int r = plane_update_core(fp, qp, m, v, outlier_cut, out, x2, kappa);
    if (r == 3) {
        out = t;
        embed_cov(fp, qp.c, out.c);
    }
    return r;
}

// ----------------------------------------------------------------- window (a8)

template <class F> struct WindowT {
    F eta, phi, deta, dphi;
};
using Window = WindowT<float>;

template <class F>
__device__ __forceinline__ WindowT<F> window(const DevLayer& L, const DevParams& P, const PredT<F>& q,
                                             const FrameT<F>& fr) {
    const F x = q.xh, y = q.yh, z = q.zh;
    const F rt2 = x * x + y * y, rt = sqrt(rt2), r3 = sqrt(rt2 + z * z);
    WindowT<F> w;
    w.eta = asinh(z / rt);
    w.phi = atan2(y, x);
    const F c = x / rt, sn = y / rt;
    // gradients in (r-hat, phi-hat, z-hat) at the predicted point
    const F ge_r = -z / (rt * r3), ge_z = F(1) / r3;
    const F gp_p = F(1) / rt;
    const F sr2 = F(L.sig[0]) * F(L.sig[0]), sp2 = F(L.sig[1]) * F(L.sig[1]), sz2 = F(L.sig[2]) * F(L.sig[2]);
    F ve = ge_r * ge_r * sr2 + ge_z * ge_z * sz2;
    F vp = gp_p * gp_p * sp2;
    // surface part: gradient components along e1, e2
    const F geg[3] = {ge_r * c, ge_r * sn, ge_z};       // eta gradient, global
    const F gpg[3] = {-gp_p * sn, gp_p * c, F(0)};      // phi gradient, global
    const F ge1 = dot3(fr.e1, geg), ge2 = dot3(fr.e2, geg);
    const F gp1 = dot3(fr.e1, gpg), gp2 = dot3(fr.e2, gpg);
    ve += ge1 * ge1 * q.c[0] + F(2) * ge1 * ge2 * q.c[1] + ge2 * ge2 * q.c[2];
    vp += gp1 * gp1 * q.c[0] + F(2) * gp1 * gp2 * q.c[1] + gp2 * gp2 * q.c[2];
    w.deta = fmin(fmax(F(P.nsig) * sqrt(fmax(ve, F(0))), F(P.deta_min)), F(P.deta_max));
    w.dphi = fmin(fmax(F(P.nsig) * sqrt(fmax(vp, F(0))), F(P.dphi_min)), F(P.dphi_max));
    return w;
}

// ----------------------------------------------------------------- chi2 (a9) and update (a11)

// Cholesky of a packed 3x3; inv[] gets 1/L_ii.  Returns false if not positive definite.
template <class F> __device__ __forceinline__ bool chol3(const F S[6], F L[6], F inv[3]) {
    if (!(S[0] > F(0))) return false;
    inv[0] = rsq(S[0]);
    const F l10 = S[1] * inv[0], l20 = S[3] * inv[0];
    const F d1 = S[2] - l10 * l10;
    if (!(d1 > F(0))) return false;
    inv[1] = rsq(d1);
    const F l21 = (S[4] - l20 * l10) * inv[1];
    const F d2 = S[5] - l20 * l20 - l21 * l21;
    if (!(d2 > F(0))) return false;
    inv[2] = rsq(d2);
    L[0] = S[0] * inv[0]; L[1] = l10; L[2] = d1 * inv[1]; L[3] = l20; L[4] = l21; L[5] = d2 * inv[2];
    return true;
}

// Residual m - x' (compensated position) and hit covariance in the local frame; S = V + C_surface.
// dm (optional): a small displacement of the hit (alignment), added to the residual after the
// compensated subtraction so that it is not rounded to the hit's own ulp.
template <class F>
__device__ __forceinline__ void local_meas(const FrameT<F>& f, const PredT<F>& q, F mx, F my, F mz, const F v[6],
                                           F rl[3], F vl[6], F S[6], const F* dm = nullptr) {
    F r[3] = {sub_rn(sub_rn(mx, q.xh), q.xl), sub_rn(sub_rn(my, q.yh), q.yl), sub_rn(sub_rn(mz, q.zh), q.zl)};
    if (dm) {
        r[0] += dm[0]; r[1] += dm[1]; r[2] += dm[2];
    }
    to_local3(f, r, rl);
    to_local_sym3(f, v, vl);
    S[0] = vl[0]; S[1] = vl[1]; S[3] = vl[3];
    S[2] = vl[2] + q.c[0]; S[4] = vl[4] + q.c[1]; S[5] = vl[5] + q.c[2];
}

template <class F>
__device__ __forceinline__ bool chi2_hit(const FrameT<F>& f, const PredT<F>& q, F mx, F my, F mz, const F v[6],
                                         F& chi2, const F* dm = nullptr) {
    F rl[3], vl[6], S[6], L[6], inv[3];
    local_meas(f, q, mx, my, mz, v, rl, vl, S, dm);
    if (!chol3(S, L, inv)) return false;
    const F y0 = rl[0] * inv[0];
    const F y1 = (rl[1] - L[1] * y0) * inv[1];
    const F y2 = (rl[2] - L[3] * y0 - L[4] * y1) * inv[2];
    chi2 = y0 * y0 + y1 * y1 + y2 * y2;
    return true;
}

template <class F>
__device__ __forceinline__ bool chi2_hit(int kind, const PredT<F>& q, F mx, F my, F mz, const F v[6], F& chi2,
                                         const F* dm = nullptr) {
    return chi2_hit(frame_of(kind, q), q, mx, my, mz, v, chi2, dm);
}

// Kalman update of a predicted state with one hit, Joseph form in the surface frame:
// K = C H^T S^-1 (H picks u1, u2 into measurement rows e1, e2; the normal row is zero),
// C+ = (I - K H) C (I - K H)^T + K V K^T; the result is returned as a global-frame state.
// Returns false if S is not positive definite or theta leaves (0, pi).
// kappa (optional) gets (max L_ii / min L_ii)^2 of the Cholesky factor of S, an estimate of its
// condition number.
// JOSEPH = false takes the equal (in exact arithmetic) short form C+ = (I - K H) C, lower
// triangle only: 30 instead of ~170 multiply-adds.  For FP64 steps only, where rounding of the
// short form (relative error ~ kappa(S) x 1e-16) stays far below the tolerances; FP32 steps keep
// the Joseph form, whose result stays symmetric positive definite under rounding.
template <class F, bool JOSEPH = true>
__device__ __forceinline__ bool kalman_update_f(const FrameT<F>& f, const PredT<F>& q, F mx, F my, F mz,
                                                const F v[6], StateT<F>& out, float* kappa = nullptr,
                                                const F* dm = nullptr) {
    F rl[3], vl[6], S[6], L[6], inv[3];
    local_meas(f, q, mx, my, mz, v, rl, vl, S, dm);
    if (!chol3(S, L, inv)) return false;
    if (kappa) {
        const F lmax = fmax(fmax(L[0], L[2]), L[5]), lmin = fmin(fmin(L[0], L[2]), L[5]);
        *kappa = float((lmax / lmin) * (lmax / lmin));
    }
    // W = S^-1 = L^-T L^-1
    const F i00 = inv[0], i11 = inv[1], i22 = inv[2];
    const F i10 = -L[1] * i00 * i11;
    const F i21 = -L[4] * i11 * i22;
    const F i20 = -(L[3] * i00 + L[4] * i10) * i22;
    const F W[3][3] = {{i00 * i00 + i10 * i10 + i20 * i20, i10 * i11 + i20 * i21, i20 * i22},
                       {i10 * i11 + i20 * i21, i11 * i11 + i21 * i21, i21 * i22},
                       {i20 * i22, i21 * i22, i22 * i22}};
    F K[5][3];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a) K[i][a] = fma(q.c[ix(i, 0)], W[1][a], q.c[ix(i, 1)] * W[2][a]);
    F dp[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) dp[i] = fma(K[i][0], rl[0], fma(K[i][1], rl[1], K[i][2] * rl[2]));
    F cn[15];
    if constexpr (JOSEPH) {
        // T = (I - K H) C : row i minus K_i1 * row u1 minus K_i2 * row u2
        F T[5][5];
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = 0; j < 5; ++j)
                T[i][j] = fma(-K[i][1], q.c[ix(0, j)], fma(-K[i][2], q.c[ix(1, j)], q.c[ix(i, j)]));
        const F V[3][3] = {{vl[0], vl[1], vl[3]}, {vl[1], vl[2], vl[4]}, {vl[3], vl[4], vl[5]}};
        F KV[5][3];
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int a = 0; a < 3; ++a) KV[i][a] = fma(K[i][0], V[0][a], fma(K[i][1], V[1][a], K[i][2] * V[2][a]));
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) {
                F acc = fma(-T[i][0], K[j][1], fma(-T[i][1], K[j][2], T[i][j]));
#pragma unroll
                for (int a = 0; a < 3; ++a) acc = fma(KV[i][a], K[j][a], acc);
                cn[ix(i, j)] = acc;
            }
    } else {
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j)
                cn[ix(i, j)] = fma(-K[i][1], q.c[ix(0, j)], fma(-K[i][2], q.c[ix(1, j)], q.c[ix(i, j)]));
    }
    F dg[3];
    surface_to_global(f, dp[0], dp[1], dg);
    out.xh = q.xh; out.xl = q.xl; out.yh = q.yh; out.yl = q.yl; out.zh = q.zh; out.zl = q.zl;
    add_ff(out.xh, out.xl, dg[0]);
    add_ff(out.yh, out.yl, dg[1]);
    add_ff(out.zh, out.zl, dg[2]);
    out.k = q.k + dp[2];
    out.phi = q.phi;
    out.pl = q.pl;
    add_ff(out.phi, out.pl, dp[3]);
    wrap_pi_ff(out.phi, out.pl);
    out.th = q.th;
    out.tl = q.tl;
    add_ff(out.th, out.tl, dp[4]);
    embed_cov(f, cn, out.c);
    return out.th > F(0) && out.th < Phys<F>::pi;
}

// The same with the surface frame built from the prediction.
template <class F>
__device__ __forceinline__ bool kalman_update(int kind, const PredT<F>& q, F mx, F my, F mz, const F v[6],
                                              StateT<F>& out, float* kappa = nullptr, const F* dm = nullptr) {
    return kalman_update_f(frame_of(kind, q), q, mx, my, mz, v, out, kappa, dm);
}

// Kalman update of a global-frame state that is not constrained to a surface (the first hit of
// a seed, whose starting covariance is a diagonal prior): Joseph form in global coordinates.
template <class F>
__device__ __forceinline__ bool state_update(StateT<F>& t, F mx, F my, F mz, const F v[6], F* chi2 = nullptr) {
    F S[6], L[6], inv[3];
#pragma unroll
    for (int i = 0; i < 6; ++i) S[i] = t.c[i] + v[i];
    if (!chol3(S, L, inv)) return false;
    const F r[3] = {sub_rn(sub_rn(mx, t.xh), t.xl), sub_rn(sub_rn(my, t.yh), t.yl), sub_rn(sub_rn(mz, t.zh), t.zl)};
    if (chi2) {   // r^T S^-1 r = |L^-1 r|^2
        const F y0 = r[0] * inv[0];
        const F y1 = (r[1] - L[1] * y0) * inv[1];
        const F y2 = (r[2] - L[3] * y0 - L[4] * y1) * inv[2];
        *chi2 = y0 * y0 + y1 * y1 + y2 * y2;
    }
    const F i00 = inv[0], i11 = inv[1], i22 = inv[2];
    const F i10 = -L[1] * i00 * i11;
    const F i21 = -L[4] * i11 * i22;
    const F i20 = -(L[3] * i00 + L[4] * i10) * i22;
    const F W[3][3] = {{i00 * i00 + i10 * i10 + i20 * i20, i10 * i11 + i20 * i21, i20 * i22},
                       {i10 * i11 + i20 * i21, i11 * i11 + i21 * i21, i21 * i22},
                       {i20 * i22, i21 * i22, i22 * i22}};
    F K[6][3];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            F acc = F(0);
#pragma unroll
            for (int b = 0; b < 3; ++b) acc = fma(t.c[ix(i, b)], W[b][a], acc);
            K[i][a] = acc;
        }
    F dp[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) dp[i] = fma(K[i][0], r[0], fma(K[i][1], r[1], K[i][2] * r[2]));
    F T[6][6];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            F acc = t.c[ix(i, j)];
#pragma unroll
            for (int a = 0; a < 3; ++a) acc = fma(-K[i][a], t.c[ix(a, j)], acc);
            T[i][j] = acc;
        }
    const F V[3][3] = {{v[0], v[1], v[3]}, {v[1], v[2], v[4]}, {v[3], v[4], v[5]}};
    F KV[6][3];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a) KV[i][a] = fma(K[i][0], V[0][a], fma(K[i][1], V[1][a], K[i][2] * V[2][a]));
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            F acc = T[i][j];
#pragma unroll
            for (int a = 0; a < 3; ++a) acc = fma(KV[i][a] - T[i][a], K[j][a], acc);
            t.c[ix(i, j)] = acc;
        }
    add_ff(t.xh, t.xl, dp[0]);
    add_ff(t.yh, t.yl, dp[1]);
    add_ff(t.zh, t.zl, dp[2]);
    t.k += dp[3];
    add_ff(t.phi, t.pl, dp[4]);
    wrap_pi_ff(t.phi, t.pl);
    add_ff(t.th, t.tl, dp[5]);
    return t.th > F(0) && t.th < Phys<F>::pi;
}

// ----------------------------------------------------------------- state I/O and conversion

template <class F, class G> __device__ __forceinline__ void load_state6(const G* p, const G* c, StateT<F>& t) {
    t.xh = F(p[0]); t.yh = F(p[1]); t.zh = F(p[2]);
    t.xl = F(0); t.yl = F(0); t.zl = F(0);
    t.k = F(p[3]); t.phi = F(p[4]); t.th = F(p[5]); t.tl = F(0); t.pl = F(0);
#pragma unroll
    for (int i = 0; i < 21; ++i) t.c[i] = F(c[i]);
}

template <class F> __device__ __forceinline__ void store_state6(const StateT<F>& t, float* p, float* c) {
    p[0] = float(t.xh + t.xl); p[1] = float(t.yh + t.yl); p[2] = float(t.zh + t.zl);
    p[3] = float(t.k); p[4] = float(t.phi + t.pl); p[5] = float(t.th + t.tl);
#pragma unroll
    for (int i = 0; i < 21; ++i) c[i] = float(t.c[i]);
}

// double state -> float state: positions split into hi + lo
__device__ __forceinline__ void narrow_state(const StateT<double>& d, State& t) {
    const double x = d.xh + d.xl, y = d.yh + d.yl, z = d.zh + d.zl;
    t.xh = float(x); t.xl = float(x - double(t.xh));
    t.yh = float(y); t.yl = float(y - double(t.yh));
    t.zh = float(z); t.zl = float(z - double(t.zh));
    const double th = d.th + d.tl, ph = d.phi + d.pl;
    t.k = float(d.k); t.th = float(th); t.tl = float(th - double(t.th));
    t.phi = float(ph); t.pl = float(ph - double(t.phi));
#pragma unroll
    for (int i = 0; i < 21; ++i) t.c[i] = float(d.c[i]);
}

// Hit payload: 3 x float4 = (x, y, z, id) (v0, v1, v2, v3) (v4, v5, module, -); module -1: the hit
// lies on its layer's own surface
template <class F>
__device__ __forceinline__ void load_hit(const float4* __restrict__ pay, long long q, F m[3], F v[6], int* id,
                                         int* mod = nullptr) {
    const float4 a = __ldg(pay + 3 * q), b = __ldg(pay + 3 * q + 1), c = __ldg(pay + 3 * q + 2);
    m[0] = F(a.x); m[1] = F(a.y); m[2] = F(a.z);
    if (id) *id = __float_as_int(a.w);
    if (mod) *mod = __float_as_int(c.z);
    v[0] = F(b.x); v[1] = F(b.y); v[2] = F(b.z); v[3] = F(b.w); v[4] = F(c.x); v[5] = F(c.y);
}

}  // namespace mk

namespace mk {
// The FP32 image of a state of any precision (a float state is copied).
__device__ __forceinline__ void narrow_to_fp32(const StateT<double>& d, State& t) { narrow_state(d, t); }
__device__ __forceinline__ void narrow_to_fp32(const State& d, State& t) { t = d; }
template <class T, int K> __device__ __forceinline__ void narrow_to_fp32(const StateT<Dual<T, K>>& d, State& t) {
    t.xh = float(d.xh); t.yh = float(d.yh); t.zh = float(d.zh);
    t.xl = float(d.xl); t.yl = float(d.yl); t.zl = float(d.zl);
    t.k = float(d.k); t.phi = float(d.phi); t.th = float(d.th); t.tl = float(d.tl); t.pl = float(d.pl);
#pragma unroll
    for (int i = 0; i < 21; ++i) t.c[i] = float(d.c[i]);
}
}  // namespace mk

namespace mk {
template <class F>
__device__ __forceinline__ int propagate_refined(const DevLayer& L, float cBf, int material, const StateT<F>& t,
                                                 PredT<F>& q, int& newton_it, bool fast, F* dir) {
    F sg = F(0);
    bool have = false;
    if (fast) {
        State t32;
        narrow_to_fp32(t, t32);
        Pred q32;
        float s32 = 0.0f;
        int nw = 0;
        if (propagate_core<float, float>(L, cBf, 0, t32, t32.c, q32, q32.c, nw, nullptr, nullptr, nullptr, &s32) == 1) {
            sg = F(s32);
            have = true;
        }
    }
    return propagate_core<F, F>(L, cBf, material, t, t.c, q, q.c, newton_it, dir, nullptr, have ? &sg : nullptr,
                                nullptr, fast);
}
}  // namespace mk

namespace mk {
// Kalman update with a hit at the state's own position under a prior whose position block is
// diagonal and uncorrelated with the other parameters (the seed fit's first hit): the residual is
// zero and only the position block changes, to C' = C0 S^-1 V with S = C0 + V (the same matrix
// as C0 - C0 S^-1 C0, without its cancellation).  Returns false if S is not positive definite.
template <class F> __device__ __forceinline__ bool prior_update_at_hit(StateT<F>& t, const F v[6]) {
    const F c0[3] = {t.c[ix(0, 0)], t.c[ix(1, 1)], t.c[ix(2, 2)]};
    F S[6], L[6], inv[3];
#pragma unroll
    for (int i = 0; i < 6; ++i) S[i] = v[i];
    S[ix(0, 0)] += c0[0]; S[ix(1, 1)] += c0[1]; S[ix(2, 2)] += c0[2];
    if (!chol3(S, L, inv)) return false;
    const F Vm[3][3] = {{v[0], v[1], v[3]}, {v[1], v[2], v[4]}, {v[3], v[4], v[5]}};
    F X[3][3];   // S^-1 V by forward and back substitution with L (L[0], L[2], L[5] diagonal)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const F y0 = Vm[0][c] * inv[0];
        const F y1 = (Vm[1][c] - L[1] * y0) * inv[1];
        const F y2 = (Vm[2][c] - L[3] * y0 - L[4] * y1) * inv[2];
        X[2][c] = y2 * inv[2];
        X[1][c] = (y1 - L[4] * X[2][c]) * inv[1];
        X[0][c] = (y0 - L[1] * X[1][c] - L[3] * X[2][c]) * inv[0];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) t.c[ix(i, j)] = F(0.5) * (c0[i] * X[i][j] + c0[j] * X[j][i]);
    return true;
}
}  // namespace mk
