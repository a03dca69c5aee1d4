// Device-side Kalman step for one track candidate per CUDA lane (sm_103a, FP32).
//
// Propagation to a barrel cylinder or endcap disk in a uniform solenoid field with its
// 6x6 Jacobian, covariance transport J C J^T, multiple scattering and mean energy loss
// (a4-a7), the eta-phi window (a8), the 3D chi2 (a9) and the Joseph-form gain/update
// (a11).  The paper (Sec. 3.1) names propagation, hit selection and the Kalman filter
// calculations as the per-layer work; the formulas are the textbook ones it cites.
//
// Precision: all arithmetic is FP32 except the track position, which is carried as an
// unevaluated sum hi + lo of two floats.  Positions reach |z| = 275 cm where one FP32 ulp
// is 15 nm, comparable to the 1e-3 chi2 tolerance on 30 um hits; the compensated sum keeps
// the predicted residual m - x' exact to ~1e-12 relative, and the crossing equation is
// written relative to the current position so its terms stay small.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mkgb.h"

namespace mk {

constexpr float kCLight = 0.00299792458f;   // curvature [1/cm] per (T / GeV)
constexpr float kMPion = 0.13957039f;        // GeV
constexpr float kMElec = 0.51099895e-3f;     // GeV
constexpr float kSiK = 0.307075f;            // MeV cm^2/mol
constexpr float kSiZA = 0.49848f;
constexpr float kSiRho = 2.329f;             // g/cm^3
constexpr float kSiX0 = 9.37f;               // cm
constexpr float kSiI = 173.0e-9f;            // GeV
constexpr float kIncCap = 10.0f;
constexpr float kPi = 3.14159265358979f;
constexpr float kTwoPi = 6.28318530717959f;

struct DevLayer {
    int kind;
    float pos, lo, hi, xx0;
    float sig[3];
    int n_eta, n_phi;
    float eta_lo, eta_scale;   // bin = floor((eta - eta_lo) * eta_scale)
    int bin_base;              // first bin of this layer inside an event's bin block
    int pad;
};

struct DevGeom {
    int n_layers, n_regions, bins_per_event, max_plan;
    float bz, cB, barrel_eta_max, pad;
    DevLayer layers[MKGB_MAX_LAYERS];
    int plan_off[MKGB_MAX_REGIONS + 1];
    int plan[MKGB_MAX_REGIONS * MKGB_MAX_PLAN];
};

struct DevParams {
    float chi2_cut;
    int max_cands, max_holes, material;
    float nsig, deta_min, deta_max, dphi_min, dphi_max;
    float score_hit, score_hole, barrel_eta_max;
};

// Packed lower-triangle index of a symmetric 6x6 (i, j in 0..5).
__host__ __device__ constexpr int ix(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

struct State {
    float xh, yh, zh;   // position, high part
    float xl, yl, zl;   // position, low part (|lo| <= ulp(hi)/2)
    float k, phi, th;   // q/pT, direction phi, polar angle
    float c[21];        // covariance of (x, y, z, k, phi, theta), packed
};

// ----------------------------------------------------------------- compensated sums

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) += d, renormalised.
__device__ __forceinline__ void add_ff(float& hi, float& lo, float d) {
    float s, e;
    two_sum(hi, d, s, e);
    e = __fadd_rn(e, lo);
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// R^2 - (x^2 + y^2) for x = xh + xl, y = yh + yl, with the squares split exactly by FMA.
__device__ __forceinline__ float r2_gap(float R, float xh, float xl, float yh, float yl) {
    float pR = __fmul_rn(R, R), eR = __fmaf_rn(R, R, -pR);
    float p1 = __fmul_rn(xh, xh), e1 = __fmaf_rn(xh, xh, -p1);
    float p2 = __fmul_rn(yh, yh), e2 = __fmaf_rn(yh, yh, -p2);
    float s1, t1, s2, t2;
    two_sum(pR, -p1, s1, t1);
    two_sum(s1, -p2, s2, t2);
    float tail = __fadd_rn(__fadd_rn(t1, t2), __fsub_rn(__fsub_rn(eR, e1), e2));
    tail = __fsub_rn(tail, 2.0f * (xh * xl + yh * yl));
    return __fadd_rn(s2, tail);
}

__device__ __forceinline__ float wrap_pi(float a) {
    // into (-pi, pi]
    a = a - kTwoPi * rintf(a * (1.0f / kTwoPi));
    if (a <= -kPi) a += kTwoPi;
    if (a > kPi) a -= kTwoPi;
    return a;
}

// sin(a)/a and (1 - cos a)/a.
__device__ __forceinline__ void s1c1(float a, float& S1, float& C1) {
    if (fabsf(a) < 1e-4f) {
        S1 = 1.0f - a * a * (1.0f / 6.0f);
        C1 = a * (0.5f - a * a * (1.0f / 24.0f));
    } else {
        float sh, ch;
        sincosf(0.5f * a, &sh, &ch);
        float inv = 1.0f / a;
        S1 = 2.0f * sh * ch * inv;
        C1 = 2.0f * sh * sh * inv;
    }
}

// sin(a/2) / (a/2)
__device__ __forceinline__ float sinc_half(float a) {
    const float h = 0.5f * a;
    if (fabsf(h) < 0.05f) {
        const float h2 = h * h;
        return 1.0f + h2 * (-1.0f / 6.0f + h2 * (1.0f / 120.0f - h2 * (1.0f / 5040.0f)));
    }
    return sinf(h) / h;
}

// Derivatives of S1 and C1 with respect to a (power series below |a| = 0.3).
__device__ __forceinline__ void s1c1_deriv(float a, float S1, float C1, float& dS1, float& dC1) {
    if (fabsf(a) < 0.3f) {
        float a2 = a * a;
        dS1 = a * (-1.0f / 3.0f + a2 * (1.0f / 30.0f + a2 * (-1.0f / 840.0f + a2 * (1.0f / 45360.0f - a2 * (1.0f / 3991680.0f)))));
        dC1 = 0.5f + a2 * (-1.0f / 8.0f + a2 * (1.0f / 144.0f + a2 * (-1.0f / 5760.0f + a2 * (1.0f / 403200.0f))));
    } else {
        float inv = 1.0f / a;
        float sa = S1 * a, ca = 1.0f - C1 * a;   // sin(a), cos(a)
        dS1 = (ca - S1) * inv;
        dC1 = (sa - C1) * inv;
    }
}

// ----------------------------------------------------------------- predicted state in the surface frame
//
// At a layer surface the predicted position has no spread along the surface normal (the
// crossing is constrained to the surface).  With a large spread along the surface (a grazing
// crossing of a curling track) a global FP32 covariance carries rounding of ~1e-7 of that
// spread in the normal direction, comparable to the hit's own normal variance.  The
// predicted covariance is therefore kept in surface coordinates (u1, u2, k, phi, theta),
// 15 packed floats whose normal row is exactly zero, and the chi2 and the update are
// evaluated in the local measurement frame (n, e1, e2):
//   barrel: n = (x, y, 0)/r, e1 = (-y, x, 0)/r, e2 = z-hat;   disk: n = z-hat, e1 = x-hat, e2 = y-hat.

struct Pred {
    float xh, yh, zh, xl, yl, zl, k, phi, th;
    float c[15];   // covariance of (u1, u2, k, phi, theta), packed like ix()
};

struct Frame {
    float c, s;    // barrel: n = (c, s, 0); unused for disks
    int disk;
};

__device__ __forceinline__ Frame frame_of(int kind, float x, float y) {
    Frame f;
    f.disk = kind == MKGB_DISK;
    const float ir = rsqrtf(x * x + y * y);
    f.c = x * ir;
    f.s = y * ir;
    return f;
}

// global 3-vector -> local (n, e1, e2) components
__device__ __forceinline__ void to_local3(const Frame& f, const float g[3], float l[3]) {
    if (f.disk) {
        l[0] = g[2]; l[1] = g[0]; l[2] = g[1];
    } else {
        l[0] = f.c * g[0] + f.s * g[1];
        l[1] = -f.s * g[0] + f.c * g[1];
        l[2] = g[2];
    }
}

// surface displacement (d1 along e1, d2 along e2) -> global
__device__ __forceinline__ void surface_to_global(const Frame& f, float d1, float d2, float g[3]) {
    if (f.disk) {
        g[0] = d1; g[1] = d2; g[2] = 0.0f;
    } else {
        g[0] = -f.s * d1; g[1] = f.c * d1; g[2] = d2;
    }
}

// packed 3x3 symmetric (xx, yx, yy, zx, zy, zz) global -> local frame
__device__ __forceinline__ void to_local_sym3(const Frame& f, const float v[6], float w[6]) {
    if (f.disk) {   // (n, e1, e2) = (z, x, y)
        w[0] = v[5]; w[1] = v[3]; w[2] = v[0]; w[3] = v[4]; w[4] = v[1]; w[5] = v[2];
    } else {
        const float c = f.c, s = f.s, cc = c * c, ss = s * s, cs = c * s;
        w[0] = cc * v[0] + 2.0f * cs * v[1] + ss * v[2];              // nn
        w[1] = cs * (v[2] - v[0]) + (cc - ss) * v[1];                 // e1 n
        w[2] = ss * v[0] - 2.0f * cs * v[1] + cc * v[2];              // e1 e1
        w[3] = c * v[3] + s * v[4];                                   // e2 n
        w[4] = -s * v[3] + c * v[4];                                  // e2 e1
        w[5] = v[5];                                                  // e2 e2
    }
}

// Surface-frame covariance (15) -> global state covariance (21).
__device__ __forceinline__ void embed_cov(const Frame& f, const float q[15], float c[21]) {
    // columns of E (3x2): e1, e2
    float E[3][2];
    if (f.disk) {
        E[0][0] = 1.0f; E[0][1] = 0.0f; E[1][0] = 0.0f; E[1][1] = 1.0f; E[2][0] = 0.0f; E[2][1] = 0.0f;
    } else {
        E[0][0] = -f.s; E[0][1] = 0.0f; E[1][0] = f.c; E[1][1] = 0.0f; E[2][0] = 0.0f; E[2][1] = 1.0f;
    }
    const float cuu[2][2] = {{q[0], q[1]}, {q[1], q[2]}};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float m0 = E[i][0] * cuu[0][0] + E[i][1] * cuu[1][0];
        const float m1 = E[i][0] * cuu[0][1] + E[i][1] * cuu[1][1];
#pragma unroll
        for (int j = 0; j <= i; ++j) c[ix(i, j)] = m0 * E[j][0] + m1 * E[j][1];
        // position x (k, phi, theta): local indices 2, 3, 4
#pragma unroll
        for (int o = 0; o < 3; ++o) c[ix(3 + o, i)] = E[i][0] * q[ix(2 + o, 0)] + E[i][1] * q[ix(2 + o, 1)];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) c[ix(3 + a, 3 + b)] = q[ix(2 + a, 2 + b)];
}

__device__ __forceinline__ void pred_to_state(int kind, const Pred& q, State& t) {
    t.xh = q.xh; t.yh = q.yh; t.zh = q.zh; t.xl = q.xl; t.yl = q.yl; t.zl = q.zl;
    t.k = q.k; t.phi = q.phi; t.th = q.th;
    embed_cov(frame_of(kind, q.xh, q.yh), q.c, t.c);
}

// ----------------------------------------------------------------- propagation (a4-a7)

__device__ __forceinline__ float R_of(const DevLayer& L) { return L.pos; }

// Material of layer L at the predicted state: Highland Q on (k, phi, theta) and mean energy loss
// scaling k and its row/column.  Returns false if the particle stops.
__device__ __forceinline__ bool apply_material(const DevLayer& L, Pred& q, float st, float ct, float sfp,
                                               float cfp) {
    float cosi;
    if (L.kind == MKGB_BARREL) {
        const float ir = rsqrtf(q.xh * q.xh + q.yh * q.yh);
        cosi = fabsf((q.xh * cfp + q.yh * sfp) * st * ir);
    } else {
        cosi = fabsf(ct);
    }
    const float fac = (cosi * kIncCap > 1.0f) ? 1.0f / cosi : kIncCap;
    const float tt = L.xx0 * fac;
    const float k = q.k;
    if (!(tt > 0.0f) || k == 0.0f) return true;
    const float pm = 1.0f / (fabsf(k) * st);
    const float e2 = pm * pm + kMPion * kMPion;
    const float beta2 = pm * pm / e2;
    const float beta = sqrtf(beta2);
    const float th0 = 0.0136f / (beta * pm) * sqrtf(tt) * (1.0f + 0.038f * logf(tt / beta2));
    const float th02 = th0 * th0;
    const float kc = k * (ct / st);
    q.c[ix(3, 3)] += th02 / (st * st);
    q.c[ix(4, 4)] += th02;
    q.c[ix(2, 2)] += kc * kc * th02;
    q.c[ix(4, 2)] -= kc * th02;
    // PDG Bethe-Bloch mean energy loss in silicon (no density effect)
    const float e = sqrtf(e2);
    const float bg2 = pm * pm * (1.0f / (kMPion * kMPion));
    const float gam = e * (1.0f / kMPion);
    const float rme = kMElec / kMPion;
    const float tmax = 2.0f * kMElec * bg2 / (1.0f + 2.0f * gam * rme + rme * rme);
    const float dedx = kSiK * kSiZA / beta2 * (0.5f * logf(2.0f * kMElec * bg2 * tmax / (kSiI * kSiI)) - beta2);
    const float de = dedx * kSiRho * (tt * kSiX0) * 1e-3f;
    const float en = e - de;
    if (!(en > kMPion)) return false;
    const float a = pm / sqrtf((en - kMPion) * (en + kMPion));
    q.k = k * a;
    q.c[ix(2, 0)] *= a; q.c[ix(2, 1)] *= a; q.c[ix(3, 2)] *= a; q.c[ix(4, 2)] *= a;
    q.c[ix(2, 2)] *= a * a;
    return true;
}

// Propagates t to layer L.  Returns 1 (crossed; q holds the predicted state with material),
// 0 (not crossed) or -1 (particle stopped in the material).  newton_it counts iterations.
__device__ __forceinline__ int propagate(const DevLayer& L, float cB, int material, const State& t, Pred& q,
                                         int& newton_it) {
    float sf, cf, st, ct;
    sincosf(t.phi, &sf, &cf);
    sincosf(t.th, &st, &ct);
    const float om = -cB * t.k;
    const float ux = t.xh + t.xl, uy = t.yh + t.yl;
    float s, S1, C1, dx, dy;
    if (L.kind == MKGB_BARREL) {
        const float R = L.pos;
        const float c0 = r2_gap(R, t.xh, t.xl, t.yh, t.yl);   // R^2 - |u|^2
        if (!(c0 > 0.0f)) return 0;
        const float b = ux * cf + uy * sf;
        const float sq = sqrtf(b * b + c0);
        const float s0 = (b > 0.0f) ? c0 / (b + sq) : sq - b;
        float lo = 0.0f, hi = 3.0e38f;
        if (fabsf(om) > 1e-12f) {
            const float inv = 1.0f / om;
            const float cx = ux - sf * inv, cy = uy + cf * inv;
            const float rho = fabsf(inv);
            const float reach = sqrtf(cx * cx + cy * cy) + rho - R;
            if (reach < 0.0f) return 0;
            const float sg = om > 0.0f ? 1.0f : -1.0f;
            float turn = (atan2f(sg * cx, -sg * cy) - t.phi) * sg;
            turn -= kTwoPi * floorf(turn * (1.0f / kTwoPi));
            hi = turn * rho;
        }
        s = (s0 > lo && s0 < hi) ? s0 : 0.5f * (lo + hi);
        for (int it = 0; it < 40; ++it) {
            ++newton_it;
            s1c1(om * s, S1, C1);
            dx = s * (cf * S1 - sf * C1);
            dy = s * (sf * S1 + cf * C1);
            // g(s) = |u + d|^2 - R^2 = 2 u.d + |d|^2 - c0 (terms of size |u||d|, not R^2)
            const float g = 2.0f * (ux * dx + uy * dy) + (dx * dx + dy * dy) - c0;
            if (g == 0.0f) break;
            if (g < 0.0f) lo = s; else hi = s;
            float spn, cpn;
            sincosf(t.phi + om * s, &spn, &cpn);
            const float dg = 2.0f * ((ux + dx) * cpn + (uy + dy) * spn);
            float sn = (dg > 0.0f) ? s - g / dg : 0.5f * (lo + hi);
            if (!(sn >= lo && sn <= hi)) sn = 0.5f * (lo + hi);
            const float ds = sn - s;
            s = sn;
            if (fabsf(ds) <= 1e-6f * s) break;
        }
    } else {
        if (fabsf(ct) < 1e-7f) return 0;
        const float dzp = __fsub_rn(__fsub_rn(L.pos, t.zh), t.zl);
        s = dzp * st / ct;
        if (!(s > 0.0f)) return 0;
        // loopers are followed on the outgoing part of their current turn only: the disk must be
        // reached before the next point of largest radius (and moving outward, checked below)
        if (fabsf(om) > 1e-12f) {
            const float inv = 1.0f / om;
            const float cx = ux - sf * inv, cy = uy + cf * inv;
            const float sg = om > 0.0f ? 1.0f : -1.0f;
            float turn = (atan2f(sg * cx, -sg * cy) - t.phi) * sg;
            turn -= kTwoPi * floorf(turn * (1.0f / kTwoPi));
            if (s > turn * fabsf(inv)) return 0;
        }
    }
    const float a = om * s;
    s1c1(a, S1, C1);
    {
        // chord form: d = s sinc(a/2) (cos psi, sin psi) with psi = phi + a/2 kept as an unrounded
        // sum; sin and cos of psi get the first-order correction for its low part
        float psh, psl;
        two_sum(t.phi, 0.5f * a, psh, psl);
        float sp, cp;
        sincosf(psh, &sp, &cp);
        const float chord = s * sinc_half(a);
        const float cpc = fmaf(-sp, psl, cp), spc = fmaf(cp, psl, sp);
        dx = chord * cpc;
        dy = chord * spc;
    }
    const float cot = ct / st;
    const float dz = (L.kind == MKGB_BARREL) ? s * cot : __fsub_rn(__fsub_rn(L.pos, t.zh), t.zl);
    float xh = t.xh, xl = t.xl, yh = t.yh, yl = t.yl, zh = t.zh, zl = t.zl;
    add_ff(xh, xl, dx);
    add_ff(yh, yl, dy);
    add_ff(zh, zl, dz);
    if (L.kind == MKGB_BARREL) {
        // polish: the FP32 Newton residual carries ~1e-7 |u||d| of rounding, i.e. the point sits
        // up to a few 1e-6 cm off the cylinder along the normal (where the hit error is 30 um);
        // the gap R^2 - r'^2 of the compensated position is exact to ~1e-10, so one more step
        // along the track puts the predicted point on the surface
        float spn, cpn;
        sincosf(t.phi + a, &spn, &cpn);
        const float gap = r2_gap(R_of(L), xh, xl, yh, yl);
        const float dsp = gap / (2.0f * (xh * cpn + yh * spn));
        add_ff(xh, xl, dsp * cpn);
        add_ff(yh, yl, dsp * spn);
        add_ff(zh, zl, dsp * cot);
        if (!(zh >= L.lo && zh <= L.hi)) return 0;
    } else {
        const float r = sqrtf(xh * xh + yh * yh);
        if (!(r >= L.lo && r <= L.hi)) return 0;
    }
    const float phin = t.phi + a;
    float sfp, cfp;
    sincosf(phin, &sfp, &cfp);
    if (L.kind == MKGB_DISK && xh * cfp + yh * sfp < 0.0f) return 0;   // moving inward: past the apex

    // ---- Jacobian rows x, y, z, phi: J = A + (df/ds)(ds/dp); rows k, theta are identity
    float dS1, dC1;
    s1c1_deriv(a, S1, C1, dS1, dC1);
    const float A03 = -cB * s * s * (cf * dS1 - sf * dC1);
    const float A13 = -cB * s * s * (sf * dS1 + cf * dC1);
    const float A04 = -dy, A14 = dx;
    const float A25 = -s / (st * st);
    const float A43 = -cB * s;
    const Frame fr = frame_of(L.kind, xh, yh);
    float ds[6];
    if (L.kind == MKGB_BARREL) {
        const float ig = -1.0f / (xh * cfp + yh * sfp);
        ds[0] = xh * ig; ds[1] = yh * ig; ds[2] = 0.0f;
        ds[3] = (xh * A03 + yh * A13) * ig;
        ds[4] = (xh * A04 + yh * A14) * ig;
        ds[5] = 0.0f;
    } else {
        const float ig = -1.0f / cot;
        ds[0] = 0.0f; ds[1] = 0.0f; ds[2] = ig;
        ds[3] = 0.0f; ds[4] = 0.0f; ds[5] = A25 * ig;
    }
    // surface rows: barrel u1 = -s x + c y (along e1), u2 = z; disk u1 = x, u2 = y.  The row
    // along the normal vanishes by the surface constraint and is not formed.
    const float f1 = fr.disk ? cfp : (-fr.s * cfp + fr.c * sfp);
    const float f2 = fr.disk ? sfp : cot;
    const float fs[3] = {f1, f2, om};   // df/ds along u1, u2, phi
    float J[3][6];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int j = 0; j < 6; ++j) J[r][j] = fs[r] * ds[j];
    if (fr.disk) {
        J[0][0] += 1.0f; J[0][3] += A03; J[0][4] += A04;
        J[1][1] += 1.0f; J[1][3] += A13; J[1][4] += A14;
    } else {
        J[0][0] -= fr.s; J[0][1] += fr.c; J[0][3] += -fr.s * A03 + fr.c * A13; J[0][4] += -fr.s * A04 + fr.c * A14;
        J[1][2] += 1.0f; J[1][5] += A25;
    }
    J[2][3] += A43; J[2][4] += 1.0f;

    // ---- transport into the surface frame: rows (u1, u2, phi) dense, (k, theta) identity
    constexpr int D[3] = {0, 1, 3};   // local indices of the dense rows
    float T[3][6];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            float acc = 0.0f;
#pragma unroll
            for (int l = 0; l < 6; ++l) acc = fmaf(J[r][l], t.c[ix(l, j)], acc);
            T[r][j] = acc;
        }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int p = 0; p <= r; ++p) {
            float acc = 0.0f;
#pragma unroll
            for (int l = 0; l < 6; ++l) acc = fmaf(T[r][l], J[p][l], acc);
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
    q.phi = wrap_pi(phin);
    q.th = t.th;
    if (material && !apply_material(L, q, st, ct, sfp, cfp)) return -1;
    return 1;
}

// ----------------------------------------------------------------- window (a8)

struct Window {
    float eta, phi, deta, dphi;
};

__device__ __forceinline__ Window window(const DevLayer& L, const DevParams& P, const Pred& q) {
    const float x = q.xh, y = q.yh, z = q.zh;
    const float rt2 = x * x + y * y, rt = sqrtf(rt2), r3 = sqrtf(rt2 + z * z);
    Window w;
    w.eta = asinhf(z / rt);
    w.phi = atan2f(y, x);
    const float c = x / rt, sn = y / rt;
    // gradients in (r-hat, phi-hat, z-hat) at the predicted point
    const float ge_r = -z / (rt * r3), ge_z = 1.0f / r3;
    const float gp_p = 1.0f / rt;
    const float sr2 = L.sig[0] * L.sig[0], sp2 = L.sig[1] * L.sig[1], sz2 = L.sig[2] * L.sig[2];
    float ve = ge_r * ge_r * sr2 + ge_z * ge_z * sz2;
    float vp = gp_p * gp_p * sp2;
    // surface part: gradient components along e1, e2
    float ge1, ge2, gp1, gp2;
    if (L.kind == MKGB_DISK) {         // e1 = x-hat, e2 = y-hat
        ge1 = ge_r * c; ge2 = ge_r * sn;
        gp1 = -gp_p * sn; gp2 = gp_p * c;
    } else {                           // e1 = phi-hat, e2 = z-hat
        ge1 = 0.0f; ge2 = ge_z;
        gp1 = gp_p; gp2 = 0.0f;
    }
    ve += ge1 * ge1 * q.c[0] + 2.0f * ge1 * ge2 * q.c[1] + ge2 * ge2 * q.c[2];
    vp += gp1 * gp1 * q.c[0] + 2.0f * gp1 * gp2 * q.c[1] + gp2 * gp2 * q.c[2];
    w.deta = fminf(fmaxf(P.nsig * sqrtf(fmaxf(ve, 0.0f)), P.deta_min), P.deta_max);
    w.dphi = fminf(fmaxf(P.nsig * sqrtf(fmaxf(vp, 0.0f)), P.dphi_min), P.dphi_max);
    return w;
}

// ----------------------------------------------------------------- chi2 (a9) and update (a11)

// Cholesky of a packed 3x3; inv[] gets 1/L_ii.  Returns false if not positive definite.
__device__ __forceinline__ bool chol3(const float S[6], float L[6], float inv[3]) {
    if (!(S[0] > 0.0f)) return false;
    inv[0] = rsqrtf(S[0]);
    const float l10 = S[1] * inv[0], l20 = S[3] * inv[0];
    const float d1 = S[2] - l10 * l10;
    if (!(d1 > 0.0f)) return false;
    inv[1] = rsqrtf(d1);
    const float l21 = (S[4] - l20 * l10) * inv[1];
    const float d2 = S[5] - l20 * l20 - l21 * l21;
    if (!(d2 > 0.0f)) return false;
    inv[2] = rsqrtf(d2);
    L[0] = S[0] * inv[0]; L[1] = l10; L[2] = d1 * inv[1]; L[3] = l20; L[4] = l21; L[5] = d2 * inv[2];
    return true;
}

// Residual m - x' (compensated position) and hit covariance in the local frame; S = V + C_surface.
__device__ __forceinline__ void local_meas(const Frame& f, const Pred& q, float mx, float my, float mz,
                                           const float v[6], float rl[3], float vl[6], float S[6]) {
    const float r[3] = {__fsub_rn(__fsub_rn(mx, q.xh), q.xl), __fsub_rn(__fsub_rn(my, q.yh), q.yl),
                        __fsub_rn(__fsub_rn(mz, q.zh), q.zl)};
    to_local3(f, r, rl);
    to_local_sym3(f, v, vl);
    S[0] = vl[0]; S[1] = vl[1]; S[3] = vl[3];
    S[2] = vl[2] + q.c[0]; S[4] = vl[4] + q.c[1]; S[5] = vl[5] + q.c[2];
}

__device__ __forceinline__ bool chi2_hit(int kind, const Pred& q, float mx, float my, float mz, const float v[6],
                                         float& chi2) {
    const Frame f = frame_of(kind, q.xh, q.yh);
    float rl[3], vl[6], S[6], L[6], inv[3];
    local_meas(f, q, mx, my, mz, v, rl, vl, S);
    if (!chol3(S, L, inv)) return false;
    const float y0 = rl[0] * inv[0];
    const float y1 = (rl[1] - L[1] * y0) * inv[1];
    const float y2 = (rl[2] - L[3] * y0 - L[4] * y1) * inv[2];
    chi2 = y0 * y0 + y1 * y1 + y2 * y2;
    return true;
}

// Kalman update of a predicted state with one hit, Joseph form in the surface frame:
// K = C H^T S^-1 (H picks u1, u2 into measurement rows e1, e2; the normal row is zero),
// C+ = (I - K H) C (I - K H)^T + K V K^T; the result is returned as a global-frame State.
// Returns false if S is not positive definite or theta leaves (0, pi).
__device__ __forceinline__ bool kalman_update(int kind, const Pred& q, float mx, float my, float mz,
                                              const float v[6], State& out) {
    const Frame f = frame_of(kind, q.xh, q.yh);
    float rl[3], vl[6], S[6], L[6], inv[3];
    local_meas(f, q, mx, my, mz, v, rl, vl, S);
    if (!chol3(S, L, inv)) return false;
    // W = S^-1 = L^-T L^-1
    const float i00 = inv[0], i11 = inv[1], i22 = inv[2];
    const float i10 = -L[1] * i00 * i11;
    const float i21 = -L[4] * i11 * i22;
    const float i20 = -(L[3] * i00 + L[4] * i10) * i22;
    const float W[3][3] = {{i00 * i00 + i10 * i10 + i20 * i20, i10 * i11 + i20 * i21, i20 * i22},
                           {i10 * i11 + i20 * i21, i11 * i11 + i21 * i21, i21 * i22},
                           {i20 * i22, i21 * i22, i22 * i22}};
    float K[5][3];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a) K[i][a] = fmaf(q.c[ix(i, 0)], W[1][a], q.c[ix(i, 1)] * W[2][a]);
    float dp[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) dp[i] = fmaf(K[i][0], rl[0], fmaf(K[i][1], rl[1], K[i][2] * rl[2]));
    // T = (I - K H) C : row i minus K_i1 * row u1 minus K_i2 * row u2
    float T[5][5];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j)
            T[i][j] = fmaf(-K[i][1], q.c[ix(0, j)], fmaf(-K[i][2], q.c[ix(1, j)], q.c[ix(i, j)]));
    const float V[3][3] = {{vl[0], vl[1], vl[3]}, {vl[1], vl[2], vl[4]}, {vl[3], vl[4], vl[5]}};
    float KV[5][3];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a) KV[i][a] = fmaf(K[i][0], V[0][a], fmaf(K[i][1], V[1][a], K[i][2] * V[2][a]));
    float cn[15];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            float acc = fmaf(-T[i][0], K[j][1], fmaf(-T[i][1], K[j][2], T[i][j]));
#pragma unroll
            for (int a = 0; a < 3; ++a) acc = fmaf(KV[i][a], K[j][a], acc);
            cn[ix(i, j)] = acc;
        }
    float dg[3];
    surface_to_global(f, dp[0], dp[1], dg);
    out.xh = q.xh; out.xl = q.xl; out.yh = q.yh; out.yl = q.yl; out.zh = q.zh; out.zl = q.zl;
    add_ff(out.xh, out.xl, dg[0]);
    add_ff(out.yh, out.yl, dg[1]);
    add_ff(out.zh, out.zl, dg[2]);
    out.k = q.k + dp[2];
    out.phi = wrap_pi(q.phi + dp[3]);
    out.th = q.th + dp[4];
    embed_cov(f, cn, out.c);
    return out.th > 0.0f && out.th < kPi;
}

// Kalman update of a global-frame state that is not constrained to a surface (the first hit of
// a seed, whose starting covariance is a diagonal prior): Joseph form in global coordinates.
__device__ __forceinline__ bool state_update(State& t, float mx, float my, float mz, const float v[6]) {
    float S[6], L[6], inv[3];
#pragma unroll
    for (int i = 0; i < 6; ++i) S[i] = t.c[i] + v[i];
    if (!chol3(S, L, inv)) return false;
    const float r[3] = {__fsub_rn(__fsub_rn(mx, t.xh), t.xl), __fsub_rn(__fsub_rn(my, t.yh), t.yl),
                        __fsub_rn(__fsub_rn(mz, t.zh), t.zl)};
    const float i00 = inv[0], i11 = inv[1], i22 = inv[2];
    const float i10 = -L[1] * i00 * i11;
    const float i21 = -L[4] * i11 * i22;
    const float i20 = -(L[3] * i00 + L[4] * i10) * i22;
    const float W[3][3] = {{i00 * i00 + i10 * i10 + i20 * i20, i10 * i11 + i20 * i21, i20 * i22},
                           {i10 * i11 + i20 * i21, i11 * i11 + i21 * i21, i21 * i22},
                           {i20 * i22, i21 * i22, i22 * i22}};
    float K[6][3];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float acc = 0.0f;
#pragma unroll
            for (int b = 0; b < 3; ++b) acc = fmaf(t.c[ix(i, b)], W[b][a], acc);
            K[i][a] = acc;
        }
    float dp[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) dp[i] = fmaf(K[i][0], r[0], fmaf(K[i][1], r[1], K[i][2] * r[2]));
    float T[6][6];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            float acc = t.c[ix(i, j)];
#pragma unroll
            for (int a = 0; a < 3; ++a) acc = fmaf(-K[i][a], t.c[ix(a, j)], acc);
            T[i][j] = acc;
        }
    const float V[3][3] = {{v[0], v[1], v[3]}, {v[1], v[2], v[4]}, {v[3], v[4], v[5]}};
    float KV[6][3];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a) KV[i][a] = fmaf(K[i][0], V[0][a], fmaf(K[i][1], V[1][a], K[i][2] * V[2][a]));
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            float acc = T[i][j];
#pragma unroll
            for (int a = 0; a < 3; ++a) acc = fmaf(KV[i][a] - T[i][a], K[j][a], acc);
            t.c[ix(i, j)] = acc;
        }
    add_ff(t.xh, t.xl, dp[0]);
    add_ff(t.yh, t.yl, dp[1]);
    add_ff(t.zh, t.zl, dp[2]);
    t.k += dp[3];
    t.phi = wrap_pi(t.phi + dp[4]);
    t.th += dp[5];
    return t.th > 0.0f && t.th < kPi;
}

// ----------------------------------------------------------------- state I/O

__device__ __forceinline__ void load_state6(const float* p, const float* c, State& t) {
    t.xh = p[0]; t.yh = p[1]; t.zh = p[2];
    t.xl = 0.0f; t.yl = 0.0f; t.zl = 0.0f;
    t.k = p[3]; t.phi = p[4]; t.th = p[5];
#pragma unroll
    for (int i = 0; i < 21; ++i) t.c[i] = c[i];
}

__device__ __forceinline__ void store_state6(const State& t, float* p, float* c) {
    p[0] = t.xh + t.xl; p[1] = t.yh + t.yl; p[2] = t.zh + t.zl;
    p[3] = t.k; p[4] = t.phi; p[5] = t.th;
#pragma unroll
    for (int i = 0; i < 21; ++i) c[i] = t.c[i];
}

// Hit payload: 3 x float4 = (x, y, z, id) (v0, v1, v2, v3) (v4, v5, -, -)
__device__ __forceinline__ void load_hit(const float4* __restrict__ pay, long long q, float m[3], float v[6],
                                         int* id) {
    const float4 a = __ldg(pay + 3 * q), b = __ldg(pay + 3 * q + 1), c = __ldg(pay + 3 * q + 2);
    m[0] = a.x; m[1] = a.y; m[2] = a.z;
    if (id) *id = __float_as_int(a.w);
    v[0] = b.x; v[1] = b.y; v[2] = b.z; v[3] = b.w; v[4] = c.x; v[5] = c.y;
}

}  // namespace mk
