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

// ----------------------------------------------------------------- propagation (a4-a7)

struct PropWork {
    int newton_it;
};

// Material of layer L at the (already propagated) state: Highland Q and mean energy loss.
// Returns false if the particle stops.
__device__ __forceinline__ bool apply_material(const DevLayer& L, State& t, float st, float ct,
                                               float sfp, float cfp) {
    float cosi;
    if (L.kind == MKGB_BARREL) {
        float r = sqrtf(t.xh * t.xh + t.yh * t.yh);
        cosi = fabsf((t.xh * cfp + t.yh * sfp) * st / r);
    } else {
        cosi = fabsf(ct);
    }
    float fac = (cosi * kIncCap > 1.0f) ? 1.0f / cosi : kIncCap;
    float tt = L.xx0 * fac;
    float k = t.k;
    if (!(tt > 0.0f) || k == 0.0f) return true;
    float pm = 1.0f / (fabsf(k) * st);
    float e2 = pm * pm + kMPion * kMPion;
    float beta2 = pm * pm / e2;
    float beta = sqrtf(beta2);
    float th0 = 0.0136f / (beta * pm) * sqrtf(tt) * (1.0f + 0.038f * logf(tt / beta2));
    float th02 = th0 * th0;
    float cot = ct / st;
    float kc = k * cot;
    t.c[ix(4, 4)] += th02 / (st * st);
    t.c[ix(5, 5)] += th02;
    t.c[ix(3, 3)] += kc * kc * th02;
    t.c[ix(5, 3)] -= kc * th02;
    // PDG Bethe-Bloch mean energy loss in silicon (no density effect)
    float e = sqrtf(e2);
    float bg2 = pm * pm * (1.0f / (kMPion * kMPion));
    float gam = e * (1.0f / kMPion);
    float rme = kMElec / kMPion;
    float tmax = 2.0f * kMElec * bg2 / (1.0f + 2.0f * gam * rme + rme * rme);
    float dedx = kSiK * kSiZA / beta2 * (0.5f * logf(2.0f * kMElec * bg2 * tmax / (kSiI * kSiI)) - beta2);
    float de = dedx * kSiRho * (tt * kSiX0) * 1e-3f;
    float en = e - de;
    if (!(en > kMPion)) return false;
    float p2 = sqrtf((en - kMPion) * (en + kMPion));
    float a = pm / p2;
    t.k = k * a;
#pragma unroll
    for (int j = 0; j < 6; ++j)
        if (j != 3) t.c[ix(3, j)] *= a;
    t.c[ix(3, 3)] *= a * a;
    return true;
}

// Propagates t to layer L.  Returns 1 (crossed; t holds the predicted state with material),
// 0 (not crossed; t unchanged) or -1 (particle stopped in the material).
__device__ __forceinline__ int propagate(const DevLayer& L, float cB, int material, State& t, int& newton_it) {
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
    }
    const float a = om * s;
    s1c1(a, S1, C1);
    dx = s * (cf * S1 - sf * C1);
    dy = s * (sf * S1 + cf * C1);
    const float cot = ct / st;
    const float dz = (L.kind == MKGB_BARREL) ? s * cot : __fsub_rn(__fsub_rn(L.pos, t.zh), t.zl);
    float xh = t.xh, xl = t.xl, yh = t.yh, yl = t.yl, zh = t.zh, zl = t.zl;
    add_ff(xh, xl, dx);
    add_ff(yh, yl, dy);
    add_ff(zh, zl, dz);
    if (L.kind == MKGB_BARREL) {
        if (!(zh >= L.lo && zh <= L.hi)) return 0;
    } else {
        const float r = sqrtf(xh * xh + yh * yh);
        if (!(r >= L.lo && r <= L.hi)) return 0;
    }
    const float phin = t.phi + a;
    float sfp, cfp;
    sincosf(phin, &sfp, &cfp);

    // ---- Jacobian: J = A + (df/ds)(ds/dp), rows x, y, z, phi dense; k, theta identity
    float dS1, dC1;
    s1c1_deriv(a, S1, C1, dS1, dC1);
    const float A03 = -cB * s * s * (cf * dS1 - sf * dC1);
    const float A13 = -cB * s * s * (sf * dS1 + cf * dC1);
    const float A04 = -dy, A14 = dx;
    const float A25 = -s / (st * st);
    const float A43 = -cB * s;
    float ds[6];
    if (L.kind == MKGB_BARREL) {
        const float gs = xh * cfp + yh * sfp;
        const float ig = -1.0f / gs;
        ds[0] = xh * ig; ds[1] = yh * ig; ds[2] = 0.0f;
        ds[3] = (xh * A03 + yh * A13) * ig;
        ds[4] = (xh * A04 + yh * A14) * ig;
        ds[5] = 0.0f;
    } else {
        const float ig = -1.0f / cot;
        ds[0] = 0.0f; ds[1] = 0.0f; ds[2] = ig;
        ds[3] = 0.0f; ds[4] = 0.0f; ds[5] = A25 * ig;
    }
    const float fs[4] = {cfp, sfp, cot, om};   // df/ds for rows x, y, z, phi
    float J[4][6];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int j = 0; j < 6; ++j) J[r][j] = fs[r] * ds[j];
    J[0][0] += 1.0f; J[0][3] += A03; J[0][4] += A04;
    J[1][1] += 1.0f; J[1][3] += A13; J[1][4] += A14;
    J[2][2] += 1.0f; J[2][5] += A25;
    J[3][3] += A43; J[3][4] += 1.0f;

    // ---- transport C' = J C J^T (dense rows D = {x, y, z, phi})
    constexpr int D[4] = {0, 1, 2, 4};
    float T[4][6];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            float acc = 0.0f;
#pragma unroll
            for (int l = 0; l < 6; ++l) acc = fmaf(J[r][l], t.c[ix(l, j)], acc);
            T[r][j] = acc;
        }
    float cn[21];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q <= r; ++q) {
            float acc = 0.0f;
#pragma unroll
            for (int l = 0; l < 6; ++l) acc = fmaf(T[r][l], J[q][l], acc);
            cn[ix(D[r], D[q])] = acc;
        }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        cn[ix(D[r], 3)] = T[r][3];
        cn[ix(D[r], 5)] = T[r][5];
    }
    cn[ix(3, 3)] = t.c[ix(3, 3)];
    cn[ix(5, 3)] = t.c[ix(5, 3)];
    cn[ix(5, 5)] = t.c[ix(5, 5)];
#pragma unroll
    for (int i = 0; i < 21; ++i) t.c[i] = cn[i];
    t.xh = xh; t.xl = xl; t.yh = yh; t.yl = yl; t.zh = zh; t.zl = zl;
    t.phi = wrap_pi(phin);
    if (material && !apply_material(L, t, st, ct, sfp, cfp)) return -1;
    return 1;
}

// ----------------------------------------------------------------- window (a8)

struct Window {
    float eta, phi, deta, dphi;
};

__device__ __forceinline__ Window window(const DevLayer& L, const DevParams& P, const State& t) {
    const float x = t.xh, y = t.yh, z = t.zh;
    const float rt2 = x * x + y * y, rt = sqrtf(rt2), r3 = sqrtf(rt2 + z * z);
    Window w;
    w.eta = asinhf(z / rt);
    w.phi = atan2f(y, x);
    const float irr = 1.0f / (rt2 * r3);
    const float ge0 = -z * x * irr, ge1 = -z * y * irr, ge2 = 1.0f / r3;
    const float gp0 = -y / rt2, gp1 = x / rt2;
    const float c = x / rt, sn = y / rt;
    const float sr2 = L.sig[0] * L.sig[0], sp2 = L.sig[1] * L.sig[1], sz2 = L.sig[2] * L.sig[2];
    const float m00 = t.c[0] + sr2 * c * c + sp2 * sn * sn;
    const float m10 = t.c[1] + (sr2 - sp2) * c * sn;
    const float m11 = t.c[2] + sr2 * sn * sn + sp2 * c * c;
    const float m20 = t.c[3], m21 = t.c[4], m22 = t.c[5] + sz2;
    const float ve = ge0 * ge0 * m00 + ge1 * ge1 * m11 + ge2 * ge2 * m22 +
                     2.0f * (ge0 * ge1 * m10 + ge0 * ge2 * m20 + ge1 * ge2 * m21);
    const float vp = gp0 * gp0 * m00 + gp1 * gp1 * m11 + 2.0f * gp0 * gp1 * m10;
    w.deta = fminf(fmaxf(P.nsig * sqrtf(fmaxf(ve, 0.0f)), P.deta_min), P.deta_max);
    w.dphi = fminf(fmaxf(P.nsig * sqrtf(fmaxf(vp, 0.0f)), P.dphi_min), P.dphi_max);
    return w;
}

// ----------------------------------------------------------------- chi2 (a9) and update (a11)

// Cholesky of S = C_pos + V.  Returns false if S is not positive definite.
__device__ __forceinline__ bool chol3(const float* c, const float v[6], float L[6], float inv[3]) {
    const float s00 = c[0] + v[0], s10 = c[1] + v[1], s11 = c[2] + v[2];
    const float s20 = c[3] + v[3], s21 = c[4] + v[4], s22 = c[5] + v[5];
    if (!(s00 > 0.0f)) return false;
    inv[0] = rsqrtf(s00);
    const float l00 = s00 * inv[0];
    const float l10 = s10 * inv[0], l20 = s20 * inv[0];
    const float d1 = s11 - l10 * l10;
    if (!(d1 > 0.0f)) return false;
    inv[1] = rsqrtf(d1);
    const float l11 = d1 * inv[1];
    const float l21 = (s21 - l20 * l10) * inv[1];
    const float d2 = s22 - l20 * l20 - l21 * l21;
    if (!(d2 > 0.0f)) return false;
    inv[2] = rsqrtf(d2);
    L[0] = l00; L[1] = l10; L[2] = l11; L[3] = l20; L[4] = l21; L[5] = d2 * inv[2];
    return true;
}

// Residual m - x' with the compensated position.
__device__ __forceinline__ void residual(const State& t, float mx, float my, float mz, float r[3]) {
    r[0] = __fsub_rn(__fsub_rn(mx, t.xh), t.xl);
    r[1] = __fsub_rn(__fsub_rn(my, t.yh), t.yl);
    r[2] = __fsub_rn(__fsub_rn(mz, t.zh), t.zl);
}

__device__ __forceinline__ bool chi2_hit(const State& t, float mx, float my, float mz, const float v[6],
                                         float& chi2) {
    float L[6], inv[3], r[3];
    if (!chol3(t.c, v, L, inv)) return false;
    residual(t, mx, my, mz, r);
    const float y0 = r[0] * inv[0];
    const float y1 = (r[1] - L[1] * y0) * inv[1];
    const float y2 = (r[2] - L[3] * y0 - L[4] * y1) * inv[2];
    chi2 = y0 * y0 + y1 * y1 + y2 * y2;
    return true;
}

// Kalman update with the Joseph form C+ = (I - K H) C (I - K H)^T + K V K^T.
// Returns false if S is not positive definite or theta leaves (0, pi).
__device__ __forceinline__ bool kalman_update(State& t, float mx, float my, float mz, const float v[6]) {
    float L[6], inv[3], r[3];
    if (!chol3(t.c, v, L, inv)) return false;
    residual(t, mx, my, mz, r);
    // W = S^-1 = L^-T L^-1
    const float i00 = inv[0], i11 = inv[1], i22 = inv[2];
    const float i10 = -L[1] * i00 * i11;
    const float i21 = -L[4] * i11 * i22;
    const float i20 = -(L[3] * i00 + L[4] * i10) * i22;
    const float w00 = i00 * i00 + i10 * i10 + i20 * i20;
    const float w10 = i10 * i11 + i20 * i21;
    const float w11 = i11 * i11 + i21 * i21;
    const float w20 = i20 * i22;
    const float w21 = i21 * i22;
    const float w22 = i22 * i22;
    const float W[3][3] = {{w00, w10, w20}, {w10, w11, w21}, {w20, w21, w22}};
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
    // T = (I - K H) C  (row i: C_i - sum_a K_ia C_a)
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
    // KV = K V
    const float V[3][3] = {{v[0], v[1], v[3]}, {v[1], v[2], v[4]}, {v[3], v[4], v[5]}};
    float KV[6][3];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float acc = 0.0f;
#pragma unroll
            for (int b = 0; b < 3; ++b) acc = fmaf(K[i][b], V[b][a], acc);
            KV[i][a] = acc;
        }
    // C+_ij = T_ij - sum_a T_ia K_ja + sum_a KV_ia K_ja   (lower triangle)
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
