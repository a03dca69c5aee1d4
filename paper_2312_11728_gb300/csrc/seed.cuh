// Seed fit device functions (a1), shared by the seed kernels.
#pragma once

#include "internal.h"

namespace mk {

// Hits of seed i and the prior of its fit (a1): the circle through the three transverse points
// gives |curvature|, the charge (turning sign) and phi at hit 1; dz over the arc length gives
// cot(theta); the covariance is diagonal and diffuse.  Returns ok (valid hits of one event).
template <class F>
__device__ __forceinline__ bool seed_prior(const DevGeom& g, const HitStore& H, const int* __restrict__ seed_hits,
                                           int i, F m[3][3], F v[3][6], int lay[3], int& event, StateT<F>& t,
                                           int mod[3]) {
    int id[3], ev[3];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        id[j] = seed_hits[3 * i + j];
        if (id[j] < 0 || id[j] >= H.n_hits) {
            ok = false;
            id[j] = 0;
        }
        const int seg = H.hit_seg[id[j]];
        ev[j] = seg / H.n_layers;
        lay[j] = seg - ev[j] * H.n_layers;
        load_hit(H.pay, id[j], m[j], v[j], nullptr, &mod[j]);   // mod: the hit's module, -1 none
        if (!g.mods) mod[j] = -1;
    }
    event = ev[0];
    ok = ok && ev[0] == ev[1] && ev[1] == ev[2];
    // circle through the three transverse points, relative to hit 1
    const F ax = m[1][0] - m[0][0], ay = m[1][1] - m[0][1];
    const F bx = m[2][0] - m[0][0], by = m[2][1] - m[0][1];
    const F cross = ax * by - ay * bx;
    const F chord2 = bx * bx + by * by;
    F k, phi1, arc;
    if (fabs(cross) < F(1e-12) * chord2) {   // three points on a line: no curvature
        k = F(0);
        phi1 = atan2(by, bx);
        arc = sqrt(chord2);
    } else {
        const F a2 = ax * ax + ay * ay;
        const F inv2c = F(0.5) / cross;
        const F ux = (by * a2 - ay * chord2) * inv2c;
        const F uy = (ax * chord2 - bx * a2) * inv2c;
        const F rho = sqrt(ux * ux + uy * uy);
        const F sg = cross > F(0) ? F(1) : F(-1);
        k = -(sg / rho) / F(g.cB);
        phi1 = atan2(-sg * ux, sg * uy);
        const F v1x = -ux, v1y = -uy, v3x = bx - ux, v3y = by - uy;
        arc = fabs(atan2(v1x * v3y - v1y * v3x, v1x * v3x + v1y * v3y)) * rho;
    }
    const F cot = (m[2][2] - m[0][2]) / arc;
    t.xh = m[0][0]; t.yh = m[0][1]; t.zh = m[0][2];
    t.xl = F(0); t.yl = F(0); t.zl = F(0);
    t.k = k; t.phi = phi1; t.th = atan2(F(1), cot);
#pragma unroll
    for (int q = 0; q < 21; ++q) t.c[q] = F(0);
    const F sk = F(0.5) * fabs(k) + F(0.05);
    t.c[ix(0, 0)] = F(0.01); t.c[ix(1, 1)] = F(0.01); t.c[ix(2, 2)] = F(0.01);
    t.c[ix(3, 3)] = sk * sk; t.c[ix(4, 4)] = F(0.0025); t.c[ix(5, 5)] = F(0.0025);
    return ok;
}

// The seed fit's precision modes.  kSeedPlain: every step in F (the all-FP64 path).
// kSeedAssisted (FP64 with FP32 help): the first update in closed form (zero residual, diagonal
// prior), FP32 crossings refined by FP64 Newton iterations (propagate_refined), the update's frame
// from the propagation's direction and the short covariance update (I - K H) C.  kSeedMixed (the
// seeds of the FP32 path): as kSeedAssisted, but each step's trajectory (float-float positions and
// angles), Jacobian and material in FP32, with the FP64 covariance transported in FP64 by that
// Jacobian: the update's cancellation, the ill-conditioned part of the seed fit, stays in FP64,
// and an FP32 Jacobian only perturbs the problem by ~1e-7 relative.  The FP32 trajectory leaves
// ~2e-6 cm in a 30 cm step's transverse position, ~1e-6 of q/pT on a short lever arm: seeds with
// |q/pT| below kSeedKappaRedo, whose q/pT tolerance is that small, are fitted again in
// kSeedAssisted.
enum : int { kSeedPlain = 0, kSeedAssisted = 1, kSeedMixed = 2 };
constexpr double kSeedKappaRedo = 0.03;   // 1/GeV: |q/pT| below which a mixed seed fit is redone

// Seed fit of seed i in precision F: update with hit 1, then propagate to and update with hits
// 2 and 3 (MOD: a hit measured on a module is used on its module's plane, reached from its
// layer's surface; hit 1 needs no step, the estimate sits on it).  Returns ok.
template <class F, int MODE = kSeedPlain, bool MOD = false>
__device__ __forceinline__ bool seed_fit(const DevGeom& g, const DevParams& P, const HitStore& H,
                                         const int* __restrict__ seed_hits, int i, StateT<F>& t, int lay[3],
                                         int& event) {
    F m[3][3], v[3][6];
    int mod[3];
    bool ok = seed_prior(g, H, seed_hits, i, m, v, lay, event, t, mod);
    if constexpr (!MOD) ok = ok && mod[0] < 0 && mod[1] < 0 && mod[2] < 0;
    int newton = 0;
    constexpr bool fast = MODE != kSeedPlain && sizeof(F) == 8;
    if constexpr (fast)
        ok = ok && prior_update_at_hit(t, v[0]);
    else
        ok = ok && state_update(t, m[0][0], m[0][1], m[0][2], v[0]);
#pragma unroll
    for (int j = 1; j < 3; ++j) {
        PredT<F> q;
        const DevLayer& L = g.layers[lay[j]];
        F dir[4];
        if constexpr (fast && MODE == kSeedMixed) {
            State t32;
            narrow_to_fp32(t, t32);
            Pred q32;
            float d32[4];
            ok = ok && propagate_core<float, F>(L, g.cB, P.material, t32, t.c, q32, q.c, newton, d32) == 1;
            q.xh = F(q32.xh); q.yh = F(q32.yh); q.zh = F(q32.zh);
            q.xl = F(q32.xl); q.yl = F(q32.yl); q.zl = F(q32.zl);
            q.k = F(q32.k); q.phi = F(q32.phi); q.pl = F(q32.pl); q.th = F(q32.th); q.tl = F(q32.tl);
#pragma unroll
            for (int c = 0; c < 4; ++c) dir[c] = F(d32[c]);
        } else {
            ok = ok && propagate_refined(L, g.cB, P.material, t, q, newton, fast, dir) == 1;
        }
        if constexpr (MOD) {
            if (ok && mod[j] >= 0) {   // a module hit: the update on its module's plane (Sec. 3.1)
                F x2u;
                float kap;
                ok = module_update(L.kind, q, g.mods, mod[j], g.cB, m[j], v[j], 0.0f, t, x2u, kap) == 0;
                continue;
            }
        }
        if constexpr (fast)
            ok = ok && kalman_update_f<F, false>(frame_of(L.kind, q.xh, q.yh, dir[0], dir[1], dir[2], dir[3]), q,
                                                 m[j][0], m[j][1], m[j][2], v[j], t);
        else
            ok = ok && kalman_update(L.kind, q, m[j][0], m[j][1], m[j][2], v[j], t);
    }
    return ok;
}

__device__ __forceinline__ void seed_region(const DevGeom& g, const DevParams& P, float th, int lay3, bool ok,
                                            int& region, int& start) {
    const float eta = -logf(tanf(0.5f * th));
    region = 0;
    if (g.n_regions > 1 && !(fabsf(eta) < P.barrel_eta_max)) region = eta > 0.0f ? 1 : 2;
    if (region >= g.n_regions) region = 0;
    start = -1;
    for (int q = g.plan_off[region]; q < g.plan_off[region + 1]; ++q)
        if (g.plan[q] == lay3) start = q - g.plan_off[region] + 1;
    if (!ok || start < 0) {
        region = -1;
        start = -1;
    }
}

}  // namespace mk
