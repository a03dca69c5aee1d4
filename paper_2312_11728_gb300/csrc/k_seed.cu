// Seed states (a1) and their ordering keys (a3), one seed per lane.
//
// Sec. 2.2: the input to track finding is a list of seeds, each a list of hits with a
// parameter estimate at its outermost point.  The estimate here: the circle through the
// transverse positions of the three hits gives |curvature| and, from the turning sign,
// the charge; the tangent at hit 1 gives phi; dz over the arc length from hit 1 to hit 3
// gives cot(theta).  From that estimate at hit 1 with a diffuse diagonal covariance, a
// Kalman fit through hits 1, 2, 3 (propagation with material between them) gives the
// state at hit 3.  The seed's region (layer plan) follows from its eta, and the search
// starts at the plan step after hit 3's layer.
#include "internal.h"

namespace mk {

namespace {

constexpr int kThreads = 128;

__global__ void __launch_bounds__(kThreads) k_seed(const DevGeom* __restrict__ gp, DevParams P, HitStore H, int n,
                                                   const int* __restrict__ seed_hits, float* __restrict__ state,
                                                   int4* __restrict__ info, int* __restrict__ key_of,
                                                   int* __restrict__ key_counts, float* state6, float* cov21,
                                                   int* info3) {
    __shared__ DevGeom g;
    {
        const int4* src = reinterpret_cast<const int4*>(gp);
        int4* dst = reinterpret_cast<int4*>(&g);
        for (int i = threadIdx.x; i < (int)(sizeof(DevGeom) / 16); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int id[3], lay[3], ev[3];
    float m[3][3], v[3][6];
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
        load_hit(H.pay, id[j], m[j], v[j], nullptr);
    }
    ok = ok && ev[0] == ev[1] && ev[1] == ev[2];

    // circle through the three transverse points, relative to hit 1
    const float ax = m[1][0] - m[0][0], ay = m[1][1] - m[0][1];
    const float bx = m[2][0] - m[0][0], by = m[2][1] - m[0][1];
    const float cross = ax * by - ay * bx;
    const float chord2 = bx * bx + by * by;
    float k, phi1, arc;
    if (fabsf(cross) < 1e-7f * chord2) {
        k = 0.0f;
        phi1 = atan2f(by, bx);
        arc = sqrtf(chord2);
    } else {
        const float a2 = ax * ax + ay * ay;
        const float inv2c = 0.5f / cross;
        const float ux = (by * a2 - ay * chord2) * inv2c;
        const float uy = (ax * chord2 - bx * a2) * inv2c;
        const float rho = sqrtf(ux * ux + uy * uy);
        const float sg = cross > 0.0f ? 1.0f : -1.0f;
        k = -(sg / rho) / g.cB;
        phi1 = atan2f(-sg * ux, sg * uy);
        const float v1x = -ux, v1y = -uy, v3x = bx - ux, v3y = by - uy;
        arc = fabsf(atan2f(v1x * v3y - v1y * v3x, v1x * v3x + v1y * v3y)) * rho;
    }
    const float cot = (m[2][2] - m[0][2]) / arc;
    State t;
    t.xh = m[0][0]; t.yh = m[0][1]; t.zh = m[0][2];
    t.xl = 0.0f; t.yl = 0.0f; t.zl = 0.0f;
    t.k = k; t.phi = phi1; t.th = atan2f(1.0f, cot);
#pragma unroll
    for (int q = 0; q < 21; ++q) t.c[q] = 0.0f;
    const float sk = 0.5f * fabsf(k) + 0.05f;
    t.c[ix(0, 0)] = 0.01f; t.c[ix(1, 1)] = 0.01f; t.c[ix(2, 2)] = 0.01f;
    t.c[ix(3, 3)] = sk * sk; t.c[ix(4, 4)] = 0.0025f; t.c[ix(5, 5)] = 0.0025f;
    int newton = 0;
    ok = ok && state_update(t, m[0][0], m[0][1], m[0][2], v[0]);
#pragma unroll
    for (int j = 1; j < 3; ++j) {
        Pred q;
        ok = ok && propagate(g.layers[lay[j]], g.cB, P.material, t, q, newton) == 1;
        ok = ok && kalman_update(g.layers[lay[j]].kind, q, m[j][0], m[j][1], m[j][2], v[j], t);
    }
    // region and first search step
    const float eta = -logf(tanf(0.5f * t.th));
    int region = 0;
    if (g.n_regions > 1 && !(fabsf(eta) < P.barrel_eta_max)) region = eta > 0.0f ? 1 : 2;
    if (region >= g.n_regions) region = 0;
    int start = -1;
    for (int q = g.plan_off[region]; q < g.plan_off[region + 1]; ++q)
        if (g.plan[q] == lay[2]) start = q - g.plan_off[region] + 1;
    const int status = (ok && start >= 0) ? 0 : 1;

    float* o = state + (int64_t)i * kSeedStateStride;
    o[0] = t.xh; o[1] = t.yh; o[2] = t.zh; o[3] = t.xl; o[4] = t.yl; o[5] = t.zl;
    o[6] = t.k; o[7] = t.phi; o[8] = t.th;
#pragma unroll
    for (int q = 0; q < 21; ++q) o[9 + q] = t.c[q];
    info[i] = make_int4(region, start, ev[0], status);
    if (state6) store_state6(t, state6 + 6 * (int64_t)i, cov21 + 21 * (int64_t)i);
    if (info3) {
        info3[3 * i] = region;
        info3[3 * i + 1] = start;
        info3[3 * i + 2] = status;
    }
    // (event, eta cell, phi cell) key for the hit-coherent processing order
    int ce = (int)floorf((eta + 4.0f) * (kSeedEtaCells / 8.0f));
    ce = ce < 0 ? 0 : (ce >= kSeedEtaCells ? kSeedEtaCells - 1 : ce);
    int cp = (int)floorf((t.phi + kPi) * (kSeedPhiCells / kTwoPi));
    cp = cp < 0 ? 0 : (cp >= kSeedPhiCells ? kSeedPhiCells - 1 : cp);
    const int key = (ev[0] * kSeedEtaCells + ce) * kSeedPhiCells + cp;
    key_of[i] = key;
    atomicAdd(key_counts + key, 1);
}

}  // namespace

cudaError_t launch_seed(cudaStream_t st, const DevGeom* g, DevParams P, HitStore H, int n, const int* seed_hits,
                        float* state, int4* info, int* key_of, int* key_counts, float* state6, float* cov21,
                        int* info3) {
    if (n == 0) return cudaSuccess;
    k_seed<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(g, P, H, n, seed_hits, state, info, key_of,
                                                              key_counts, state6, cov21, info3);
    return cudaGetLastError();
}

}  // namespace mk
