// Derivative of the fit's total chi2 (growth row G1 of the fit over a known assignment, Sec. 4).
//
// d(sum of the predicted chi2 over tracks and layers) / d(per-layer alignment, per-layer material
// thickness scale, per-track starting parameters).  Alignment of layer l moves its hits,
// h' = h + d_l + w_l x (h - c_l), with c_l the origin for a cylinder and (0, 0, z_l) for a disk;
// the layer surfaces stay nominal.  The thickness scale multiplies x/X0 of the layer.
//
// One thread per track runs the FP32 fit on dual numbers (dual.cuh) that carry KD directional
// derivatives: the track's parameters (6 starting parameters, then 7 per listed layer) are
// taken KD at a time, so a track with L layers takes ceil((6 + 7 L) / KD) passes, each a full
// fit.  Forward mode needs no stored states (memory stays one track's registers and stack);
// the cost grows with the parameter count instead.  Per-layer derivatives are summed in shared
// memory per block, then added to the global arrays.
#include "internal.h"

namespace mk {

namespace {

constexpr int kThreads = 64;
constexpr int KD = 4;   // derivative directions per pass
using D = Dual<float, KD>;

__device__ __forceinline__ void load_geom(const DevGeom* __restrict__ gp, DevGeom& g) {
    const int4* src = reinterpret_cast<const int4*>(gp);
    int4* dst = reinterpret_cast<int4*>(&g);
    for (int i = threadIdx.x; i < (int)(sizeof(DevGeom) / 16); i += blockDim.x) dst[i] = src[i];
}

__device__ __forceinline__ D seeded(float v, int comp, int base) {
    D r(v);
    const int k = comp - base;
    if (k >= 0 && k < KD) r.d[k] = 1.0f;
    return r;
}

__global__ void __launch_bounds__(kThreads) k_fit_grad(const DevGeom* __restrict__ gp, DevParams P,
                                                       const float4* __restrict__ pay, int64_t n_hits, int n,
                                                       int max_steps, const int* __restrict__ layers,
                                                       const int* __restrict__ hits, const float* __restrict__ p0,
                                                       const float* __restrict__ c0, const float* __restrict__ align,
                                                       const float* __restrict__ xscale, float* __restrict__ chi2_out,
                                                       float* __restrict__ d_p0, float* __restrict__ d_align,
                                                       float* __restrict__ d_xscale, int* __restrict__ status_out) {
    __shared__ DevGeom g;
    __shared__ float acc[MKGB_MAX_LAYERS * 7];
    load_geom(gp, g);
    for (int q = threadIdx.x; q < MKGB_MAX_LAYERS * 7; q += blockDim.x) acc[q] = 0.0f;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int* lrow = layers + (int64_t)i * max_steps;
        const int* hrow = hits + (int64_t)i * max_steps;
        int nl = 0;
        while (nl < max_steps && lrow[nl] >= 0 && lrow[nl] < g.n_layers) ++nl;
        const int ncomp = 6 + 7 * nl;
        const float* pi = p0 + 6 * (int64_t)i;
        const float* ci = c0 + 21 * (int64_t)i;
        int status = 0;
        float chi2v = 0.0f;
        for (int base = 0; base < ncomp && status == 0; base += KD) {
            StateT<D> t;
            t.xh = seeded(pi[0], 0, base); t.yh = seeded(pi[1], 1, base); t.zh = seeded(pi[2], 2, base);
            t.xl = D(0.0f); t.yl = D(0.0f); t.zl = D(0.0f);
            t.k = seeded(pi[3], 3, base); t.phi = seeded(pi[4], 4, base); t.th = seeded(pi[5], 5, base);
#pragma unroll 1
            for (int q = 0; q < 21; ++q) t.c[q] = D(ci[q]);
            D sum(0.0f);
            int newton = 0;
            for (int j = 0; j < nl; ++j) {
                const int l = lrow[j];
                const DevLayer& L = g.layers[l];
                const int cj = 6 + 7 * j;
                const D xs = seeded(xscale[l], cj + 6, base);
                PredT<D> q;
                const int r = propagate_core<D, D>(L, g.cB, P.material, t, t.c, q, q.c, newton, nullptr, &xs);
                if (r != 1) {
                    status = r == 0 ? 1 : 2;
                    break;
                }
                const int h = hrow[j];
                if (h >= n_hits) {
                    status = 4;
                    break;
                }
                if (h >= 0) {
                    float mf[3], vf[6];
                    load_hit(pay, h, mf, vf, nullptr);
                    const float* al = align + 6 * l;
                    D sh[3], w[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        sh[c] = seeded(al[c], cj + c, base);
                        w[c] = seeded(al[3 + c], cj + 3 + c, base);
                    }
                    // alignment displacement d + w x (h - c), added to the residual (not to the
                    // FP32 hit position, whose ulp at 1 m is 0.08 um)
                    const float cz = L.kind == MKGB_DISK ? L.pos : 0.0f;
                    const D r0(mf[0]), r1(mf[1]), r2(mf[2] - cz);
                    const D dm[3] = {sh[0] + (w[1] * r2 - w[2] * r1), sh[1] + (w[2] * r0 - w[0] * r2),
                                     sh[2] + (w[0] * r1 - w[1] * r0)};
                    const D mx(mf[0]), my(mf[1]), mz(mf[2]);
                    D v[6];
#pragma unroll
                    for (int c = 0; c < 6; ++c) v[c] = D(vf[c]);
                    D x2;
                    if (!chi2_hit(L.kind, q, mx, my, mz, v, x2, dm) ||
                        !kalman_update(L.kind, q, mx, my, mz, v, t, nullptr, dm)) {
                        status = 3;
                        break;
                    }
                    sum += x2;
                } else {
                    pred_to_state(L.kind, q, t);
                }
            }
            if (status != 0) break;
            if (base == 0) chi2v = sum.v;
#pragma unroll
            for (int k = 0; k < KD; ++k) {
                const int comp = base + k;
                if (comp >= ncomp) break;
                if (comp < 6) {
                    d_p0[6 * (int64_t)i + comp] = sum.d[k];
                } else {
                    const int j = (comp - 6) / 7, qq = (comp - 6) % 7;
                    atomicAdd(acc + lrow[j] * 7 + qq, sum.d[k]);
                }
            }
        }
        if (status != 0) {
            chi2v = 0.0f;
#pragma unroll
            for (int c = 0; c < 6; ++c) d_p0[6 * (int64_t)i + c] = 0.0f;
        }
        chi2_out[i] = chi2v;
        if (status_out) status_out[i] = status;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < g.n_layers * 7; q += blockDim.x) {
        const float v = acc[q];
        if (v != 0.0f) {
            const int l = q / 7, c = q % 7;
            atomicAdd(c < 6 ? d_align + 6 * l + c : d_xscale + l, v);
        }
    }
}

}  // namespace

cudaError_t launch_fit_grad(cudaStream_t st, const DevGeom* g, DevParams P, const float4* pay, int64_t n_hits, int n,
                            int max_steps, const int* layers, const int* hits, const float* p0, const float* c0,
                            const float* align, const float* xscale, float* chi2_out, float* d_p0, float* d_align,
                            float* d_xscale, int* status_out) {
    if (n == 0) return cudaSuccess;
    k_fit_grad<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(g, P, pay, n_hits, n, max_steps, layers, hits, p0,
                                                                   c0, align, xscale, chi2_out, d_p0, d_align,
                                                                   d_xscale, status_out);
    return cudaGetLastError();
}

}  // namespace mk
