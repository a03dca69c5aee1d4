// Backward fit (Sec. 2.2: each found track re-traversed backwards, refitting its parameters).
//
// One track per lane, as the forward fit.  The track's state on its last listed layer (the
// forward fit's result there) has its covariance scaled by cov_scale, so that the forward fit's
// information is released, and is fitted through the listed layers from the last to the first:
// the hit on the last layer first (the state taken in that layer's surface frame, as every
// prediction, so the update is the same local-frame one), then for each earlier layer the crossing
// behind the state (propagate_core with BACKWARD: negative path length, material adding the
// energy loss back), chi2 and update.  The result is the state on the innermost listed layer for
// the segment inside it (its material included).  Traversing the trajectory backwards with s < 0
// equals traversing the reversed trajectory (k -> -k, phi -> phi + pi, theta -> pi - theta)
// forwards, the reading the oracle writes out; in FP32 it avoids rounding phi + pi.
//
// Mixed precision as the forward fit: tracks whose largest kappa(S) exceeds kappa_fp64 are refit
// in FP64 by the same kernel instantiated for double; precision = MKGB_FP64 fits all in FP64.
#include "internal.h"

namespace mk {

namespace {

constexpr int kThreads = 128;

__device__ __forceinline__ void load_geom(const DevGeom* __restrict__ gp, DevGeom& g) {
    const int4* src = reinterpret_cast<const int4*>(gp);
    int4* dst = reinterpret_cast<int4*>(&g);
    for (int i = threadIdx.x; i < (int)(sizeof(DevGeom) / 16); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
}

// One track in precision F; its status and the largest kappa(S).  MOD: module hits loaded (used on
// their module planes).
template <class F, bool MOD>
__device__ __forceinline__ int bkfit_track(const DevGeom& g, const DevParams& P, const float4* __restrict__ pay,
                                           int64_t n_hits, int max_steps, const int* __restrict__ lrow,
                                           const int* __restrict__ hrow, const float* p_start, const float* c_start,
                                           float cov_scale, StateT<F>& t, F& sum, float& kmax,
                                           unsigned long long& c_steps, unsigned long long& c_upd, int& c_newton) {
    load_state6(p_start, c_start, t);
#pragma unroll
    for (int q = 0; q < 21; ++q) t.c[q] *= F(cov_scale);
    sum = F(0);
    kmax = 0.0f;
    int nl = 0;
    while (nl < max_steps && __ldg(lrow + nl) >= 0 && __ldg(lrow + nl) < g.n_layers) ++nl;
    for (int j = nl - 1; j >= 0; --j) {
        const int l = __ldg(lrow + j);
        const int h = __ldg(hrow + j);
        if (h >= n_hits) return 4;   // hit index outside the loaded hits
        const DevLayer& L = g.layers[l];
        F m[3], v[6], x2;
        int md = -1;
        if (h >= 0) {
            if constexpr (MOD)
                load_hit(pay, h, m, v, nullptr, &md);
            else
                load_hit(pay, h, m, v, nullptr);
        }
        if (MOD && md >= 0) {   // a module hit (Sec. 3.1): on its module's plane
            float kap = 0.0f;
            int r;
            if (j == nl - 1) {   // the start state lies on that plane
                r = module_update_on_plane(t, g.mods, md, m, v, P.fit_outlier_chi2, t, x2, kap);
            } else {
                PredT<F> q;
                const int rp = propagate_core<F, F, true>(L, g.cB, P.material, t, t.c, q, q.c, c_newton);
                if (rp != 1) return rp == 0 ? 1 : 2;
                ++c_steps;
                r = module_update(L.kind, q, g.mods, md, g.cB, m, v, P.fit_outlier_chi2, t, x2, kap);
                if (r == 1 || r == 3) pred_to_state(L.kind, q, t);   // not reached; outlier: not used
                if (r == 1) return 1;
            }
            if (r == 2) return 3;
            if (r == 0) {
                kmax = fmaxf(kmax, kap);
                sum += x2;
                ++c_upd;
            }
            continue;
        }
        if (j == nl - 1) {
            // the start state lies on this layer: taken in the layer's surface frame (its
            // covariance without variance along the normal), then updated as every other step
            PredT<F> q;
            q.xh = t.xh; q.yh = t.yh; q.k = t.k; q.phi = t.phi; q.th = t.th;
            const FrameT<F> fr = frame_of(L.kind, q);
            state_to_pred(fr, t, q);
            if (h >= 0) {
                float kap = 0.0f;
                if (!chi2_hit(fr, q, m[0], m[1], m[2], v, x2)) return 3;
                if (!(P.fit_outlier_chi2 > 0.0f && x2 > F(P.fit_outlier_chi2))) {   // else an outlier
                    if (!kalman_update_f(fr, q, m[0], m[1], m[2], v, t, &kap)) return 3;
                    kmax = fmaxf(kmax, kap);
                    sum += x2;
                    ++c_upd;
                    continue;
                }
            }
            pred_to_state(L.kind, q, t);
            continue;
        }
        PredT<F> q;
        const int r = propagate_core<F, F, true>(L, g.cB, P.material, t, t.c, q, q.c, c_newton);
        if (r != 1) return r == 0 ? 1 : 2;
        ++c_steps;
        if (h >= 0) {
            float kap = 0.0f;
            if (!chi2_hit(L.kind, q, m[0], m[1], m[2], v, x2)) return 3;
            if (P.fit_outlier_chi2 > 0.0f && x2 > F(P.fit_outlier_chi2)) {   // outlier: not used
                pred_to_state(L.kind, q, t);
                continue;
            }
            if (!kalman_update(L.kind, q, m[0], m[1], m[2], v, t, &kap)) return 3;
            kmax = fmaxf(kmax, kap);
            sum += x2;
            ++c_upd;
        } else {
            pred_to_state(L.kind, q, t);
        }
    }
    return 0;
}

// All tracks (list == nullptr) or the listed ones (the FP64 refit of the flagged FP32 fits).
template <class F, bool MOD>
__global__ void __launch_bounds__(kThreads) k_bkfit(const DevGeom* __restrict__ gp, DevParams P,
                                                    const float4* __restrict__ pay, int64_t n_hits, int n,
                                                    int max_steps, const int* __restrict__ layers,
                                                    const int* __restrict__ hits, const float* __restrict__ p_start,
                                                    const float* __restrict__ c_start, float cov_scale,
                                                    float* __restrict__ p_out, float* __restrict__ c_out,
                                                    float* __restrict__ chi2_out, int* __restrict__ status_out,
                                                    unsigned long long* counters, int* rescue_list, int* rescue_count,
                                                    const int* __restrict__ list, const int* __restrict__ count) {
    __shared__ DevGeom g;
    load_geom(gp, g);
    const int cnt = list ? *count : n;
    unsigned long long c_steps = 0, c_upd = 0;
    int c_newton = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < cnt; r += gridDim.x * blockDim.x) {
        const int i = list ? list[r] : r;
        StateT<F> t;
        F sum;
        float kmax;
        const int status = bkfit_track<F, MOD>(g, P, pay, n_hits, max_steps, layers + (int64_t)i * max_steps,
                                          hits + (int64_t)i * max_steps, p_start + 6 * (int64_t)i,
                                          c_start + 21 * (int64_t)i, cov_scale, t, sum, kmax, c_steps, c_upd,
                                          c_newton);
        store_state6(t, p_out + 6 * (int64_t)i, c_out + 21 * (int64_t)i);
        chi2_out[i] = float(sum);
        if (status_out) status_out[i] = status;
        if (rescue_list && P.kappa_fp64 > 0.0f && kmax > P.kappa_fp64) rescue_list[atomicAdd(rescue_count, 1)] = i;
    }
    if (counters && !list) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            c_steps += __shfl_xor_sync(0xffffffffu, c_steps, off);
            c_upd += __shfl_xor_sync(0xffffffffu, c_upd, off);
            c_newton += __shfl_xor_sync(0xffffffffu, c_newton, off);
        }
        if ((threadIdx.x & 31) == 0 && c_steps + c_upd) {
            atomicAdd(counters + 0, c_steps);
            atomicAdd(counters + 1, c_upd);
            atomicAdd(counters + 2, c_upd);
            atomicAdd(counters + 4, (unsigned long long)c_newton);
        }
    }
}

}  // namespace

cudaError_t launch_bkfit(cudaStream_t st, const DevGeom* g, DevParams P, const float4* pay, int64_t n_hits, int n,
                         int max_steps, const int* layers, const int* hits, const float* p_start, const float* c_start,
                         float cov_scale, float* p_out, float* c_out, float* chi2_out, int* status_out,
                         unsigned long long* counters, int* rescue_list, int* rescue_count, int n_sms, bool modular) {
    if (n == 0) return cudaSuccess;
    const int blocks = (n + kThreads - 1) / kThreads;
    auto fit64 = modular ? k_bkfit<double, true> : k_bkfit<double, false>;
    auto fit32 = modular ? k_bkfit<float, true> : k_bkfit<float, false>;
    if (P.precision == MKGB_FP64) {
        fit64<<<blocks, kThreads, 0, st>>>(g, P, pay, n_hits, n, max_steps, layers, hits, p_start, c_start,
                                                     cov_scale, p_out, c_out, chi2_out, status_out, counters,
                                                     nullptr, nullptr, nullptr, nullptr);
        return cudaGetLastError();
    }
    fit32<<<blocks, kThreads, 0, st>>>(g, P, pay, n_hits, n, max_steps, layers, hits, p_start, c_start,
                                                cov_scale, p_out, c_out, chi2_out, status_out, counters, rescue_list,
                                                rescue_count, nullptr, nullptr);
    if (P.kappa_fp64 > 0.0f && rescue_list) {
        const int rb = blocks < 2 * n_sms ? blocks : 2 * n_sms;
        fit64<<<rb, kThreads, 0, st>>>(g, P, pay, n_hits, n, max_steps, layers, hits, p_start, c_start,
                                                 cov_scale, p_out, c_out, chi2_out, status_out, counters, nullptr,
                                                 nullptr, rescue_list, rescue_count);
    }
    return cudaGetLastError();
}

}  // namespace mk
