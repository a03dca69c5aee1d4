// Kalman fit over a known hit assignment (a12) and single-step kernels.
//
// Sec. 4: with faster building, the final fit becomes a comparably expensive step.  One
// track per lane, the state stays in registers across all its layers; per step the lane
// reads one 48-byte hit payload.  FP32-bound (a few hundred FMA per 52 bytes read).
//
// Mixed precision: the FP32 pass estimates the condition number of every innovation
// covariance S from its Cholesky factor.  An update with kappa(S) near 1/eps_FP32 (a grazing
// crossing whose along-track spread dwarfs the hit error) leaves FP32 rounding in the
// posterior, so tracks above a threshold are appended to a list and a second kernel refits
// them entirely in FP64 (the same code for double).  The default threshold is 2^24, where the
// innovation covariance's condition reaches 1/eps of FP32.
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

// One track in precision F; returns its status and the largest kappa(S) of its updates.  MOD:
// module hits loaded (used on their module planes).
template <class F, bool MOD>
__device__ __forceinline__ int fit_track(const DevGeom& g, const DevParams& P, const float4* __restrict__ pay,
                                         int64_t n_hits, int max_steps, const int* __restrict__ lrow,
                                         const int* __restrict__ hrow, const float* p0, const float* c0,
                                         StateT<F>& t, F& sum, float& kmax, unsigned long long& c_steps,
                                         unsigned long long& c_upd, int& c_newton) {
    load_state6(p0, c0, t);
    sum = F(0);
    kmax = 0.0f;
    for (int j = 0; j < max_steps; ++j) {
        const int l = __ldg(lrow + j);
        if (l < 0 || l >= g.n_layers) break;
        const DevLayer& L = g.layers[l];
        PredT<F> q;
        const int r = propagate_refined(L, g.cB, P.material, t, q, c_newton, sizeof(F) == 8 && P.precision != MKGB_FP64);
        if (r != 1) return r == 0 ? 1 : 2;
        ++c_steps;
        const int h = __ldg(hrow + j);
        if (h >= n_hits) {
            pred_to_state(L.kind, q, t);
            return 4;   // hit index outside the loaded hits
        }
        if (h >= 0) {
            F m[3], v[6], x2;
            float kap = 0.0f;
            int md = -1;
            if constexpr (MOD)
                load_hit(pay, h, m, v, nullptr, &md);
            else
                load_hit(pay, h, m, v, nullptr);
            if (MOD && md >= 0) {   // a module hit is used on its module's plane (Sec. 3.1)
                const int r = module_update(L.kind, q, g.mods, md, g.cB, m, v, P.fit_outlier_chi2, t, x2, kap);
                if (r == 1 || r == 3) pred_to_state(L.kind, q, t);   // not reached; outlier: not used
                if (r == 1) return 1;
                if (r == 2) return 3;
                if (r == 3) continue;
                kmax = fmaxf(kmax, kap);
                sum += x2;
                ++c_upd;
                continue;
            }
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

template <bool MOD>
__global__ void __launch_bounds__(kThreads) k_fit(const DevGeom* __restrict__ gp, DevParams P,
                                                  const float4* __restrict__ pay, int64_t n_hits, int n, int max_steps,
                                                  const int* __restrict__ layers, const int* __restrict__ hits,
                                                  const float* __restrict__ p0, const float* __restrict__ c0,
                                                  float* __restrict__ p_out, float* __restrict__ c_out,
                                                  float* __restrict__ chi2_out, int* __restrict__ status_out,
                                                  unsigned long long* counters, int* rescue_list,
                                                  int* rescue_count) {
    __shared__ DevGeom g;
    load_geom(gp, g);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c_steps = 0, c_upd = 0;
    int c_newton = 0;
    if (i < n) {
        State t;
        float sum, kmax;
        const int status = fit_track<float, MOD>(g, P, pay, n_hits, max_steps, layers + (int64_t)i * max_steps,
                                            hits + (int64_t)i * max_steps, p0 + 6 * (int64_t)i, c0 + 21 * (int64_t)i,
                                            t, sum, kmax, c_steps, c_upd, c_newton);
        store_state6(t, p_out + 6 * (int64_t)i, c_out + 21 * (int64_t)i);
        chi2_out[i] = sum;
        if (status_out) status_out[i] = status;
        if (rescue_list && P.kappa_fp64 > 0.0f && kmax > P.kappa_fp64) rescue_list[atomicAdd(rescue_count, 1)] = i;
    }
    if (counters) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            c_steps += __shfl_xor_sync(0xffffffffu, c_steps, off);
            c_upd += __shfl_xor_sync(0xffffffffu, c_upd, off);
            c_newton += __shfl_xor_sync(0xffffffffu, c_newton, off);
        }
        if ((threadIdx.x & 31) == 0 && c_steps) {
            atomicAdd(counters + 0, c_steps);
            atomicAdd(counters + 1, c_upd);
            atomicAdd(counters + 2, c_upd);
            atomicAdd(counters + 4, (unsigned long long)c_newton);
        }
    }
}

// FP64 refit of the listed tracks (kappa rescue) or of all tracks (all-FP64 path, list == null).
template <bool MOD>
__global__ void __launch_bounds__(kThreads) k_fit64(const DevGeom* __restrict__ gp, DevParams P,
                                                    const float4* __restrict__ pay, int64_t n_hits, int n,
                                                    int max_steps, const int* __restrict__ layers,
                                                    const int* __restrict__ hits, const float* __restrict__ p0,
                                                    const float* __restrict__ c0, float* __restrict__ p_out,
                                                    float* __restrict__ c_out, float* __restrict__ chi2_out,
                                                    int* __restrict__ status_out, unsigned long long* counters,
                                                    const int* __restrict__ list, const int* __restrict__ count) {
    __shared__ DevGeom g;
    load_geom(gp, g);
    const int cnt = list ? *count : n;
    unsigned long long c_steps = 0, c_upd = 0;
    int c_newton = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < cnt; r += gridDim.x * blockDim.x) {
        const int i = list ? list[r] : r;
        StateT<double> t;
        double sum;
        float kmax;
        const int status = fit_track<double, MOD>(g, P, pay, n_hits, max_steps, layers + (int64_t)i * max_steps,
                                             hits + (int64_t)i * max_steps, p0 + 6 * (int64_t)i, c0 + 21 * (int64_t)i,
                                             t, sum, kmax, c_steps, c_upd, c_newton);
        store_state6(t, p_out + 6 * (int64_t)i, c_out + 21 * (int64_t)i);
        chi2_out[i] = float(sum);
        if (status_out) status_out[i] = status;
    }
    if (counters && !list) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            c_steps += __shfl_xor_sync(0xffffffffu, c_steps, off);
            c_upd += __shfl_xor_sync(0xffffffffu, c_upd, off);
            c_newton += __shfl_xor_sync(0xffffffffu, c_newton, off);
        }
        if ((threadIdx.x & 31) == 0 && c_steps) {
            atomicAdd(counters + 0, c_steps);
            atomicAdd(counters + 1, c_upd);
            atomicAdd(counters + 2, c_upd);
            atomicAdd(counters + 4, (unsigned long long)c_newton);
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_step_propagate(const DevGeom* __restrict__ gp, DevParams P, int n,
                                                             const int* __restrict__ layers,
                                                             const float* __restrict__ p_in,
                                                             const float* __restrict__ c_in, float* p_out,
                                                             float* c_out, int* crossed) {
    __shared__ DevGeom g;
    load_geom(gp, g);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    State t;
    load_state6(p_in + 6 * (int64_t)i, c_in + 21 * (int64_t)i, t);
    const int l = layers[i];
    int it = 0;
    int r = 0;
    if (l >= 0 && l < g.n_layers) {
        Pred q;
        r = propagate(g.layers[l], g.cB, P.material, t, q, it);
        if (r == 1) pred_to_state(g.layers[l].kind, q, t);
    }
    store_state6(t, p_out + 6 * (int64_t)i, c_out + 21 * (int64_t)i);
    crossed[i] = r;
}

__global__ void __launch_bounds__(kThreads) k_step_update(int n, const float* __restrict__ p_in,
                                                          const float* __restrict__ c_in,
                                                          const float* __restrict__ hxyz,
                                                          const float* __restrict__ hcov, float* p_out,
                                                          float* c_out, float* chi2, int* ok) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    State t;
    load_state6(p_in + 6 * (int64_t)i, c_in + 21 * (int64_t)i, t);
    float v[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) v[j] = hcov[6 * (int64_t)i + j];
    const float mx = hxyz[3 * (int64_t)i], my = hxyz[3 * (int64_t)i + 1], mz = hxyz[3 * (int64_t)i + 2];
    float x2 = 0.0f;
    // a state given in the global frame is updated without a surface constraint
    float S[6], Lc[6], inv[3];
    bool good = true;
#pragma unroll
    for (int j = 0; j < 6; ++j) S[j] = t.c[j] + v[j];
    if (chol3(S, Lc, inv)) {
        const float r0 = mx - t.xh, r1 = my - t.yh, r2 = mz - t.zh;
        const float y0 = r0 * inv[0], y1 = (r1 - Lc[1] * y0) * inv[1], y2 = (r2 - Lc[3] * y0 - Lc[4] * y1) * inv[2];
        x2 = y0 * y0 + y1 * y1 + y2 * y2;
    } else {
        good = false;
    }
    good = good && state_update(t, mx, my, mz, v);
    store_state6(t, p_out + 6 * (int64_t)i, c_out + 21 * (int64_t)i);
    chi2[i] = x2;
    ok[i] = good ? 1 : 0;
}

}  // namespace

cudaError_t launch_fit(cudaStream_t st, const DevGeom* g, DevParams P, const float4* pay, int64_t n_hits, int n,
                       int max_steps, const int* layers, const int* hits, const float* p0, const float* c0,
                       float* p_out, float* c_out, float* chi2_out, int* status_out, unsigned long long* counters,
                       int* rescue_list, int* rescue_count, int n_sms, bool modular) {
    if (n == 0) return cudaSuccess;
    const int blocks = (n + kThreads - 1) / kThreads;
    auto fit64 = modular ? k_fit64<true> : k_fit64<false>;
    if (P.precision == MKGB_FP64) {
        fit64<<<blocks, kThreads, 0, st>>>(g, P, pay, n_hits, n, max_steps, layers, hits, p0, c0, p_out, c_out,
                                          chi2_out, status_out, counters, nullptr, nullptr);
        return cudaGetLastError();
    }
    auto fit = modular ? k_fit<true> : k_fit<false>;
    fit<<<blocks, kThreads, 0, st>>>(g, P, pay, n_hits, n, max_steps, layers, hits, p0, c0, p_out, c_out, chi2_out,
                                    status_out, counters, rescue_list, rescue_count);
    if (P.kappa_fp64 > 0.0f && rescue_list) {
        const int rb = blocks < 2 * n_sms ? blocks : 2 * n_sms;
        fit64<<<rb, kThreads, 0, st>>>(g, P, pay, n_hits, n, max_steps, layers, hits, p0, c0, p_out, c_out,
                                      chi2_out, status_out, counters, rescue_list, rescue_count);
    }
    return cudaGetLastError();
}

// Scratch of mkgb_fit_static, the fit entry point that allocates nothing: a file-scope device
// array holding the work counters, the FP64 refit counter and the refit list for at most
// kFitStaticMaxTracks tracks (layout in internal.h).  Its address is looked up, not allocated.
static __device__ __align__(256) unsigned char g_fit_static_scratch[kFitStaticScratchBytes];

cudaError_t fit_static_scratch_address(void** base) {
    return cudaGetSymbolAddress(base, g_fit_static_scratch);
}

cudaError_t launch_step_propagate(cudaStream_t st, const DevGeom* g, DevParams P, int n, const int* layers,
                                  const float* p_in, const float* c_in, float* p_out, float* c_out, int* crossed) {
    if (n == 0) return cudaSuccess;
    k_step_propagate<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(g, P, n, layers, p_in, c_in, p_out, c_out,
                                                                        crossed);
    return cudaGetLastError();
}

cudaError_t launch_step_update(cudaStream_t st, int n, const float* p_in, const float* c_in, const float* hxyz,
                               const float* hcov, float* p_out, float* c_out, float* chi2, int* ok) {
    if (n == 0) return cudaSuccess;
    k_step_update<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(n, p_in, c_in, hxyz, hcov, p_out, c_out, chi2,
                                                                     ok);
    return cudaGetLastError();
}

}  // namespace mk
