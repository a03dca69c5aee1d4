// Derivative of the fit's total chi2 (growth row G1 of the fit over a known assignment, Sec. 4).
//
// d(sum of the predicted chi2 over tracks and layers) / d(per-layer alignment, per-layer material
// thickness scale, per-track starting parameters).  Alignment of layer l moves its hits,
// h' = h + d_l + w_l x (h - c_l), with c_l the origin for a cylinder and (0, 0, z_l) for a disk;
// the layer surfaces stay nominal.  The thickness scale multiplies x/X0 of the layer.
//
// Both kernels run the FP32 fit step (fit_step below) on dual numbers (dual.cuh) carrying KD
// directional derivatives, one thread per track.
//
// k_fit_adjoint (reverse sweep, the default): a plain FP32 pass stores the input state of every
// step (a checkpoint per layer); then, from the last step back to the first, the step is redone
// from its checkpoint with its 34 inputs (27 state words, 6 alignment, 1 thickness scale) seeded
// KD at a time, and the adjoint of its output (d total / d output, starting at zero after the
// last step; the step's own chi2 enters with weight 1) is contracted with the output
// derivatives: d total / d input = dchi2_j / d input + lambda . d out / d input.  The state part
// becomes the adjoint for the previous step, the layer part is summed per layer, and the adjoint
// at the first step's input is d chi2 / d p0.  Cost ~ L x ceil(34 / KD) dual steps per track.
//
// k_fit_grad (forward mode): all 6 + 7 L parameters of a track are seeded KD at a time over a
// whole fit, ceil((6 + 7 L) / KD) fits per track (about 4x the work of the reverse sweep at 22
// layers) but no checkpoint memory.
//
// Per-layer derivatives are summed in shared memory per block, then added to the global arrays.
#include "internal.h"

namespace mk {

namespace {

constexpr int kThreads = 64;
constexpr int KD = 2;   // derivative directions per pass (at 4 the dual state spilled 1.4 KB of stack per thread)
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

// A module hit's chi2 and update on its module's plane (Sec. 3.1) with the alignment
// displacement dm in the residual; 0 ok, 1 plane not reached, 3 update failed.  Not inlined: the
// dual-number kernels keep their registers for the layers without modules.
template <class T>
__device__ __noinline__ int grad_module_update(int kind, const PredT<T>& q, const float4* __restrict__ mods, int mod,
                                               float cB, T mx, T my, T mz, const T v[6], const T dm[3], StateT<T>& t,
                                               T& x2) {
    PredT<T> qp;
    FrameT<T> fp;
    if (!to_module_plane(kind, q, mods, mod, cB, qp, fp)) return 1;
    if (!chi2_hit(fp, qp, mx, my, mz, v, x2, dm) || !kalman_update_f(fp, qp, mx, my, mz, v, t, nullptr, dm))
        return 3;
    return 0;
}

// One step of the fit in scalar T: propagate to layer l (its thickness scaled by xs), then, with
// hit h >= 0, chi2 and update with the hit displaced by the alignment al (the displacement
// d + w x (h - c) enters the residual, not the FP32 hit position, whose ulp at 1 m is 0.08 um);
// h < 0 propagates only.  Returns 0 (ok; x2 = the step's chi2) or the fit's status code.
template <class T, bool MOD>
__device__ __forceinline__ int fit_step(const DevGeom& g, const DevParams& P, const float4* __restrict__ pay,
                                        int64_t n_hits, int l, int h, StateT<T>& t, const T al[6], const T& xs,
                                        T& x2) {
    const DevLayer& L = g.layers[l];
    PredT<T> q;
    int newton = 0;
    const int r = propagate_core<T, T>(L, g.cB, P.material, t, t.c, q, q.c, newton, nullptr, &xs);
    if (r != 1) return r == 0 ? 1 : 2;
    if (h >= n_hits) return 4;
    x2 = T(0.0f);
    if (h < 0) {
        pred_to_state(L.kind, q, t);
        return 0;
    }
    float mf[3], vf[6];
    int md = -1;
    if constexpr (MOD)
        load_hit(pay, h, mf, vf, nullptr, &md);
    else
        load_hit(pay, h, mf, vf, nullptr);
    const float cz = L.kind == MKGB_DISK ? L.pos : 0.0f;
    const T r0(mf[0]), r1(mf[1]), r2(mf[2] - cz);
    const T dm[3] = {al[0] + (al[4] * r2 - al[5] * r1), al[1] + (al[5] * r0 - al[3] * r2),
                     al[2] + (al[3] * r1 - al[4] * r0)};
    const T mx(mf[0]), my(mf[1]), mz(mf[2]);
    T v[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) v[c] = T(vf[c]);
    if (MOD && md >= 0) {   // a module hit, on its module's plane (not reached: status 1, as the fit)
        const int rm = grad_module_update(L.kind, q, g.mods, md, g.cB, mx, my, mz, v, dm, t, x2);
        if (rm == 1) pred_to_state(L.kind, q, t);
        return rm;
    }
    if (!chi2_hit(L.kind, q, mx, my, mz, v, x2, dm) || !kalman_update(L.kind, q, mx, my, mz, v, t, nullptr, dm))
        return 3;
    return 0;
}

template <bool MOD>
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
            for (int j = 0; j < nl; ++j) {
                const int l = lrow[j];
                const int cj = 6 + 7 * j;
                const float* al = align + 6 * l;
                D ald[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) ald[c] = seeded(al[c], cj + c, base);
                const D xs = seeded(xscale[l], cj + 6, base);
                D x2;
                status = fit_step<D, MOD>(g, P, pay, n_hits, l, hrow[j], t, ald, xs, x2);
                if (status != 0) break;
                sum += x2;
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

// Checkpoint of a step's input state: 32 floats (hi positions, lo positions, k, phi, theta, 21
// covariance words, theta's and phi's low parts), record j of track i at ((j * n + i) * 32).
__device__ __forceinline__ void store_ck(float* __restrict__ p, const State& t) {
    float4* v = reinterpret_cast<float4*>(p);
    v[0] = make_float4(t.xh, t.yh, t.zh, t.xl);
    v[1] = make_float4(t.yl, t.zl, t.k, t.phi);
    v[2] = make_float4(t.th, t.c[0], t.c[1], t.c[2]);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[3 + q] = make_float4(t.c[3 + 4 * q], t.c[4 + 4 * q], t.c[5 + 4 * q], t.c[6 + 4 * q]);
    v[7] = make_float4(t.c[19], t.c[20], t.tl, t.pl);
}

__device__ __forceinline__ void load_ck(const float* __restrict__ p, State& t) {
    const float4* v = reinterpret_cast<const float4*>(p);
    float4 a = v[0];
    t.xh = a.x; t.yh = a.y; t.zh = a.z; t.xl = a.w;
    a = v[1];
    t.yl = a.x; t.zl = a.y; t.k = a.z; t.phi = a.w;
    a = v[2];
    t.th = a.x; t.c[0] = a.y; t.c[1] = a.z; t.c[2] = a.w;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        a = v[3 + q];
        t.c[3 + 4 * q] = a.x; t.c[4 + 4 * q] = a.y; t.c[5 + 4 * q] = a.z; t.c[6 + 4 * q] = a.w;
    }
    a = v[7];
    t.c[19] = a.x; t.c[20] = a.y; t.tl = a.z; t.pl = a.w;
}

// Inputs of one step, in the adjoint's order: x, y, z, k, phi, theta, the 21 covariance words,
// the layer's 6 alignment parameters, its thickness scale.
constexpr int kStateIn = 27, kStepIn = 34;

template <bool MOD>
__global__ void __launch_bounds__(kThreads) k_fit_adjoint(
    const DevGeom* __restrict__ gp, DevParams P, const float4* __restrict__ pay, int64_t n_hits, int n,
    int max_steps, const int* __restrict__ layers, const int* __restrict__ hits, const float* __restrict__ p0,
    const float* __restrict__ c0, const float* __restrict__ align, const float* __restrict__ xscale,
    float* __restrict__ chi2_out, float* __restrict__ d_p0, float* __restrict__ d_align,
    float* __restrict__ d_xscale, int* __restrict__ status_out, float* __restrict__ ck) {
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
        // ---- plain pass, checkpointing the input of every step
        State t;
        {
            const float* pi = p0 + 6 * (int64_t)i;
            const float* ci = c0 + 21 * (int64_t)i;
            t.xh = pi[0]; t.yh = pi[1]; t.zh = pi[2];
            t.xl = 0.0f; t.yl = 0.0f; t.zl = 0.0f;
            t.k = pi[3]; t.phi = pi[4]; t.th = pi[5];
#pragma unroll 1
            for (int q = 0; q < 21; ++q) t.c[q] = ci[q];
        }
        int status = 0;
        float chi2v = 0.0f;
        for (int j = 0; j < nl && status == 0; ++j) {
            const int l = lrow[j];
            store_ck(ck + ((int64_t)j * n + i) * 32, t);
            float x2 = 0.0f;
            status = fit_step<float, MOD>(g, P, pay, n_hits, l, hrow[j], t, align + 6 * l, xscale[l], x2);
            chi2v += x2;
        }
        // ---- reverse sweep
        float lam[kStateIn];   // d total / d (state after step j)
#pragma unroll
        for (int c = 0; c < kStateIn; ++c) lam[c] = 0.0f;
        for (int j = nl - 1; j >= 0 && status == 0; --j) {
            const int l = lrow[j], h = hrow[j];
            State t0;
            load_ck(ck + ((int64_t)j * n + i) * 32, t0);
            const float* al = align + 6 * l;
            float lnew[kStateIn];
            for (int base = 0; base < kStepIn; base += KD) {
                // without a hit the alignment has no effect: skip passes that seed only it
                if (h < 0 && base >= kStateIn + 1 && base + KD <= kStepIn - 1) continue;
                StateT<D> td;
                td.xh = seeded(t0.xh, 0, base); td.yh = seeded(t0.yh, 1, base); td.zh = seeded(t0.zh, 2, base);
                td.xl = D(t0.xl); td.yl = D(t0.yl); td.zl = D(t0.zl);
                td.k = seeded(t0.k, 3, base); td.phi = seeded(t0.phi, 4, base); td.th = seeded(t0.th, 5, base);
                td.tl = D(t0.tl);
                td.pl = D(t0.pl);
#pragma unroll 1
                for (int q = 0; q < 21; ++q) td.c[q] = seeded(t0.c[q], 6 + q, base);
                D ald[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) ald[c] = seeded(al[c], kStateIn + c, base);
                const D xs = seeded(xscale[l], kStepIn - 1, base);
                D x2;
                if (fit_step<D, MOD>(g, P, pay, n_hits, l, h, td, ald, xs, x2) != 0) {
                    status = 5;   // the redone step failed where the plain pass did not
                    break;
                }
#pragma unroll
                for (int k = 0; k < KD; ++k) {
                    const int comp = base + k;
                    if (comp >= kStepIn) break;
                    float a = x2.d[k];
                    a = fmaf(lam[0], td.xh.d[k] + td.xl.d[k], a);
                    a = fmaf(lam[1], td.yh.d[k] + td.yl.d[k], a);
                    a = fmaf(lam[2], td.zh.d[k] + td.zl.d[k], a);
                    a = fmaf(lam[3], td.k.d[k], a);
                    a = fmaf(lam[4], td.phi.d[k] + td.pl.d[k], a);
                    a = fmaf(lam[5], td.th.d[k] + td.tl.d[k], a);
#pragma unroll
                    for (int q = 0; q < 21; ++q) a = fmaf(lam[6 + q], td.c[q].d[k], a);
                    if (comp < kStateIn)
                        lnew[comp] = a;
                    else if (a != 0.0f)
                        atomicAdd(acc + l * 7 + (comp - kStateIn), a);
                }
            }
#pragma unroll
            for (int c = 0; c < kStateIn; ++c) lam[c] = lnew[c];
        }
        if (status != 0) {
            chi2v = 0.0f;
#pragma unroll
            for (int c = 0; c < 6; ++c) lam[c] = 0.0f;
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) d_p0[6 * (int64_t)i + c] = lam[c];
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
                            float* d_xscale, int* status_out, float* ck, bool modular) {
    if (n == 0) return cudaSuccess;
    const int blocks = (n + kThreads - 1) / kThreads;
    auto adjoint = modular ? k_fit_adjoint<true> : k_fit_adjoint<false>;
    auto forward = modular ? k_fit_grad<true> : k_fit_grad<false>;
    if (ck)
        adjoint<<<blocks, kThreads, 0, st>>>(g, P, pay, n_hits, n, max_steps, layers, hits, p0, c0, align,
                                                   xscale, chi2_out, d_p0, d_align, d_xscale, status_out, ck);
    else
        forward<<<blocks, kThreads, 0, st>>>(g, P, pay, n_hits, n, max_steps, layers, hits, p0, c0, align, xscale,
                                                chi2_out, d_p0, d_align, d_xscale, status_out);
    return cudaGetLastError();
}

}  // namespace mk
