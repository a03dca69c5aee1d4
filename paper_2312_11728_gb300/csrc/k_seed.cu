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
//
// Precision: the seed fit's covariance arithmetic runs in FP64.  Its diffuse prior makes every
// update badly conditioned (the innovation covariance S has a condition number of ~1e6 at the
// median seed): the posterior variance along a precisely measured direction is a small
// difference of numbers that FP32 rounding has already perturbed.  The trajectory and Jacobian
// of each step are FP32 in the FP32 path (seed.cuh, kSeedMixed); seeds whose q/pT is too small
// for the FP32 trajectory's accuracy are fitted again in FP64 from a device list.  Another
// kernel computes the (event, eta, phi) ordering keys.
#include "seed.cuh"

namespace mk {

namespace {

constexpr int kThreads = 128;

__device__ __forceinline__ void load_geom(const DevGeom* __restrict__ gp, DevGeom& g) {
    const int4* src = reinterpret_cast<const int4*>(gp);
    int4* dst = reinterpret_cast<int4*>(&g);
    for (int i = threadIdx.x; i < (int)(sizeof(DevGeom) / 16); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
}

__device__ __forceinline__ void write_seed(const State& t, int i, int region, int start, int event, float* state,
                                           int4* info, float* state6, float* cov21, int* info3) {
    float* o = state + (int64_t)i * kSeedStateStride;
    o[0] = t.xh; o[1] = t.yh; o[2] = t.zh; o[3] = t.xl; o[4] = t.yl; o[5] = t.zl;
    o[6] = t.k; o[7] = t.phi; o[8] = t.th;
#pragma unroll
    for (int q = 0; q < 21; ++q) o[9 + q] = t.c[q];
    o[30] = t.tl;
    o[31] = t.pl;
    const int status = region >= 0 ? 0 : 1;
    info[i] = make_int4(region, start, event, status);
    if (state6) store_state6(t, state6 + 6 * (int64_t)i, cov21 + 21 * (int64_t)i);
    if (info3) {
        info3[3 * i] = region;
        info3[3 * i + 1] = start;
        info3[3 * i + 2] = status;
    }
}

// The chunk of a hit id among the range's chunk offsets (-1: outside them all).
__device__ __forceinline__ int chunk_of(const SeedRange& r, int h) {
    for (int k = 0; k < r.n_chunks; ++k)
        if (h >= r.off[k] && h < r.off[k + 1]) return k;
    return -1;
}

// MOD: module hits loaded (seed hits on modules are used on their planes); the plain
// instantiation keeps the layers-only registers.  MODE: the seed fit's precision mode (seed.cuh).
// redo_in (may be nullptr): the seeds to fit, a list of redo_in[0] seed indices at redo_in + 1
// (grid-stride); else seed i = the thread.  redo_out (kSeedMixed only, may be nullptr): seeds whose
// |q/pT| falls below kSeedKappaRedo are appended there in the same layout, to be fitted again.
template <int MODE, bool MOD>
__global__ void __launch_bounds__(kThreads) k_seed(const DevGeom* __restrict__ gp, DevParams P, HitStore H, int n,
                                                   const int* __restrict__ seed_hits, float* __restrict__ state,
                                                   double* __restrict__ state64, int4* __restrict__ info,
                                                   float* state6, float* cov21, int* info3, SeedRange range,
                                                   const int* __restrict__ redo_in, int* __restrict__ redo_out) {
    __shared__ DevGeom g;
    load_geom(gp, g);
    const int n_items = redo_in ? redo_in[0] : n;
    for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < n_items; item += gridDim.x * blockDim.x) {
        const int i = redo_in ? redo_in[1 + item] : item;
        if (range.which >= 0) {   // hits arriving in chunks: the seeds of one chunk, or the rest
            const int c0 = chunk_of(range, seed_hits[3 * i]), c1 = chunk_of(range, seed_hits[3 * i + 1]),
                      c2 = chunk_of(range, seed_hits[3 * i + 2]);
            const bool in_one = c0 >= 0 && c0 == c1 && c1 == c2;
            if (range.which < range.n_chunks ? !(in_one && c0 == range.which) : in_one) continue;
        }
        StateT<double> td;
        int lay[3], event, region, start;
        const bool ok = seed_fit<double, MODE, MOD>(g, P, H, seed_hits, i, td, lay, event);
        if (MODE == kSeedMixed && redo_out && ok && fabs(td.k) < kSeedKappaRedo) {
            redo_out[1 + atomicAdd(redo_out, 1)] = i;
            continue;   // written by the redo
        }
        State t;
        narrow_state(td, t);
        seed_region(g, P, t.th, lay[2], ok, region, start);
        write_seed(t, i, region, start, event, state, info, state6, cov21, info3);
        if (state64) {   // the FP64 state for the all-FP64 search
            double* o = state64 + (int64_t)i * kSeedStateStride;
            o[0] = td.xh; o[1] = td.yh; o[2] = td.zh; o[3] = td.xl; o[4] = td.yl; o[5] = td.zl;
            o[6] = td.k; o[7] = td.phi; o[8] = td.th;
#pragma unroll
            for (int q = 0; q < 21; ++q) o[9 + q] = td.c[q];
            o[30] = td.tl; o[31] = td.pl;
        }
    }
}

// (event, eta cell, phi cell) key of every seed and its histogram, for the hit-coherent order
__global__ void __launch_bounds__(kThreads) k_seed_key(int n, const float* __restrict__ state,
                                                       const int4* __restrict__ info, int* __restrict__ key_of,
                                                       int* __restrict__ key_counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* o = state + (int64_t)i * kSeedStateStride;
    const float eta = -logf(tanf(0.5f * o[8]));
    int ce = (int)floorf((eta + 4.0f) * (kSeedEtaCells / 8.0f));
    ce = ce < 0 ? 0 : (ce >= kSeedEtaCells ? kSeedEtaCells - 1 : ce);
    int cp = (int)floorf((o[7] + kPi) * (kSeedPhiCells / kTwoPi));
    cp = cp < 0 ? 0 : (cp >= kSeedPhiCells ? kSeedPhiCells - 1 : cp);
    const int key = (info[i].z * kSeedEtaCells + ce) * kSeedPhiCells + cp;
    key_of[i] = key;
    atomicAdd(key_counts + key, 1);
}

}  // namespace

cudaError_t launch_seed_fit(cudaStream_t st, const DevGeom* g, DevParams P, HitStore H, int n, const int* seed_hits,
                            float* state, double* state64, int4* info, float* state6, float* cov21, int* info3,
                            const SeedRange& range, bool modular, int* redo) {
    if (n == 0) return cudaSuccess;
    const int blocks = (n + kThreads - 1) / kThreads;
    if (P.precision == MKGB_FP64) {   // the plain all-FP64 path
        auto kern = modular ? k_seed<kSeedPlain, true> : k_seed<kSeedPlain, false>;
        kern<<<blocks, kThreads, 0, st>>>(g, P, H, n, seed_hits, state, state64, info, state6, cov21, info3, range,
                                          nullptr, nullptr);
        return cudaGetLastError();
    }
    // the FP32 path: mixed-precision seed fits, the low-|q/pT| ones redone FP32-assisted in FP64
    // when a redo list is given (redo[0] must be zero before the first launch of a batch)
    auto kern = modular ? k_seed<kSeedMixed, true> : k_seed<kSeedMixed, false>;
    kern<<<blocks, kThreads, 0, st>>>(g, P, H, n, seed_hits, state, state64, info, state6, cov21, info3, range,
                                      nullptr, redo);
    return cudaGetLastError();
}

cudaError_t launch_seed_redo(cudaStream_t st, const DevGeom* g, DevParams P, HitStore H, int n, const int* seed_hits,
                             float* state, int4* info, float* state6, float* cov21, int* info3, bool modular,
                             const int* redo, int n_sms) {
    if (n == 0 || P.precision == MKGB_FP64) return cudaSuccess;
    const int need = (n + kThreads - 1) / kThreads, cap = 8 * n_sms;
    const int blocks = need < cap ? need : cap;   // grid-stride over the list, whose length the device holds
    auto kern = modular ? k_seed<kSeedAssisted, true> : k_seed<kSeedAssisted, false>;
    kern<<<blocks, kThreads, 0, st>>>(g, P, H, n, seed_hits, state, nullptr, info, state6, cov21, info3, SeedRange(),
                                      redo, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_seed_keys(cudaStream_t st, int n, const float* state, const int4* info, int* key_of,
                             int* key_counts) {
    if (n == 0) return cudaSuccess;
    k_seed_key<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(n, state, info, key_of, key_counts);
    return cudaGetLastError();
}

}  // namespace mk
