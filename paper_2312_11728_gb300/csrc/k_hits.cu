// Layer-hit binning (a2) and seed ordering (a3).
//
// Sec. 3.1: a layer aggregates hits so that track search proceeds uniformly; Sec. 2.2:
// seeds are sorted in (eta, phi) to improve hit-access coherency.  Each (event, layer)
// segment of hits gets an eta-phi bin index built by a counting sort: per-hit bin ids
// and an atomic histogram, one device-wide exclusive scan of the histogram (which gives
// every bin's first position, segments following each other in input order), then an
// atomic-cursor scatter of (eta, phi) and the 48-byte payload into bin order.  Order
// inside a bin is not fixed; no result depends on it (selection ties break on hit id).
// HBM-bound: ~36 B read + ~104 B written per hit, plus the histogram.
#include "internal.h"

namespace mk {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int upper_seg(const int64_t* __restrict__ off, int n_seg, int64_t i) {
    // largest s in [0, n_seg) with off[s] <= i
    int lo = 0, hi = n_seg;   // off[lo] <= i < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// Hits [h0, h1) of the n_seg segments (a chunk of whole events, or all of them).
__global__ void __launch_bounds__(kThreads) k_hit_prep(const DevGeom* __restrict__ g, int n_layers,
                                                       const int64_t* __restrict__ seg_off, int n_seg,
                                                       int64_t h0, int64_t h1, const float* __restrict__ xyz,
                                                       const float* __restrict__ cov,
                                                       const int* __restrict__ hit_mod, int bins_per_event,
                                                       float4* __restrict__ pay, float2* __restrict__ ep_tmp,
                                                       int* __restrict__ bin_of_hit, int* __restrict__ hit_seg,
                                                       int* __restrict__ counts) {
    for (int64_t i = h0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < h1;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int seg = upper_seg(seg_off, n_seg, i);
        const int e = seg / n_layers, l = seg - e * n_layers;
        const DevLayer& L = g->layers[l];
        const float x = __ldg(xyz + 3 * i), y = __ldg(xyz + 3 * i + 1), z = __ldg(xyz + 3 * i + 2);
        float v[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) v[j] = __ldg(cov + 6 * i + j);
        pay[3 * i] = make_float4(x, y, z, __int_as_float((int)i));
        pay[3 * i + 1] = make_float4(v[0], v[1], v[2], v[3]);
        pay[3 * i + 2] = make_float4(v[4], v[5], __int_as_float(hit_mod ? __ldg(hit_mod + i) : -1), 0.0f);
        const float eta = asinhf(z / sqrtf(x * x + y * y));
        const float phi = atan2f(y, x);
        const float fe = (eta - L.eta_lo) * L.eta_scale;
        int ie = fe >= 0.0f ? (int)fminf(floorf(fe), (float)(L.n_eta - 1)) : 0;
        const float fp = (phi + kPi) * (L.n_phi * (1.0f / kTwoPi));
        int ip = fp >= 0.0f ? (int)fminf(floorf(fp), (float)(L.n_phi - 1)) : 0;
        const int gb = e * bins_per_event + L.bin_base + ie * L.n_phi + ip;
        ep_tmp[i] = make_float2(eta, phi);
        bin_of_hit[i] = gb;
        hit_seg[i] = seg;
        atomicAdd(counts + gb, 1);
    }
}

__global__ void __launch_bounds__(kThreads) k_hit_scatter(int64_t n_hits, const float4* __restrict__ pay,
                                                          const float2* __restrict__ ep_tmp,
                                                          const int* __restrict__ bin_of_hit, int* cursor,
                                                          float2* __restrict__ hb_ep, float4* __restrict__ hb_pay) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_hits;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int pos = atomicAdd(cursor + bin_of_hit[i], 1);
        hb_ep[pos] = ep_tmp[i];
        hb_pay[3 * (int64_t)pos] = pay[3 * i];
        hb_pay[3 * (int64_t)pos + 1] = pay[3 * i + 1];
        hb_pay[3 * (int64_t)pos + 2] = pay[3 * i + 2];
    }
}

// ---- device-wide exclusive scan (block scan + recursive scan of block totals)
constexpr int kScanT = 256, kScanI = 8, kScanB = kScanT * kScanI;

__global__ void __launch_bounds__(kScanT) k_scan_block(const int* in, int* out, int64_t n, int* bsum) {
    __shared__ int sh[kScanB];
    __shared__ int wsum[kScanT / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanB;
    for (int j = threadIdx.x; j < kScanB; j += kScanT) {
        const int64_t k = base + j;
        sh[j] = k < n ? in[k] : 0;
    }
    __syncthreads();
    int v[kScanI];
    int tot = 0;
#pragma unroll
    for (int i = 0; i < kScanI; ++i) {
        v[i] = sh[threadIdx.x * kScanI + i];
        tot += v[i];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = tot;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < kScanT / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += y;
        }
        if (lane < kScanT / 32) wsum[lane] = s;
    }
    __syncthreads();
    int run = x - tot + (w > 0 ? wsum[w - 1] : 0);
#pragma unroll
    for (int i = 0; i < kScanI; ++i) {
        sh[threadIdx.x * kScanI + i] = run;
        run += v[i];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kScanB; j += kScanT) {
        const int64_t k = base + j;
        if (k < n) out[k] = sh[j];
    }
    if (threadIdx.x == kScanT - 1) bsum[blockIdx.x] = run;
}

__global__ void __launch_bounds__(kScanT) k_scan_add(int* out, int64_t n, const int* boff) {
    const int add = boff[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kScanB;
    for (int j = threadIdx.x; j < kScanB; j += kScanT) {
        const int64_t k = base + j;
        if (k < n) out[k] += add;
    }
}

__global__ void k_copy_int(const int* src, int* dst) { *dst = *src; }

__global__ void __launch_bounds__(kThreads) k_seed_scatter(int n, const int* __restrict__ key_of, int* cursor,
                                                           int* __restrict__ order) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) order[atomicAdd(cursor + key_of[i], 1)] = i;
}

int grid_for(int64_t n) {
    const int64_t b = (n + kThreads - 1) / kThreads;
    return (int)(b < 1 ? 1 : (b > 152 * 64 ? 152 * 64 : b));
}

// Hits whose module does not fit their layer: a module hit on a layer without modules or on another
// layer's module, a hit without module on a modular layer, a module index out of range.
__global__ void __launch_bounds__(kThreads) k_check_modules(const DevGeom* __restrict__ g, int n_layers,
                                                            int64_t n_hits, const int* __restrict__ hit_seg,
                                                            const int* __restrict__ hit_mod, int* bad) {
    int nb = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_hits;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int l = hit_seg[i] % n_layers;
        const int m = hit_mod[i];
        const bool modular = g->layers[l].modular != 0;
        bool ok;
        if (m < 0) {
            ok = m == -1 && !modular;
        } else {
            ok = modular && m < g->n_mods && __float_as_int(__ldg(g->mods + 2 * m).w) == l;
        }
        nb += ok ? 0 : 1;
    }
    if (nb) atomicAdd(bad, nb);
}

}  // namespace

cudaError_t launch_check_modules(cudaStream_t st, const DevGeom* g, int n_layers, int64_t n_hits,
                                 const int* hit_seg, const int* hit_mod, int* bad) {
    if (n_hits == 0) return cudaSuccess;
    k_check_modules<<<grid_for(n_hits), kThreads, 0, st>>>(g, n_layers, n_hits, hit_seg, hit_mod, bad);
    return cudaGetLastError();
}

cudaError_t launch_hit_prep(cudaStream_t st, const DevGeom* g, int n_layers, const int64_t* seg_off, int n_seg,
                            int64_t n_hits, const float* xyz, const float* cov, const int* hit_mod,
                            int bins_per_event, float4* pay, float2* ep_tmp, int* bin_of_hit, int* hit_seg,
                            int* counts, int64_t h0, int64_t h1) {
    if (h1 < 0) h1 = n_hits;
    if (h1 <= h0) return cudaSuccess;
    k_hit_prep<<<grid_for(h1 - h0), kThreads, 0, st>>>(g, n_layers, seg_off, n_seg, h0, h1, xyz, cov, hit_mod,
                                                       bins_per_event, pay, ep_tmp, bin_of_hit, hit_seg, counts);
    return cudaGetLastError();
}

cudaError_t launch_hit_scatter(cudaStream_t st, int64_t n_hits, const float4* pay, const float2* ep_tmp,
                               const int* bin_of_hit, int* cursor, float2* hb_ep, float4* hb_pay) {
    if (n_hits == 0) return cudaSuccess;
    k_hit_scatter<<<grid_for(n_hits), kThreads, 0, st>>>(n_hits, pay, ep_tmp, bin_of_hit, cursor, hb_ep, hb_pay);
    return cudaGetLastError();
}

size_t scan_tmp_ints(int64_t n) {
    size_t tot = 0;
    int64_t m = n;
    while (m > kScanB) {
        const int64_t nb = (m + kScanB - 1) / kScanB;
        tot += 2 * nb + 1;
        m = nb;
    }
    return tot + 16;
}

cudaError_t exclusive_scan(cudaStream_t st, const int* in, int* out, int64_t n, int* tmp) {
    const int64_t nb = (n + kScanB - 1) / kScanB;
    if (nb <= 1) {
        k_scan_block<<<1, kScanT, 0, st>>>(in, out, n, out + n);
        return cudaGetLastError();
    }
    int* bsum = tmp;
    int* boff = tmp + nb;
    k_scan_block<<<(unsigned)nb, kScanT, 0, st>>>(in, out, n, bsum);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = exclusive_scan(st, bsum, boff, nb, tmp + 2 * nb + 1);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)nb, kScanT, 0, st>>>(out, n, boff);
    k_copy_int<<<1, 1, 0, st>>>(boff + nb, out + n);
    return cudaGetLastError();
}

cudaError_t launch_seed_scatter(cudaStream_t st, int n, const int* key_of, int* cursor, int* order) {
    if (n == 0) return cudaSuccess;
    k_seed_scatter<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(n, key_of, cursor, order);
    return cudaGetLastError();
}

}  // namespace mk
