// Arithmetic-throughput probes: the FP32 and FP64 fused multiply-add rates this device sustains,
// the denominators of the search's and the seed fit's rooflines (the method itself has no such
// step).  Each thread runs kChains independent multiply-add chains (enough independent work per
// warp to cover the pipeline latency at full occupancy); the result is folded into one word per
// thread so that no chain is dead code.
#include "internal.h"

namespace mk {

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

template <class T>
__global__ void __launch_bounds__(kThreads) k_probe_fma(int iters, T b, T c, T* __restrict__ sink) {
    T acc[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc[j] = T(threadIdx.x + j);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int j = 0; j < kChains; ++j) acc[j] = fma(acc[j], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += acc[j];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

cudaError_t launch_probe_fma(cudaStream_t st, int kind, int n_sms, int iters, void* sink, int64_t* fma_count) {
    int per_sm = 0;
    const void* k = kind == 0 ? (const void*)k_probe_fma<float> : (const void*)k_probe_fma<double>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int blocks = n_sms * per_sm;
    *fma_count = (int64_t)blocks * kThreads * iters * 16 * kChains;
    // b slightly below 1 and c small keep the chains finite for any iteration count
    if (kind == 0)
        k_probe_fma<float><<<blocks, kThreads, 0, st>>>(iters, 0.999999f, 1e-6f, static_cast<float*>(sink));
    else
        k_probe_fma<double><<<blocks, kThreads, 0, st>>>(iters, 0.999999, 1e-6, static_cast<double*>(sink));
    return cudaGetLastError();
}

size_t probe_sink_bytes(int n_sms) { return (size_t)n_sms * 32 * kThreads * sizeof(double); }

}  // namespace mk
