// Seed cleaning and the quality filter with duplicate removal (Sec. 2.2: seeds are processed in
// parallel, so hits consumed by earlier tracks cannot be masked; duplicates are removed from the
// resulting tracks).
//
// Both compare items (rows of hit ids; < 0 = none) that share hits.  An index of the items on
// each hit (counting sort by hit id: counts, scan, fill) lists, for every hit of an item, the
// other items on it; one thread per item walks those and counts the hits it shares with each
// better item by comparing the two rows.  The decision is an OR over the better items, so it does
// not depend on the order in which the index lists them.
//   seeds: a seed is dropped if a seed of lower index shares at least two of its three hits;
//   tracks: a track with fewer than min_hits hits is dropped, and a track is dropped if a better
//   track (higher score, equal score and lower index) shares at least frac x the smaller hit
//   count.  Every item is judged against all others (not transitively).
#include "internal.h"

namespace mk {

namespace {

constexpr int kThreads = 256;

__global__ void k_item_hit_count(int64_t n_entries, const int* __restrict__ hits, int64_t n_hits, int* cnt) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_entries; q += (int64_t)gridDim.x * blockDim.x) {
        const int h = hits[q];
        if (h >= 0 && h < n_hits) atomicAdd(cnt + h, 1);
    }
}

__global__ void k_item_hit_fill(int n, int width, const int* __restrict__ hits, int64_t n_hits, int* cursor,
                                int* items) {
    const int64_t total = (int64_t)n * width;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int h = hits[q];
        if (h >= 0 && h < n_hits) items[atomicAdd(cursor + h, 1)] = (int)(q / width);
    }
}

__device__ __forceinline__ int row_hits(const int* __restrict__ a, int width, int64_t n_hits) {
    int c = 0;
    for (int i = 0; i < width; ++i) c += (a[i] >= 0 && a[i] < n_hits);
    return c;
}

__device__ __forceinline__ int row_shared(const int* __restrict__ a, const int* __restrict__ b, int width,
                                          int64_t n_hits) {
    int s = 0;
    for (int i = 0; i < width; ++i) {
        const int h = a[i];
        if (h < 0 || h >= n_hits) continue;
        for (int j = 0; j < width; ++j)
            if (b[j] == h) {
                ++s;
                break;
            }
    }
    return s;
}

// mode 0: seeds (better = lower index, drop at >= 2 shared); mode 1: tracks (score, frac, min_hits)
__global__ void __launch_bounds__(kThreads) k_item_decide(int mode, int n, int width, const int* __restrict__ hits,
                                                          const float* __restrict__ score, int64_t n_hits,
                                                          int min_hits, float frac, const int* __restrict__ off,
                                                          const int* __restrict__ items, int* keep) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int* a = hits + (int64_t)t * width;
    const int na = row_hits(a, width, n_hits);
    bool k = mode == 0 || na >= min_hits;
    const float st = mode == 1 ? score[t] : 0.0f;
    for (int i = 0; i < width && k; ++i) {
        const int h = a[i];
        if (h < 0 || h >= n_hits) continue;
        for (int q = off[h]; q < off[h + 1] && k; ++q) {
            const int u = items[q];
            if (u == t) continue;
            const int* b = hits + (int64_t)u * width;
            if (mode == 0) {
                if (u < t && row_shared(a, b, width, n_hits) >= 2) k = false;
            } else {
                const float su = score[u];
                if (!(su > st || (su == st && u < t))) continue;
                const int nb = row_hits(b, width, n_hits);
                const int s = row_shared(a, b, width, n_hits);
                if ((double)s >= (double)frac * (double)(na < nb ? na : nb)) k = false;
            }
        }
    }
    keep[t] = k ? 1 : 0;
}

}  // namespace

size_t clean_scratch_ints(int n, int width, int64_t n_hits) {
    // counts/offsets (n_hits + 1), cursor (n_hits + 1), items (n x width), scan scratch
    return 2 * ((size_t)n_hits + 1) + (size_t)n * width + scan_tmp_ints(n_hits) + 64;
}

cudaError_t launch_item_decide(cudaStream_t st, int mode, int n, int width, const int* hits, const float* score,
                               int64_t n_hits, int min_hits, float frac, int* scratch, int* keep, int n_sms) {
    if (n == 0) return cudaSuccess;
    int* off = scratch;
    int* cursor = off + (n_hits + 1);
    int* items = cursor + (n_hits + 1);
    int* tmp = items + (int64_t)n * width;
    cudaError_t e = cudaMemsetAsync(off, 0, 4 * ((size_t)n_hits + 1), st);
    if (e != cudaSuccess) return e;
    const int64_t entries = (int64_t)n * width;
    const int grid = 8 * n_sms;
    k_item_hit_count<<<grid, kThreads, 0, st>>>(entries, hits, n_hits, off);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = exclusive_scan(st, off, off, n_hits, tmp)) != cudaSuccess) return e;   // off[n_hits] = total
    if ((e = cudaMemcpyAsync(cursor, off, 4 * ((size_t)n_hits + 1), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return e;
    k_item_hit_fill<<<grid, kThreads, 0, st>>>(n, width, hits, n_hits, cursor, items);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_item_decide<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(mode, n, width, hits, score, n_hits, min_hits,
                                                                        frac, off, items, keep);
    return cudaGetLastError();
}

}  // namespace mk
