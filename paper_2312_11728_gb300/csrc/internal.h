// Internal interfaces between the C-ABI layer (api.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kalman.cuh"

namespace mk {

// Child kinds of a candidate at one layer (a10).
enum : int { K_NONE = 0, K_HIT = 1, K_MISS = 2, K_SKIP = 3, K_STOP = 4, K_CARRY = 5 };

constexpr int kSeedStateStride = 32;   // xh,yh,zh,xl,yl,zl,k,phi,th,c[21],pad,pad
constexpr int kSeedEtaCells = 32;      // coarse eta-phi cells for the seed order (a3)
constexpr int kSeedPhiCells = 64;

// Hits after mkgb_load_hits: original order (payload) and the binned copy (a2).
struct HitStore {
    const int64_t* seg_off;    // E*L + 1 (device)
    int n_events, n_layers;
    int64_t n_hits;
    const float4* pay;         // 3 float4 per hit, original order: (x,y,z,id) (v0..v3) (v4,v5,-,-)
    const float2* hb_ep;       // binned order: (eta, phi)
    const float4* hb_pay;      // binned order payload
    const int* bin_start;      // E*bins_per_event + 1 offsets into the binned arrays
    const int* hit_seg;        // per hit: segment e*L + l
};

struct SeedStore {
    int n;
    const float* state;        // n x kSeedStateStride
    const double* state64;     // n x kSeedStateStride, FP64 states (precision MKGB_FP64 only)
    const int4* info;          // n: (region, first plan step, event, status)
    const int* order;          // n: seeds sorted by (event, eta cell, phi cell)
};

struct BuildOutDev {
    float* params;
    float* cov;
    float* chi2;
    float* score;
    int* nfound;
    int* nholes;
    int* hits;
    int max_plan;
    int* ovl = nullptr;   // n x max_plan overlap hit ids (-1 none), nullptr: not wanted
};

// Work buffers of the search (k_build.cu): per seed 8 candidate slots, double-buffered.
struct BuildWork {
    unsigned char* st[2];   // slot states, 32 words (FP32 or FP64 per the precision)
    int4* meta[2];    // slot (score, chi2 sum, nfound | nholes << 8 | stopped << 16, alive)
    unsigned char* pr;      // slot predictions at the round's layer, 28 words
    // slot children: (n hits, non-hit kind, non-hit score, b2) + 4 x (chi2, hit, chi2, hit); b2: with
    // module hits, the best accepted hit on another module than the first entry's (-1 none)
    int4* ls;
    int* live[2];     // work list of live candidate slots per round
    int* seeds[2];    // work list of seeds with a live candidate per round
    int4* sinfo;      // per ordered seed: (plan position of its first step, first step, steps, event)
    int* fin;         // per ordered seed: buffer holding its final slots | (rounds searched << 1), -1 none
    int* trail;       // per ordered seed: longest plan x 8 ints ((code + 4) << 3 | parent slot)
    int* otrail;      // the same layout: overlap hit id of the step (-1 none); nullptr without modules
    int* rescue;      // kept children of the round whose update is redone in FP64
    int* counts;      // [live0, live1, seeds0, seeds1, rescue]
    // fused rounds: [tau] length of round tau's live list, [kRescueCountBase + tau] its FP64 redo list
    int* rcounts;
};
constexpr int kRescueCountBase = MKGB_MAX_PLAN + 2;
constexpr int kRoundCountInts = 2 * kRescueCountBase;

// counters (64-bit): [0] steps, [1] chi2 evaluations, [2] updates, [3] hits tested, [4] Newton iterations
constexpr int kNumCounters = 5;

// ---- k_hits.cu
// hit_mod (may be nullptr: every hit on its layer's own surface) goes into the payload.  Prepares
// hits [h0, h1) (h1 < 0: up to n_hits), so that a batch arriving in chunks is prepared per chunk.
cudaError_t launch_hit_prep(cudaStream_t st, const DevGeom* g, int n_layers, const int64_t* seg_off, int n_seg,
                            int64_t n_hits, const float* xyz, const float* cov, const int* hit_mod,
                            int bins_per_event, float4* pay, float2* ep_tmp, int* bin_of_hit, int* hit_seg,
                            int* counts, int64_t h0 = 0, int64_t h1 = -1);
// Counts into *bad the hits whose module does not fit their layer (a module hit on a layer without
// modules or on another layer's module, a hit without module on a modular layer, an index out of range).
cudaError_t launch_check_modules(cudaStream_t st, const DevGeom* g, int n_layers, int64_t n_hits,
                                 const int* hit_seg, const int* hit_mod, int* bad);
cudaError_t launch_hit_scatter(cudaStream_t st, int64_t n_hits, const float4* pay, const float2* ep_tmp,
                               const int* bin_of_hit, int* cursor, float2* hb_ep, float4* hb_pay);
// Exclusive scan of n ints (out[n] gets the total); tmp must hold scan_tmp_ints(n) ints.
size_t scan_tmp_ints(int64_t n);
cudaError_t exclusive_scan(cudaStream_t st, const int* in, int* out, int64_t n, int* tmp);
cudaError_t launch_seed_scatter(cudaStream_t st, int n, const int* key_of, int* cursor, int* order);

// ---- k_seed.cu
// The seeds one launch of the seed fit takes: which < 0 all of them; with the hits arriving in
// n_chunks chunks of whole events (hit ids [off[k], off[k + 1])), which = k the seeds whose three
// hits lie in chunk k, which = n_chunks the rest (hits in several chunks or invalid ids), fitted
// once every chunk has been prepared.
constexpr int kMaxSeedChunks = 8;
struct SeedRange {
    int which = -1;
    int n_chunks = 0;
    int off[kMaxSeedChunks + 1] = {};
};
// modular: module hits loaded (a seed hit on a module is used on its module's plane).  The FP32
// path's seed fits are mixed-precision; those with |q/pT| below a limit are left to
// launch_seed_redo through redo (n + 1 ints: the count, zeroed before the batch's first launch,
// then the seed indices).  The all-FP64 path fits every seed in FP64 and ignores redo.
cudaError_t launch_seed_fit(cudaStream_t st, const DevGeom* g, DevParams P, HitStore H, int n, const int* seed_hits,
                            float* state, double* state64, int4* info, float* state6, float* cov21, int* info3,
                            const SeedRange& range, bool modular, int* redo);
// The FP64 (FP32-assisted) fits of the seeds listed in redo, after every launch_seed_fit of the batch.
cudaError_t launch_seed_redo(cudaStream_t st, const DevGeom* g, DevParams P, HitStore H, int n, const int* seed_hits,
                             float* state, int4* info, float* state6, float* cov21, int* info3, bool modular,
                             const int* redo, int n_sms);
cudaError_t launch_seed_keys(cudaStream_t st, int n, const float* state, const int4* info, int* key_of,
                             int* key_counts);

// ---- k_build.cu
// with_ovl: room for the overlap hits of modular layers (the otrail array)
size_t build_work_bytes(int n_seeds, int max_plan_len, int precision, bool with_ovl = false);
BuildWork carve_build_work(void* base, int n_seeds, int max_plan_len, int precision, bool with_ovl = false);
struct BuildGraph;
BuildGraph* build_graph_create();
void build_graph_destroy(BuildGraph* gph);
// find_shape / select_shape: launch shapes of the round kernels (0 default; 1, 2 alternatives the
// autotuner tries); gph: graph cache of the context (nullptr: plain launches).
cudaError_t launch_build(cudaStream_t st, const DevGeom* g, int max_plan_len, DevParams P, HitStore H, SeedStore S,
                         BuildOutDev out, BuildWork w, unsigned long long* counters, int n_sms, int find_shape,
                         int select_shape, BuildGraph* gph, bool backward = false);
// Start records of the backward search; g holds the geometry with every region's plan reversed.
cudaError_t launch_bw_seed(cudaStream_t st, const DevGeom* g, DevParams P, int n, const float* p, const float* c,
                           const int* first_layer, const int* event, float* state, int4* info, int* order);

// ---- k_fit.cu
// ---- k_grad.cu
// FMA-throughput probe (kind 0 FP32, 1 FP64): one resident grid of iters x 16 x 8 chained
// multiply-adds per thread into sink (probe_sink_bytes); fma_count gets the multiply-adds issued.
cudaError_t launch_probe_fma(cudaStream_t st, int kind, int n_sms, int iters, void* sink, int64_t* fma_count);
size_t probe_sink_bytes(int n_sms);

// Derivative of the fit's total chi2: reverse sweep when ck (n x max_steps x 32 floats of
// checkpoints) is given, forward mode when it is nullptr.
cudaError_t launch_fit_grad(cudaStream_t st, const DevGeom* g, DevParams P, const float4* pay, int64_t n_hits, int n,
                            int max_steps, const int* layers, const int* hits, const float* p0, const float* c0,
                            const float* align, const float* xscale, float* chi2_out, float* d_p0, float* d_align,
                            float* d_xscale, int* status_out, float* ck, bool modular = false);

// Static scratch of mkgb_fit_static: [0, 64) work counters (kNumCounters x u64), [64, 80) the
// FP64 refit counter, [256, 256 + 4 * kFitStaticMaxTracks) the refit list.  The counters and the
// refit counter must be zero when a fit starts; the list needs no initial value.
constexpr int kFitStaticMaxTracks = 1 << 16;
constexpr size_t kFitStaticCountersOff = 0, kFitStaticRescueCountOff = 64, kFitStaticListOff = 256;
constexpr size_t kFitStaticZeroBytes = 128;
constexpr size_t kFitStaticScratchBytes = kFitStaticListOff + 4 * (size_t)kFitStaticMaxTracks;
static_assert(8 * kNumCounters <= (int)kFitStaticRescueCountOff, "counters overlap the refit counter");
// Device address of that scratch on the current device (cudaGetSymbolAddress).
cudaError_t fit_static_scratch_address(void** base);

cudaError_t launch_fit(cudaStream_t st, const DevGeom* g, DevParams P, const float4* pay, int64_t n_hits, int n,
                       int max_steps, const int* layers, const int* hits, const float* p0, const float* c0,
                       float* p_out, float* c_out, float* chi2_out, int* status_out, unsigned long long* counters,
                       int* rescue_list, int* rescue_count, int n_sms, bool modular = false);
// Backward fit (Sec. 2.2) of n tracks listed in forward order from their state on the last
// listed layer (covariance scaled by cov_scale); FP64 refit of tracks above kappa_fp64.
cudaError_t launch_bkfit(cudaStream_t st, const DevGeom* g, DevParams P, const float4* pay, int64_t n_hits, int n,
                         int max_steps, const int* layers, const int* hits, const float* p_start, const float* c_start,
                         float cov_scale, float* p_out, float* c_out, float* chi2_out, int* status_out,
                         unsigned long long* counters, int* rescue_list, int* rescue_count, int n_sms,
                         bool modular = false);
// Seed cleaning (mode 0) and quality filter + duplicate removal (mode 1) over n rows of `width`
// hit ids; scratch holds clean_scratch_ints(n, width, n_hits) ints; keep gets 0/1 per row.
size_t clean_scratch_ints(int n, int width, int64_t n_hits);
cudaError_t launch_item_decide(cudaStream_t st, int mode, int n, int width, const int* hits, const float* score,
                               int64_t n_hits, int min_hits, float frac, int* scratch, int* keep, int n_sms);
cudaError_t launch_step_propagate(cudaStream_t st, const DevGeom* g, DevParams P, int n, const int* layers,
                                  const float* p_in, const float* c_in, float* p_out, float* c_out, int* crossed);
cudaError_t launch_step_update(cudaStream_t st, int n, const float* p_in, const float* c_in, const float* hxyz,
                               const float* hcov, float* p_out, float* c_out, float* chi2, int* ok);

}  // namespace mk
