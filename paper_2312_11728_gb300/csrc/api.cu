// C ABI of libmkgb.so: context, device buffers, host staging and kernel launches.
// Declarations and argument contracts: include/mkgb.h.
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

using namespace mk;

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

cudaError_t ensure(DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.p && b.bytes >= bytes) return cudaSuccess;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e == cudaSuccess) b.bytes = bytes;
    return e;
}

void release(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DevGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

enum Stage { S_A, S_B, S_C, S_D, S_E, S_F, S_G, S_H, S_I, S_J, S_K, S_L, S_COUNT };

}  // namespace

struct mkgb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // side stream for the hit binning (needed by the search only), forked after the hit
    // preparation and joined by the next user of the binned hits
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_prep = nullptr, ev_bins = nullptr;
    bool bins_pending = false;   // ev_bins recorded and not yet waited for on the context's stream
    // side stream and events of mkgb_run's fit
    cudaStream_t fit_st = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_fit = nullptr;
    // mkgb_run_host: host-to-device copy stream, per-chunk and per-input events, device copies
    static constexpr int kHostChunks = 8;
    cudaStream_t cp_in = nullptr;
    cudaEvent_t ev_chunk[kHostChunks] = {}, ev_seedin = nullptr, ev_fitin = nullptr, ev_start = nullptr;
    DevBuf host_run;
    int n_sms = 0;
    std::string err;
    bool has_geom = false, has_params = false, has_hits = false, has_seeds = false, seeds_fp64 = false;
    DevGeom geom_h;
    DevBuf geom_d;
    int max_plan_len = 0;
    DevParams params;
    int n_events = 0, n_layers = 0;
    int64_t n_hits = 0;
    std::vector<int64_t> seg_off_h;
    DevBuf seg_off, in_xyz, in_cov, pay, ep_tmp, bin_of_hit, hit_seg, bins, hb_ep, hb_pay, cursor, scan_tmp;
    int n_seeds = 0;
    DevBuf seed_hits, seed_state, seed_state64, seed_info, seed_key, key_counts, key_cursor, seed_order, seed_scan_tmp;
    DevBuf seed_redo;   // the seeds whose mixed-precision fit is redone in FP64: count, then indices
    DevBuf counters_build, counters_fit, queue, rescue_list, rescue_count, build_work, probe_sink, grad_ck;
    // backward search: the geometry with reversed plans and the tracks' start records
    DevBuf geom_bwd_d, bw_state, bw_info, bw_order;
    DevBuf clean_scratch;   // seed cleaning / duplicate removal index
    // module planes (Sec. 3.1) and whether the loaded hits carry module ids
    DevBuf mods_d, in_mod, mod_bad;
    bool mod_hits = false;
    DevBuf stage[S_COUNT];
    // launch shapes of the search rounds and the graph cache replaying them
    int find_shape = 1, select_shape = 0;   // two kernels per round: find 64 x 8, select 128 x 5
    bool use_graph = true;
    BuildGraph* graph = nullptr;
};

namespace {

int fail(mkgb_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? MKGB_ENOMEM : MKGB_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                       \
    } while (0)

HitStore hit_store(const mkgb_ctx* c) {
    HitStore H;
    H.seg_off = (const int64_t*)c->seg_off.p;
    H.n_events = c->n_events;
    H.n_layers = c->n_layers;
    H.n_hits = c->n_hits;
    H.pay = (const float4*)c->pay.p;
    H.hb_ep = (const float2*)c->hb_ep.p;
    H.hb_pay = (const float4*)c->hb_pay.p;
    H.bin_start = (const int*)c->bins.p;
    H.hit_seg = (const int*)c->hit_seg.p;
    return H;
}

// Device view of an input array: the pointer itself (on_device) or a staged copy.
cudaError_t stage_in(mkgb_ctx* c, Stage s, const void* src, size_t bytes, bool on_device, const void** out) {
    if (on_device || src == nullptr) {
        *out = src;
        return cudaSuccess;
    }
    cudaError_t e = ensure(c->stage[s], bytes);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(c->stage[s].p, src, bytes, cudaMemcpyHostToDevice, c->stream);
    *out = c->stage[s].p;
    return e;
}

cudaError_t stage_out(mkgb_ctx* c, Stage s, void* dst, size_t bytes, bool on_device, void** out) {
    if (on_device || dst == nullptr) {
        *out = dst;
        return cudaSuccess;
    }
    cudaError_t e = ensure(c->stage[s], bytes);
    *out = c->stage[s].p;
    return e;
}

// A library-owned device buffer of the given bytes (outputs nobody reads back).
cudaError_t stage_buf(mkgb_ctx* c, Stage s, size_t bytes, void** out) {
    cudaError_t e = ensure(c->stage[s], bytes);
    *out = c->stage[s].p;
    return e;
}

cudaError_t copy_back(mkgb_ctx* c, void* dst, const void* dev, size_t bytes, bool on_device) {
    if (on_device || dst == nullptr || bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, dev, bytes, cudaMemcpyDeviceToHost, c->stream);
}

// Device buffers of n seeds: the seed fit's states and infos, and the ordering's keys and scratch.
int seed_buffers(mkgb_ctx* ctx, int n) {
    const int64_t nkeys = (int64_t)ctx->n_events * kSeedEtaCells * kSeedPhiCells;
    CK(ensure(ctx->seed_state, 4 * (size_t)kSeedStateStride * n));
    if (ctx->params.precision == MKGB_FP64) CK(ensure(ctx->seed_state64, 8 * (size_t)kSeedStateStride * n));
    CK(ensure(ctx->seed_info, 16 * (size_t)n));
    CK(ensure(ctx->seed_key, 4 * (size_t)n));
    CK(ensure(ctx->seed_order, 4 * (size_t)n));
    CK(ensure(ctx->key_counts, 4 * (nkeys + 1)));
    CK(ensure(ctx->key_cursor, 4 * (nkeys + 1)));
    CK(ensure(ctx->seed_scan_tmp, 4 * scan_tmp_ints(nkeys + 1)));
    CK(ensure(ctx->seed_redo, 4 * ((size_t)n + 1)));
    return MKGB_OK;
}

// The (event, eta, phi) order of the n fitted seeds (a3): keys, their histogram, scan, scatter;
// marks the seeds as loaded.
int seed_order(mkgb_ctx* ctx, cudaStream_t st, int n) {
    const int64_t nkeys = (int64_t)ctx->n_events * kSeedEtaCells * kSeedPhiCells;
    CK(cudaMemsetAsync(ctx->key_counts.p, 0, 4 * (nkeys + 1), st));
    CK(launch_seed_keys(st, n, (const float*)ctx->seed_state.p, (const int4*)ctx->seed_info.p, (int*)ctx->seed_key.p,
                        (int*)ctx->key_counts.p));
    CK(exclusive_scan(st, (const int*)ctx->key_counts.p, (int*)ctx->key_counts.p, nkeys, (int*)ctx->seed_scan_tmp.p));
    CK(cudaMemcpyAsync(ctx->key_cursor.p, ctx->key_counts.p, 4 * nkeys, cudaMemcpyDeviceToDevice, st));
    CK(launch_seed_scatter(st, n, (const int*)ctx->seed_key.p, (int*)ctx->key_cursor.p, (int*)ctx->seed_order.p));
    ctx->n_seeds = n;
    ctx->has_seeds = true;
    ctx->seeds_fp64 = ctx->params.precision == MKGB_FP64;
    return MKGB_OK;
}

// The search of mkgb_build on the context's stream into device outputs d (seeds and binned hits
// loaded); the rounds go through the context's graph cache unless graphs are switched off.
int enqueue_build(mkgb_ctx* ctx, const BuildOutDev& d, int find_shape, int select_shape) {
    cudaStream_t st = ctx->stream;
    SeedStore S{ctx->n_seeds, (const float*)ctx->seed_state.p, (const double*)ctx->seed_state64.p,
                (const int4*)ctx->seed_info.p, (const int*)ctx->seed_order.p};
    if (ctx->bins_pending) {   // the binned hits (mkgb_load_hits)
        CK(cudaStreamWaitEvent(st, ctx->ev_bins, 0));
        ctx->bins_pending = false;
    }
    const int prec = ctx->params.precision;
    if (prec == MKGB_FP64 && !ctx->seeds_fp64)
        return fail(ctx, MKGB_ESTATE, "FP64 search needs seeds made under the FP64 precision");
    const bool ovl = ctx->mod_hits;   // overlap hits need their own trail
    CK(ensure(ctx->build_work, build_work_bytes(ctx->n_seeds, ctx->max_plan_len, prec, ovl)));
    const BuildWork w = carve_build_work(ctx->build_work.p, ctx->n_seeds, ctx->max_plan_len, prec, ovl);
    CK(cudaMemsetAsync(ctx->counters_build.p, 0, 8 * kNumCounters, st));
    if (ctx->use_graph && !ctx->graph) ctx->graph = build_graph_create();
    CK(launch_build(st, (const DevGeom*)ctx->geom_d.p, ctx->max_plan_len, ctx->params, hit_store(ctx), S, d, w,
                    (unsigned long long*)ctx->counters_build.p, ctx->n_sms, find_shape, select_shape,
                    ctx->use_graph ? ctx->graph : nullptr));
    return MKGB_OK;
}

// Copies the host geometry to the device, and the same geometry with every region's plan in
// reverse order (the backward search); synchronises the context's stream.
int upload_geometry(mkgb_ctx* ctx) {
    CK(cudaMemcpyAsync(ctx->geom_d.p, &ctx->geom_h, sizeof(DevGeom), cudaMemcpyHostToDevice, ctx->stream));
    CK(ensure(ctx->geom_bwd_d, sizeof(DevGeom)));
    DevGeom gb = ctx->geom_h;
    for (int r = 0; r < gb.n_regions; ++r) std::reverse(gb.plan + gb.plan_off[r], gb.plan + gb.plan_off[r + 1]);
    CK(cudaMemcpyAsync(ctx->geom_bwd_d.p, &gb, sizeof(DevGeom), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));   // gb lives on this stack frame
    return MKGB_OK;
}

}  // namespace

extern "C" {

const char* mkgb_version(void) { return "mkgb 0.1 sm_103a"; }

const char* mkgb_last_error(const mkgb_ctx* ctx) {
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

int mkgb_create(mkgb_ctx** out, int device, void* stream) {
    mkgb_ctx* ctx = nullptr;
    if (!out) return MKGB_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return MKGB_ECUDA;
    ctx = new mkgb_ctx();
    ctx->device = device;
    DevGuard guard(device);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete ctx;
        return MKGB_ECUDA;
    }
    ctx->n_sms = prop.multiProcessorCount;
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return MKGB_ECUDA;
        }
        ctx->own_stream = true;
    }
    if (ensure(ctx->counters_build, 8 * kNumCounters) != cudaSuccess ||
        ensure(ctx->counters_fit, 8 * kNumCounters) != cudaSuccess || ensure(ctx->queue, 16) != cudaSuccess ||
        ensure(ctx->geom_d, sizeof(DevGeom)) != cudaSuccess) {
        mkgb_destroy(ctx);
        return MKGB_ENOMEM;
    }
    cudaMemsetAsync(ctx->counters_build.p, 0, 8 * kNumCounters, ctx->stream);
    cudaMemsetAsync(ctx->counters_fit.p, 0, 8 * kNumCounters, ctx->stream);
    *out = ctx;
    return MKGB_OK;
}

void mkgb_destroy(mkgb_ctx* ctx) {
    if (!ctx) return;
    {
        DevGuard guard(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        if (ctx->aux) {
            cudaStreamSynchronize(ctx->aux);
            cudaStreamDestroy(ctx->aux);
        }
        if (ctx->ev_prep) cudaEventDestroy(ctx->ev_prep);
        if (ctx->ev_bins) cudaEventDestroy(ctx->ev_bins);
        if (ctx->fit_st) {
            cudaStreamSynchronize(ctx->fit_st);
            cudaStreamDestroy(ctx->fit_st);
        }
        if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
        if (ctx->ev_fit) cudaEventDestroy(ctx->ev_fit);
        if (ctx->cp_in) {
            cudaStreamSynchronize(ctx->cp_in);
            cudaStreamDestroy(ctx->cp_in);
        }
        for (cudaEvent_t e : ctx->ev_chunk)
            if (e) cudaEventDestroy(e);
        if (ctx->ev_seedin) cudaEventDestroy(ctx->ev_seedin);
        if (ctx->ev_fitin) cudaEventDestroy(ctx->ev_fitin);
        if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
        DevBuf* all[] = {&ctx->host_run, &ctx->geom_d, &ctx->seg_off, &ctx->in_xyz, &ctx->in_cov, &ctx->pay, &ctx->ep_tmp,
                         &ctx->bin_of_hit, &ctx->hit_seg, &ctx->bins, &ctx->hb_ep, &ctx->hb_pay, &ctx->cursor,
                         &ctx->scan_tmp, &ctx->seed_hits, &ctx->seed_state, &ctx->seed_state64, &ctx->seed_info, &ctx->seed_key,
                         &ctx->key_counts, &ctx->key_cursor, &ctx->seed_order, &ctx->seed_scan_tmp, &ctx->seed_redo,
                         &ctx->counters_build, &ctx->counters_fit, &ctx->queue, &ctx->rescue_list,
                         &ctx->rescue_count, &ctx->build_work, &ctx->probe_sink, &ctx->grad_ck,
                         &ctx->geom_bwd_d, &ctx->bw_state, &ctx->bw_info, &ctx->bw_order,
                         &ctx->clean_scratch, &ctx->mods_d, &ctx->in_mod, &ctx->mod_bad};
        for (DevBuf* b : all) release(*b);
        for (auto& b : ctx->stage) release(b);
        build_graph_destroy(ctx->graph);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    }
    delete ctx;
}

int mkgb_load_geometry(mkgb_ctx* ctx, const mkgb_layer* layers, int n_layers, const int32_t* plan,
                       const int32_t* plan_off, int n_regions, float bz_tesla) {
    if (!ctx) return MKGB_EINVAL;
    if (!layers || !plan || !plan_off) return fail(ctx, MKGB_EINVAL, "null geometry array");
    if (n_layers < 1 || n_layers > MKGB_MAX_LAYERS) return fail(ctx, MKGB_EINVAL, "n_layers %d outside 1..%d", n_layers, MKGB_MAX_LAYERS);
    if (n_regions < 1 || n_regions > MKGB_MAX_REGIONS) return fail(ctx, MKGB_EINVAL, "n_regions %d outside 1..%d", n_regions, MKGB_MAX_REGIONS);
    if (!(bz_tesla != 0.0f) || !(bz_tesla == bz_tesla)) return fail(ctx, MKGB_EINVAL, "bz must be non-zero");
    DevGeom g;
    memset(&g, 0, sizeof(g));
    g.n_layers = n_layers;
    g.n_regions = n_regions;
    g.bz = bz_tesla;
    g.cB = kCLight * bz_tesla;
    int64_t bins = 0;
    for (int l = 0; l < n_layers; ++l) {
        const mkgb_layer& s = layers[l];
        DevLayer& d = g.layers[l];
        if (s.kind != MKGB_BARREL && s.kind != MKGB_DISK) return fail(ctx, MKGB_EINVAL, "layer %d: bad kind %d", l, s.kind);
        if (!(s.hi > s.lo)) return fail(ctx, MKGB_EINVAL, "layer %d: empty extent", l);
        if (s.kind == MKGB_BARREL && !(s.pos > 0.0f)) return fail(ctx, MKGB_EINVAL, "layer %d: radius must be > 0", l);
        if (s.kind == MKGB_DISK && !(s.lo > 0.0f)) return fail(ctx, MKGB_EINVAL, "layer %d: disk rmin must be > 0", l);
        if (s.n_eta_bins < 1 || s.n_phi_bins < 1 || s.n_eta_bins > 4096 || s.n_phi_bins > 4096)
            return fail(ctx, MKGB_EINVAL, "layer %d: bin counts outside 1..4096", l);
        if (!(s.eta_hi > s.eta_lo)) return fail(ctx, MKGB_EINVAL, "layer %d: empty eta range", l);
        if (!(s.x_over_x0 >= 0.0f)) return fail(ctx, MKGB_EINVAL, "layer %d: negative material", l);
        d.kind = s.kind;
        d.pos = s.pos;
        d.lo = s.lo;
        d.hi = s.hi;
        d.xx0 = s.x_over_x0;
        for (int j = 0; j < 3; ++j) d.sig[j] = s.sig_local[j];
        d.n_eta = s.n_eta_bins;
        d.n_phi = s.n_phi_bins;
        d.eta_lo = s.eta_lo;
        d.eta_scale = (float)s.n_eta_bins / (s.eta_hi - s.eta_lo);
        d.bin_base = (int)bins;
        bins += (int64_t)s.n_eta_bins * s.n_phi_bins;
    }
    if (bins > (1 << 26)) return fail(ctx, MKGB_EINVAL, "too many bins per event (%lld)", (long long)bins);
    g.bins_per_event = (int)bins;
    if (plan_off[0] != 0) return fail(ctx, MKGB_EINVAL, "plan_off[0] must be 0");
    int maxp = 0;
    for (int r = 0; r < n_regions; ++r) {
        const int len = plan_off[r + 1] - plan_off[r];
        if (len < 1 || len > MKGB_MAX_PLAN) return fail(ctx, MKGB_EINVAL, "plan %d length %d outside 1..%d", r, len, MKGB_MAX_PLAN);
        maxp = len > maxp ? len : maxp;
    }
    const int total = plan_off[n_regions];
    if (total > MKGB_MAX_REGIONS * MKGB_MAX_PLAN) return fail(ctx, MKGB_EINVAL, "plans too long");
    for (int r = 0; r <= n_regions; ++r) g.plan_off[r] = plan_off[r];
    for (int q = 0; q < total; ++q) {
        if (plan[q] < 0 || plan[q] >= n_layers) return fail(ctx, MKGB_EINVAL, "plan entry %d = %d out of range", q, plan[q]);
        g.plan[q] = plan[q];
    }
    g.max_plan = maxp;
    DevGuard guard(ctx->device);
    ctx->geom_h = g;
    const int rc = upload_geometry(ctx);
    if (rc != MKGB_OK) return rc;
    ctx->max_plan_len = maxp;
    ctx->n_layers = n_layers;
    ctx->has_geom = true;
    ctx->has_hits = false;
    ctx->has_seeds = false;
    ctx->mod_hits = false;
    return MKGB_OK;
}

int mkgb_load_modules(mkgb_ctx* ctx, int n_modules, const int32_t* layer, const float* pos, const float* normal) {
    if (!ctx) return MKGB_EINVAL;
    if (!ctx->has_geom) return fail(ctx, MKGB_ESTATE, "load_modules before load_geometry");
    if (n_modules < 0 || (n_modules > 0 && (!layer || !pos || !normal))) return fail(ctx, MKGB_EINVAL, "bad module arrays");
    if (n_modules >= (1 << 30)) return fail(ctx, MKGB_EINVAL, "too many modules");
    std::vector<float4> tab(2 * (size_t)n_modules);
    bool modular[MKGB_MAX_LAYERS] = {false};
    for (int m = 0; m < n_modules; ++m) {
        const int l = layer[m];
        if (l < 0 || l >= ctx->n_layers) return fail(ctx, MKGB_EINVAL, "module %d: layer %d out of range", m, l);
        const float nx = normal[3 * m], ny = normal[3 * m + 1], nz = normal[3 * m + 2];
        const float n2 = nx * nx + ny * ny + nz * nz;
        if (!(fabsf(n2 - 1.0f) < 1e-4f)) return fail(ctx, MKGB_EINVAL, "module %d: normal is not a unit vector", m);
        if (!(pos[3 * m] == pos[3 * m] && pos[3 * m + 1] == pos[3 * m + 1] && pos[3 * m + 2] == pos[3 * m + 2]))
            return fail(ctx, MKGB_EINVAL, "module %d: bad position", m);
        int li = l;
        float lw;
        memcpy(&lw, &li, 4);
        tab[2 * m] = make_float4(pos[3 * m], pos[3 * m + 1], pos[3 * m + 2], lw);
        tab[2 * m + 1] = make_float4(nx, ny, nz, 0.0f);
        modular[l] = true;
    }
    DevGuard guard(ctx->device);
    if (n_modules > 0) {
        CK(ensure(ctx->mods_d, 32 * (size_t)n_modules));
        CK(cudaMemcpyAsync(ctx->mods_d.p, tab.data(), 32 * (size_t)n_modules, cudaMemcpyHostToDevice, ctx->stream));
    }
    ctx->geom_h.mods = n_modules > 0 ? (const float4*)ctx->mods_d.p : nullptr;
    ctx->geom_h.n_mods = n_modules;
    for (int l = 0; l < ctx->n_layers; ++l) ctx->geom_h.layers[l].modular = modular[l] ? 1 : 0;
    const int rc = upload_geometry(ctx);   // synchronises: tab may go
    if (rc != MKGB_OK) return rc;
    ctx->has_hits = false;   // hits are matched to the modules when they are loaded
    ctx->has_seeds = false;
    ctx->mod_hits = false;
    return MKGB_OK;
}

int mkgb_set_params(mkgb_ctx* ctx, const mkgb_params* p) {
    if (!ctx) return MKGB_EINVAL;
    if (!p) return fail(ctx, MKGB_EINVAL, "null params");
    if (p->max_cands < 1 || p->max_cands > MKGB_MAX_CANDS) return fail(ctx, MKGB_EINVAL, "max_cands %d outside 1..%d", p->max_cands, MKGB_MAX_CANDS);
    if (p->max_holes < 0) return fail(ctx, MKGB_EINVAL, "max_holes < 0");
    if (!(p->deta_min >= 0.0f && p->dphi_min >= 0.0f && p->deta_max >= p->deta_min && p->dphi_max >= p->dphi_min))
        return fail(ctx, MKGB_EINVAL, "bad window bounds");
    if (!(p->dphi_max < 1.5f)) return fail(ctx, MKGB_EINVAL, "dphi_max must be < 1.5 rad");
    if (!(p->win_nsigma >= 0.0f) || !(p->chi2_cut > 0.0f)) return fail(ctx, MKGB_EINVAL, "bad n_sigma or chi2_cut");
    DevParams& d = ctx->params;
    d.chi2_cut = p->chi2_cut;
    d.max_cands = p->max_cands;
    d.max_holes = p->max_holes;
    d.material = p->material ? 1 : 0;
    d.nsig = p->win_nsigma;
    d.deta_min = p->deta_min;
    d.deta_max = p->deta_max;
    d.dphi_min = p->dphi_min;
    d.dphi_max = p->dphi_max;
    d.score_hit = p->score_hit;
    d.score_hole = p->score_hole;
    d.barrel_eta_max = p->barrel_eta_max;
    if (p->precision != MKGB_FP32 && p->precision != MKGB_FP64) return fail(ctx, MKGB_EINVAL, "bad precision %d", p->precision);
    d.precision = p->precision;
    if (!(p->kappa_fp64 >= 0.0f)) return fail(ctx, MKGB_EINVAL, "kappa_fp64 must be >= 0");
    d.kappa_fp64 = p->kappa_fp64;
    if (!(p->fit_outlier_chi2 >= 0.0f)) return fail(ctx, MKGB_EINVAL, "fit_outlier_chi2 must be >= 0");
    d.fit_outlier_chi2 = p->fit_outlier_chi2;
    if (!(p->score_overlap == p->score_overlap) || !(fabsf(p->score_overlap) < 1e30f))
        return fail(ctx, MKGB_EINVAL, "score_overlap must be finite");
    d.score_overlap = p->score_overlap;
    ctx->has_params = true;
    return MKGB_OK;
}

namespace {

// Hits arriving in chunks of whole events: the preparation of chunk k, hits [hit_off[k],
// hit_off[k + 1]), waits for ready[k] (recorded after the chunk's copy).
struct HitChunks {
    int n = 0;
    const int64_t* hit_off = nullptr;
    const cudaEvent_t* ready = nullptr;
    // enqueued on the context's stream after chunk k's preparation (nullptr: nothing)
    std::function<int(int k)> after;
};

int load_hits_impl(mkgb_ctx* ctx, int n_events, const int64_t* seg_off, const float* xyz, const float* cov6,
                   const int32_t* hit_module, int on_device, const HitChunks* chunks = nullptr) {
    if (!ctx->has_geom) return fail(ctx, MKGB_ESTATE, "load_hits before load_geometry");
    if (n_events < 1 || !seg_off) return fail(ctx, MKGB_EINVAL, "need n_events >= 1 and seg_off");
    const int L = ctx->n_layers;
    const int64_t nseg = (int64_t)n_events * L;
    if (seg_off[0] != 0) return fail(ctx, MKGB_EINVAL, "seg_off[0] must be 0");
    for (int64_t s = 0; s < nseg; ++s)
        if (seg_off[s + 1] < seg_off[s]) return fail(ctx, MKGB_EINVAL, "seg_off decreases at %lld", (long long)s);
    const int64_t n = seg_off[nseg];
    if (n > ((int64_t)1 << 28) - 8) return fail(ctx, MKGB_EINVAL, "too many hits (%lld)", (long long)n);
    if (n > 0 && (!xyz || !cov6)) return fail(ctx, MKGB_EINVAL, "null hit arrays");
    const int64_t nbins = (int64_t)n_events * ctx->geom_h.bins_per_event;
    if (nbins > ((int64_t)1 << 31) - 2) return fail(ctx, MKGB_EINVAL, "too many bins (%lld)", (long long)nbins);
    DevGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;
    if (!ctx->aux) {
        CK(cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ctx->ev_prep, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->ev_bins, cudaEventDisableTiming));
    }
    // the previous call's binning must be done before its inputs and outputs are rewritten
    if (ctx->bins_pending) {
        CK(cudaStreamWaitEvent(st, ctx->ev_bins, 0));
        ctx->bins_pending = false;
    }
    // The offsets are copied only when they change (a repeated batch costs no host round trip).
    // A copy from pageable memory returns once the source has been staged, so the host vector
    // may be rewritten after the call.
    const bool same = ctx->seg_off_h.size() == (size_t)(nseg + 1) && ctx->seg_off.p &&
                      std::equal(seg_off, seg_off + nseg + 1, ctx->seg_off_h.begin());
    if (!same) {
        ctx->seg_off_h.assign(seg_off, seg_off + nseg + 1);
        CK(ensure(ctx->seg_off, 8 * (nseg + 1)));
        CK(cudaMemcpyAsync(ctx->seg_off.p, ctx->seg_off_h.data(), 8 * (nseg + 1), cudaMemcpyHostToDevice, st));
    }
    const float* dx = xyz;
    const float* dc = cov6;
    if (!on_device && n > 0) {
        CK(ensure(ctx->in_xyz, 12 * n));
        CK(ensure(ctx->in_cov, 24 * n));
        CK(cudaMemcpyAsync(ctx->in_xyz.p, xyz, 12 * n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ctx->in_cov.p, cov6, 24 * n, cudaMemcpyHostToDevice, st));
        dx = (const float*)ctx->in_xyz.p;
        dc = (const float*)ctx->in_cov.p;
    }
    CK(ensure(ctx->pay, 48 * n));
    CK(ensure(ctx->ep_tmp, 8 * n));
    CK(ensure(ctx->bin_of_hit, 4 * n));
    CK(ensure(ctx->hit_seg, 4 * n));
    CK(ensure(ctx->hb_ep, 8 * n));
    CK(ensure(ctx->hb_pay, 48 * n));
    CK(ensure(ctx->bins, 4 * (nbins + 1)));
    CK(ensure(ctx->cursor, 4 * (nbins + 1)));
    CK(ensure(ctx->scan_tmp, 4 * scan_tmp_ints(nbins + 1)));
    const int* dm = hit_module;
    if (hit_module && !on_device && n > 0) {
        CK(ensure(ctx->in_mod, 4 * n));
        CK(cudaMemcpyAsync(ctx->in_mod.p, hit_module, 4 * n, cudaMemcpyHostToDevice, st));
        dm = (const int*)ctx->in_mod.p;
    }
    CK(cudaMemsetAsync(ctx->bins.p, 0, 4 * (nbins + 1), st));
    if (chunks && chunks->n > 0) {
        for (int k = 0; k < chunks->n; ++k) {
            CK(cudaStreamWaitEvent(st, chunks->ready[k], 0));
            CK(launch_hit_prep(st, (const DevGeom*)ctx->geom_d.p, L, (const int64_t*)ctx->seg_off.p, (int)nseg, n, dx,
                               dc, n > 0 ? dm : nullptr, ctx->geom_h.bins_per_event, (float4*)ctx->pay.p,
                               (float2*)ctx->ep_tmp.p, (int*)ctx->bin_of_hit.p, (int*)ctx->hit_seg.p,
                               (int*)ctx->bins.p, chunks->hit_off[k], chunks->hit_off[k + 1]));
            if (chunks->after) {
                const int rc = chunks->after(k);
                if (rc != MKGB_OK) return rc;
            }
        }
    } else {
        CK(launch_hit_prep(st, (const DevGeom*)ctx->geom_d.p, L, (const int64_t*)ctx->seg_off.p, (int)nseg, n, dx, dc,
                           n > 0 ? dm : nullptr, ctx->geom_h.bins_per_event, (float4*)ctx->pay.p,
                           (float2*)ctx->ep_tmp.p, (int*)ctx->bin_of_hit.p, (int*)ctx->hit_seg.p, (int*)ctx->bins.p));
    }
    ctx->has_hits = false;
    if (hit_module && n > 0) {   // every module id must fit its hit's layer (synchronises)
        CK(ensure(ctx->mod_bad, 16));
        CK(cudaMemsetAsync(ctx->mod_bad.p, 0, 4, st));
        CK(launch_check_modules(st, (const DevGeom*)ctx->geom_d.p, L, n, (const int*)ctx->hit_seg.p, dm,
                                (int*)ctx->mod_bad.p));
        int bad = 0;
        CK(cudaMemcpyAsync(&bad, ctx->mod_bad.p, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (bad) return fail(ctx, MKGB_EINVAL, "%d hits with a module that does not fit their layer", bad);
    }
    // The binned copy is used by the search only: it is built on the side stream, overlapping
    // the seed fit and the fit on the context's stream, and mkgb_build waits for it.
    CK(cudaEventRecord(ctx->ev_prep, st));
    CK(cudaStreamWaitEvent(ctx->aux, ctx->ev_prep, 0));
    CK(exclusive_scan(ctx->aux, (const int*)ctx->bins.p, (int*)ctx->bins.p, nbins, (int*)ctx->scan_tmp.p));
    CK(cudaMemcpyAsync(ctx->cursor.p, ctx->bins.p, 4 * nbins, cudaMemcpyDeviceToDevice, ctx->aux));
    CK(launch_hit_scatter(ctx->aux, n, (const float4*)ctx->pay.p, (const float2*)ctx->ep_tmp.p,
                          (const int*)ctx->bin_of_hit.p, (int*)ctx->cursor.p, (float2*)ctx->hb_ep.p,
                          (float4*)ctx->hb_pay.p));
    CK(cudaEventRecord(ctx->ev_bins, ctx->aux));
    ctx->bins_pending = true;
    if (!on_device) CK(cudaStreamSynchronize(st));
    ctx->n_events = n_events;
    ctx->n_hits = n;
    ctx->has_hits = true;
    ctx->has_seeds = false;
    ctx->mod_hits = hit_module != nullptr && n > 0;
    return MKGB_OK;
}

}  // namespace

int mkgb_load_hits(mkgb_ctx* ctx, int n_events, const int64_t* seg_off, const float* xyz, const float* cov6,
                   int on_device) {
    if (!ctx) return MKGB_EINVAL;
    return load_hits_impl(ctx, n_events, seg_off, xyz, cov6, nullptr, on_device);
}

int mkgb_load_hits_modular(mkgb_ctx* ctx, int n_events, const int64_t* seg_off, const float* xyz, const float* cov6,
                           const int32_t* hit_module, int on_device) {
    if (!ctx) return MKGB_EINVAL;
    if (!hit_module) return fail(ctx, MKGB_EINVAL, "null hit_module");
    if (ctx->has_geom && ctx->geom_h.n_mods == 0) return fail(ctx, MKGB_ESTATE, "load_hits_modular before load_modules");
    return load_hits_impl(ctx, n_events, seg_off, xyz, cov6, hit_module, on_device);
}

int mkgb_seed(mkgb_ctx* ctx, int n_seeds, const int32_t* seed_hits, int on_device, float* state_out,
              float* cov_out, int32_t* info_out) {
    if (!ctx) return MKGB_EINVAL;
    if (!ctx->has_hits) return fail(ctx, MKGB_ESTATE, "seed before load_hits");
    if (!ctx->has_params) return fail(ctx, MKGB_ESTATE, "seed before set_params");
    if (n_seeds < 0 || (n_seeds > 0 && !seed_hits)) return fail(ctx, MKGB_EINVAL, "bad seeds");
    if (n_seeds > 0 && ctx->n_hits == 0) return fail(ctx, MKGB_EINVAL, "seeds given but no hits loaded");
    if ((state_out == nullptr) != (cov_out == nullptr)) return fail(ctx, MKGB_EINVAL, "state_out and cov_out go together");
    DevGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;
    const int n = n_seeds;
    const void* sh = nullptr;
    CK(stage_in(ctx, S_A, seed_hits, 12 * (size_t)n, on_device, &sh));
    int rc = seed_buffers(ctx, n);
    if (rc != MKGB_OK) return rc;
    void *s6 = nullptr, *c21 = nullptr, *i3 = nullptr;
    CK(stage_out(ctx, S_B, state_out, 24 * (size_t)n, on_device, &s6));
    CK(stage_out(ctx, S_C, cov_out, 84 * (size_t)n, on_device, &c21));
    CK(stage_out(ctx, S_D, info_out, 12 * (size_t)n, on_device, &i3));
    const bool fp64 = ctx->params.precision == MKGB_FP64;
    CK(cudaMemsetAsync(ctx->seed_redo.p, 0, 4, st));
    CK(launch_seed_fit(st, (const DevGeom*)ctx->geom_d.p, ctx->params, hit_store(ctx), n, (const int*)sh,
                       (float*)ctx->seed_state.p, fp64 ? (double*)ctx->seed_state64.p : nullptr,
                       (int4*)ctx->seed_info.p, (float*)s6, (float*)c21, (int*)i3, SeedRange(), ctx->mod_hits,
                       (int*)ctx->seed_redo.p));
    CK(launch_seed_redo(st, (const DevGeom*)ctx->geom_d.p, ctx->params, hit_store(ctx), n, (const int*)sh,
                        (float*)ctx->seed_state.p, (int4*)ctx->seed_info.p, (float*)s6, (float*)c21, (int*)i3,
                        ctx->mod_hits, (const int*)ctx->seed_redo.p, ctx->n_sms));
    rc = seed_order(ctx, st, n);
    if (rc != MKGB_OK) return rc;
    CK(copy_back(ctx, state_out, s6, 24 * (size_t)n, on_device));
    CK(copy_back(ctx, cov_out, c21, 84 * (size_t)n, on_device));
    CK(copy_back(ctx, info_out, i3, 12 * (size_t)n, on_device));
    if (!on_device) CK(cudaStreamSynchronize(st));
    return MKGB_OK;
}

int mkgb_build(mkgb_ctx* ctx, const mkgb_tracks* out, int on_device) {
    if (!ctx) return MKGB_EINVAL;
    if (!ctx->has_seeds) return fail(ctx, MKGB_ESTATE, "build before seed");
    if (!out || !out->params || !out->cov || !out->chi2 || !out->score || !out->nfound || !out->nholes || !out->hits)
        return fail(ctx, MKGB_EINVAL, "null output array");
    if (out->max_plan < ctx->max_plan_len) return fail(ctx, MKGB_EINVAL, "max_plan %d < longest plan %d", out->max_plan, ctx->max_plan_len);
    if (ctx->n_hits >= ((int64_t)1 << 28) - 8)
        return fail(ctx, MKGB_EINVAL, "%lld hits loaded: the search takes fewer than 2^28 - 8",
                    (long long)ctx->n_hits);
    DevGuard guard(ctx->device);
    const size_t n = (size_t)ctx->n_seeds;
    BuildOutDev d;
    void* p;
    CK(stage_out(ctx, S_A, out->params, 24 * n, on_device, &p)); d.params = (float*)p;
    CK(stage_out(ctx, S_B, out->cov, 84 * n, on_device, &p)); d.cov = (float*)p;
    CK(stage_out(ctx, S_C, out->chi2, 4 * n, on_device, &p)); d.chi2 = (float*)p;
    CK(stage_out(ctx, S_D, out->score, 4 * n, on_device, &p)); d.score = (float*)p;
    CK(stage_out(ctx, S_E, out->nfound, 4 * n, on_device, &p)); d.nfound = (int*)p;
    CK(stage_out(ctx, S_F, out->nholes, 4 * n, on_device, &p)); d.nholes = (int*)p;
    CK(stage_out(ctx, S_G, out->hits, 4 * n * out->max_plan, on_device, &p)); d.hits = (int*)p;
    d.max_plan = out->max_plan;
    if (out->ovl_hits) {
        CK(stage_out(ctx, S_H, out->ovl_hits, 4 * n * out->max_plan, on_device, &p));
        d.ovl = (int*)p;
    }
    const int rc = enqueue_build(ctx, d, ctx->find_shape, ctx->select_shape);
    if (rc != MKGB_OK) return rc;
    cudaStream_t st = ctx->stream;
    CK(copy_back(ctx, out->params, d.params, 24 * n, on_device));
    CK(copy_back(ctx, out->cov, d.cov, 84 * n, on_device));
    CK(copy_back(ctx, out->chi2, d.chi2, 4 * n, on_device));
    CK(copy_back(ctx, out->score, d.score, 4 * n, on_device));
    CK(copy_back(ctx, out->nfound, d.nfound, 4 * n, on_device));
    CK(copy_back(ctx, out->nholes, d.nholes, 4 * n, on_device));
    CK(copy_back(ctx, out->hits, d.hits, 4 * n * out->max_plan, on_device));
    if (d.ovl) CK(copy_back(ctx, out->ovl_hits, d.ovl, 4 * n * out->max_plan, on_device));
    if (!on_device) CK(cudaStreamSynchronize(st));
    return MKGB_OK;
}

int mkgb_build_backward(mkgb_ctx* ctx, int n, const int32_t* track_event, const int32_t* first_layer,
                        const float* p_start, const float* c_start, const mkgb_tracks* out, int on_device) {
    if (!ctx) return MKGB_EINVAL;
    if (!ctx->has_geom || !ctx->has_params) return fail(ctx, MKGB_ESTATE, "build_backward before geometry/params");
    if (!ctx->has_hits) return fail(ctx, MKGB_ESTATE, "build_backward before load_hits");
    if (n < 0) return fail(ctx, MKGB_EINVAL, "negative size");
    if (ctx->params.precision == MKGB_FP64)
        return fail(ctx, MKGB_EINVAL, "the backward search runs in FP32 (precision MKGB_FP32)");
    if (n > 0 && (!track_event || !first_layer || !p_start || !c_start)) return fail(ctx, MKGB_EINVAL, "null input");
    if (!out || !out->params || !out->cov || !out->chi2 || !out->score || !out->nfound || !out->nholes || !out->hits)
        return fail(ctx, MKGB_EINVAL, "null output array");
    if (out->max_plan < ctx->max_plan_len) return fail(ctx, MKGB_EINVAL, "max_plan %d < longest plan %d", out->max_plan, ctx->max_plan_len);
    if (ctx->n_hits >= ((int64_t)1 << 28) - 8)
        return fail(ctx, MKGB_EINVAL, "%lld hits loaded: the search takes fewer than 2^28 - 8", (long long)ctx->n_hits);
    if (!on_device)
        for (int i = 0; i < n; ++i) {
            if (track_event[i] < 0 || track_event[i] >= ctx->n_events)
                return fail(ctx, MKGB_EINVAL, "track %d: event %d outside the loaded events", i, track_event[i]);
            if (first_layer[i] < 0 || first_layer[i] >= ctx->n_layers)
                return fail(ctx, MKGB_EINVAL, "track %d: layer %d outside the geometry", i, first_layer[i]);
        }
    if (n == 0) return MKGB_OK;
    DevGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;
    const size_t N = (size_t)n;
    const void *dev_ev, *dfl, *dp, *dc;
    CK(stage_in(ctx, S_H, track_event, 4 * N, on_device, &dev_ev));
    CK(stage_in(ctx, S_I, first_layer, 4 * N, on_device, &dfl));
    CK(stage_in(ctx, S_J, p_start, 24 * N, on_device, &dp));
    CK(stage_in(ctx, S_K, c_start, 84 * N, on_device, &dc));
    BuildOutDev d;
    void* p;
    CK(stage_out(ctx, S_A, out->params, 24 * N, on_device, &p)); d.params = (float*)p;
    CK(stage_out(ctx, S_B, out->cov, 84 * N, on_device, &p)); d.cov = (float*)p;
    CK(stage_out(ctx, S_C, out->chi2, 4 * N, on_device, &p)); d.chi2 = (float*)p;
    CK(stage_out(ctx, S_D, out->score, 4 * N, on_device, &p)); d.score = (float*)p;
    CK(stage_out(ctx, S_E, out->nfound, 4 * N, on_device, &p)); d.nfound = (int*)p;
    CK(stage_out(ctx, S_F, out->nholes, 4 * N, on_device, &p)); d.nholes = (int*)p;
    CK(stage_out(ctx, S_G, out->hits, 4 * N * out->max_plan, on_device, &p)); d.hits = (int*)p;
    d.max_plan = out->max_plan;
    if (out->ovl_hits) {
        CK(stage_out(ctx, S_L, out->ovl_hits, 4 * N * out->max_plan, on_device, &p));
        d.ovl = (int*)p;
    }
    CK(ensure(ctx->bw_state, 4 * (size_t)kSeedStateStride * N));
    CK(ensure(ctx->bw_info, 16 * N));
    CK(ensure(ctx->bw_order, 4 * N));
    CK(launch_bw_seed(st, (const DevGeom*)ctx->geom_bwd_d.p, ctx->params, n, (const float*)dp, (const float*)dc,
                      (const int*)dfl, (const int*)dev_ev, (float*)ctx->bw_state.p, (int4*)ctx->bw_info.p,
                      (int*)ctx->bw_order.p));
    if (ctx->bins_pending) {   // the binned hits (mkgb_load_hits)
        CK(cudaStreamWaitEvent(st, ctx->ev_bins, 0));
        ctx->bins_pending = false;
    }
    SeedStore S{n, (const float*)ctx->bw_state.p, nullptr, (const int4*)ctx->bw_info.p, (const int*)ctx->bw_order.p};
    CK(ensure(ctx->build_work, build_work_bytes(n, ctx->max_plan_len, MKGB_FP32, ctx->mod_hits)));
    const BuildWork w = carve_build_work(ctx->build_work.p, n, ctx->max_plan_len, MKGB_FP32, ctx->mod_hits);
    CK(cudaMemsetAsync(ctx->counters_build.p, 0, 8 * kNumCounters, st));
    CK(launch_build(st, (const DevGeom*)ctx->geom_bwd_d.p, ctx->max_plan_len, ctx->params, hit_store(ctx), S, d, w,
                    (unsigned long long*)ctx->counters_build.p, ctx->n_sms, ctx->find_shape >= 3 ? 3 : 0, 0, nullptr, true));
    CK(copy_back(ctx, out->params, d.params, 24 * N, on_device));
    CK(copy_back(ctx, out->cov, d.cov, 84 * N, on_device));
    CK(copy_back(ctx, out->chi2, d.chi2, 4 * N, on_device));
    CK(copy_back(ctx, out->score, d.score, 4 * N, on_device));
    CK(copy_back(ctx, out->nfound, d.nfound, 4 * N, on_device));
    CK(copy_back(ctx, out->nholes, d.nholes, 4 * N, on_device));
    CK(copy_back(ctx, out->hits, d.hits, 4 * N * out->max_plan, on_device));
    if (d.ovl) CK(copy_back(ctx, out->ovl_hits, d.ovl, 4 * N * out->max_plan, on_device));
    if (!on_device) CK(cudaStreamSynchronize(st));
    return MKGB_OK;
}

namespace {

int item_decide(mkgb_ctx* ctx, int mode, int n, int width, const int32_t* hits, const float* score, int min_hits,
                float frac, int32_t* keep_out, int on_device, const char* what) {
    if (!ctx->has_hits) return fail(ctx, MKGB_ESTATE, "%s before load_hits (hit ids index the loaded hits)", what);
    if (n < 0 || width < 1) return fail(ctx, MKGB_EINVAL, "%s: bad sizes", what);
    if (n > 0 && (!hits || !keep_out || (mode == 1 && !score))) return fail(ctx, MKGB_EINVAL, "%s: null array", what);
    if (!on_device)
        for (size_t q = 0; q < (size_t)n * width; ++q)
            if (hits[q] >= ctx->n_hits) return fail(ctx, MKGB_EINVAL, "%s: hit id %d beyond the loaded hits", what, hits[q]);
    if (n == 0) return MKGB_OK;
    DevGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;
    const size_t N = (size_t)n;
    const void *dh, *ds = nullptr;
    CK(stage_in(ctx, S_A, hits, 4 * N * width, on_device, &dh));
    if (mode == 1) CK(stage_in(ctx, S_B, score, 4 * N, on_device, &ds));
    void* ko;
    CK(stage_out(ctx, S_C, keep_out, 4 * N, on_device, &ko));
    CK(ensure(ctx->clean_scratch, 4 * clean_scratch_ints(n, width, ctx->n_hits)));
    CK(launch_item_decide(st, mode, n, width, (const int*)dh, (const float*)ds, ctx->n_hits, min_hits, frac,
                          (int*)ctx->clean_scratch.p, (int*)ko, ctx->n_sms));
    CK(copy_back(ctx, keep_out, ko, 4 * N, on_device));
    if (!on_device) CK(cudaStreamSynchronize(st));
    return MKGB_OK;
}

}  // namespace

int mkgb_clean_seeds(mkgb_ctx* ctx, int n, const int32_t* seed_hits, int32_t* keep_out, int on_device) {
    if (!ctx) return MKGB_EINVAL;
    return item_decide(ctx, 0, n, 3, seed_hits, nullptr, 0, 0.0f, keep_out, on_device, "clean_seeds");
}

int mkgb_remove_duplicates(mkgb_ctx* ctx, int n, int width, const int32_t* hits, const float* score, int min_hits,
                           float frac, int32_t* keep_out, int on_device) {
    if (!ctx) return MKGB_EINVAL;
    if (!(frac > 0.0f && frac <= 1.0f)) return fail(ctx, MKGB_EINVAL, "remove_duplicates: frac %g outside (0, 1]", frac);
    return item_decide(ctx, 1, n, width, hits, score, min_hits, frac, keep_out, on_device, "remove_duplicates");
}

int mkgb_fit(mkgb_ctx* ctx, int n, int max_steps, const int32_t* layers, const int32_t* hits, const float* p0,
             const float* c0, float* p_out, float* c_out, float* chi2_out, int32_t* status_out, int on_device) {
    if (!ctx) return MKGB_EINVAL;
    if (!ctx->has_geom || !ctx->has_params) return fail(ctx, MKGB_ESTATE, "fit before geometry/params");
    if (n < 0 || max_steps < 0) return fail(ctx, MKGB_EINVAL, "negative size");
    if (n > 0 && (!layers || !hits || !p0 || !c0 || !p_out || !c_out || !chi2_out))
        return fail(ctx, MKGB_EINVAL, "null fit array");
    bool any_hit = false;
    if (!on_device)
        for (size_t q = 0; q < (size_t)n * max_steps && !any_hit; ++q) any_hit = hits[q] >= 0;
    if ((on_device || any_hit) && !ctx->has_hits) return fail(ctx, MKGB_ESTATE, "fit with hits before load_hits");
    if (!on_device)
        for (size_t q = 0; q < (size_t)n * max_steps; ++q)
            if (hits[q] >= ctx->n_hits) return fail(ctx, MKGB_EINVAL, "hit index %d out of range", hits[q]);
    DevGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;
    const size_t N = (size_t)n, M = (size_t)max_steps;
    const void *dl, *dh, *dp0, *dc0;
    CK(stage_in(ctx, S_A, layers, 4 * N * M, on_device, &dl));
    CK(stage_in(ctx, S_B, hits, 4 * N * M, on_device, &dh));
    CK(stage_in(ctx, S_C, p0, 24 * N, on_device, &dp0));
    CK(stage_in(ctx, S_D, c0, 84 * N, on_device, &dc0));
    void *po, *co, *xo, *so;
    CK(stage_out(ctx, S_E, p_out, 24 * N, on_device, &po));
    CK(stage_out(ctx, S_F, c_out, 84 * N, on_device, &co));
    CK(stage_out(ctx, S_G, chi2_out, 4 * N, on_device, &xo));
    CK(stage_out(ctx, S_H, status_out, 4 * N, on_device, &so));
    CK(cudaMemsetAsync(ctx->counters_fit.p, 0, 8 * kNumCounters, st));
    CK(ensure(ctx->rescue_list, 4 * (N > 0 ? N : 1)));
    CK(ensure(ctx->rescue_count, 16));
    CK(cudaMemsetAsync(ctx->rescue_count.p, 0, 16, st));
    CK(launch_fit(st, (const DevGeom*)ctx->geom_d.p, ctx->params, (const float4*)ctx->pay.p,
                  ctx->has_hits ? ctx->n_hits : 0, n, max_steps, (const int*)dl, (const int*)dh, (const float*)dp0,
                  (const float*)dc0, (float*)po, (float*)co, (float*)xo, (int*)so,
                  (unsigned long long*)ctx->counters_fit.p, (int*)ctx->rescue_list.p, (int*)ctx->rescue_count.p,
                  ctx->n_sms, ctx->mod_hits));
    CK(copy_back(ctx, p_out, po, 24 * N, on_device));
    CK(copy_back(ctx, c_out, co, 84 * N, on_device));
    CK(copy_back(ctx, chi2_out, xo, 4 * N, on_device));
    CK(copy_back(ctx, status_out, so, 4 * N, on_device));
    if (!on_device) CK(cudaStreamSynchronize(st));
    return MKGB_OK;
}

int mkgb_fit_backward(mkgb_ctx* ctx, int n, int max_steps, const int32_t* layers, const int32_t* hits,
                      const float* p_start, const float* c_start, float cov_scale, float* p_out, float* c_out,
                      float* chi2_out, int32_t* status_out, int on_device) {
    if (!ctx) return MKGB_EINVAL;
    if (!ctx->has_geom || !ctx->has_params) return fail(ctx, MKGB_ESTATE, "fit_backward before geometry/params");
    if (n < 0 || max_steps < 0) return fail(ctx, MKGB_EINVAL, "negative size");
    if (!(cov_scale > 0.0f) || !(cov_scale < 3.0e38f)) return fail(ctx, MKGB_EINVAL, "cov_scale must be positive");
    if (n > 0 && (!layers || !hits || !p_start || !c_start || !p_out || !c_out || !chi2_out))
        return fail(ctx, MKGB_EINVAL, "null fit array");
    bool any_hit = false;
    if (!on_device)
        for (size_t q = 0; q < (size_t)n * max_steps && !any_hit; ++q) any_hit = hits[q] >= 0;
    if ((on_device || any_hit) && !ctx->has_hits) return fail(ctx, MKGB_ESTATE, "fit_backward with hits before load_hits");
    if (!on_device)
        for (size_t q = 0; q < (size_t)n * max_steps; ++q)
            if (hits[q] >= ctx->n_hits) return fail(ctx, MKGB_EINVAL, "hit index %d out of range", hits[q]);
    DevGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;
    const size_t N = (size_t)n, M = (size_t)max_steps;
    const void *dl, *dh, *dp0, *dc0;
    CK(stage_in(ctx, S_A, layers, 4 * N * M, on_device, &dl));
    CK(stage_in(ctx, S_B, hits, 4 * N * M, on_device, &dh));
    CK(stage_in(ctx, S_C, p_start, 24 * N, on_device, &dp0));
    CK(stage_in(ctx, S_D, c_start, 84 * N, on_device, &dc0));
    void *po, *co, *xo, *so;
    CK(stage_out(ctx, S_E, p_out, 24 * N, on_device, &po));
    CK(stage_out(ctx, S_F, c_out, 84 * N, on_device, &co));
    CK(stage_out(ctx, S_G, chi2_out, 4 * N, on_device, &xo));
    CK(stage_out(ctx, S_H, status_out, 4 * N, on_device, &so));
    CK(cudaMemsetAsync(ctx->counters_fit.p, 0, 8 * kNumCounters, st));
    CK(ensure(ctx->rescue_list, 4 * (N > 0 ? N : 1)));
    CK(ensure(ctx->rescue_count, 16));
    CK(cudaMemsetAsync(ctx->rescue_count.p, 0, 16, st));
    CK(launch_bkfit(st, (const DevGeom*)ctx->geom_d.p, ctx->params, (const float4*)ctx->pay.p,
                    ctx->has_hits ? ctx->n_hits : 0, n, max_steps, (const int*)dl, (const int*)dh, (const float*)dp0,
                    (const float*)dc0, cov_scale, (float*)po, (float*)co, (float*)xo, (int*)so,
                    (unsigned long long*)ctx->counters_fit.p, (int*)ctx->rescue_list.p, (int*)ctx->rescue_count.p,
                    ctx->n_sms, ctx->mod_hits));
    CK(copy_back(ctx, p_out, po, 24 * N, on_device));
    CK(copy_back(ctx, c_out, co, 84 * N, on_device));
    CK(copy_back(ctx, chi2_out, xo, 4 * N, on_device));
    CK(copy_back(ctx, status_out, so, 4 * N, on_device));
    if (!on_device) CK(cudaStreamSynchronize(st));
    return MKGB_OK;
}

int mkgb_fit_grad(mkgb_ctx* ctx, int n, int max_steps, const int32_t* layers, const int32_t* hits, const float* p0,
                  const float* c0, const float* align, const float* xscale, float* chi2_out, float* d_p0,
                  float* d_align, float* d_xscale, int32_t* status_out, int mode, int on_device) {
    if (!ctx) return MKGB_EINVAL;
    if (mode != 0 && mode != 1) return fail(ctx, MKGB_EINVAL, "fit_grad mode %d (0 reverse sweep, 1 forward)", mode);
    if (!ctx->has_geom || !ctx->has_params) return fail(ctx, MKGB_ESTATE, "fit_grad before geometry/params");
    if (!ctx->has_hits) return fail(ctx, MKGB_ESTATE, "fit_grad before load_hits");
    if (n < 0 || max_steps < 0) return fail(ctx, MKGB_EINVAL, "negative size");
    if (!align || !xscale || !d_align || !d_xscale) return fail(ctx, MKGB_EINVAL, "null alignment/material array");
    if (n > 0 && (!layers || !hits || !p0 || !c0 || !chi2_out || !d_p0)) return fail(ctx, MKGB_EINVAL, "null fit array");
    if (!on_device)
        for (size_t q = 0; q < (size_t)n * max_steps; ++q)
            if (hits[q] >= ctx->n_hits) return fail(ctx, MKGB_EINVAL, "hit index %d out of range", hits[q]);
    DevGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;
    const size_t N = (size_t)n, M = (size_t)max_steps, NL = (size_t)ctx->n_layers;
    const void *dl, *dh, *dp0, *dc0, *dal, *dxs;
    CK(stage_in(ctx, S_A, layers, 4 * N * M, on_device, &dl));
    CK(stage_in(ctx, S_B, hits, 4 * N * M, on_device, &dh));
    CK(stage_in(ctx, S_C, p0, 24 * N, on_device, &dp0));
    CK(stage_in(ctx, S_D, c0, 84 * N, on_device, &dc0));
    CK(stage_in(ctx, S_E, align, 24 * NL, on_device, &dal));
    CK(stage_in(ctx, S_F, xscale, 4 * NL, on_device, &dxs));
    void *xo, *gp, *ga, *gx, *so;
    CK(stage_out(ctx, S_G, chi2_out, 4 * N, on_device, &xo));
    CK(stage_out(ctx, S_H, d_p0, 24 * N, on_device, &gp));
    CK(stage_out(ctx, S_I, d_align, 24 * NL, on_device, &ga));
    CK(stage_out(ctx, S_J, d_xscale, 4 * NL, on_device, &gx));
    CK(stage_out(ctx, S_K, status_out, 4 * N, on_device, &so));
    CK(cudaMemsetAsync(ga, 0, 24 * NL, st));   // summed over tracks by the kernel
    CK(cudaMemsetAsync(gx, 0, 4 * NL, st));
    float* ck = nullptr;
    if (mode == 0) {   // checkpoints of the reverse sweep: 128 bytes per track and step
        CK(ensure(ctx->grad_ck, 128 * N * std::max<size_t>(M, 1)));
        ck = (float*)ctx->grad_ck.p;
    }
    CK(launch_fit_grad(st, (const DevGeom*)ctx->geom_d.p, ctx->params, (const float4*)ctx->pay.p, ctx->n_hits, n,
                       max_steps, (const int*)dl, (const int*)dh, (const float*)dp0, (const float*)dc0,
                       (const float*)dal, (const float*)dxs, (float*)xo, (float*)gp, (float*)ga, (float*)gx, (int*)so,
                       ck, ctx->mod_hits));
    CK(copy_back(ctx, chi2_out, xo, 4 * N, on_device));
    CK(copy_back(ctx, d_p0, gp, 24 * N, on_device));
    CK(copy_back(ctx, d_align, ga, 24 * NL, on_device));
    CK(copy_back(ctx, d_xscale, gx, 4 * NL, on_device));
    CK(copy_back(ctx, status_out, so, 4 * N, on_device));
    if (!on_device) CK(cudaStreamSynchronize(st));
    return MKGB_OK;
}

namespace {

// Per-device address of the static fit scratch, looked up on the first mkgb_fit_static call on
// that device and kept for the life of the process.
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_base[kMaxDevices] = {};

cudaError_t static_scratch(int device, void** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_base[device]) {
        void* p = nullptr;
        const cudaError_t e = fit_static_scratch_address(&p);
        if (e != cudaSuccess) return e;
        g_static_base[device] = p;
    }
    *out = g_static_base[device];
    return cudaSuccess;
}

}  // namespace

int mkgb_fit_static(mkgb_ctx* ctx, int n, int max_steps, const int32_t* layers, const int32_t* hits,
                    const float* p0, const float* c0, float* p_out, float* c_out, float* chi2_out,
                    int32_t* status_out) {
    if (!ctx) return MKGB_EINVAL;
    if (!ctx->has_geom || !ctx->has_params) return fail(ctx, MKGB_ESTATE, "fit before geometry/params");
    if (!ctx->has_hits) return fail(ctx, MKGB_ESTATE, "fit with device hit indices before load_hits");
    if (n < 0 || max_steps < 0) return fail(ctx, MKGB_EINVAL, "negative size");
    if (n > kFitStaticMaxTracks)
        return fail(ctx, MKGB_EINVAL, "mkgb_fit_static: %d tracks exceed its static scratch limit of %d; "
                    "split the batch or call mkgb_fit", n, kFitStaticMaxTracks);
    if (n > 0 && (!layers || !hits || !p0 || !c0 || !p_out || !c_out || !chi2_out))
        return fail(ctx, MKGB_EINVAL, "null fit array");
    DevGuard guard(ctx->device);
    void* base = nullptr;
    CK(static_scratch(ctx->device, &base));
    if (n == 0) return MKGB_OK;
    unsigned char* b = static_cast<unsigned char*>(base);
    cudaStream_t st = ctx->stream;
    // the work counters and the refit counter start at zero on every call
    CK(cudaMemsetAsync(b, 0, kFitStaticZeroBytes, st));
    CK(launch_fit(st, (const DevGeom*)ctx->geom_d.p, ctx->params, (const float4*)ctx->pay.p, ctx->n_hits, n,
                  max_steps, layers, hits, p0, c0, p_out, c_out, chi2_out, status_out,
                  reinterpret_cast<unsigned long long*>(b + kFitStaticCountersOff),
                  reinterpret_cast<int*>(b + kFitStaticListOff), reinterpret_cast<int*>(b + kFitStaticRescueCountOff),
                  ctx->n_sms, ctx->mod_hits));
    return MKGB_OK;
}

}  // extern "C"

namespace {

// The fit's stream in a one-call pass: the highest priority, so that its blocks are scheduled
// as soon as SM resources free up beside the FP64-bound seed fit and the latency-bound search
// (28.03 against 28.13 ms per 64-event pass at the default priority).
cudaError_t create_fit_stream(cudaStream_t* st) {
    int least = 0, greatest = 0;
    const cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e != cudaSuccess) return e;
    return cudaStreamCreateWithPriority(st, cudaStreamNonBlocking, greatest);
}

int run_impl(mkgb_ctx* ctx, int n_events, const int64_t* seg_off, const float* xyz, const float* cov6,
             const int32_t* hit_module, int n_seeds, const int32_t* seed_hits, const mkgb_tracks* out, int n_fit,
             int max_steps, const int32_t* layers, const int32_t* hits, const float* p0, const float* c0,
             float* p_out, float* c_out, float* chi2_out, int32_t* status_out) {
    DevGuard guard(ctx->device);
    const cudaStream_t main_st = ctx->stream;
    if (!ctx->fit_st) {
        CK(create_fit_stream(&ctx->fit_st));
        CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->ev_fit, cudaEventDisableTiming));
    }
    int rc = hit_module ? mkgb_load_hits_modular(ctx, n_events, seg_off, xyz, cov6, hit_module, 1)
                        : mkgb_load_hits(ctx, n_events, seg_off, xyz, cov6, 1);
    if (rc != MKGB_OK) return rc;
    // the fit needs the prepared hits only: it runs on its own stream beside the seed fit and
    // the search, and the context's stream waits for it before the call ends
    CK(cudaEventRecord(ctx->ev_fork, main_st));
    CK(cudaStreamWaitEvent(ctx->fit_st, ctx->ev_fork, 0));
    ctx->stream = ctx->fit_st;
    rc = mkgb_fit(ctx, n_fit, max_steps, layers, hits, p0, c0, p_out, c_out, chi2_out, status_out, 1);
    ctx->stream = main_st;
    CK(cudaEventRecord(ctx->ev_fit, ctx->fit_st));
    if (rc == MKGB_OK) rc = mkgb_seed(ctx, n_seeds, seed_hits, 1, nullptr, nullptr, nullptr);
    if (rc == MKGB_OK) rc = mkgb_build(ctx, out, 1);
    CK(cudaStreamWaitEvent(main_st, ctx->ev_fit, 0));
    return rc;
}

// mkgb_run with host arrays.  The inputs go to the device on a copy stream: the hits in up to
// kHostChunks chunks of whole events, each prepared as soon as it has arrived, then the seeds and
// the fit's inputs, which arrive while the hits are prepared and the seeds fitted; the fit runs
// on its own stream and its outputs go back while the search runs; the search's outputs go back
// at the end.  Every copy is one cudaMemcpyAsync; with page-locked host arrays they overlap the
// kernels.
int run_host_impl(mkgb_ctx* ctx, int n_events, const int64_t* seg_off, const float* xyz, const float* cov6,
                  int n_seeds, const int32_t* seed_hits, const mkgb_tracks* out, int n_fit, int max_steps,
                  const int32_t* layers, const int32_t* hits, const float* p0, const float* c0, float* p_out,
                  float* c_out, float* chi2_out, int32_t* status_out) {
    if (!ctx->has_geom) return fail(ctx, MKGB_ESTATE, "run before load_geometry");
    if (n_events < 1 || !seg_off) return fail(ctx, MKGB_EINVAL, "need n_events >= 1 and seg_off");
    if (!out) return fail(ctx, MKGB_EINVAL, "null track outputs");
    if (n_seeds < 0 || n_fit < 0 || max_steps < 0) return fail(ctx, MKGB_EINVAL, "negative size");
    if (n_seeds > 0 && !seed_hits) return fail(ctx, MKGB_EINVAL, "null seed hits");
    if (n_fit > 0 && (!layers || !hits || !p0 || !c0 || !p_out || !c_out || !chi2_out))
        return fail(ctx, MKGB_EINVAL, "null fit array");
    const int L = ctx->n_layers;
    const int64_t nseg = (int64_t)n_events * L;
    if (seg_off[0] != 0) return fail(ctx, MKGB_EINVAL, "seg_off[0] must be 0");
    for (int64_t q = 0; q < nseg; ++q)
        if (seg_off[q + 1] < seg_off[q]) return fail(ctx, MKGB_EINVAL, "seg_off decreases at %lld", (long long)q);
    const int64_t n = seg_off[nseg];
    if (n > ((int64_t)1 << 28) - 8) return fail(ctx, MKGB_EINVAL, "too many hits (%lld)", (long long)n);
    if (n > 0 && (!xyz || !cov6)) return fail(ctx, MKGB_EINVAL, "null hit arrays");
    DevGuard guard(ctx->device);
    const cudaStream_t main_st = ctx->stream;
    if (!ctx->fit_st) {
        CK(create_fit_stream(&ctx->fit_st));
        CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->ev_fit, cudaEventDisableTiming));
    }
    if (!ctx->cp_in) {
        CK(cudaStreamCreateWithFlags(&ctx->cp_in, cudaStreamNonBlocking));
        for (int k = 0; k < mkgb_ctx::kHostChunks; ++k)
            CK(cudaEventCreateWithFlags(&ctx->ev_chunk[k], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->ev_seedin, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->ev_fitin, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming));
    }
    // device copies of the inputs and outputs, carved from one buffer (256-byte aligned pieces)
    const size_t NS = (size_t)n_seeds, NF = (size_t)n_fit, MS = (size_t)max_steps, MP = (size_t)out->max_plan;
    const bool ovl = out->ovl_hits != nullptr;
    const size_t sizes[] = {12 * (size_t)n, 24 * (size_t)n, 12 * NS, 4 * NF * MS, 4 * NF * MS, 24 * NF, 84 * NF,
                            24 * NF, 84 * NF, 4 * NF, 4 * NF, 24 * NS, 84 * NS, 4 * NS, 4 * NS, 4 * NS, 4 * NS,
                            4 * NS * MP, ovl ? 4 * NS * MP : 0};
    constexpr int kParts = sizeof(sizes) / sizeof(sizes[0]);
    size_t offs[kParts], total = 0;
    for (int q = 0; q < kParts; ++q) {
        offs[q] = total;
        total += (sizes[q] + 255) & ~(size_t)255;
    }
    CK(ensure(ctx->host_run, total > 0 ? total : 256));
    char* base = static_cast<char*>(ctx->host_run.p);
    auto part = [&](int q) { return static_cast<void*>(base + offs[q]); };
    float *d_xyz = (float*)part(0), *d_cov = (float*)part(1);
    int32_t* d_seeds = (int32_t*)part(2);
    int32_t *d_layers = (int32_t*)part(3), *d_hits = (int32_t*)part(4);
    float *d_p0 = (float*)part(5), *d_c0 = (float*)part(6);
    float *d_po = (float*)part(7), *d_co = (float*)part(8), *d_x2 = (float*)part(9);
    int32_t* d_st = (int32_t*)part(10);
    mkgb_tracks dout;
    dout.params = (float*)part(11); dout.cov = (float*)part(12); dout.chi2 = (float*)part(13);
    dout.score = (float*)part(14); dout.nfound = (int32_t*)part(15); dout.nholes = (int32_t*)part(16);
    dout.hits = (int32_t*)part(17); dout.max_plan = out->max_plan;
    dout.ovl_hits = ovl ? (int32_t*)part(18) : nullptr;

    // the copies start once the context's stream has passed everything enqueued before this call
    CK(cudaEventRecord(ctx->ev_start, main_st));
    CK(cudaStreamWaitEvent(ctx->cp_in, ctx->ev_start, 0));
    const int K = n_events < mkgb_ctx::kHostChunks ? n_events : mkgb_ctx::kHostChunks;
    int64_t hoff[mkgb_ctx::kHostChunks + 1];
    for (int k = 0; k <= K; ++k) hoff[k] = seg_off[(int64_t)((int64_t)n_events * k / K) * L];
    // the seeds first (each chunk's seeds are fitted as soon as its hits are prepared), then the
    // hits chunk by chunk, then the fit's inputs
    if (NS > 0) CK(cudaMemcpyAsync(d_seeds, seed_hits, 12 * NS, cudaMemcpyHostToDevice, ctx->cp_in));
    CK(cudaEventRecord(ctx->ev_seedin, ctx->cp_in));
    for (int k = 0; k < K; ++k) {
        const int64_t h0 = hoff[k], nh = hoff[k + 1] - hoff[k];
        if (nh > 0) {
            CK(cudaMemcpyAsync(d_xyz + 3 * h0, xyz + 3 * h0, 12 * nh, cudaMemcpyHostToDevice, ctx->cp_in));
            CK(cudaMemcpyAsync(d_cov + 6 * h0, cov6 + 6 * h0, 24 * nh, cudaMemcpyHostToDevice, ctx->cp_in));
        }
        CK(cudaEventRecord(ctx->ev_chunk[k], ctx->cp_in));
    }
    if (NF > 0) {
        if (MS > 0) {
            CK(cudaMemcpyAsync(d_layers, layers, 4 * NF * MS, cudaMemcpyHostToDevice, ctx->cp_in));
            CK(cudaMemcpyAsync(d_hits, hits, 4 * NF * MS, cudaMemcpyHostToDevice, ctx->cp_in));
        }
        CK(cudaMemcpyAsync(d_p0, p0, 24 * NF, cudaMemcpyHostToDevice, ctx->cp_in));
        CK(cudaMemcpyAsync(d_c0, c0, 84 * NF, cudaMemcpyHostToDevice, ctx->cp_in));
    }
    CK(cudaEventRecord(ctx->ev_fitin, ctx->cp_in));

    if (!ctx->has_params) return fail(ctx, MKGB_ESTATE, "run before set_params");
    ctx->n_events = n_events;   // sizes the seed ordering's keys
    int rc = seed_buffers(ctx, n_seeds);
    if (rc != MKGB_OK) return rc;
    const bool fp64 = ctx->params.precision == MKGB_FP64;
    SeedRange range;
    range.n_chunks = K;
    for (int k = 0; k <= K; ++k) range.off[k] = (int)hoff[k];
    auto seed_launch = [&](int which) -> int {
        HitStore H;
        memset(&H, 0, sizeof(H));
        H.seg_off = (const int64_t*)ctx->seg_off.p;
        H.n_events = n_events;
        H.n_layers = L;
        H.n_hits = n;
        H.pay = (const float4*)ctx->pay.p;
        H.hit_seg = (const int*)ctx->hit_seg.p;
        range.which = which;
        CK(launch_seed_fit(main_st, (const DevGeom*)ctx->geom_d.p, ctx->params, H, n_seeds, d_seeds,
                           (float*)ctx->seed_state.p, fp64 ? (double*)ctx->seed_state64.p : nullptr,
                           (int4*)ctx->seed_info.p, nullptr, nullptr, nullptr, range, false, (int*)ctx->seed_redo.p));
        if (which == K)   // every chunk's seeds are fitted: the FP64 redo of the listed ones
            CK(launch_seed_redo(main_st, (const DevGeom*)ctx->geom_d.p, ctx->params, H, n_seeds, d_seeds,
                                (float*)ctx->seed_state.p, (int4*)ctx->seed_info.p, nullptr, nullptr, nullptr, false,
                                (const int*)ctx->seed_redo.p, ctx->n_sms));
        return MKGB_OK;
    };
    CK(cudaMemsetAsync(ctx->seed_redo.p, 0, 4, main_st));
    CK(cudaStreamWaitEvent(main_st, ctx->ev_seedin, 0));
    HitChunks hc;
    hc.n = K;
    hc.hit_off = hoff;
    hc.ready = ctx->ev_chunk;
    hc.after = seed_launch;
    rc = load_hits_impl(ctx, n_events, seg_off, d_xyz, d_cov, nullptr, 1, &hc);
    if (rc != MKGB_OK) {
        cudaStreamSynchronize(ctx->cp_in);
        return rc;
    }
    // the seeds not inside one chunk (hits of several events, invalid ids), then their order
    rc = seed_launch(K);
    if (rc == MKGB_OK) rc = seed_order(ctx, main_st, n_seeds);
    if (rc != MKGB_OK) {
        cudaStreamSynchronize(ctx->cp_in);
        return rc;
    }
    // the fit: after the hit preparation and its inputs' arrival, on its own stream; its outputs
    // go back on that stream while the search runs
    CK(cudaEventRecord(ctx->ev_fork, main_st));
    CK(cudaStreamWaitEvent(ctx->fit_st, ctx->ev_fork, 0));
    CK(cudaStreamWaitEvent(ctx->fit_st, ctx->ev_fitin, 0));
    ctx->stream = ctx->fit_st;
    rc = mkgb_fit(ctx, n_fit, max_steps, d_layers, d_hits, d_p0, d_c0, d_po, d_co, d_x2, d_st, 1);
    ctx->stream = main_st;
    if (rc == MKGB_OK && NF > 0) {
        CK(cudaMemcpyAsync(p_out, d_po, 24 * NF, cudaMemcpyDeviceToHost, ctx->fit_st));
        CK(cudaMemcpyAsync(c_out, d_co, 84 * NF, cudaMemcpyDeviceToHost, ctx->fit_st));
        CK(cudaMemcpyAsync(chi2_out, d_x2, 4 * NF, cudaMemcpyDeviceToHost, ctx->fit_st));
        if (status_out) CK(cudaMemcpyAsync(status_out, d_st, 4 * NF, cudaMemcpyDeviceToHost, ctx->fit_st));
    }
    CK(cudaEventRecord(ctx->ev_fit, ctx->fit_st));
    if (rc == MKGB_OK) rc = mkgb_build(ctx, &dout, 1);
    if (rc == MKGB_OK && NS > 0) {
        CK(cudaMemcpyAsync(out->params, dout.params, 24 * NS, cudaMemcpyDeviceToHost, main_st));
        CK(cudaMemcpyAsync(out->cov, dout.cov, 84 * NS, cudaMemcpyDeviceToHost, main_st));
        CK(cudaMemcpyAsync(out->chi2, dout.chi2, 4 * NS, cudaMemcpyDeviceToHost, main_st));
        CK(cudaMemcpyAsync(out->score, dout.score, 4 * NS, cudaMemcpyDeviceToHost, main_st));
        CK(cudaMemcpyAsync(out->nfound, dout.nfound, 4 * NS, cudaMemcpyDeviceToHost, main_st));
        CK(cudaMemcpyAsync(out->nholes, dout.nholes, 4 * NS, cudaMemcpyDeviceToHost, main_st));
        if (MP > 0) CK(cudaMemcpyAsync(out->hits, dout.hits, 4 * NS * MP, cudaMemcpyDeviceToHost, main_st));
        if (ovl && MP > 0) CK(cudaMemcpyAsync(out->ovl_hits, dout.ovl_hits, 4 * NS * MP, cudaMemcpyDeviceToHost, main_st));
    }
    CK(cudaStreamWaitEvent(main_st, ctx->ev_fit, 0));
    CK(cudaStreamWaitEvent(main_st, ctx->ev_fitin, 0));
    CK(cudaStreamSynchronize(main_st));
    return rc;
}

}  // namespace

extern "C" {

int mkgb_run_host(mkgb_ctx* ctx, int n_events, const int64_t* seg_off, const float* xyz, const float* cov6,
                  int n_seeds, const int32_t* seed_hits, const mkgb_tracks* out, int n_fit, int max_steps,
                  const int32_t* layers, const int32_t* hits, const float* p0, const float* c0, float* p_out,
                  float* c_out, float* chi2_out, int32_t* status_out) {
    if (!ctx) return MKGB_EINVAL;
    return run_host_impl(ctx, n_events, seg_off, xyz, cov6, n_seeds, seed_hits, out, n_fit, max_steps, layers, hits,
                         p0, c0, p_out, c_out, chi2_out, status_out);
}

int mkgb_run(mkgb_ctx* ctx, int n_events, const int64_t* seg_off, const float* xyz, const float* cov6, int n_seeds,
             const int32_t* seed_hits, const mkgb_tracks* out, int n_fit, int max_steps, const int32_t* layers,
             const int32_t* hits, const float* p0, const float* c0, float* p_out, float* c_out, float* chi2_out,
             int32_t* status_out) {
    if (!ctx) return MKGB_EINVAL;
    return run_impl(ctx, n_events, seg_off, xyz, cov6, nullptr, n_seeds, seed_hits, out, n_fit, max_steps, layers,
                    hits, p0, c0, p_out, c_out, chi2_out, status_out);
}

int mkgb_run_modular(mkgb_ctx* ctx, int n_events, const int64_t* seg_off, const float* xyz, const float* cov6,
                     const int32_t* hit_module, int n_seeds, const int32_t* seed_hits, const mkgb_tracks* out,
                     int n_fit, int max_steps, const int32_t* layers, const int32_t* hits, const float* p0,
                     const float* c0, float* p_out, float* c_out, float* chi2_out, int32_t* status_out) {
    if (!ctx) return MKGB_EINVAL;
    if (!hit_module) return fail(ctx, MKGB_EINVAL, "null hit_module");
    return run_impl(ctx, n_events, seg_off, xyz, cov6, hit_module, n_seeds, seed_hits, out, n_fit, max_steps, layers,
                    hits, p0, c0, p_out, c_out, chi2_out, status_out);
}

int mkgb_set_launch(mkgb_ctx* ctx, int find_shape, int select_shape, int use_graph) {
    if (!ctx) return MKGB_EINVAL;
    if (find_shape < 0 || find_shape > 5 || select_shape < 0 || select_shape > 2)
        return fail(ctx, MKGB_EINVAL, "launch shapes (%d, %d) outside 0..5, 0..2", find_shape, select_shape);
    ctx->find_shape = find_shape;
    ctx->select_shape = select_shape;
    ctx->use_graph = use_graph != 0;
    return MKGB_OK;
}

int mkgb_autotune(mkgb_ctx* ctx, int reps, int* find_shape, int* select_shape, float* ms_out) {
    if (!ctx) return MKGB_EINVAL;
    if (!ctx->has_seeds) return fail(ctx, MKGB_ESTATE, "autotune before seed");
    if (reps < 1) return fail(ctx, MKGB_EINVAL, "reps %d < 1", reps);
    DevGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;
    const size_t n = (size_t)ctx->n_seeds;
    BuildOutDev d;
    void* p;
    CK(stage_buf(ctx, S_A, 24 * n, &p)); d.params = (float*)p;
    CK(stage_buf(ctx, S_B, 84 * n, &p)); d.cov = (float*)p;
    CK(stage_buf(ctx, S_C, 4 * n, &p)); d.chi2 = (float*)p;
    CK(stage_buf(ctx, S_D, 4 * n, &p)); d.score = (float*)p;
    CK(stage_buf(ctx, S_E, 4 * n, &p)); d.nfound = (int*)p;
    CK(stage_buf(ctx, S_F, 4 * n, &p)); d.nholes = (int*)p;
    CK(stage_buf(ctx, S_G, 4 * n * (size_t)ctx->max_plan_len, &p)); d.hits = (int*)p;
    d.max_plan = ctx->max_plan_len;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(ctx, MKGB_ECUDA, "event creation failed");
    }
    int best_f = ctx->find_shape, best_s = ctx->select_shape, rc = MKGB_OK;
    float best = -1.0f;
    for (int f = 0; f < 6 && rc == MKGB_OK; ++f)
        for (int s = 0; s < (f < 3 ? 3 : 1) && rc == MKGB_OK; ++s) {   // fused shapes have no select kernel
            rc = enqueue_build(ctx, d, f, s);   // warm-up (and the graph's recording)
            if (rc == MKGB_OK) cudaEventRecord(e0, st);
            for (int r = 0; r < reps && rc == MKGB_OK; ++r) rc = enqueue_build(ctx, d, f, s);
            if (rc != MKGB_OK) break;
            float ms = 0.0f;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = fail(ctx, MKGB_ECUDA, "autotune timing failed");
                break;
            }
            ms /= reps;
            if (best < 0.0f || ms < best) {
                best = ms;
                best_f = f;
                best_s = s;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MKGB_OK) return rc;
    ctx->find_shape = best_f;
    ctx->select_shape = best_s;
    if (find_shape) *find_shape = best_f;
    if (select_shape) *select_shape = best_s;
    if (ms_out) *ms_out = best;
    return MKGB_OK;
}

int mkgb_probe_peak(mkgb_ctx* ctx, int kind, double* tflops_out) {
    if (!ctx) return MKGB_EINVAL;
    if ((kind != 0 && kind != 1) || !tflops_out) return fail(ctx, MKGB_EINVAL, "probe kind %d or null output", kind);
    DevGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;
    CK(ensure(ctx->probe_sink, probe_sink_bytes(ctx->n_sms)));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(ctx, MKGB_ECUDA, "event creation failed");
    }
    // a short launch sizes the timed one to ~20 ms
    int iters = kind == 0 ? 512 : 16;
    double rate = 0.0;
    cudaError_t e = cudaSuccess;
    for (int pass = 0; pass < 3 && e == cudaSuccess; ++pass) {
        int64_t fmas = 0;
        float ms = 0.0f;
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = launch_probe_fma(st, kind, ctx->n_sms, iters, ctx->probe_sink.p, &fmas);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess || ms <= 0.0f) break;
        rate = 2.0 * (double)fmas / (ms * 1e-3) / 1e12;
        const double scale = 20.0 / ms;
        iters = (int)std::min(1e7, std::max(1.0, iters * scale));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(ctx, MKGB_ECUDA, "probe: %s", cudaGetErrorString(e));
    *tflops_out = rate;
    return MKGB_OK;
}

int mkgb_propagate(mkgb_ctx* ctx, int n, const int32_t* layers, const float* p_in, const float* c_in, float* p_out,
                   float* c_out, int32_t* crossed_out, int on_device) {
    if (!ctx) return MKGB_EINVAL;
    if (!ctx->has_geom || !ctx->has_params) return fail(ctx, MKGB_ESTATE, "propagate before geometry/params");
    if (n < 0 || (n > 0 && (!layers || !p_in || !c_in || !p_out || !c_out || !crossed_out)))
        return fail(ctx, MKGB_EINVAL, "bad propagate arguments");
    DevGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;
    const size_t N = (size_t)n;
    const void *dl, *dp, *dc;
    CK(stage_in(ctx, S_A, layers, 4 * N, on_device, &dl));
    CK(stage_in(ctx, S_B, p_in, 24 * N, on_device, &dp));
    CK(stage_in(ctx, S_C, c_in, 84 * N, on_device, &dc));
    void *po, *co, *xo;
    CK(stage_out(ctx, S_D, p_out, 24 * N, on_device, &po));
    CK(stage_out(ctx, S_E, c_out, 84 * N, on_device, &co));
    CK(stage_out(ctx, S_F, crossed_out, 4 * N, on_device, &xo));
    CK(launch_step_propagate(st, (const DevGeom*)ctx->geom_d.p, ctx->params, n, (const int*)dl, (const float*)dp,
                             (const float*)dc, (float*)po, (float*)co, (int*)xo));
    CK(copy_back(ctx, p_out, po, 24 * N, on_device));
    CK(copy_back(ctx, c_out, co, 84 * N, on_device));
    CK(copy_back(ctx, crossed_out, xo, 4 * N, on_device));
    if (!on_device) CK(cudaStreamSynchronize(st));
    return MKGB_OK;
}

int mkgb_update(mkgb_ctx* ctx, int n, const float* p_in, const float* c_in, const float* hit_xyz,
                const float* hit_cov, float* p_out, float* c_out, float* chi2_out, int32_t* ok_out, int on_device) {
    if (!ctx) return MKGB_EINVAL;
    if (n < 0 || (n > 0 && (!p_in || !c_in || !hit_xyz || !hit_cov || !p_out || !c_out || !chi2_out || !ok_out)))
        return fail(ctx, MKGB_EINVAL, "bad update arguments");
    DevGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;
    const size_t N = (size_t)n;
    const void *dp, *dc, *dx, *dv;
    CK(stage_in(ctx, S_A, p_in, 24 * N, on_device, &dp));
    CK(stage_in(ctx, S_B, c_in, 84 * N, on_device, &dc));
    CK(stage_in(ctx, S_C, hit_xyz, 12 * N, on_device, &dx));
    CK(stage_in(ctx, S_D, hit_cov, 24 * N, on_device, &dv));
    void *po, *co, *xo, *ko;
    CK(stage_out(ctx, S_E, p_out, 24 * N, on_device, &po));
    CK(stage_out(ctx, S_F, c_out, 84 * N, on_device, &co));
    CK(stage_out(ctx, S_G, chi2_out, 4 * N, on_device, &xo));
    CK(stage_out(ctx, S_H, ok_out, 4 * N, on_device, &ko));
    CK(launch_step_update(st, n, (const float*)dp, (const float*)dc, (const float*)dx, (const float*)dv, (float*)po,
                          (float*)co, (float*)xo, (int*)ko));
    CK(copy_back(ctx, p_out, po, 24 * N, on_device));
    CK(copy_back(ctx, c_out, co, 84 * N, on_device));
    CK(copy_back(ctx, chi2_out, xo, 4 * N, on_device));
    CK(copy_back(ctx, ok_out, ko, 4 * N, on_device));
    if (!on_device) CK(cudaStreamSynchronize(st));
    return MKGB_OK;
}

int mkgb_counters(mkgb_ctx* ctx, int kind, int64_t out[5]) {
    if (!ctx) return MKGB_EINVAL;
    if (!out || (kind != 0 && kind != 1)) return fail(ctx, MKGB_EINVAL, "bad counters request");
    DevGuard guard(ctx->device);
    unsigned long long h[kNumCounters];
    CK(cudaMemcpyAsync(h, kind == 0 ? ctx->counters_build.p : ctx->counters_fit.p, sizeof(h), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < kNumCounters; ++i) out[i] = (int64_t)h[i];
    return MKGB_OK;
}

}  // extern "C"
