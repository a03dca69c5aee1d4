// Combinatorial forward search (Sec. 2.2) as layer-synchronous rounds of two kernels.
//
// All seeds of all events advance together, one step of their layer plan per round (the
// paper's search processes every candidate of a layer before the next, Sec. 3.1).  A seed owns
// 8 candidate slots; per round:
//   k_find    one thread per live candidate, taken from a compacted work list: propagation with
//             Jacobian, transport and material (a4-a7), the eta-phi window (a8) and the chi2 of
//             each hit inside it (a9).  Writes the predicted state (surface frame) and the
//             candidate's children: its best hits (chi2 asc, hit id asc) and its non-hit child;
//   k_select  eight lanes per seed (lane = parent slot): merges the children of the seed's
//             candidates into the N best with 64-bit (score, parent slot) keys reduced by warp
//             shuffles (a10); lane r takes the r-th child, applies the Joseph update with its hit
//             from the parent's prediction (a11), writes slot r of the next round's buffers and
//             (parent slot, hit) to the trail, and appends the child to the next work lists.
// k_start fills round 0 from the seed states; k_finish picks each seed's best candidate and walks
// the trail back for its hit list (a13).
//
// Slot records are array-of-structures in HBM: a state is 32 floats (xh, yh, zh, xl, yl, zl, k,
// phi, theta, 21 covariance terms, theta's and phi's low parts), a prediction 28 floats, a child
// list 20 ints, the slot's (score, chi2 sum, counts, alive) one int4.  With module hits loaded
// (Sec. 3.1), the child list also names the best accepted hit on another module than its first
// entry's, and an overlap trail beside the hit trail keeps each step's overlap hit (Sec. 2.2).  Work lists are filled with warp-aggregated
// atomics, so the threads of a warp read neighbouring slots.  No kernel waits on another block;
// every loop is bounded by a list length, a window's bin range or the Newton iteration limit.
#include "internal.h"

#include <cstring>

namespace mk {

namespace {

constexpr int kGroup = 8;   // slots (lanes) per seed, >= MKGB_MAX_CANDS
constexpr int kThreads = 128;
constexpr float kBig = 3.0e38f;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long order_key(float score, int slot) {
    unsigned u = __float_as_uint(score);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | (unsigned)(kGroup - 1 - slot);
}

__device__ __forceinline__ float shfl_f(float v, int src) { return __shfl_sync(kFull, v, src); }
__device__ __forceinline__ int shfl_i(int v, int src) { return __shfl_sync(kFull, v, src); }

// ---- slot records: a state is 32 words (xh, yh, zh, xl, yl, zl, k, phi, theta, 21 covariance
// terms, theta's and phi's low parts), a prediction 28 words; words are F, moved as 16-byte vectors

__device__ __forceinline__ void unpack16(const float4& v, float* f) { f[0] = v.x; f[1] = v.y; f[2] = v.z; f[3] = v.w; }
__device__ __forceinline__ void unpack16(const double2& v, double* f) { f[0] = v.x; f[1] = v.y; }
__device__ __forceinline__ float4 pack16(const float* f) { return make_float4(f[0], f[1], f[2], f[3]); }
__device__ __forceinline__ double2 pack16(const double* f) { return make_double2(f[0], f[1]); }
template <class F> struct Vec16;
template <> struct Vec16<float> { using T = float4; };
template <> struct Vec16<double> { using T = double2; };

template <class F, int N> __device__ __forceinline__ void load_words(const unsigned char* __restrict__ p, F* f) {
    using V = typename Vec16<F>::T;
    constexpr int per = 16 / sizeof(F);
    const V* v = reinterpret_cast<const V*>(p);
#pragma unroll
    for (int i = 0; i < N / per; ++i) unpack16(v[i], f + per * i);
}

template <class F, int N> __device__ __forceinline__ void store_words(unsigned char* __restrict__ p, const F* f) {
    using V = typename Vec16<F>::T;
    constexpr int per = 16 / sizeof(F);
    V* v = reinterpret_cast<V*>(p);
#pragma unroll
    for (int i = 0; i < N / per; ++i) v[i] = pack16(f + per * i);
}

// Asynchronous 16-byte copy global -> shared (cached in L2 only), its commit and wait.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Words of a slot's state record (hi/lo positions, k, phi, theta, 21 covariance words, theta's
// and phi's low parts) and of its prediction record (the same with 15 surface-frame covariance
// words, padded to 16-byte words); layout_build_work sizes its arrays with them.
constexpr int kStateWords = 32, kPredWords = 28;
static_assert(kStateWords == kSeedStateStride, "seed records are copied into state records");
template <class F> constexpr size_t state_bytes() { return kStateWords * sizeof(F); }
template <class F> constexpr size_t pred_bytes() { return kPredWords * sizeof(F); }

template <class F> __device__ __forceinline__ void load_state_rec(const unsigned char* r, StateT<F>& t) {
    F f[kStateWords];
    load_words<F, kStateWords>(r, f);
    t.xh = f[0]; t.yh = f[1]; t.zh = f[2]; t.xl = f[3]; t.yl = f[4]; t.zl = f[5];
    t.k = f[6]; t.phi = f[7]; t.th = f[8];
#pragma unroll
    for (int i = 0; i < 21; ++i) t.c[i] = f[9 + i];
    t.tl = f[30];
    t.pl = f[31];
}

template <class F> __device__ __forceinline__ void store_state_rec(unsigned char* r, const StateT<F>& t) {
    F f[kStateWords];
    f[0] = t.xh; f[1] = t.yh; f[2] = t.zh; f[3] = t.xl; f[4] = t.yl; f[5] = t.zl;
    f[6] = t.k; f[7] = t.phi; f[8] = t.th;
#pragma unroll
    for (int i = 0; i < 21; ++i) f[9 + i] = t.c[i];
    f[30] = t.tl; f[31] = t.pl;
    store_words<F, kStateWords>(r, f);
}

template <class F> __device__ __forceinline__ void load_pred_rec(const unsigned char* r, PredT<F>& q) {
    F f[kPredWords];
    load_words<F, kPredWords>(r, f);
    q.xh = f[0]; q.yh = f[1]; q.zh = f[2]; q.xl = f[3]; q.yl = f[4]; q.zl = f[5];
    q.k = f[6]; q.phi = f[7]; q.th = f[8];
#pragma unroll
    for (int i = 0; i < 15; ++i) q.c[i] = f[9 + i];
    q.tl = f[24];
    q.pl = f[25];
}

template <class F> __device__ __forceinline__ void store_pred_rec(unsigned char* r, const PredT<F>& q) {
    F f[kPredWords];
    f[0] = q.xh; f[1] = q.yh; f[2] = q.zh; f[3] = q.xl; f[4] = q.yl; f[5] = q.zl;
    f[6] = q.k; f[7] = q.phi; f[8] = q.th;
#pragma unroll
    for (int i = 0; i < 15; ++i) f[9 + i] = q.c[i];
    f[24] = q.tl; f[25] = q.pl; f[26] = F(0); f[27] = F(0);
    store_words<F, kPredWords>(r, f);
}

template <class F> __device__ __forceinline__ void copy_state_rec(const unsigned char* src, unsigned char* dst) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int q = 0; q < (int)(state_bytes<F>() / 16); ++q) d4[q] = s4[q];
}

// slot meta: (score, chi2 sum, nfound | nholes << 8 | stopped << 16, alive)
__device__ __forceinline__ int4 pack_meta(float score, float chi2s, int nfound, int nholes, bool stopped, bool alive) {
    return make_int4(__float_as_int(score), __float_as_int(chi2s), nfound | (nholes << 8) | ((int)stopped << 16),
                     (int)alive);
}

// Appends v to list (count at *cnt) for the lanes with pred set: one atomic per warp.
__device__ __forceinline__ void warp_append(bool pred, int v, int* list, int* cnt) {
    const unsigned m = __ballot_sync(kFull, pred);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = v;
}

__device__ __forceinline__ void load_geom_smem(const DevGeom* __restrict__ gp, DevGeom& g) {
    const int4* src = reinterpret_cast<const int4*>(gp);
    int4* dst = reinterpret_cast<int4*>(&g);
    for (int i = threadIdx.x; i < (int)(sizeof(DevGeom) / 16); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
}

__device__ __forceinline__ void add_counters(unsigned long long* counters, unsigned long long c0,
                                             unsigned long long c1, unsigned long long c2, unsigned long long c3,
                                             unsigned long long c4) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        c0 += __shfl_xor_sync(kFull, c0, off);
        c1 += __shfl_xor_sync(kFull, c1, off);
        c2 += __shfl_xor_sync(kFull, c2, off);
        c3 += __shfl_xor_sync(kFull, c3, off);
        c4 += __shfl_xor_sync(kFull, c4, off);
    }
    if ((threadIdx.x & 31) == 0) {
        if (c0) atomicAdd(counters + 0, c0);
        if (c1) atomicAdd(counters + 1, c1);
        if (c2) atomicAdd(counters + 2, c2);
        if (c3) atomicAdd(counters + 3, c3);
        if (c4) atomicAdd(counters + 4, c4);
    }
}

struct BuildArgs {
    const DevGeom* geom;
    DevParams P;
    HitStore H;
    SeedStore S;
    BuildOutDev out;
    BuildWork w;
    unsigned long long* counters;
    int max_steps;   // trail rows per seed (longest plan)
    int nfound0;     // hits a track has when its search starts (3 seed hits forwards, 0 backwards)
    int fused;       // 1: one k_round per plan step (per-round list lengths in w.rcounts)
};

// ---- round 0: slot 0 of every seed with work takes the seed state
template <class F>
__global__ void __launch_bounds__(kThreads) k_start(BuildArgs a) {
    const DevGeom* __restrict__ g = a.geom;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;   // seed position in the (event, eta, phi) order
    bool work = false;
    if (i < a.S.n) {
        const int seed = a.S.order[i];
        const int4 inf = a.S.info[seed];
        int pos = 0, start = 0, nsteps = 0, event = 0;
        if (inf.w == 0) {
            const int pb = g->plan_off[inf.x];
            start = inf.y;
            pos = pb + start;
            nsteps = g->plan_off[inf.x + 1] - pos;
            if (nsteps < 0) nsteps = 0;
            event = inf.z;
        }
        a.w.sinfo[i] = make_int4(pos, start, nsteps, event);
        a.w.fin[i] = -1;
        work = nsteps > 0;
        const int4 dead = make_int4(0, 0, 0, 0);
#pragma unroll
        for (int c = 1; c < kGroup; ++c) a.w.meta[0][i * kGroup + c] = dead;
        if (work) {
            const unsigned char* src = sizeof(F) == 4
                ? reinterpret_cast<const unsigned char*>(a.S.state + (int64_t)seed * kSeedStateStride)
                : reinterpret_cast<const unsigned char*>(a.S.state64 + (int64_t)seed * kSeedStateStride);
            copy_state_rec<F>(src, a.w.st[0] + (int64_t)i * kGroup * state_bytes<F>());
            a.w.meta[0][i * kGroup] = pack_meta(0.0f, 0.0f, a.nfound0, 0, false, true);
        } else {
            a.w.meta[0][i * kGroup] = dead;
        }
    }
    warp_append(work, i * kGroup, a.w.live[0], a.fused ? a.w.rcounts + 0 : a.w.counts + 0);
    if (!a.fused) warp_append(work, i, a.w.seeds[0], a.w.counts + 2);
}

// ---- a4-a9 for every live candidate of round tau

// MOD: module hits loaded (their chi2 on the module planes, the overlap bookkeeping); the plain
// instantiation keeps the layers-only path's registers.
template <class F, int TH, int MINB, bool BWD = false, bool MOD = false>
__global__ void __launch_bounds__(TH, MINB) k_find(BuildArgs a, int tau) {
    __shared__ DevGeom g;
    // per-thread sorted list of hit children (chi2 asc, id asc), one column per thread
    __shared__ float s_x2[kGroup][TH];
    __shared__ int s_id[kGroup][TH];
    __shared__ int s_hq[kGroup][TH];
    load_geom_smem(a.geom, g);
    const int tx = threadIdx.x;
    const int cur = tau & 1, nxt = cur ^ 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {   // lists filled by this round's k_select
        a.w.counts[nxt] = 0;
        a.w.counts[2 + nxt] = 0;
        a.w.counts[4] = 0;
    }
    const DevParams& P = a.P;
    const int n = a.w.counts[cur];
    const int* __restrict__ list = a.w.live[cur];
    unsigned long long c_steps = 0, c_chi2 = 0, c_tested = 0, c_newton = 0;
    const int stride = gridDim.x * blockDim.x;
    // every lane of a warp runs the same number of iterations (warp_append inside k_select
    // needs converged warps; here it keeps the loop uniform)
    const int lane = threadIdx.x & 31;
    // The next item's records (state, meta, seed info) are copied into this thread's column of
    // s_rec while the current item is processed, so their load latency is hidden.  A column is
    // read into registers before the next copy into it is issued (the copy's shared-memory write
    // follows its global read, after these reads).  FP32 records and blocks of up to 128 threads
    // only (static shared memory); the FP64 comparison path loads directly.
    constexpr bool kPf = sizeof(F) == 4 && TH <= 128;
    constexpr int kSW = kPf ? (int)(state_bytes<F>() / 16) : 1;   // 16-byte words of a state record
    __shared__ int4 s_rec[kSW + 2][kPf ? TH : 1];
    auto fetch = [&](int slot) {
        const int4* src = reinterpret_cast<const int4*>(a.w.st[cur] + (int64_t)slot * state_bytes<F>());
#pragma unroll
        for (int j = 0; j < kSW; ++j) cp_async16(&s_rec[j][tx], src + j);
        cp_async16(&s_rec[kSW][tx], a.w.meta[cur] + slot);
        cp_async16(&s_rec[kSW + 1][tx], a.w.sinfo + slot / kGroup);
    };
    int sl_cur = -1, sl_next = -1;
    {
        const int first = blockIdx.x * blockDim.x + (threadIdx.x & ~31) + lane;
        sl_cur = first < n ? list[first] : -1;
        if constexpr (kPf) {
            if (sl_cur >= 0) fetch(sl_cur);
            cp_async_commit();
        }
        if (first + stride < n) sl_next = list[first + stride];
    }
    for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int idx = base + lane;
        const int sl = sl_cur;
        int4 si = make_int4(0, 0, 0, 0), mt = make_int4(0, 0, 0, 0);
        StateT<F> t;
        if constexpr (kPf) {
            cp_async_wait_all();
            if (sl >= 0) {
                si = s_rec[kSW + 1][tx];
                mt = s_rec[kSW][tx];
                F f[32];
#pragma unroll
                for (int j = 0; j < kSW; ++j)
                    unpack16(*reinterpret_cast<const typename Vec16<F>::T*>(&s_rec[j][tx]), f + j * (16 / sizeof(F)));
                t.xh = f[0]; t.yh = f[1]; t.zh = f[2]; t.xl = f[3]; t.yl = f[4]; t.zl = f[5];
                t.k = f[6]; t.phi = f[7]; t.th = f[8];
#pragma unroll
                for (int q = 0; q < 21; ++q) t.c[q] = f[9 + q];
                t.tl = f[30];
                t.pl = f[31];
            }
            asm volatile("" ::: "memory");
            sl_cur = sl_next;
            if (sl_cur >= 0) fetch(sl_cur);
            cp_async_commit();
        } else {
            if (sl >= 0) {
                si = a.w.sinfo[sl / kGroup];
                mt = a.w.meta[cur][sl];
                load_state_rec(a.w.st[cur] + (int64_t)sl * state_bytes<F>(), t);
            }
            sl_cur = sl_next;
        }
        sl_next = idx + 2 * stride < n ? list[idx + 2 * stride] : -1;
        if (idx >= n) continue;
        const int layer = g.plan[si.x + tau];
        const DevLayer& L = g.layers[layer];
        if (mt.w == 0) {   // dropped after the selection (its FP64 update redo failed)
            a.w.ls[(int64_t)sl * 5] = make_int4(0, K_NONE, 0, 0);
            continue;
        }
        const float score = __int_as_float(mt.x);
        const int nholes = (mt.z >> 8) & 0xff;

        PredT<F> q;
        F dir[4];
        int newton = 0;
        // BWD: the backward search (Sec. 2.2), crossing the plan's layers behind the candidate
        const int r = propagate_core<F, F, BWD>(L, g.cB, P.material, t, t.c, q, q.c, newton, dir);
        c_newton += newton;
        int nh_kind = K_NONE, n_h = 0;
        float nh_score = 0.0f;
        // overlap pickup (Sec. 2.2): the best accepted module hit b1 (the list's first entry on a
        // modular layer) and the best one on another module b2 (binned index, -1 none)
        int b1m = -1, b2 = -1, b2id = 0;
        float b1x = 0.0f, b2x = 0.0f;
        int b1id = 0, b1q = -1;
        if (r == 0) {
            nh_kind = K_SKIP;
            nh_score = score;
        } else if (r > 0) {
            ++c_steps;
            if (nholes < P.max_holes) {
                nh_kind = K_MISS;
                nh_score = score - P.score_hole;
            } else {
                nh_kind = K_STOP;
                nh_score = score;
            }
            const FrameT<F> fr = frame_of(L.kind, q.xh, q.yh, dir[0], dir[1], dir[2], dir[3]);
            const WindowT<F> w = window(L, P, q, fr);
            const float eps = 1e-5f;
            const float fe0 = (w.eta - w.deta - eps - L.eta_lo) * L.eta_scale;
            const float fe1 = (w.eta + w.deta + eps - L.eta_lo) * L.eta_scale;
            const int e0 = fe0 >= 0.0f ? (int)fminf(floorf(fe0), (float)(L.n_eta - 1)) : 0;
            const int e1 = fe1 >= 0.0f ? (int)fminf(floorf(fe1), (float)(L.n_eta - 1)) : 0;
            const float pscale = L.n_phi * (1.0f / kTwoPi);
            const int f0 = (int)floorf((w.phi - w.dphi - eps + kPi) * pscale);
            const int f1 = (int)floorf((w.phi + w.dphi + eps + kPi) * pscale);
            int nf = f1 - f0 + 1;
            int fa = f0 % L.n_phi;
            if (fa < 0) fa += L.n_phi;
            if (nf >= L.n_phi) {
                nf = L.n_phi;
                fa = 0;
            }
            const int run1 = min(nf, L.n_phi - fa), run2 = nf - run1;
            const int64_t bb = (int64_t)si.w * g.bins_per_event + L.bin_base;
            for (int ie = e0; ie <= e1; ++ie) {
                const int64_t rowb = bb + (int64_t)ie * L.n_phi;
                for (int run = 0; run < 2; ++run) {
                    const int b0 = run == 0 ? fa : 0;
                    const int nb = run == 0 ? run1 : run2;
                    if (nb <= 0) continue;
                    const int q0 = __ldg(a.H.bin_start + rowb + b0);
                    const int q1 = __ldg(a.H.bin_start + rowb + b0 + nb);
                    for (int hq = q0; hq < q1; ++hq) {
                        ++c_tested;
                        const float2 ep = __ldg(a.H.hb_ep + hq);
                        if (fabs(F(ep.x) - w.eta) <= w.deta && fabs(wrap_pi(F(ep.y) - w.phi)) <= w.dphi) {
                            ++c_chi2;
                            F m[3], v[6];
                            int id, md = -1;
                            F x2f;
                            bool okx;
                            if constexpr (MOD) {
                                load_hit(a.H.hb_pay, hq, m, v, &id, &md);
                                // a module hit: chi2 on its module's plane (Sec. 3.1)
                                okx = md >= 0 ? module_chi2_dir(q, fr, dir, g.mods, md, g.cB, m, v, x2f)
                                              : chi2_hit(fr, q, m[0], m[1], m[2], v, x2f);
                            } else {
                                load_hit(a.H.hb_pay, hq, m, v, &id);
                                okx = chi2_hit(fr, q, m[0], m[1], m[2], v, x2f);
                            }
                            if (okx && x2f < F(P.chi2_cut)) {
                                const float x2 = float(x2f);   // scores and child order in FP32
                                if (MOD && md >= 0) {
                                    if (b1m < 0 || x2 < b1x || (x2 == b1x && id < b1id)) {
                                        if (b1m >= 0 && md != b1m) {   // the previous b1 becomes b2
                                            b2 = b1q; b2x = b1x; b2id = b1id;
                                        }
                                        b1q = hq; b1x = x2; b1id = id; b1m = md;
                                    } else if (md != b1m && (b2 < 0 || x2 < b2x || (x2 == b2x && id < b2id))) {
                                        b2 = hq; b2x = x2; b2id = id;
                                    }
                                }
                                // insert into the sorted list (kept to its first kGroup entries)
                                int j = n_h < kGroup ? n_h : kGroup - 1;
                                const bool fits = n_h < kGroup ||
                                                  x2 < s_x2[j][tx] || (x2 == s_x2[j][tx] && id < s_id[j][tx]);
                                if (fits) {
                                    while (j > 0 && (x2 < s_x2[j - 1][tx] ||
                                                     (x2 == s_x2[j - 1][tx] && id < s_id[j - 1][tx]))) {
                                        s_x2[j][tx] = s_x2[j - 1][tx];
                                        s_id[j][tx] = s_id[j - 1][tx];
                                        s_hq[j][tx] = s_hq[j - 1][tx];
                                        --j;
                                    }
                                    s_x2[j][tx] = x2;
                                    s_id[j][tx] = id;
                                    s_hq[j][tx] = hq;
                                    if (n_h < kGroup) ++n_h;
                                }
                            }
                        }
                    }
                }
            }
            store_pred_rec(a.w.pr + (int64_t)sl * pred_bytes<F>(), q);
        }
        int4* lrec = a.w.ls + (int64_t)sl * 5;
        lrec[0] = make_int4(n_h, nh_kind, __float_as_int(nh_score), MOD ? b2 : -1);
        for (int j = 0; j < n_h; j += 2)
            lrec[1 + j / 2] = make_int4(__float_as_int(s_x2[j][tx]), s_hq[j][tx],
                                        __float_as_int(j + 1 < n_h ? s_x2[j + 1][tx] : kBig),
                                        j + 1 < n_h ? s_hq[j + 1][tx] : 0);
    }
    add_counters(a.counters, c_steps, c_chi2, 0ull, c_tested, c_newton);
}

// ---- a10-a11 for every seed with a live candidate in round tau
template <class F, int TH, int MINB, bool MOD = false>
__global__ void __launch_bounds__(TH, MINB) k_select(BuildArgs a, int tau) {
    __shared__ DevGeom g;
    load_geom_smem(a.geom, g);
    const int cur = tau & 1, nxt = cur ^ 1;
    const DevParams& P = a.P;
    const int lane = threadIdx.x & 31;
    const int slot = lane & 7, gbase = lane & ~7;
    const int n = a.w.counts[2 + cur];
    const int* __restrict__ list = a.w.seeds[cur];
    unsigned long long c_upd = 0;
    const int groups_per_block = TH / kGroup;
    const int gstride = gridDim.x * groups_per_block;
    // loop bound uniform over the warp: the first group index of the warp
    const int g0 = blockIdx.x * groups_per_block + (threadIdx.x >> 5) * 4;
    for (int wg = g0; wg < n; wg += gstride) {
        const int gi = wg + (lane >> 3);
        const bool gact = gi < n;
        const int i = gact ? list[gi] : 0;
        const int4 si = gact ? a.w.sinfo[i] : make_int4(0, 0, 0, 0);
        const int sl = i * kGroup + slot;
        const int4 mt = gact ? a.w.meta[cur][sl] : make_int4(0, 0, 0, 0);
        const float score = __int_as_float(mt.x);
        const bool alive = mt.w != 0;
        const bool stopped = ((mt.z >> 16) & 1) != 0;

        int nh_kind = K_NONE;
        float nh_score = -kBig;
        int b1q = -1, b2q = -1;   // the parent's best module hit and best hit on another module
        float lx[kGroup];
        int lq[kGroup];
#pragma unroll
        for (int j = 0; j < kGroup; ++j) {
            lx[j] = kBig;
            lq[j] = 0;
        }
        if (alive) {
            if (stopped) {
                nh_kind = K_CARRY;
                nh_score = score;
            } else {
                const int4* lrec = a.w.ls + (int64_t)sl * 5;
                int4 e[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) e[q] = lrec[q];   // all at once; entries past the count unused
                nh_kind = e[0].y;
                nh_score = __int_as_float(e[0].z);
#pragma unroll
                for (int j = 0; j < kGroup; j += 2) {
                    if (j < e[0].x) {
                        lx[j] = __int_as_float(e[1 + j / 2].x);
                        lq[j] = e[1 + j / 2].y;
                    }
                    if (j + 1 < e[0].x) {
                        lx[j + 1] = __int_as_float(e[1 + j / 2].z);
                        lq[j + 1] = e[1 + j / 2].w;
                    }
                }
                if constexpr (MOD) {
                    b2q = e[0].w;
                    b1q = e[0].x > 0 ? lq[0] : -1;
                }
            }
        }
        // a parent whose accepted module hits span two modules gives every hit child an overlap
        // hit (Sec. 2.2) and its score
        const float ovl_bonus = MOD && b2q >= 0 ? P.score_overlap : 0.0f;

        // ---- the N best children of the seed (a10)
        bool nh_avail = nh_kind != K_NONE;
        int my_parent = -1, my_kind = K_NONE, my_q = 0, my_b1 = -1, my_b2 = -1;
        float my_x2 = 0.0f, my_score = 0.0f;
        for (int r = 0; r < P.max_cands; ++r) {
            const bool has_hit = lx[0] < kBig;
            float hit_score = score + P.score_hit - lx[0];
            if constexpr (MOD) hit_score += ovl_bonus;
            int hk = K_NONE;
            float hs = 0.0f;
            if (has_hit && (!nh_avail || hit_score >= nh_score)) {
                hk = K_HIT;
                hs = hit_score;
            } else if (nh_avail) {
                hk = nh_kind;
                hs = nh_score;
            }
            unsigned long long best = hk != K_NONE ? order_key(hs, slot) : 0ull;
#pragma unroll
            for (int off = 1; off < kGroup; off <<= 1) {
                const unsigned long long o = __shfl_xor_sync(kFull, best, off);
                best = o > best ? o : best;
            }
            const bool valid = best != 0ull;
            const int wslot = kGroup - 1 - (int)(best & 7ull);
            const int src = gbase + wslot;
            const int w_kind = shfl_i(hk, src);
            const int w_q = shfl_i(lq[0], src);
            const float w_x2 = shfl_f(lx[0], src);
            const float w_score = shfl_f(hs, src);
            if (valid && slot == r) {
                my_parent = wslot;
                my_kind = w_kind;
                my_q = w_q;
                my_x2 = w_x2;
                my_score = w_score;
            }
            if constexpr (MOD) {
                const int w_b1 = shfl_i(b1q, src), w_b2 = shfl_i(b2q, src);
                if (valid && slot == r) {
                    my_b1 = w_b1;
                    my_b2 = w_b2;
                }
            }
            if (valid && slot == wslot) {
                if (hk == K_HIT) {
#pragma unroll
                    for (int j = 0; j < kGroup - 1; ++j) {
                        lx[j] = lx[j + 1];
                        lq[j] = lq[j + 1];
                    }
                    lx[kGroup - 1] = kBig;
                } else {
                    nh_avail = false;
                }
            }
        }

        // ---- the child's state (a11), meta, trail and next-round lists
        const int psrc = gbase + (my_parent >= 0 ? my_parent : slot);
        const int4 pm = make_int4(shfl_i(mt.x, psrc), shfl_i(mt.y, psrc), shfl_i(mt.z, psrc), shfl_i(mt.w, psrc));
        bool c_alive = false, c_stopped = false;
        float chi2s = __int_as_float(pm.y);
        int nfound = pm.z & 0xff, nholes = (pm.z >> 8) & 0xff;
        int code = MKGB_HIT_STOP;
        const int csl = i * kGroup + slot;
        bool rescue = false;
        int ovl = -1;
        if (gact && my_kind != K_NONE) {
            const int psl = i * kGroup + my_parent;
            c_alive = true;
            c_stopped = ((pm.z >> 16) & 1) != 0;
            if (my_kind == K_SKIP || my_kind == K_CARRY) {
                copy_state_rec<F>(a.w.st[cur] + (int64_t)psl * state_bytes<F>(),
                                  a.w.st[nxt] + (int64_t)csl * state_bytes<F>());
                if (my_kind == K_SKIP) code = MKGB_HIT_SKIP;
            } else {
                const DevLayer& L = g.layers[g.plan[si.x + tau]];
                PredT<F> pq;
                load_pred_rec(a.w.pr + (int64_t)psl * pred_bytes<F>(), pq);
                StateT<F> t;
                if (my_kind == K_HIT) {
                    F m[3], v[6];
                    int id, md = -1;
                    if constexpr (MOD)
                        load_hit(a.H.hb_pay, my_q, m, v, &id, &md);
                    else
                        load_hit(a.H.hb_pay, my_q, m, v, &id);
                    float kap = 0.0f;
                    bool ok;
                    if (MOD && md >= 0) {   // a module hit: the update on its module's plane (Sec. 3.1)
                        F x2u;
                        ok = module_update(L.kind, pq, g.mods, md, g.cB, m, v, 0.0f, t, x2u, kap) == 0;
                        if (my_b2 >= 0) {   // the overlap hit: b1 unless the hit is on b1's module
                            const int m1 = __float_as_int(__ldg(a.H.hb_pay + 3 * (int64_t)my_b1 + 2).z);
                            const int oq = md != m1 ? my_b1 : my_b2;
                            ovl = __float_as_int(__ldg(a.H.hb_pay + 3 * (int64_t)oq).w);
                        }
                    } else {
                        ok = kalman_update(L.kind, pq, m[0], m[1], m[2], v, t, &kap);
                    }
                    if (ok) {
                        chi2s += my_x2;
                        ++nfound;
                        ++c_upd;
                        code = id;
                        // FP32 cannot resolve an innovation covariance this ill-conditioned: the
                        // update is redone in FP64 by k_rescue (mixed precision, growth G3)
                        rescue = sizeof(F) == 4 && P.kappa_fp64 > 0.0f && kap > P.kappa_fp64;
                    } else {
                        c_alive = false;
                    }
                } else {
                    pred_to_state(L.kind, pq, t);
                    if (my_kind == K_MISS) {
                        ++nholes;
                        code = MKGB_HIT_MISS;
                    } else {   // K_STOP
                        c_stopped = true;
                    }
                }
                store_state_rec(a.w.st[nxt] + (int64_t)csl * state_bytes<F>(), t);
            }
            a.w.trail[((int64_t)i * a.max_steps + tau) * kGroup + slot] = ((code + 4) << 3) | my_parent;
            if (MOD && a.w.otrail) a.w.otrail[((int64_t)i * a.max_steps + tau) * kGroup + slot] = c_alive ? ovl : -1;
        }
        const bool more = gact && tau + 1 < si.z;
        const unsigned am = __ballot_sync(kFull, c_alive);
        const bool any = ((am >> gbase) & 0xffu) != 0u;
        const bool p_live = more && c_alive && !c_stopped, p_seed = more && any && slot == 0;
        const unsigned m0 = __ballot_sync(kFull, rescue), m1 = __ballot_sync(kFull, p_live),
                       m2 = __ballot_sync(kFull, p_seed);
        int b0 = 0, b1 = 0, b2 = 0;
        if (lane == 0) {   // the three list reservations of the warp, in flight together
            if (m0) b0 = atomicAdd(a.w.counts + 4, __popc(m0));
            if (m1) b1 = atomicAdd(a.w.counts + nxt, __popc(m1));
            if (m2) b2 = atomicAdd(a.w.counts + 2 + nxt, __popc(m2));
        }
        if (gact) a.w.meta[nxt][csl] = pack_meta(my_score, chi2s, nfound, nholes, c_stopped, c_alive);
        if (gact && slot == 0 && (!more || !any)) a.w.fin[i] = nxt | ((tau + 1) << 1);
        b0 = __shfl_sync(kFull, b0, 0);
        b1 = __shfl_sync(kFull, b1, 0);
        b2 = __shfl_sync(kFull, b2, 0);
        const unsigned below = (1u << lane) - 1u;
        if (rescue) a.w.rescue[b0 + __popc(m0 & below)] = csl;
        if (p_live) a.w.live[nxt][b1 + __popc(m1 & below)] = csl;
        if (p_seed) a.w.seeds[nxt][b2 + __popc(m2 & below)] = i;
    }
    add_counters(a.counters, 0ull, 0ull, c_upd, 0ull, 0ull);
}

// ---- fused round: a4-a11 for every live candidate of round tau in one launch
//
// A block takes a slice of the round's live list whose ends are moved to seed boundaries (the
// live candidates of a seed are contiguous in the list, at most kGroup of them), so each seed is
// handled by exactly one block.  Three phases, each with its own mapping of threads to work:
//   phase 1  one thread per candidate of the slice: propagation, window and chi2 (a4-a9); its
//            prediction (or, when it does not cross its layer, its state) and its sorted hit
//            children stay in shared memory;
//   merge    eight lanes per seed: the N best children of the seed (a10) by 64-bit (score,
//            parent slot) keys reduced with warp shuffles; every child becomes a descriptor in
//            shared memory, and the seed's next-round list entries are reserved in one go (its
//            candidates stay contiguous there);
//   update   one thread per child descriptor: the Joseph update from the parent's prediction in
//            shared memory (a11), the child's state, meta and trail.
// Against two kernels per round (a thread per candidate, then eight lanes per seed for merge and
// update) this keeps the prediction and child records (112 + 80 B per candidate) out of HBM, and
// the update no longer idles the lanes of the seed's empty slots.  A child whose update fails
// keeps its reserved list entry with a dead meta, which the next round skips.  The FP64 redo of a
// flagged update (k_rescue) finds its parent's prediction in the prediction array, written for
// flagged children only.

template <class F> constexpr int rec_vecs() { return (int)(state_bytes<F>() / 16); }
constexpr int kChildVecs(bool mod) { return mod ? 3 : 2; }   // int4 words of a child descriptor
// Shared memory of k_round for a block of th threads: records [rec_vecs][th] of 16-byte vectors,
// hit children chi2 / binned index / hit id [kGroup][th] each, per item a header and its slot
// meta (int4 each) and its slot, the first item of each seed (th + 1), and 4 th child
// descriptors (a merge chunk of th / 2 seeds has at most 4 th children).
template <class F, bool MOD> constexpr size_t round_smem_bytes(int th) {
    return (size_t)th * (16 * rec_vecs<F>() + 12 * kGroup + 16 + 16 + 8) + 16 + (size_t)4 * th * 16 * kChildVecs(MOD);
}

template <class F, int TH, int MINB, bool BWD = false, bool MOD = false>
__global__ void __launch_bounds__(TH, MINB) k_round(BuildArgs a, int tau) {
    static_assert(TH % 32 == 0 && TH >= 64, "whole warps, at least two per block");
    __shared__ DevGeom g;
    __shared__ int s_be[2];
    __shared__ int s_wsum[TH / 32];
    __shared__ int s_nchild;
    extern __shared__ __align__(16) unsigned char dsm[];
    using V = typename Vec16<F>::T;
    constexpr int RV = rec_vecs<F>();                       // 16-byte vectors of a state record
    constexpr int PV = (int)(pred_bytes<F>() / 16);         // ... of a prediction record
    constexpr int per = 16 / (int)sizeof(F);
    constexpr int CV = kChildVecs(MOD);
    constexpr int kChunkSeeds = TH / 2;                     // seeds merged before their updates
    V* s_rec = reinterpret_cast<V*>(dsm);                   // [RV][TH]
    float* s_x2 = reinterpret_cast<float*>(dsm + (size_t)16 * RV * TH);   // [kGroup][TH]
    int* s_hq = reinterpret_cast<int*>(s_x2 + kGroup * TH);
    int* s_id = s_hq + kGroup * TH;
    int4* s_hdr = reinterpret_cast<int4*>(s_id + kGroup * TH);   // (n hits, non-hit kind, its score, b2)
    int4* s_imeta = s_hdr + TH;                                  // the item's slot meta
    int4* s_child = s_imeta + TH;                                // [4 TH][CV] child descriptors
    int* s_slot = reinterpret_cast<int*>(s_child + 4 * TH * CV);
    int* s_first = s_slot + TH;                                  // TH + 1
    load_geom_smem(a.geom, g);
    const DevParams& P = a.P;
    const int tx = threadIdx.x, lane = tx & 31, wid = tx >> 5;
    const int cur = tau & 1, nxt = cur ^ 1;
    const int n = a.w.rcounts[tau];
    const int* __restrict__ list = a.w.live[cur];
    int* cnt_live = a.w.rcounts + tau + 1;
    int* cnt_resc = a.w.rcounts + kRescueCountBase + tau;
    constexpr int kSpan = TH - (kGroup - 1);   // nominal slice: at most TH items once its ends move
    const int ntiles = (n + kSpan - 1) / kSpan;
    unsigned long long c_steps = 0, c_chi2 = 0, c_tested = 0, c_newton = 0, c_upd = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (wid == 0) {
            // lanes 0-7: the eight positions from the nominal start, lanes 8-15: from the nominal
            // end; one of each eight starts a seed (or lies past the list)
            const int p = (tile + (lane >> 3)) * kSpan + (lane & 7);
            bool first = false;
            if (lane < 16) first = p >= n || p == 0 || (__ldg(list + p) >> 3) != (__ldg(list + p - 1) >> 3);
            const unsigned m = __ballot_sync(kFull, first);
            if (lane == 0) {
                s_be[0] = min(n, tile * kSpan + __ffs(m & 0xffu) - 1);
                s_be[1] = min(n, (tile + 1) * kSpan + __ffs((m >> 8) & 0xffu) - 1);
            }
        }
        __syncthreads();
        const int items = s_be[1] - s_be[0];

        // ---- phase 1: a4-a9 for the slice's candidates, one per thread
        const int sl = tx < items ? __ldg(list + s_be[0] + tx) : -1;
        s_slot[tx] = sl;
        if (sl >= 0) {
            const int4 si = __ldg(a.w.sinfo + sl / kGroup);
            const int4 mt = a.w.meta[cur][sl];
            s_imeta[tx] = mt;
            int nh_kind = K_NONE, n_h = 0, b2 = -1;
            float nh_score = 0.0f;
            if (mt.w != 0) {   // (0: dropped after the selection, its FP64 update redo failed)
                StateT<F> t;
                load_state_rec(a.w.st[cur] + (int64_t)sl * state_bytes<F>(), t);
                const DevLayer& L = g.layers[g.plan[si.x + tau]];
                const float score = __int_as_float(mt.x);
                const int nholes = (mt.z >> 8) & 0xff;
                PredT<F> q;
                F dir[4];
                int newton = 0;
                const int r = propagate_core<F, F, BWD>(L, g.cB, P.material, t, t.c, q, q.c, newton, dir);
                c_newton += newton;
                int b1m = -1, b2id = 0, b1id = 0, b1q = -1;
                float b1x = 0.0f, b2x = 0.0f;
                if (r == 0) {   // not crossed: the child is the unchanged state
                    nh_kind = K_SKIP;
                    nh_score = score;
                    F f[kStateWords];
                    f[0] = t.xh; f[1] = t.yh; f[2] = t.zh; f[3] = t.xl; f[4] = t.yl; f[5] = t.zl;
                    f[6] = t.k; f[7] = t.phi; f[8] = t.th;
#pragma unroll
                    for (int q2 = 0; q2 < 21; ++q2) f[9 + q2] = t.c[q2];
                    f[30] = t.tl; f[31] = t.pl;
#pragma unroll
                    for (int v = 0; v < RV; ++v) s_rec[v * TH + tx] = pack16(f + per * v);
                } else if (r > 0) {
                    ++c_steps;
                    if (nholes < P.max_holes) {
                        nh_kind = K_MISS;
                        nh_score = score - P.score_hole;
                    } else {
                        nh_kind = K_STOP;
                        nh_score = score;
                    }
                    const FrameT<F> fr = frame_of(L.kind, q.xh, q.yh, dir[0], dir[1], dir[2], dir[3]);
                    const WindowT<F> w = window(L, P, q, fr);
                    const float eps = 1e-5f;
                    const float fe0 = (w.eta - w.deta - eps - L.eta_lo) * L.eta_scale;
                    const float fe1 = (w.eta + w.deta + eps - L.eta_lo) * L.eta_scale;
                    const int e0 = fe0 >= 0.0f ? (int)fminf(floorf(fe0), (float)(L.n_eta - 1)) : 0;
                    const int e1 = fe1 >= 0.0f ? (int)fminf(floorf(fe1), (float)(L.n_eta - 1)) : 0;
                    const float pscale = L.n_phi * (1.0f / kTwoPi);
                    const int f0 = (int)floorf((w.phi - w.dphi - eps + kPi) * pscale);
                    const int f1 = (int)floorf((w.phi + w.dphi + eps + kPi) * pscale);
                    int nf = f1 - f0 + 1;
                    int fa = f0 % L.n_phi;
                    if (fa < 0) fa += L.n_phi;
                    if (nf >= L.n_phi) {
                        nf = L.n_phi;
                        fa = 0;
                    }
                    const int run1 = min(nf, L.n_phi - fa), run2 = nf - run1;
                    const int64_t bb = (int64_t)si.w * g.bins_per_event + L.bin_base;
                    for (int ie = e0; ie <= e1; ++ie) {
                        const int64_t rowb = bb + (int64_t)ie * L.n_phi;
                        for (int run = 0; run < 2; ++run) {
                            const int b0 = run == 0 ? fa : 0;
                            const int nb = run == 0 ? run1 : run2;
                            if (nb <= 0) continue;
                            const int q0 = __ldg(a.H.bin_start + rowb + b0);
                            const int q1 = __ldg(a.H.bin_start + rowb + b0 + nb);
                            for (int hq = q0; hq < q1; ++hq) {
                                ++c_tested;
                                const float2 ep = __ldg(a.H.hb_ep + hq);
                                if (fabs(F(ep.x) - w.eta) <= w.deta && fabs(wrap_pi(F(ep.y) - w.phi)) <= w.dphi) {
                                    ++c_chi2;
                                    F m[3], v[6];
                                    int id, md = -1;
                                    F x2f;
                                    bool okx;
                                    if constexpr (MOD) {
                                        load_hit(a.H.hb_pay, hq, m, v, &id, &md);
                                        okx = md >= 0 ? module_chi2_dir(q, fr, dir, g.mods, md, g.cB, m, v, x2f)
                                                      : chi2_hit(fr, q, m[0], m[1], m[2], v, x2f);
                                    } else {
                                        load_hit(a.H.hb_pay, hq, m, v, &id);
                                        okx = chi2_hit(fr, q, m[0], m[1], m[2], v, x2f);
                                    }
                                    if (okx && x2f < F(P.chi2_cut)) {
                                        const float x2 = float(x2f);   // scores and child order in FP32
                                        if (MOD && md >= 0) {
                                            if (b1m < 0 || x2 < b1x || (x2 == b1x && id < b1id)) {
                                                if (b1m >= 0 && md != b1m) {   // the previous b1 becomes b2
                                                    b2 = b1q; b2x = b1x; b2id = b1id;
                                                }
                                                b1q = hq; b1x = x2; b1id = id; b1m = md;
                                            } else if (md != b1m && (b2 < 0 || x2 < b2x || (x2 == b2x && id < b2id))) {
                                                b2 = hq; b2x = x2; b2id = id;
                                            }
                                        }
                                        // insert into the sorted list (kept to its first kGroup entries)
                                        int jj = n_h < kGroup ? n_h : kGroup - 1;
                                        const bool fits = n_h < kGroup || x2 < s_x2[jj * TH + tx] ||
                                                          (x2 == s_x2[jj * TH + tx] && id < s_id[jj * TH + tx]);
                                        if (fits) {
                                            while (jj > 0 && (x2 < s_x2[(jj - 1) * TH + tx] ||
                                                              (x2 == s_x2[(jj - 1) * TH + tx] &&
                                                               id < s_id[(jj - 1) * TH + tx]))) {
                                                s_x2[jj * TH + tx] = s_x2[(jj - 1) * TH + tx];
                                                s_id[jj * TH + tx] = s_id[(jj - 1) * TH + tx];
                                                s_hq[jj * TH + tx] = s_hq[(jj - 1) * TH + tx];
                                                --jj;
                                            }
                                            s_x2[jj * TH + tx] = x2;
                                            s_id[jj * TH + tx] = id;
                                            s_hq[jj * TH + tx] = hq;
                                            if (n_h < kGroup) ++n_h;
                                        }
                                    }
                                }
                            }
                        }
                    }
                    F f[kPredWords];
                    f[0] = q.xh; f[1] = q.yh; f[2] = q.zh; f[3] = q.xl; f[4] = q.yl; f[5] = q.zl;
                    f[6] = q.k; f[7] = q.phi; f[8] = q.th;
#pragma unroll
                    for (int q2 = 0; q2 < 15; ++q2) f[9 + q2] = q.c[q2];
                    f[24] = q.tl; f[25] = q.pl; f[26] = F(0); f[27] = F(0);
#pragma unroll
                    for (int v = 0; v < PV; ++v) s_rec[v * TH + tx] = pack16(f + per * v);
                }
            }
            s_hdr[tx] = make_int4(n_h, nh_kind, __float_as_int(nh_score), MOD ? b2 : -1);
        }
        __syncthreads();

        // ---- the slice's seeds: the first item of each (block-wide count of seed starts)
        int nseeds;
        {
            const bool first = sl >= 0 && (tx == 0 || (s_slot[tx - 1] >> 3) != (sl >> 3));
            const unsigned m = __ballot_sync(kFull, first);
            if (lane == 0) s_wsum[wid] = __popc(m);
            __syncthreads();
            int off = 0, tot = 0;
#pragma unroll
            for (int k = 0; k < TH / 32; ++k) {
                const int v = s_wsum[k];
                off += k < wid ? v : 0;
                tot += v;
            }
            if (first) s_first[off + __popc(m & ((1u << lane) - 1u))] = tx;
            if (tx == 0) s_first[tot] = items;
            nseeds = tot;
        }

        const int slot = lane & 7, gbase = lane & ~7;
        for (int sbase = 0; sbase < nseeds; sbase += kChunkSeeds) {
            const int send = min(nseeds, sbase + kChunkSeeds);
            if (tx == 0) s_nchild = 0;
            __syncthreads();
            // ---- merge: eight lanes per seed (lane = parent slot / child rank), a10
            for (int wg = sbase + wid * 4; wg < send; wg += TH / kGroup) {   // uniform over the warp
                const int gi = wg + (lane >> 3);
                const bool gact = gi < send;
                const int j0 = gact ? s_first[gi] : 0, j1 = gact ? s_first[gi + 1] : 0;
                const int i = gact ? (s_slot[j0] >> 3) : 0;
                const int4 si = gact ? __ldg(a.w.sinfo + i) : make_int4(0, 0, 0, 0);
                int jr = -1;   // this slot's item in the slice (live candidates only)
                for (int jj = j0; jj < j1; ++jj)
                    if ((s_slot[jj] & 7) == slot) jr = jj;
                const int4 mt = !gact ? make_int4(0, 0, 0, 0) : jr >= 0 ? s_imeta[jr] : a.w.meta[cur][i * kGroup + slot];
                const float score = __int_as_float(mt.x);
                const bool alive = mt.w != 0;
                const bool stopped = ((mt.z >> 16) & 1) != 0;

                int nh_kind = K_NONE;
                float nh_score = -kBig;
                int b1q = -1, b2q = -1;
                float lx[kGroup];
                int lq[kGroup];
#pragma unroll
                for (int jj = 0; jj < kGroup; ++jj) {
                    lx[jj] = kBig;
                    lq[jj] = 0;
                }
                if (alive) {
                    if (stopped) {
                        nh_kind = K_CARRY;
                        nh_score = score;
                    } else if (jr >= 0) {
                        const int4 h = s_hdr[jr];
                        nh_kind = h.y;
                        nh_score = __int_as_float(h.z);
#pragma unroll
                        for (int jj = 0; jj < kGroup; ++jj)
                            if (jj < h.x) {
                                lx[jj] = s_x2[jj * TH + jr];
                                lq[jj] = s_hq[jj * TH + jr];
                            }
                        if constexpr (MOD) {
                            b2q = h.w;
                            b1q = h.x > 0 ? lq[0] : -1;
                        }
                    }
                }
                const float ovl_bonus = MOD && b2q >= 0 ? P.score_overlap : 0.0f;

                bool nh_avail = nh_kind != K_NONE;
                int my_parent = -1, my_kind = K_NONE, my_q = 0, my_b1 = -1, my_b2 = -1;
                float my_x2 = 0.0f, my_score = 0.0f;
                for (int r = 0; r < P.max_cands; ++r) {
                    const bool has_hit = lx[0] < kBig;
                    float hit_score = score + P.score_hit - lx[0];
                    if constexpr (MOD) hit_score += ovl_bonus;
                    int hk = K_NONE;
                    float hs = 0.0f;
                    if (has_hit && (!nh_avail || hit_score >= nh_score)) {
                        hk = K_HIT;
                        hs = hit_score;
                    } else if (nh_avail) {
                        hk = nh_kind;
                        hs = nh_score;
                    }
                    unsigned long long best = hk != K_NONE ? order_key(hs, slot) : 0ull;
#pragma unroll
                    for (int off = 1; off < kGroup; off <<= 1) {
                        const unsigned long long o = __shfl_xor_sync(kFull, best, off);
                        best = o > best ? o : best;
                    }
                    const bool valid = best != 0ull;
                    const int wslot = kGroup - 1 - (int)(best & 7ull);
                    const int src = gbase + wslot;
                    const int w_kind = shfl_i(hk, src);
                    const int w_q = shfl_i(lq[0], src);
                    const float w_x2 = shfl_f(lx[0], src);
                    const float w_score = shfl_f(hs, src);
                    if (valid && slot == r) {
                        my_parent = wslot;
                        my_kind = w_kind;
                        my_q = w_q;
                        my_x2 = w_x2;
                        my_score = w_score;
                    }
                    if constexpr (MOD) {
                        const int w_b1 = shfl_i(b1q, src), w_b2 = shfl_i(b2q, src);
                        if (valid && slot == r) {
                            my_b1 = w_b1;
                            my_b2 = w_b2;
                        }
                    }
                    if (valid && slot == wslot) {
                        if (hk == K_HIT) {
#pragma unroll
                            for (int jj = 0; jj < kGroup - 1; ++jj) {
                                lx[jj] = lx[jj + 1];
                                lq[jj] = lq[jj + 1];
                            }
                            lx[kGroup - 1] = kBig;
                        } else {
                            nh_avail = false;
                        }
                    }
                }

                // the child of rank `slot`: its parent's meta and record, descriptor and list entry
                const int psrc = gbase + (my_parent >= 0 ? my_parent : slot);
                const int4 pm = make_int4(shfl_i(mt.x, psrc), shfl_i(mt.y, psrc), shfl_i(mt.z, psrc), shfl_i(mt.w, psrc));
                const int pj = shfl_i(jr, psrc);
                const int csl = i * kGroup + slot;
                const bool has_child = gact && my_kind != K_NONE;
                const bool more = gact && tau + 1 < si.z;
                // live next round unless stopped (its parent's stop carried, or a stop here) or its
                // update fails (its entry then meets a dead meta)
                const bool pot_live = has_child && more && my_kind != K_STOP && my_kind != K_CARRY &&
                                      ((pm.z >> 16) & 1) == 0;
                const unsigned mc = __ballot_sync(kFull, has_child), ml = __ballot_sync(kFull, pot_live);
                int bc = 0, bl = 0;
                if (lane == 0) {
                    if (mc) bc = atomicAdd(&s_nchild, __popc(mc));
                    if (ml) bl = atomicAdd(cnt_live, __popc(ml));
                }
                bc = __shfl_sync(kFull, bc, 0);
                bl = __shfl_sync(kFull, bl, 0);
                const unsigned below = (1u << lane) - 1u;
                if (pot_live) a.w.live[nxt][bl + __popc(ml & below)] = csl;
                if (has_child) {
                    const int c = bc + __popc(mc & below);
                    int4* d = s_child + c * CV;
                    d[0] = make_int4(csl, my_kind | (my_parent << 4) | ((pj + 1) << 8), my_q, __float_as_int(my_x2));
                    d[1] = make_int4(__float_as_int(my_score), pm.y, pm.z, g.plan[si.x + tau]);
                    if constexpr (MOD) d[2] = make_int4(my_b1, my_b2, 0, 0);
                } else if (gact) {
                    a.w.meta[nxt][csl] = make_int4(0, 0, 0, 0);
                }
                // no live child left (plan ended, every child stopped or none): the seed ends here
                const bool any_live = ((ml >> gbase) & 0xffu) != 0u;
                if (gact && slot == 0 && !any_live) a.w.fin[i] = nxt | ((tau + 1) << 1);
            }
            __syncthreads();

            // ---- update: one thread per child (a11)
            const int nc = s_nchild;
            for (int c0 = 0; c0 < nc; c0 += TH) {   // uniform over the block
                const int c = c0 + tx;
                const bool act = c < nc;
                int4 d0 = make_int4(0, 0, 0, 0), d1 = make_int4(0, 0, 0, 0);
                int my_b1 = -1, my_b2 = -1;
                if (act) {
                    d0 = s_child[c * CV];
                    d1 = s_child[c * CV + 1];
                    if constexpr (MOD) {
                        const int4 d2 = s_child[c * CV + 2];
                        my_b1 = d2.x;
                        my_b2 = d2.y;
                    }
                }
                const int csl = d0.x, my_kind = d0.y & 15, my_parent = (d0.y >> 4) & 15, pj = (d0.y >> 8) - 1;
                const int my_q = d0.z;
                const float my_x2 = __int_as_float(d0.w), my_score = __int_as_float(d1.x);
                const int i = csl / kGroup, cslot = csl % kGroup;
                bool c_alive = act, c_stopped = ((d1.z >> 16) & 1) != 0;
                float chi2s = __int_as_float(d1.y);
                int nfound = d1.z & 0xff, nholes = (d1.z >> 8) & 0xff;
                int code = MKGB_HIT_STOP;
                bool rescue = false;
                int ovl = -1;
                if (act) {
                    const int psl = i * kGroup + my_parent;
                    unsigned char* dst = a.w.st[nxt] + (int64_t)csl * state_bytes<F>();
                    if (my_kind == K_CARRY) {
                        copy_state_rec<F>(a.w.st[cur] + (int64_t)psl * state_bytes<F>(), dst);
                    } else if (my_kind == K_SKIP) {
                        V* d4 = reinterpret_cast<V*>(dst);
#pragma unroll
                        for (int v = 0; v < RV; ++v) d4[v] = s_rec[v * TH + pj];
                        code = MKGB_HIT_SKIP;
                    } else {
                        const DevLayer& L = g.layers[d1.w];
                        PredT<F> pq;
                        {
                            F f[kPredWords];
#pragma unroll
                            for (int v = 0; v < PV; ++v) unpack16(s_rec[v * TH + pj], f + per * v);
                            pq.xh = f[0]; pq.yh = f[1]; pq.zh = f[2]; pq.xl = f[3]; pq.yl = f[4]; pq.zl = f[5];
                            pq.k = f[6]; pq.phi = f[7]; pq.th = f[8];
#pragma unroll
                            for (int q2 = 0; q2 < 15; ++q2) pq.c[q2] = f[9 + q2];
                            pq.tl = f[24];
                            pq.pl = f[25];
                        }
                        StateT<F> t;
                        if (my_kind == K_HIT) {
                            F m[3], v[6];
                            int id, md = -1;
                            if constexpr (MOD)
                                load_hit(a.H.hb_pay, my_q, m, v, &id, &md);
                            else
                                load_hit(a.H.hb_pay, my_q, m, v, &id);
                            float kap = 0.0f;
                            bool ok;
                            if (MOD && md >= 0) {   // a module hit: the update on its module's plane (Sec. 3.1)
                                F x2u;
                                ok = module_update(L.kind, pq, g.mods, md, g.cB, m, v, 0.0f, t, x2u, kap) == 0;
                                if (my_b2 >= 0) {   // the overlap hit: b1 unless the hit is on b1's module
                                    const int m1 = __float_as_int(__ldg(a.H.hb_pay + 3 * (int64_t)my_b1 + 2).z);
                                    const int oq = md != m1 ? my_b1 : my_b2;
                                    ovl = __float_as_int(__ldg(a.H.hb_pay + 3 * (int64_t)oq).w);
                                }
                            } else {
                                ok = kalman_update(L.kind, pq, m[0], m[1], m[2], v, t, &kap);
                            }
                            if (ok) {
                                chi2s += my_x2;
                                ++nfound;
                                ++c_upd;
                                code = id;
                                // FP32 cannot resolve an innovation covariance this ill-conditioned:
                                // k_rescue redoes the update in FP64 from the parent's prediction
                                rescue = sizeof(F) == 4 && P.kappa_fp64 > 0.0f && kap > P.kappa_fp64;
                                if (rescue) store_pred_rec(a.w.pr + (int64_t)psl * pred_bytes<F>(), pq);
                            } else {
                                c_alive = false;
                            }
                        } else {
                            pred_to_state(L.kind, pq, t);
                            if (my_kind == K_MISS) {
                                ++nholes;
                                code = MKGB_HIT_MISS;
                            } else {   // K_STOP
                                c_stopped = true;
                            }
                        }
                        store_state_rec(dst, t);
                    }
                    a.w.trail[((int64_t)i * a.max_steps + tau) * kGroup + cslot] = ((code + 4) << 3) | my_parent;
                    if (MOD && a.w.otrail)
                        a.w.otrail[((int64_t)i * a.max_steps + tau) * kGroup + cslot] = c_alive ? ovl : -1;
                    a.w.meta[nxt][csl] = pack_meta(my_score, chi2s, nfound, nholes, c_stopped, c_alive);
                }
                const unsigned m0 = __ballot_sync(kFull, rescue);
                int b0 = 0;
                if (lane == 0 && m0) b0 = atomicAdd(cnt_resc, __popc(m0));
                b0 = __shfl_sync(kFull, b0, 0);
                if (rescue) a.w.rescue[b0 + __popc(m0 & ((1u << lane) - 1u))] = csl;
            }
            __syncthreads();   // the next chunk's merge reuses the descriptors
        }
    }
    add_counters(a.counters, c_steps, c_chi2, c_upd, c_tested, c_newton);
}

// ---- FP64 redo of the round's flagged updates (kept children of round tau whose innovation
// covariance had a condition estimate above kappa_fp64); one thread per child
__global__ void __launch_bounds__(kThreads) k_rescue(BuildArgs a, int tau) {
    __shared__ DevGeom g;
    load_geom_smem(a.geom, g);
    const int nxt = (tau & 1) ^ 1;
    const int n = a.fused ? a.w.rcounts[kRescueCountBase + tau] : a.w.counts[4];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int csl = a.w.rescue[r];
        const int i = csl / kGroup;
        const int slot = csl % kGroup;
        const int v = a.w.trail[((int64_t)i * a.max_steps + tau) * kGroup + slot];
        const int psl = i * kGroup + (v & 7);
        const int4 si = a.w.sinfo[i];
        const int lkind = g.layers[g.plan[si.x + tau]].kind;
        Pred pq;
        load_pred_rec(a.w.pr + (int64_t)psl * pred_bytes<float>(), pq);
        PredT<double> qd;
        qd.xh = pq.xh; qd.yh = pq.yh; qd.zh = pq.zh; qd.xl = pq.xl; qd.yl = pq.yl; qd.zl = pq.zl;
        qd.k = pq.k; qd.phi = pq.phi; qd.th = pq.th; qd.tl = pq.tl; qd.pl = pq.pl;
#pragma unroll
        for (int q = 0; q < 15; ++q) qd.c[q] = pq.c[q];
        // the hit: its binned index is not in the trail (which holds the hit id), so it is looked
        // up through the hit id in the payload's original order
        const int id = (v >> 3) - 4;
        double m[3], vv[6];
        int md;
        load_hit(a.H.pay, id, m, vv, nullptr, &md);
        StateT<double> td;
        bool ok;
        if (md >= 0) {
            double x2u;
            float kap;
            ok = module_update(lkind, qd, g.mods, md, g.cB, m, vv, 0.0f, td, x2u, kap) == 0;
        } else {
            ok = kalman_update(lkind, qd, m[0], m[1], m[2], vv, td);
        }
        if (ok) {
            State t;
            narrow_state(td, t);
            store_state_rec(a.w.st[nxt] + (int64_t)csl * state_bytes<float>(), t);
        } else {
            a.w.meta[nxt][csl].w = 0;   // dropped; k_find skips it
        }
    }
}

// ---- best candidate per seed and its hit list (a13); 8 lanes per seed
template <class F>
__global__ void __launch_bounds__(kThreads) k_finish(BuildArgs a) {
    const int lane = threadIdx.x & 31, slot = lane & 7, gbase = lane & ~7;
    const int gi = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const bool gact = gi < a.S.n;
    const int i = gact ? gi : 0;
    const int finv = gact ? a.w.fin[i] : -1;
    const int fin = finv >= 0 ? finv & 1 : -1, rounds = finv >= 0 ? finv >> 1 : 0;
    int4 mt = make_int4(0, 0, 0, 0);
    if (fin >= 0) mt = a.w.meta[fin][i * kGroup + slot];
    const unsigned am = __ballot_sync(kFull, mt.w != 0);
    const unsigned gm = (am >> gbase) & 0xffu;
    if (!gact) return;
    const int best = gm ? __ffs(gm) - 1 : -1;
    const int seed = a.S.order[i];
    int* hrow = a.out.hits + (int64_t)seed * a.out.max_plan;
    int* orow = a.out.ovl ? a.out.ovl + (int64_t)seed * a.out.max_plan : nullptr;
    for (int q = slot; q < a.out.max_plan; q += kGroup) {
        hrow[q] = MKGB_HIT_PRE;
        if (orow) orow[q] = -1;
    }
    __syncwarp(0xffu << gbase);
    if (slot != (best >= 0 ? best : 0)) return;
    float* po = a.out.params + 6 * (int64_t)seed;
    float* co = a.out.cov + 21 * (int64_t)seed;
    if (best >= 0) {
        StateT<F> t;
        load_state_rec(a.w.st[fin] + (int64_t)(i * kGroup + best) * state_bytes<F>(), t);
        store_state6(t, po, co);
        a.out.chi2[seed] = __int_as_float(mt.y);
        a.out.score[seed] = __int_as_float(mt.x);
        a.out.nfound[seed] = mt.z & 0xff;
        a.out.nholes[seed] = (mt.z >> 8) & 0xff;
        const int4 si = a.w.sinfo[i];
        // a seed whose candidates had all stopped before its plan ended (fused rounds finish it
        // then): its later plan steps are those of a stopped candidate
        for (int tau = rounds; tau < si.z; ++tau) {
            hrow[si.y + tau] = MKGB_HIT_STOP;
            if (orow) orow[si.y + tau] = -1;
        }
        int s_ = best;
        for (int tau = min(rounds, si.z) - 1; tau >= 0; --tau) {
            const int64_t at = ((int64_t)i * a.max_steps + tau) * kGroup + s_;
            const int v = a.w.trail[at];
            hrow[si.y + tau] = (v >> 3) - 4;
            if (orow && a.w.otrail) orow[si.y + tau] = a.w.otrail[at];
            s_ = v & 7;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 6; ++q) po[q] = 0.0f;
#pragma unroll
        for (int q = 0; q < 21; ++q) co[q] = 0.0f;
        a.out.chi2[seed] = 0.0f;
        a.out.score[seed] = -INFINITY;
        a.out.nfound[seed] = 0;
        a.out.nholes[seed] = 0;
    }
}

int resident_grid(const void* kernel, int n_sms, int threads = kThreads) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return n_sms * per_sm;
}

}  // namespace

namespace {

// Carves the work buffers out of one allocation (256-byte aligned pieces); with base == nullptr
// only the total size is computed.
size_t layout_build_work(char* base, int n_seeds, int max_plan_len, int word_bytes, bool with_ovl, BuildWork* w) {
    const size_t ns = (size_t)n_seeds, slots = ns * kGroup, wb = (size_t)word_bytes;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* r = base ? base + off : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return r;
    };
    BuildWork t;
    t.st[0] = reinterpret_cast<unsigned char*>(take(slots * kStateWords * wb));
    t.st[1] = reinterpret_cast<unsigned char*>(take(slots * kStateWords * wb));
    t.meta[0] = reinterpret_cast<int4*>(take(slots * 16));
    t.meta[1] = reinterpret_cast<int4*>(take(slots * 16));
    t.pr = reinterpret_cast<unsigned char*>(take(slots * kPredWords * wb));
    t.ls = reinterpret_cast<int4*>(take(slots * 80));
    t.live[0] = reinterpret_cast<int*>(take(slots * 4));
    t.live[1] = reinterpret_cast<int*>(take(slots * 4));
    t.seeds[0] = reinterpret_cast<int*>(take(ns * 4));
    t.seeds[1] = reinterpret_cast<int*>(take(ns * 4));
    t.sinfo = reinterpret_cast<int4*>(take(ns * 16));
    t.fin = reinterpret_cast<int*>(take(ns * 4));
    t.trail = reinterpret_cast<int*>(take(ns * (size_t)max_plan_len * kGroup * 4));
    t.otrail = with_ovl ? reinterpret_cast<int*>(take(ns * (size_t)max_plan_len * kGroup * 4)) : nullptr;
    t.rescue = reinterpret_cast<int*>(take(slots * 4));
    t.counts = reinterpret_cast<int*>(take(32 + 4 * kRoundCountInts));
    t.rcounts = base ? t.counts + 8 : nullptr;
    if (w) *w = t;
    return off;
}

// Start records of the backward search (Sec. 2.2): per track its state on its innermost found
// layer (p, c: 6 + 21 floats), the region from its eta as for a seed, and the first step of the
// geometry's reversed plan after that layer (info = (region, start, event, status); status 1
// when the layer is not in the plan or no layer lies inside it); the search order is the input
// order.
__global__ void __launch_bounds__(kThreads) k_bw_seed(const DevGeom* __restrict__ g, DevParams P, int n,
                                                      const float* __restrict__ p, const float* __restrict__ c,
                                                      const int* __restrict__ first_layer,
                                                      const int* __restrict__ event, float* state, int4* info,
                                                      int* order) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float* o = state + (int64_t)i * kSeedStateStride;
    const float* pi = p + 6 * (int64_t)i;
    const float* ci = c + 21 * (int64_t)i;
    o[0] = pi[0]; o[1] = pi[1]; o[2] = pi[2]; o[3] = 0.0f; o[4] = 0.0f; o[5] = 0.0f;
    o[6] = pi[3]; o[7] = pi[4]; o[8] = pi[5];
#pragma unroll
    for (int q = 0; q < 21; ++q) o[9 + q] = ci[q];
    o[30] = 0.0f; o[31] = 0.0f;
    const float eta = -logf(tanf(0.5f * pi[5]));
    int region = 0;
    if (g->n_regions > 1 && !(fabsf(eta) < P.barrel_eta_max)) region = eta > 0.0f ? 1 : 2;
    if (region >= g->n_regions) region = 0;
    int start = -1;
    const int pb = g->plan_off[region], len = g->plan_off[region + 1] - pb;
    for (int k = 0; k < len; ++k)   // g holds the reversed plans
        if (g->plan[pb + k] == first_layer[i]) start = k + 1;
    const bool ok = start > 0 && start < len;
    info[i] = make_int4(region, ok ? start : 0, event[i], ok ? 0 : 1);
    order[i] = i;
}

// Launch shapes of the round kernels (threads per block, minimum resident blocks per SM), one of
// which the autotuner picks: k_find x k_select.  The resident grid of each shape is computed once,
// before any capture.
template <class F, int TH, int MINB, bool BWD = false, bool MOD = false> struct FindShape {
    static int grid(int n_sms) {
        static int g = 0;
        if (!g) g = resident_grid((const void*)k_find<F, TH, MINB, BWD, MOD>, n_sms, TH);
        return g;
    }
    static void launch(cudaStream_t st, const BuildArgs& a, int tau, int n_sms) {
        k_find<F, TH, MINB, BWD, MOD><<<grid(n_sms), TH, 0, st>>>(a, tau);
    }
};
template <class F, int TH, int MINB, bool MOD = false> struct SelectShape {
    static int grid(int n_sms) {
        static int g = 0;
        if (!g) g = resident_grid((const void*)k_select<F, TH, MINB, MOD>, n_sms, TH);
        return g;
    }
    static void launch(cudaStream_t st, const BuildArgs& a, int tau, int n_sms) {
        k_select<F, TH, MINB, MOD><<<grid(n_sms), TH, 0, st>>>(a, tau);
    }
};

// The fused round kernel: dynamic shared memory set once per instantiation, resident grid.
template <class F, int TH, int MINB, bool BWD = false, bool MOD = false> struct RoundShape {
    static int grid(int n_sms) {
        static int g = 0;
        if (!g) {
            const void* k = (const void*)k_round<F, TH, MINB, BWD, MOD>;
            const size_t smem = round_smem_bytes<F, MOD>(TH);
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, TH, smem) != cudaSuccess || per_sm < 1)
                per_sm = 1;
            g = n_sms * per_sm;
        }
        return g;
    }
    static void launch(cudaStream_t st, const BuildArgs& a, int tau, int n_sms) {
        k_round<F, TH, MINB, BWD, MOD><<<grid(n_sms), TH, round_smem_bytes<F, MOD>(TH), st>>>(a, tau);
    }
};

template <class F, bool MOD> void prime_shapes_of(int n_sms) {
    RoundShape<F, 128, 4, false, MOD>::grid(n_sms);
    RoundShape<F, 128, 3, false, MOD>::grid(n_sms);
    RoundShape<F, 256, 2, false, MOD>::grid(n_sms);
    FindShape<F, 64, 8, false, MOD>::grid(n_sms);
    FindShape<F, 128, 1, false, MOD>::grid(n_sms);
    FindShape<F, 256, 1, false, MOD>::grid(n_sms);
    SelectShape<F, 64, 10, MOD>::grid(n_sms);
    SelectShape<F, 128, 5, MOD>::grid(n_sms);
    SelectShape<F, 256, 2, MOD>::grid(n_sms);
}

template <class F> void prime_shapes(int n_sms) {
    if (sizeof(F) == 4) {
        FindShape<float, 128, 1, true>::grid(n_sms);
        FindShape<float, 128, 1, true, true>::grid(n_sms);
        RoundShape<float, 128, 4, true>::grid(n_sms);
        RoundShape<float, 128, 4, true, true>::grid(n_sms);
    }
    prime_shapes_of<F, false>(n_sms);
    prime_shapes_of<F, true>(n_sms);
}

template <class F, bool BWD = false, bool MOD = false>
void launch_find(int shape, cudaStream_t st, const BuildArgs& a, int tau, int n_sms) {
    if constexpr (BWD) {   // the backward search: one shape, FP32 only
        FindShape<F, 128, 1, true, MOD>::launch(st, a, tau, n_sms);
        return;
    }
    switch (shape) {
        case 1: FindShape<F, 64, 8, false, MOD>::launch(st, a, tau, n_sms); break;
        case 2: FindShape<F, 256, 1, false, MOD>::launch(st, a, tau, n_sms); break;
        default: FindShape<F, 128, 1, false, MOD>::launch(st, a, tau, n_sms); break;
    }
}

// Fused round shapes: find_shape 3, 4, 5 = blocks of 128 x 4, 128 x 3, 256 x 2 (threads x resident
// blocks per SM); the backward search takes 128 x 4.
template <class F, bool BWD = false, bool MOD = false>
void launch_round(int shape, cudaStream_t st, const BuildArgs& a, int tau, int n_sms) {
    if constexpr (BWD) {
        RoundShape<F, 128, 4, true, MOD>::launch(st, a, tau, n_sms);
        return;
    }
    switch (shape) {
        case 4: RoundShape<F, 128, 3, false, MOD>::launch(st, a, tau, n_sms); break;
        case 5: RoundShape<F, 256, 2, false, MOD>::launch(st, a, tau, n_sms); break;
        default: RoundShape<F, 128, 4, false, MOD>::launch(st, a, tau, n_sms); break;
    }
}

template <class F, bool MOD = false>
void launch_select(int shape, cudaStream_t st, const BuildArgs& a, int tau, int n_sms) {
    switch (shape) {
        case 1: SelectShape<F, 64, 10, MOD>::launch(st, a, tau, n_sms); break;
        case 2: SelectShape<F, 256, 2, MOD>::launch(st, a, tau, n_sms); break;
        default: SelectShape<F, 128, 5, MOD>::launch(st, a, tau, n_sms); break;
    }
}

template <class F, bool BWD = false, bool MOD = false>
cudaError_t launch_rounds(cudaStream_t st, const BuildArgs& a, int n, int max_plan_len, int n_sms, int find_shape,
                          int select_shape) {
    cudaError_t e = cudaMemsetAsync(a.w.counts, 0, 32 + 4 * kRoundCountInts, st);
    if (e != cudaSuccess) return e;
    const int nb = (n + kThreads - 1) / kThreads;
    k_start<F><<<nb, kThreads, 0, st>>>(a);
    for (int tau = 0; tau < max_plan_len; ++tau) {
        if (a.fused) {
            launch_round<F, BWD, MOD>(find_shape, st, a, tau, n_sms);
        } else {
            launch_find<F, BWD, MOD>(find_shape, st, a, tau, n_sms);
            launch_select<F, MOD>(select_shape, st, a, tau, n_sms);
        }
        if (sizeof(F) == 4 && a.P.kappa_fp64 > 0.0f) k_rescue<<<n_sms, kThreads, 0, st>>>(a, tau);
    }
    k_finish<F><<<(n * kGroup + kThreads - 1) / kThreads, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t enqueue_rounds(cudaStream_t st, const BuildArgs& a, int n, int max_plan_len, int n_sms, int find_shape,
                           int select_shape, bool backward = false) {
    // module hits loaded (their overlap trail exists): the module-aware kernels
    const bool mod = a.w.otrail != nullptr;
    if (backward)
        return mod ? launch_rounds<float, true, true>(st, a, n, max_plan_len, n_sms, find_shape, select_shape)
                   : launch_rounds<float, true>(st, a, n, max_plan_len, n_sms, find_shape, select_shape);
    // MKGB_FP64: the plain all-FP64 comparison path (same rounds, every Kalman step in FP64)
    if (a.P.precision == MKGB_FP64)
        return mod ? launch_rounds<double, false, true>(st, a, n, max_plan_len, n_sms, find_shape, select_shape)
                   : launch_rounds<double>(st, a, n, max_plan_len, n_sms, find_shape, select_shape);
    return mod ? launch_rounds<float, false, true>(st, a, n, max_plan_len, n_sms, find_shape, select_shape)
               : launch_rounds<float>(st, a, n, max_plan_len, n_sms, find_shape, select_shape);
}

bool capturable(cudaStream_t st) {
    if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
    return cs == cudaStreamCaptureStatusNone;   // inside a caller's capture: plain launches join it
}

}  // namespace

size_t build_work_bytes(int n_seeds, int max_plan_len, int precision, bool with_ovl) {
    return layout_build_work(nullptr, n_seeds, max_plan_len, precision == MKGB_FP64 ? 8 : 4, with_ovl, nullptr);
}

BuildWork carve_build_work(void* base, int n_seeds, int max_plan_len, int precision, bool with_ovl) {
    BuildWork w;
    layout_build_work(static_cast<char*>(base), n_seeds, max_plan_len, precision == MKGB_FP64 ? 8 : 4, with_ovl,
                      &w);
    return w;
}

// The search of one call as a CUDA graph: the ~70 launches of the rounds (counters reset, k_start,
// per plan step k_find, k_select and k_rescue, k_finish) are captured once and replayed while the
// arguments, the launch shapes and the stream stay the same.
struct BuildGraph {
    cudaGraphExec_t exec = nullptr;
    BuildArgs key;
    int n = -1, max_plan = -1, find_shape = -1, select_shape = -1;
    cudaStream_t st = nullptr;
    bool disabled = false;
};

BuildGraph* build_graph_create() { return new BuildGraph(); }

void build_graph_destroy(BuildGraph* gph) {
    if (!gph) return;
    if (gph->exec) cudaGraphExecDestroy(gph->exec);
    delete gph;
}

cudaError_t launch_build(cudaStream_t st, const DevGeom* g, int max_plan_len, DevParams P, HitStore H, SeedStore S,
                         BuildOutDev out, BuildWork w, unsigned long long* counters, int n_sms, int find_shape,
                         int select_shape, BuildGraph* gph, bool backward) {
    if (S.n == 0) return cudaSuccess;
    BuildArgs a;
    memset(&a, 0, sizeof(a));   // padding included: the graph cache compares arguments bytewise
    a.geom = g; a.P = P; a.H = H; a.S = S; a.out = out; a.w = w; a.counters = counters; a.max_steps = max_plan_len;
    a.nfound0 = backward ? 0 : 3;
    a.fused = find_shape >= 3 ? 1 : 0;
    if (a.P.precision == MKGB_FP64)
        prime_shapes<double>(n_sms);
    else
        prime_shapes<float>(n_sms);
    if (backward) {   // plain launches (the search's graph cache serves the forward search)
        if (P.precision == MKGB_FP64) return cudaErrorInvalidValue;
        return enqueue_rounds(st, a, S.n, max_plan_len, n_sms, find_shape, select_shape, true);
    }
    if (!gph || gph->disabled || !capturable(st))
        return enqueue_rounds(st, a, S.n, max_plan_len, n_sms, find_shape, select_shape);
    const bool same = gph->exec && gph->st == st && gph->n == S.n && gph->max_plan == max_plan_len &&
                      gph->find_shape == find_shape && gph->select_shape == select_shape &&
                      memcmp(&gph->key, &a, sizeof(a)) == 0;
    if (!same) {
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            gph->disabled = true;
            return enqueue_rounds(st, a, S.n, max_plan_len, n_sms, find_shape, select_shape);
        }
        const cudaError_t le = enqueue_rounds(st, a, S.n, max_plan_len, n_sms, find_shape, select_shape);
        e = cudaStreamEndCapture(st, &graph);
        if (le != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return le;
        }
        if (e != cudaSuccess) return e;
        if (gph->exec) {
            cudaGraphExecDestroy(gph->exec);
            gph->exec = nullptr;
        }
        e = cudaGraphInstantiate(&gph->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            gph->exec = nullptr;
            return e;
        }
        gph->key = a;
        gph->st = st;
        gph->n = S.n;
        gph->max_plan = max_plan_len;
        gph->find_shape = find_shape;
        gph->select_shape = select_shape;
    }
    return cudaGraphLaunch(gph->exec, st);
}

cudaError_t launch_bw_seed(cudaStream_t st, const DevGeom* g, DevParams P, int n, const float* p, const float* c,
                           const int* first_layer, const int* event, float* state, int4* info, int* order) {
    if (n == 0) return cudaSuccess;
    k_bw_seed<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(g, P, n, p, c, first_layer, event, state, info,
                                                                  order);
    return cudaGetLastError();
}

}  // namespace mk
