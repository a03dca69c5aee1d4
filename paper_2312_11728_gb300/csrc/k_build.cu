// Combinatorial forward search (Sec. 2.2), one persistent fused kernel.
//
// Work unit: a group of 8 lanes owns one seed and holds its (at most 8) candidates, one
// per lane, in registers for the whole layer plan; a warp serves 4 seeds at a time and
// takes the next 4 from a global atomic work counter, in the (event, eta, phi) order of
// the seeds so that neighbouring warps read neighbouring hit bins.  Per plan step:
//   1. each live candidate propagates to the step's layer with Jacobian, transport and
//      material (a4-a7);
//   2. it scans the eta-phi bins overlapping its window, tests each hit against the
//      window and computes the 3D chi2 of the hits inside (a8-a9), keeping its best
//      hit children in a sorted register list;
//   3. the group merges its lanes' children into the N best of the seed with 64-bit
//      (score, parent slot) keys reduced by warp shuffles (a10);
//   4. lane r takes the r-th child: pulls the parent's predicted state by shuffles and
//      applies the Joseph update with the child's hit (a11);
//   5. (parent slot, hit) of every kept child goes to a shared-memory trail, walked back
//      at the end for the best candidate's hit list (a13).
// No global state is read or written between layers: per seed, the only HBM traffic is
// the hit bins it scans, the seed state in and the result out.  There are no waits on
// other warps or CTAs; every loop is bounded by the plan length, the window's bin range
// or a fixed Newton iteration limit.
#include "internal.h"

namespace mk {

namespace {

constexpr int kGroup = 8;                  // lanes per seed (>= MKGB_MAX_CANDS)
constexpr int kWarps = 4;                  // warps per CTA
constexpr int kThreads = kWarps * 32;
constexpr float kBig = 3.0e38f;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long order_key(float score, int slot) {
    unsigned u = __float_as_uint(score);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | (unsigned)(kGroup - 1 - slot);
}

__device__ __forceinline__ float shfl_f(float v, int src) { return __shfl_sync(kFull, v, src); }
__device__ __forceinline__ int shfl_i(int v, int src) { return __shfl_sync(kFull, v, src); }

struct BuildArgs {
    const DevGeom* geom;
    DevParams P;
    HitStore H;
    SeedStore S;
    BuildOutDev out;
    int* queue;
    unsigned long long* counters;
    int max_steps;   // longest plan (trail rows)
};

__global__ void __launch_bounds__(kThreads) k_build(BuildArgs a) {
    __shared__ DevGeom g;
    extern __shared__ int trail_smem[];
    {
        const int4* src = reinterpret_cast<const int4*>(a.geom);
        int4* dst = reinterpret_cast<int4*>(&g);
        for (int i = threadIdx.x; i < (int)(sizeof(DevGeom) / 16); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane >> 3, slot = lane & 7, gbase = grp << 3;
    int* trail = trail_smem + (warp * 4 + grp) * a.max_steps * kGroup;
    const DevParams& P = a.P;
    unsigned long long c_steps = 0, c_chi2 = 0, c_upd = 0, c_tested = 0;
    int c_newton = 0;

    for (;;) {
        __syncwarp();
        int base = 0;
        if (lane == 0) base = atomicAdd(a.queue, 4);
        base = shfl_i(base, 0);
        if (base >= a.S.n) break;
        const int sidx = base + grp;
        int seed = -1, plan_base = 0, start = 0, event = 0, nsteps = 0;
        if (sidx < a.S.n) {
            seed = a.S.order[sidx];
            const int4 inf = a.S.info[seed];
            if (inf.w == 0) {
                plan_base = g.plan_off[inf.x];
                start = inf.y;
                event = inf.z;
                nsteps = g.plan_off[inf.x + 1] - plan_base - start;
                if (nsteps < 0) nsteps = 0;
            }
        }
        const int nsteps_w = __reduce_max_sync(kFull, nsteps);

        State t;
        float score = 0.0f, chi2s = 0.0f;
        int nfound = 3, nholes = 0;
        bool stopped = false;
        bool alive = seed >= 0 && nsteps > 0 && slot == 0;
        {
            const float* o = a.S.state + (int64_t)(seed >= 0 ? seed : 0) * kSeedStateStride;
            t.xh = o[0]; t.yh = o[1]; t.zh = o[2]; t.xl = o[3]; t.yl = o[4]; t.zl = o[5];
            t.k = o[6]; t.phi = o[7]; t.th = o[8];
#pragma unroll
            for (int q = 0; q < 21; ++q) t.c[q] = o[9 + q];
        }

        for (int tau = 0; tau < nsteps_w; ++tau) {
            const bool gact = tau < nsteps;
            const int layer = gact ? g.plan[plan_base + start + tau] : 0;
            const DevLayer& L = g.layers[layer];

            // ---- 1. propagation (a4-a7)
            int nh_kind = K_NONE;
            float nh_score = -kBig;
            bool crossed = false;
            Pred q;
            float dir[4];
            if (gact && alive) {
                if (stopped) {
                    nh_kind = K_CARRY;
                    nh_score = score;
                } else {
                    const int r = propagate(L, g.cB, P.material, t, q, c_newton, dir);
                    if (r < 0) {
                        alive = false;
                    } else if (r == 0) {
                        nh_kind = K_SKIP;
                        nh_score = score;
                    } else {
                        crossed = true;
                        ++c_steps;
                        if (nholes < P.max_holes) {
                            nh_kind = K_MISS;
                            nh_score = score - P.score_hole;
                        } else {
                            nh_kind = K_STOP;
                            nh_score = score;
                        }
                    }
                }
            }

            // ---- 2. window and chi2 of the hits inside (a8-a9); sorted list (chi2 asc, id asc)
            float lx[kGroup];
            int lid[kGroup], lq[kGroup];
#pragma unroll
            for (int j = 0; j < kGroup; ++j) {
                lx[j] = kBig;
                lid[j] = 0x7fffffff;
                lq[j] = 0;
            }
            if (crossed) {
                const FrameT<float> fr = frame_of(L.kind, q.xh, q.yh, dir[0], dir[1], dir[2], dir[3]);
                const Window w = window(L, P, q, fr);
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
                const int64_t bb = (int64_t)event * g.bins_per_event + L.bin_base;
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
                            if (fabsf(ep.x - w.eta) <= w.deta && fabsf(wrap_pi(ep.y - w.phi)) <= w.dphi) {
                                ++c_chi2;
                                float m[3], v[6];
                                int id;
                                load_hit(a.H.hb_pay, hq, m, v, &id);
                                float x2;
                                if (chi2_hit(fr, q, m[0], m[1], m[2], v, x2) && x2 < P.chi2_cut) {
                                    int qq = hq;
#pragma unroll
                                    for (int j = 0; j < kGroup; ++j) {
                                        const bool better = x2 < lx[j] || (x2 == lx[j] && id < lid[j]);
                                        const float tx = lx[j];
                                        const int ti = lid[j], tq = lq[j];
                                        if (better) {
                                            lx[j] = x2;
                                            lid[j] = id;
                                            lq[j] = qq;
                                            x2 = tx;
                                            id = ti;
                                            qq = tq;
                                        }
                                    }
                                }
                            }
                        }
                    }
                }
            }

            // ---- 3. the N best children of the seed (a10)
            bool nh_avail = nh_kind != K_NONE;
            int my_parent = -1, my_kind = K_NONE, my_id = -1, my_q = 0;
            float my_x2 = 0.0f, my_score = 0.0f;
            for (int r = 0; r < P.max_cands; ++r) {
                const bool has_hit = lx[0] < kBig;
                const float hit_score = score + P.score_hit - lx[0];
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
                const int w_id = shfl_i(lid[0], src);
                const int w_q = shfl_i(lq[0], src);
                const float w_x2 = shfl_f(lx[0], src);
                const float w_score = shfl_f(hs, src);
                if (valid && slot == r) {
                    my_parent = wslot;
                    my_kind = w_kind;
                    my_id = w_id;
                    my_q = w_q;
                    my_x2 = w_x2;
                    my_score = w_score;
                }
                if (valid && slot == wslot) {
                    if (hk == K_HIT) {
#pragma unroll
                        for (int j = 0; j < kGroup - 1; ++j) {
                            lx[j] = lx[j + 1];
                            lid[j] = lid[j + 1];
                            lq[j] = lq[j + 1];
                        }
                        lx[kGroup - 1] = kBig;
                    } else {
                        nh_avail = false;
                    }
                }
            }

            // ---- 4. pull the parent's state and update (a11); 5. trail
            // Payload of a lane: its predicted state (surface frame) if it crossed, else its state.
            float R[30];
            R[0] = crossed ? q.xh : t.xh; R[1] = crossed ? q.yh : t.yh; R[2] = crossed ? q.zh : t.zh;
            R[3] = crossed ? q.xl : t.xl; R[4] = crossed ? q.yl : t.yl; R[5] = crossed ? q.zl : t.zl;
            R[6] = crossed ? q.k : t.k; R[7] = crossed ? q.phi : t.phi; R[8] = crossed ? q.th : t.th;
#pragma unroll
            for (int i = 0; i < 15; ++i) R[9 + i] = crossed ? q.c[i] : t.c[i];
#pragma unroll
            for (int i = 15; i < 21; ++i) R[9 + i] = t.c[i];
            const int psrc = gbase + (my_parent >= 0 ? my_parent : slot);
#pragma unroll
            for (int i = 0; i < 30; ++i) R[i] = shfl_f(R[i], psrc);
            const float p_chi2 = shfl_f(chi2s, psrc);
            const int p_nfound = shfl_i(nfound, psrc);
            const int p_nholes = shfl_i(nholes, psrc);
            const int p_stopped = shfl_i((int)stopped, psrc);
            if (gact) {
                if (my_kind != K_NONE) {
                    chi2s = p_chi2;
                    nfound = p_nfound;
                    nholes = p_nholes;
                    stopped = p_stopped != 0;
                    score = my_score;
                    alive = true;
                    int code = MKGB_HIT_STOP;
                    if (my_kind == K_SKIP || my_kind == K_CARRY) {
                        t.xh = R[0]; t.yh = R[1]; t.zh = R[2]; t.xl = R[3]; t.yl = R[4]; t.zl = R[5];
                        t.k = R[6]; t.phi = R[7]; t.th = R[8];
#pragma unroll
                        for (int i = 0; i < 21; ++i) t.c[i] = R[9 + i];
                        if (my_kind == K_SKIP) code = MKGB_HIT_SKIP;
                    } else {
                        Pred pq;
                        pq.xh = R[0]; pq.yh = R[1]; pq.zh = R[2]; pq.xl = R[3]; pq.yl = R[4]; pq.zl = R[5];
                        pq.k = R[6]; pq.phi = R[7]; pq.th = R[8];
#pragma unroll
                        for (int i = 0; i < 15; ++i) pq.c[i] = R[9 + i];
                        if (my_kind == K_HIT) {
                            float m[3], v[6];
                            load_hit(a.H.hb_pay, my_q, m, v, nullptr);
                            if (kalman_update(L.kind, pq, m[0], m[1], m[2], v, t)) {
                                chi2s += my_x2;
                                ++nfound;
                                ++c_upd;
                                code = my_id;
                            } else {
                                alive = false;
                            }
                        } else {
                            pred_to_state(L.kind, pq, t);
                            if (my_kind == K_MISS) {
                                ++nholes;
                                code = MKGB_HIT_MISS;
                            } else {   // K_STOP
                                stopped = true;
                            }
                        }
                    }
                    trail[tau * kGroup + slot] = ((code + 4) << 3) | my_parent;
                } else {
                    alive = false;
                }
            }
        }

        // ---- best candidate and its hit list (a13)
        __syncwarp();
        const unsigned am = __ballot_sync(kFull, alive);
        const unsigned gm = (am >> gbase) & 0xffu;
        const int best_slot = gm ? __ffs(gm) - 1 : -1;
        if (seed >= 0) {
            int* hrow = a.out.hits + (int64_t)seed * a.out.max_plan;
            if (slot == 0) {
                for (int q = 0; q < a.out.max_plan; ++q) hrow[q] = MKGB_HIT_PRE;
            }
            __syncwarp(0xffu << gbase);
            if (slot == (best_slot >= 0 ? best_slot : 0)) {
                float* po = a.out.params + 6 * (int64_t)seed;
                float* co = a.out.cov + 21 * (int64_t)seed;
                if (best_slot >= 0) {
                    store_state6(t, po, co);
                    a.out.chi2[seed] = chi2s;
                    a.out.score[seed] = score;
                    a.out.nfound[seed] = nfound;
                    a.out.nholes[seed] = nholes;
                    int s_ = best_slot;
                    for (int tau = nsteps - 1; tau >= 0; --tau) {
                        const int v = trail[tau * kGroup + s_];
                        hrow[start + tau] = (v >> 3) - 4;
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
        }
    }
    // ---- counters
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        c_steps += __shfl_xor_sync(kFull, c_steps, off);
        c_chi2 += __shfl_xor_sync(kFull, c_chi2, off);
        c_upd += __shfl_xor_sync(kFull, c_upd, off);
        c_tested += __shfl_xor_sync(kFull, c_tested, off);
        c_newton += __shfl_xor_sync(kFull, c_newton, off);
    }
    if (lane == 0) {
        atomicAdd(a.counters + 0, c_steps);
        atomicAdd(a.counters + 1, c_chi2);
        atomicAdd(a.counters + 2, c_upd);
        atomicAdd(a.counters + 3, c_tested);
        atomicAdd(a.counters + 4, (unsigned long long)c_newton);
    }
}

}  // namespace

cudaError_t launch_build(cudaStream_t st, const DevGeom* g, int max_plan_len, DevParams P, HitStore H, SeedStore S,
                         BuildOutDev out, int* queue, unsigned long long* counters, int n_sms) {
    if (S.n == 0) return cudaSuccess;
    BuildArgs a{g, P, H, S, out, queue, counters, max_plan_len};
    const size_t smem = (size_t)kWarps * 4 * max_plan_len * kGroup * sizeof(int);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int64_t want = ((int64_t)S.n + 4 * kWarps - 1) / (4 * kWarps);
    int64_t grid = (int64_t)n_sms * per_sm;
    if (grid > want) grid = want;
    k_build<<<(unsigned)grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mk
