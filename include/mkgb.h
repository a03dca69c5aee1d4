/* mkgb — batched Kalman track building and fitting on one GB300 (sm_103a).
 *
 * C ABI of libmkgb.so.  The calls follow the paper's statement of the problem
 * (arXiv:2312.11728): a detector geometry with material, set up once (Sec. 3.1);
 * hits aggregated per layer (Sec. 3.1); seeds with parameters at their outermost
 * hit (Sec. 2.2); iteration parameters (Sec. 3.2, IterationParams and
 * IterationLayerConfig); a combinatorial forward search returning the
 * best-scoring candidate per seed (Sec. 2.2, forward search); and a plain Kalman
 * fit over a known hit assignment (Sec. 4, final fit).
 *
 * Conventions
 *  - Units: cm, GeV, tesla, radians.  Track state p = (x, y, z, q/pT, phi, theta),
 *    phi in (-pi, pi], theta in (0, pi).  Covariances are packed lower triangles:
 *    index(i, j) = i(i+1)/2 + j for i >= j (21 floats for the state, 6 for a hit
 *    in the order xx, yx, yy, zx, zy, zz).
 *  - Every call returns MKGB_OK (0) or a negative code; mkgb_last_error() gives
 *    the message.  No call keeps a pointer it was given after it returns.
 *  - The caller owns every array it passes.  `on_device` = 1: array arguments
 *    are device pointers (e.g. torch CUDA tensors) and the call is asynchronous
 *    on the context's stream; 0: host pointers, copied in and out, and the call
 *    returns after its outputs are written.
 *  - All state lives in the context (the paper's rule of no non-constant global
 *    state, Sec. 3): contexts are independent; one context is not thread-safe.
 */
#ifndef MKGB_H
#define MKGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MKGB_OK 0
#define MKGB_EINVAL (-1)   /* bad argument or size */
#define MKGB_ENOMEM (-2)   /* device allocation failed */
#define MKGB_ECUDA (-3)    /* a CUDA call failed */
#define MKGB_ESTATE (-5)   /* call out of order (no geometry, no hits, no seeds) */

#define MKGB_BARREL 0
#define MKGB_DISK 1

#define MKGB_MAX_LAYERS 64
#define MKGB_MAX_REGIONS 8
#define MKGB_MAX_PLAN 48       /* layers in one layer plan */
#define MKGB_MAX_CANDS 8       /* candidates kept per seed */

/* hit codes per plan step in mkgb_tracks.hits */
#define MKGB_HIT_MISS (-1)     /* layer crossed, no hit taken (a hole) */
#define MKGB_HIT_SKIP (-2)     /* layer not crossed */
#define MKGB_HIT_STOP (-3)     /* candidate had reached the hole limit */
#define MKGB_HIT_PRE (-4)      /* plan step before the search (seed layers) or after the plan */

typedef struct mkgb_ctx mkgb_ctx;

/* A layer: an r-z bounding box in cylindrical space that aggregates hits (Sec. 3.1). */
typedef struct {
    int32_t kind;          /* MKGB_BARREL: cylinder of radius pos; MKGB_DISK: plane z = pos */
    float pos;             /* radius or z [cm] */
    float lo, hi;          /* barrel: z extent; disk: r extent [cm] */
    float x_over_x0;       /* thickness at normal incidence in radiation lengths (Sec. 3.1 material) */
    float sig_local[3];    /* hit resolution along (r-hat, phi-hat, z-hat) [cm], used for the window */
    int32_t n_eta_bins;    /* eta-phi index of the layer's hits (Sec. 2.2: eta-phi sorting for coherency) */
    int32_t n_phi_bins;
    float eta_lo, eta_hi;  /* eta range covered by the bins (hits outside go to the edge bins) */
} mkgb_layer;

/* Search parameters (Sec. 3.2: maximum missed layers, chi2 cut, hit-search parameters). */
typedef struct {
    float chi2_cut;        /* accept a hit if its predicted chi2 < chi2_cut */
    int32_t max_cands;     /* N: candidates kept per seed, 1..MKGB_MAX_CANDS */
    int32_t max_holes;     /* missed layers allowed per candidate */
    float win_nsigma;      /* window half-width = n_sigma * sigma(eta or phi) ... */
    float deta_min, deta_max, dphi_min, dphi_max;   /* ... clamped to [min, max] */
    float score_hit;       /* candidate score = score_hit * n_found - score_hole * n_holes - sum chi2 */
    float score_hole;
    float barrel_eta_max;  /* region choice with >1 plan: |eta_seed| < this -> plan 0, else 1 (eta>0) / 2 */
    int32_t material;      /* 1: multiple scattering and energy loss at every crossed layer */
    int32_t precision;     /* MKGB_FP32: Kalman steps of the search and the fit in FP32 (seed fits with
                              FP32 trajectories and FP64 covariance transport and updates, and all in
                              FP64 for seeds with |q/pT| < 0.03 /GeV);
                              MKGB_FP64: every step in FP64 (the plain comparison path) */
    float kappa_fp64;      /* an update whose innovation covariance S has a condition estimate above this
                              is redone in FP64: the search redoes that update, the fit refits the whole
                              track; 0 = never (both only in the FP32 precision) */
    float fit_outlier_chi2;/* fits over a known assignment (mkgb_fit, mkgb_fit_static, mkgb_fit_backward;
                              the final fit's outlier rejection, Sec. 2.2): a listed hit whose predicted chi2
                              exceeds this is not used (the layer is crossed, the state is not updated);
                              0 = every listed hit is used.  mkgb_fit_grad ignores it */
    float score_overlap;   /* search on modular layers (mkgb_load_modules): score added to a child that picks
                              up an overlap hit (Sec. 2.2: a single additional detector-overlap hit) */
} mkgb_params;

#define MKGB_FP32 0
#define MKGB_FP64 2

/* Output of mkgb_build: caller-allocated arrays (device or host per on_device). */
typedef struct {
    float* params;         /* n_seeds x 6: best candidate's state at its last layer */
    float* cov;            /* n_seeds x 21 */
    float* chi2;           /* n_seeds: sum of chi2 of the hits added by the search */
    float* score;          /* n_seeds: -inf if the seed failed */
    int32_t* nfound;       /* n_seeds: hits including the 3 seed hits */
    int32_t* nholes;       /* n_seeds */
    int32_t* hits;         /* n_seeds x max_plan: global hit index or MKGB_HIT_* per plan step */
    int32_t max_plan;      /* row stride of hits, >= the longest plan */
    int32_t* ovl_hits;     /* n_seeds x max_plan (NULL to skip): overlap hit index per plan step, -1 none */
} mkgb_tracks;

/* Creates a context on `device` that launches on `stream` (a cudaStream_t, including
 * cudaStreamLegacy or cudaStreamPerThread; NULL = a non-blocking stream the context creates).
 * Errors: MKGB_EINVAL (out == NULL), MKGB_ECUDA. */
int mkgb_create(mkgb_ctx** out, int device, void* stream);
void mkgb_destroy(mkgb_ctx* ctx);
/* Message of the last failing call on this context (static text for a NULL context). */
const char* mkgb_last_error(const mkgb_ctx* ctx);
/* Version string of the library build. */
const char* mkgb_version(void);

/* Detector geometry and layer plans (Sec. 3.1: layers, layer plans per tracking region,
 * material).  `plan` holds n_regions plans back to back, plan_off[r]..plan_off[r+1].
 * Host arrays.  Errors: MKGB_EINVAL on sizes beyond the MKGB_MAX_* limits, bad kinds,
 * plan entries out of range or empty extents. */
int mkgb_load_geometry(mkgb_ctx* ctx, const mkgb_layer* layers, int n_layers,
                       const int32_t* plan, const int32_t* plan_off, int n_regions, float bz_tesla);

/* Flat detector modules (Sec. 3.1: module position, normal and phi-direction vectors; the Phase-2
 * tilted modules and the overlap hits of neighbouring modules).  Module m lies on layer[m] and is
 * the plane through pos[3m..3m+2] [cm] with unit normal normal[3m..3m+2]; its phi-direction lies in
 * the plane and enters through the hit covariances, which carry the module's measurement axes.  A
 * layer with at least one module is modular: its hits lie on module planes, and its own cylinder
 * or disk stays the reference surface of the window, the material and the eta-phi bins.  The search
 * and mkgb_fit move a candidate from that surface to the plane of each module hit (the helix to
 * the plane, its Jacobian and the covariance transport; no material) before the chi2 and update.
 * Host arrays; n_modules = 0 removes the modules.  Loaded hits are dropped (load them again with
 * mkgb_load_hits_modular).  Errors: MKGB_ESTATE before mkgb_load_geometry; MKGB_EINVAL for a layer
 * out of range, a normal that is not a unit vector (|n|^2 off 1 by 1e-4 or more) or a NaN position. */
int mkgb_load_modules(mkgb_ctx* ctx, int n_modules, const int32_t* layer, const float* pos, const float* normal);

/* Iteration parameters (Sec. 3.2).  Host struct.  Errors: MKGB_EINVAL if max_cands is outside
 * 1..MKGB_MAX_CANDS, max_holes < 0 or a window bound is negative. */
int mkgb_set_params(mkgb_ctx* ctx, const mkgb_params* params);

/* Hits of n_events events, grouped by (event, layer): segment e*n_layers + l holds hits
 * seg_off[e*n_layers + l] .. seg_off[e*n_layers + l + 1] - 1 (host array, n_events*n_layers+1
 * entries, non-decreasing, seg_off[0] = 0).  xyz: n x 3, cov6: n x 6 (n = seg_off[last]).
 * The library builds each segment's eta-phi bin index (counting sort).  Hit indices used by
 * mkgb_seed, mkgb_build and mkgb_fit are positions in these arrays.
 * Errors: MKGB_ESTATE without geometry, MKGB_EINVAL on bad offsets, MKGB_ENOMEM. */
int mkgb_load_hits(mkgb_ctx* ctx, int n_events, const int64_t* seg_off,
                   const float* xyz, const float* cov6, int on_device);

/* mkgb_load_hits with the module of every hit: hit_module (n ints, host or device per on_device)
 * gives the module index of each hit on a modular layer and -1 for every other hit.  The search
 * then tests and updates module hits on their planes and picks up overlap hits (mkgb_build,
 * mkgb_tracks.ovl_hits: with the best accepted module hit b1 of a candidate's window and the best
 * one b2 on a module other than b1's, a child taking module hit h also takes b1 if h is not on b1's
 * module, else b2, and scores params.score_overlap more; its update uses h only).  mkgb_seed
 * uses a seed hit on a module on its module's plane (the seed's state is then the one on hit 3's
 * plane; status 1 if a plane is not reached).  mkgb_fit and
 * mkgb_fit_backward use module hits on their planes (status 1 if a plane is not reached within
 * 10 cm, or only at grazing incidence; the backward fit's start state is taken on the plane of its
 * last hit's module); mkgb_build_backward tests and picks up module hits as mkgb_build does (its
 * out->ovl_hits likewise); mkgb_fit_grad uses them on their planes as mkgb_fit (the alignment
 * moves the hits, the module planes stay nominal).  Synchronises the
 * stream (the module ids are checked on the device).  Errors: those of mkgb_load_hits; MKGB_ESTATE
 * without modules; MKGB_EINVAL for a NULL hit_module or a hit whose module does not fit its layer. */
int mkgb_load_hits_modular(mkgb_ctx* ctx, int n_events, const int64_t* seg_off, const float* xyz,
                           const float* cov6, const int32_t* hit_module, int on_device);

/* Seeds (Sec. 2.2): n_seeds x 3 hit indices on three consecutive crossed layers of one event,
 * innermost first.  Computes each seed's state at its third hit (circle estimate + 3-hit
 * Kalman fit; precision as params.precision states), its region and first search step, and
 * orders seeds by (event, eta, phi) for hit-access coherency.  Optional outputs (NULL to skip): state n x 6, cov n x 21, info n x 3
 * (region, first plan step, status 0 = ok).  Errors: MKGB_ESTATE without hits, MKGB_EINVAL. */
int mkgb_seed(mkgb_ctx* ctx, int n_seeds, const int32_t* seed_hits, int on_device,
              float* state_out, float* cov_out, int32_t* info_out);

/* Combinatorial forward search (Sec. 2.2) for the seeds of the last mkgb_seed call: along the
 * seed's layer plan, every candidate is propagated, hits in its eta-phi window get a chi2, the
 * N best children per seed are kept and updated; the best candidate is returned with its hit
 * list.  Errors: MKGB_ESTATE without seeds or params, MKGB_EINVAL on a short max_plan or with
 * 2^28 - 8 or more hits loaded (the hit trail packs hit indices in 28 bits). */
int mkgb_build(mkgb_ctx* ctx, const mkgb_tracks* out, int on_device);

/* Combinatorial backward search (Sec. 2.2: when the seeding region does not reach the vertex
 * region, a backward search inwards from the first known hit).  n tracks, each with its event
 * (track_event[i], an event of the loaded hits), its innermost found layer (first_layer[i]) and
 * its state on that layer (p_start n x 6, c_start n x 21: the backward fit's output there,
 * mkgb_fit_backward).  The region comes from the state's eta as for a seed; the search runs
 * through that region's plan in reverse order (inner layers last), from the step after
 * first_layer, with the crossing behind each candidate (negative path length, the energy loss
 * added back) and otherwise the forward search's rules (windows, chi2 cut, best-N, holes),
 * from score 0 and no hits.  out: as mkgb_build, one row per track, out->hits indexed by the
 * steps of the reversed plan (MKGB_HIT_PRE before the first searched step); nfound counts the
 * hits found by this search.  A track whose first_layer is not in its region's plan, or is its
 * innermost layer, gets score -inf.  FP32 (with the FP64 redo of ill-conditioned updates);
 * MKGB_EINVAL under precision MKGB_FP64.  Errors: MKGB_ESTATE without geometry, params or hits;
 * MKGB_EINVAL for a negative size, NULL arrays, max_plan short of the longest plan, or (host
 * arrays) an event or layer index out of range. */
int mkgb_build_backward(mkgb_ctx* ctx, int n, const int32_t* track_event, const int32_t* first_layer,
                        const float* p_start, const float* c_start, const mkgb_tracks* out, int on_device);

/* Seed cleaning (Sec. 2.2: seeds are processed in parallel, so hits consumed by earlier tracks
 * cannot be masked).  seed_hits: n x 3 global hit ids of the loaded hits.  keep_out[i] = 0 if
 * seed i shares at least two of its three hits with a seed of lower index, else 1 (each seed is
 * judged against all others, not transitively; the index order stands for the order sequential
 * processing would use).  Errors: MKGB_ESTATE before mkgb_load_hits; MKGB_EINVAL for n < 0, NULL
 * arrays or (host arrays) a hit id beyond the loaded hits; device arrays: such ids are not hits. */
int mkgb_clean_seeds(mkgb_ctx* ctx, int n, const int32_t* seed_hits, int32_t* keep_out, int on_device);

/* Quality filter and duplicate removal on found tracks (Sec. 2.2).  hits: n x width global hit
 * ids per track (< 0: none; e.g. the seed hits followed by mkgb_tracks.hits), score: n.  keep_out
 * [i] = 0 if track i has fewer than min_hits hits, or if a better track (higher score; equal score
 * and lower index) shares at least frac x min(hits of the two) hits with it (each track judged
 * against all others, not transitively), else 1.  Errors: MKGB_ESTATE before mkgb_load_hits;
 * MKGB_EINVAL for n < 0, width < 1, frac outside (0, 1], NULL arrays or (host arrays) a hit id
 * beyond the loaded hits. */
int mkgb_remove_duplicates(mkgb_ctx* ctx, int n, int width, const int32_t* hits, const float* score,
                           int min_hits, float frac, int32_t* keep_out, int on_device);

/* Kalman fit over a known assignment (Sec. 4): n tracks, each from p0/c0 through up to
 * max_steps layers (layers[i*max_steps + j], -1 ends the list) taking hits[i*max_steps + j]
 * (-1: propagate only).  Outputs: p_out n x 6, c_out n x 21, chi2_out (sum of predicted chi2),
 * status_out (0 ok, 1 a listed layer was not crossed, 2 particle stopped, 3 update failed,
 * 4 hit index outside the loaded hits; tracks above params.kappa_fp64 are refit in FP64;
 * NULL to skip).  Errors: MKGB_ESTATE without geometry/params, MKGB_EINVAL. */
int mkgb_fit(mkgb_ctx* ctx, int n, int max_steps, const int32_t* layers, const int32_t* hits,
             const float* p0, const float* c0, float* p_out, float* c_out, float* chi2_out,
             int32_t* status_out, int on_device);

/* Backward fit (Sec. 2.2: each found track re-traversed backwards, refitting its parameters).
 * n tracks listed as for mkgb_fit, in the forward (outward) order: layers[i*max_steps + j] (-1
 * ends the list), hits[i*max_steps + j] (-1: no hit on that layer).  p_start (n x 6) and
 * c_start (n x 21) give each track's state on its LAST listed layer (the forward fit's output
 * there); the covariance is multiplied by cov_scale (> 0; 100 releases the forward fit's
 * information) before the fit.  The track is then fitted from the last listed layer to the
 * first: the hit on the last layer is used first (global-frame update, the state lies on that
 * layer), then for each earlier layer the inward crossing along the reversed trajectory (the
 * mean energy loss in each crossed layer's material is added back; the scattering variance is
 * added as forward), chi2 and the update.  Outputs: p_out, c_out (n x 6, n x 21): the state on
 * the FIRST listed layer describing the segment inside that layer (its material included);
 * chi2_out (n): the sum of the predicted chi2 of the backward updates; status_out (n, may be
 * NULL): 0 ok, 1 a listed layer not crossed inwards, 2 stopped, 3 update failed, 4 hit index
 * beyond the loaded hits.  Tracks whose largest kappa(S) exceeds params.kappa_fp64 are refit in
 * FP64; precision = MKGB_FP64 fits all tracks in FP64.  mkgb_counters kind 1 reports the call.
 * Errors: MKGB_ESTATE without geometry/params (or hits, when a hit is listed), MKGB_EINVAL for
 * a negative size, a NULL array, cov_scale <= 0 or a hit index beyond the loaded hits (host
 * arrays). */
int mkgb_fit_backward(mkgb_ctx* ctx, int n, int max_steps, const int32_t* layers, const int32_t* hits,
                      const float* p_start, const float* c_start, float cov_scale, float* p_out,
                      float* c_out, float* chi2_out, int32_t* status_out, int on_device);

/* One pass of the hot path in one call (Sec. 2.2 search and Sec. 4 fit on one batch of events):
 * mkgb_load_hits, mkgb_seed (no optional outputs), mkgb_build and mkgb_fit with the same
 * arguments as those calls, every array a device pointer (their on_device = 1 rules).  Inside,
 * the fit runs on a second stream beside the seed fit and the search (it needs the prepared hits
 * only); the context's stream waits for it, so all outputs are complete when the context's
 * stream passes the call.  Errors: those of the four calls (the first failing one is returned;
 * the work already enqueued stays enqueued). */
int mkgb_run(mkgb_ctx* ctx, int n_events, const int64_t* seg_off, const float* xyz, const float* cov6,
             int n_seeds, const int32_t* seed_hits, const mkgb_tracks* out, int n_fit, int max_steps,
             const int32_t* layers, const int32_t* hits, const float* p0, const float* c0, float* p_out,
             float* c_out, float* chi2_out, int32_t* status_out);

/* mkgb_run with every array in host memory (the call a host program makes with its event data):
 * the same arguments, inputs and outputs as mkgb_run, and the same results bit for bit.  The
 * library copies the inputs to the device and the outputs back, overlapping the copies with the
 * kernels: the hits travel in up to 8 chunks of whole events (each chunk's hits are prepared as
 * soon as it has arrived), the seeds and the fit's inputs follow while the seeds are fitted, the
 * fit's outputs return while the search runs and the search's outputs at the end.  The overlap
 * needs page-locked host arrays (cudaHostAlloc / cudaHostRegister); pageable arrays give the
 * same results with the copies serialised.  The call returns when every output is in host
 * memory (it synchronises the context's stream); device copies of the inputs and outputs are
 * kept in one library buffer, reused by the next call.  Hit indices are checked on the device as
 * in mkgb_run (a seed or fitted track with a hit index beyond the loaded hits gets a failure
 * status instead of an error code).  Errors: MKGB_EINVAL for a NULL array with a nonzero size,
 * negative sizes or bad seg_off, and those of mkgb_run. */
int mkgb_run_host(mkgb_ctx* ctx, int n_events, const int64_t* seg_off, const float* xyz, const float* cov6,
                  int n_seeds, const int32_t* seed_hits, const mkgb_tracks* out, int n_fit, int max_steps,
                  const int32_t* layers, const int32_t* hits, const float* p0, const float* c0, float* p_out,
                  float* c_out, float* chi2_out, int32_t* status_out);

/* mkgb_run for modular layers: the hits loaded with mkgb_load_hits_modular (hit_module, a device
 * array of n ints, its module per hit), then mkgb_seed, mkgb_build (out->ovl_hits as there) and
 * mkgb_fit as in mkgb_run.  Errors: those of mkgb_run and mkgb_load_hits_modular. */
int mkgb_run_modular(mkgb_ctx* ctx, int n_events, const int64_t* seg_off, const float* xyz, const float* cov6,
                     const int32_t* hit_module, int n_seeds, const int32_t* seed_hits, const mkgb_tracks* out,
                     int n_fit, int max_steps, const int32_t* layers, const int32_t* hits, const float* p0,
                     const float* c0, float* p_out, float* c_out, float* chi2_out, int32_t* status_out);

/* Launch configuration of the search rounds (mkgb_build, mkgb_run).  The paper has no
 * counterpart: this is a library service that changes neither results nor arithmetic.
 * find_shape picks how a round of the search runs: 0, 1, 2 as two kernels per plan step (one
 * thread per candidate for propagation, window and chi2; eight lanes per seed for the merge and
 * the update) with blocks of 128, 64 or 256 threads for the first kernel and select_shape (0, 1,
 * 2: 128, 64, 256 threads) for the second; 3, 4, 5 as one fused kernel per plan step (blocks of
 * 128 threads with 4 or 3 resident per SM, or 256 threads with 2; select_shape is ignored).
 * Each kernel launches as many blocks as stay resident on the device.  use_graph = 1 (the
 * default) records the launches of one search as a CUDA graph on the first call and replays it
 * while the arguments, shapes and stream stay the same (a change re-records); the graph is used
 * only on a stream created by the caller or the library (not the legacy or per-thread default
 * stream) and not while the stream is being captured by the caller, where the launches are made
 * one by one and join the caller's capture.  Results are identical for every choice.  Errors:
 * MKGB_EINVAL for find_shape outside 0..5 or select_shape outside 0..2. */
int mkgb_set_launch(mkgb_ctx* ctx, int find_shape, int select_shape, int use_graph);

/* Autotuner of the search launch shapes (library service, no counterpart in the paper): runs
 * the search over the seeds loaded now (mkgb_seed) once per launch configuration (the 3 x 3
 * two-kernel pairs and the 3 fused shapes of mkgb_set_launch), each warmed once and then timed
 * reps times with CUDA events on the context's stream, keeps the fastest as the context's
 * shapes (mkgb_set_launch) and writes it to find_shape / select_shape (may be NULL) and its mean
 * time per search to ms_out (may be NULL).  The outputs of these searches go to the library's
 * own buffers; loaded hits and seeds are not changed.  Synchronises the stream.  Errors:
 * MKGB_ESTATE without seeds, MKGB_EINVAL for reps < 1, the errors of mkgb_build. */
int mkgb_autotune(mkgb_ctx* ctx, int reps, int* find_shape, int* select_shape, float* ms_out);

/* Derivative of the fit (growth of Sec. 4's final fit): the fit over a known assignment with
 * per-layer alignment and material applied, and the derivatives of its total chi2.  Alignment:
 * align[l*6 + (0..5)] = (dx, dy, dz, wx, wy, wz) moves every hit of layer l as
 * h' = h + d + w x (h - c_l), c_l = (0, 0, 0) for a cylinder and (0, 0, z_l) for a disk (the
 * layer surfaces stay nominal); xscale[l] multiplies the layer's x/X0.  Arguments as mkgb_fit
 * (layers, hits, p0, c0: n tracks x max_steps), plus align (n_layers x 6) and xscale (n_layers).
 * Outputs: chi2_out (n: the track's summed predicted chi2 at these parameters, 0 if it failed),
 * d_p0 (n x 6: d chi2_i / d p0_i), d_align (n_layers x 6) and d_xscale (n_layers): derivatives
 * of the total chi2 over the tracks with status 0; status_out (n, optional) as mkgb_fit, plus
 * 5 = a step redone by the reverse sweep failed where the plain pass passed it (a rounding
 * difference at a layer edge; the track is left out).  The derivatives are exact for the FP32
 * arithmetic of the fit (dual numbers; no FP64 refit).
 * mode 0: reverse sweep (one plain pass storing each step's input state, then the steps from
 * the last to the first, each redone with its 34 inputs seeded, contracting the adjoint of its
 * output; device scratch of 128 bytes per track and step, kept by the context).  mode 1: forward
 * mode over all 6 + 7 L parameters of a track (no scratch, ~4x the arithmetic at 22 layers).
 * Errors: MKGB_ESTATE without geometry, params or hits; MKGB_EINVAL on a mode other than 0 or 1,
 * NULL arrays or a hit index beyond the loaded hits (host arrays); MKGB_ENOMEM if the scratch
 * cannot be allocated. */
int mkgb_fit_grad(mkgb_ctx* ctx, int n, int max_steps, const int32_t* layers, const int32_t* hits,
                  const float* p0, const float* c0, const float* align, const float* xscale,
                  float* chi2_out, float* d_p0, float* d_align, float* d_xscale, int32_t* status_out,
                  int mode, int on_device);

/* Kalman fit over a known assignment that allocates nothing.  The paper has no counterpart:
 * this is a library service, not a step of the method.  Same arguments, outputs and
 * arithmetic as mkgb_fit with on_device = 1 (every array a device pointer on the context's
 * device; status_out may be NULL), but the call makes no device allocation or free: its
 * scratch (work counters, the FP64 refit counter and the refit list) is a fixed file-scope
 * device array of about 256 KB per device, sized for at most 65536 tracks per call.  It is
 * meant for callers that must not allocate while they run: cudaMalloc and cudaFree can
 * synchronise the whole device and can fail while a caching allocator (PyTorch's, a serving
 * pool) holds the free memory, so a stream-ordered loop that fits batch after batch keeps its
 * memory footprint fixed by calling this entry point instead.
 * Setup: the first call on a device looks up the scratch address (cudaGetSymbolAddress) and
 * keeps it for the process; make that first call before any stream capture begins.  The kept
 * address belongs to the device's primary context: after cudaDeviceReset in the same process it
 * is stale, and calling this entry point again in that process is not supported.
 * Zero state: the work counters and the refit counter must be zero when a fit starts; the call
 * clears them itself (cudaMemsetAsync on the context's stream) before its kernels, and the
 * refit list needs no initial value.
 * Concurrency: all calls on one device share the one scratch array, so two calls whose work
 * overlaps in time (other streams, other contexts, other host threads) race on it and give
 * wrong results; order them on one stream or synchronise between them.
 * The call is asynchronous with respect to the host (outputs are ready when the context's
 * stream reaches them); mkgb_counters does not report it.
 * Errors: MKGB_EINVAL for n > 65536 (the message names the limit; split the batch or use
 * mkgb_fit), a negative size or a NULL array; MKGB_ESTATE without geometry, params or hits;
 * MKGB_ECUDA if the scratch lookup or a launch fails. */
int mkgb_fit_static(mkgb_ctx* ctx, int n, int max_steps, const int32_t* layers, const int32_t* hits,
                    const float* p0, const float* c0, float* p_out, float* c_out, float* chi2_out,
                    int32_t* status_out);

/* Arithmetic-throughput probe (library service, no counterpart in the paper): the fused
 * multiply-add rate of this device, kind 0 = FP32, kind 1 = FP64, in TFLOP/s (2 flops per
 * multiply-add) written to tflops_out.  One resident grid of independent multiply-add chains,
 * timed with CUDA events on the context's stream after a sizing launch (~20 ms timed); it is the
 * measured denominator beside the nominal one in the rooflines of the FP32 search and the FP64
 * seed fit.  Synchronises the stream.  Errors: MKGB_EINVAL for another kind or a NULL output,
 * MKGB_ECUDA if a launch fails. */
int mkgb_probe_peak(mkgb_ctx* ctx, int kind, double* tflops_out);

/* Single propagation step (Sec. 3.1 propagation; a4-a7): n states to the given layers.
 * crossed_out: 1 crossed, 0 not crossed (state copied through), -1 stopped. */
int mkgb_propagate(mkgb_ctx* ctx, int n, const int32_t* layers, const float* p_in,
                   const float* c_in, float* p_out, float* c_out, int32_t* crossed_out, int on_device);

/* Single chi2 + Kalman update (a9, a11): n predicted states with one hit each (xyz n x 3,
 * cov6 n x 6).  ok_out: 1 ok, 0 update rejected (S not positive definite or theta left (0, pi)). */
int mkgb_update(mkgb_ctx* ctx, int n, const float* p_in, const float* c_in, const float* hit_xyz,
                const float* hit_cov, float* p_out, float* c_out, float* chi2_out, int32_t* ok_out,
                int on_device);

/* Work counters of the last mkgb_build (kind 0) or mkgb_fit / mkgb_fit_backward (kind 1), after the call's stream
 * work has finished: [0] candidate-layer (build) or track-layer (fit) steps on crossed layers,
 * [1] chi2 evaluations of hits inside windows, [2] Kalman updates, [3] hits tested against a
 * window, [4] Newton iterations of the barrel crossing.  Synchronises the stream. */
int mkgb_counters(mkgb_ctx* ctx, int kind, int64_t out[5]);

#ifdef __cplusplus
}
#endif
#endif
