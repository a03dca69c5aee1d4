/* Plain FP64 CPU oracle for the batched Kalman step of mkFit-style track building
 * and fitting (arXiv:2312.11728, Sec. 2.2 forward search, Sec. 3.1 layers and
 * layer plans, Sec. 4 final fit).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, __graft_entry__.smoke() and the CPU
 * baseline legs of bench.py may load this library.  It shares no code, header,
 * table or constant with the CUDA library and includes nothing from it.
 *
 * The paper names the steps (propagation, hit selection, Kalman filter
 * calculations, combinatorial search with a candidate limit and a missed-layer
 * limit, best-scoring candidate) but prints no formula.  Each function below
 * states the textbook formula it writes out: helix motion in a uniform field,
 * the Kalman filter (Fruhwirth 1987), the PDG Highland formula and the PDG
 * Bethe-Bloch mean energy loss.
 *
 * State p = (x, y, z, k = q/pT, phi, theta); covariance packed lower triangle,
 * index(i,j) = i(i+1)/2 + j for i >= j.  Hit = (x, y, z) with a packed 3x3
 * covariance (xx, yx, yy, zx, zy, zz).  Measurement H = [I3 | 0].
 */
#ifndef MKORACLE_H
#define MKORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_BARREL 0
#define ORC_DISK 1
#define ORC_MAX_PLAN 64
#define ORC_MAX_CANDS 64

/* hit codes per plan step in build output */
#define ORC_MISS (-1)
#define ORC_SKIP (-2)
#define ORC_STOP (-3)
#define ORC_PRE (-4)

typedef struct {
    int kind, n_eta, n_phi, pad;
    double pos, lo, hi, x_over_x0;
    double sig[3];
    double eta_lo, eta_hi;
} orc_layer;

/* Flat detector modules (Sec. 3.1: module position, normal and phi-direction vectors, needed
 * for the Phase-2 tilted modules and for picking up hits of overlapping modules).  A module is
 * the plane through c with unit normal n; its phi-direction lies in the plane and is carried by
 * the hit covariance, so the filter needs c and n only.  hit_mod gives each global hit id its
 * module (-1: the hit lies on its layer's own cylinder or disk). */
typedef struct {
    int n;
    const double* c;       /* n x 3 [cm] */
    const double* nrm;     /* n x 3 unit normals */
    const int* hit_mod;    /* per global hit id */
} orc_modules;

typedef struct {
    double bz, barrel_eta_max;
    int n_layers, n_regions;
    const orc_layer* layers;
    const int* plan;       /* concatenated layer plans */
    const int* plan_off;   /* n_regions + 1 */
    const orc_modules* mods;   /* NULL: no module hits */
} orc_geom;

typedef struct {
    double chi2_cut, win_nsigma, deta_min, deta_max, dphi_min, dphi_max;
    double score_hit, score_hole;
    int max_cands, max_holes, material, binned;
    double score_overlap;  /* score added to a candidate that picks up an overlap hit */
} orc_params;

/* near-tie thresholds (selection decisions that finite precision may take either way) */
typedef struct {
    double chi2_rel;      /* |chi2 - cut| < chi2_rel * cut */
    double win_abs;       /* | |d| - half_width | < win_abs + win_rel * half_width */
    double win_rel;
    double score_abs;     /* score gap < max(score_abs, score_rel * |score|) */
    double score_rel;
    double edge_rel;      /* crossing point within edge_rel * |edge| of a layer boundary */
    double kappa;         /* a kept child whose innovation covariance S = C_pos + V has a Frobenius
                             condition number above this (default 2^24 = 1/eps of FP32, where an FP32
                             update cannot resolve the posterior) */
} orc_tie;

typedef struct {
    double* params;     /* S x 6 */
    double* cov;        /* S x 21 */
    double* score;      /* S */
    double* chi2;       /* S: sum of chi2 of hits added by the search */
    int* nfound;        /* S: hits on the track including the 3 seed hits */
    int* nholes;        /* S */
    int* hits;          /* S x max_plan: global hit id or ORC_MISS/SKIP/STOP/PRE per plan step */
    int max_plan;
    int* tie_step;      /* S: first plan step with a near-tie, -1 if none */
    int* region;        /* S */
    int* start;         /* S: first plan step of the search */
    long long* counters;/* [0] crossed candidate-layer visits, [1] chi2 evaluations,
                           [2] updates, [3] hits tested against a window */
    int* ovl;           /* S x max_plan: overlap hit id per plan step, -1 none (may be NULL) */
} orc_build_out;

/* --- single steps --- */
void orc_helix(double bz, const double p[6], double s, double out[6]);
int  orc_path(const orc_geom* g, int layer, const double p[6], double* s_out, double* edge_margin);
void orc_jacobian(const orc_geom* g, int layer, const double p[6], double s, double J[36]);
void orc_jacobian_fixed_s(double bz, const double p[6], double s, double A[36]);
void orc_transport(const double J[36], const double C[21], double Cout[21]);
int  orc_material(const orc_layer* L, double p[6], double C[21], double direction);
void orc_ms_theta0(double pmag, double t, double* theta0);
double orc_eloss(double pmag, double t);
int  orc_propagate(const orc_geom* g, int layer, const double p[6], const double C[21],
                   int material, double pout[6], double Cout[21], double* s_out);
int  orc_path_inward(const orc_geom* g, int layer, const double p[6], double* s_out, double* edge_margin);
void orc_reverse(const double p[6], const double C[21], double pr[6], double Cr[21]);
int  orc_propagate_backward(const orc_geom* g, int layer, const double p[6], const double C[21],
                            int material, double pout[6], double Cout[21], double* s_out);
/* module planes: crossing nearest to the state, Jacobian, propagation (no material) */
int  orc_path_plane(double bz, const double p[6], const double c[3], const double n[3], double* s_out,
                    double* margin);
void orc_jacobian_plane(double bz, const double p[6], double s, const double n[3], double J[36]);
int  orc_propagate_plane(double bz, const double p[6], const double C[21], const double c[3],
                         const double n[3], double pout[6], double Cout[21], double* s_out);
void orc_window(const orc_layer* L, const orc_params* P, const double p[6], const double C[21],
                double out[4]);
void orc_hit_eta_phi(const double m[3], double* eta, double* phi);
int  orc_chi2(const double p[6], const double C[21], const double m[3], const double V[6],
              double* chi2);
int  orc_update(const double p[6], const double C[21], const double m[3], const double V[6],
                int joseph, double pout[6], double Cout[21], double* chi2);
int  orc_seed(const orc_geom* g, int material, const double h[9], const double V[18],
              const int layers[3], double p[6], double C[21], double pinit[6]);
int  orc_select_region(const orc_geom* g, const double p[6]);

/* --- batches --- */
void orc_seed_batch(const orc_geom* g, int material, int n, const int* seed_hits,
                    const int* seed_layers, const double* xyz, const double* cov,
                    double* p, double* C, double* pinit, int* region, int* start, int* status);
/* outlier_chi2 > 0: a hit whose predicted chi2 exceeds it is not used (the final fit's outlier
 * rejection, Sec. 2.2 / Sec. 4); near_cut (may be NULL) flags tracks with a chi2 within 1e-3 of
 * the cut, where FP32 and FP64 may decide differently. */
void orc_fit_batch(const orc_geom* g, int material, int n, int max_steps, const int* layers,
                   const int* hits, const double* xyz, const double* cov, const double* p0,
                   const double* C0, double outlier_chi2, double* p, double* C, double* chi2, int* nupd,
                   int* status, int* near_cut, long long* counters);
void orc_bkfit_batch(const orc_geom* g, int material, int n, int max_steps, const int* layers,
                     const int* hits, const double* xyz, const double* cov, const double* p_start,
                     const double* C_start, double cov_scale, double outlier_chi2, double* p, double* C,
                     double* chi2, int* nupd, int* status, int* near_cut, long long* counters);
int  orc_build_backward_event(const orc_geom* g, const orc_params* P, const orc_tie* T,
                              const long long* layer_off, const double* xyz, const double* cov,
                              int n, const double* p_start, const double* C_start, const int* first_layer,
                              orc_build_out* out);
int  orc_build_event(const orc_geom* g, const orc_params* P, const orc_tie* T,
                     const long long* layer_off, const double* xyz, const double* cov,
                     int n_seeds, const int* seed_hits, const int* seed_layers,
                     orc_build_out* out);

/* --- seed cleaning, quality filter and duplicate removal (Sec. 2.2) --- */
void orc_clean_seeds(int n, const int* seed_hits, long long n_hits, int* keep);
void orc_remove_duplicates(int n, int width, const int* hits, const double* score, long long n_hits,
                           int min_hits, double frac, int* keep);

#ifdef __cplusplus
}
#endif
#endif
