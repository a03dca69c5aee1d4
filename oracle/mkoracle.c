/* Plain FP64 CPU oracle: see mkoracle.h.  TEST INFRASTRUCTURE ONLY.
 *
 * Written for a reader checking it against the textbook formulas: no blocking,
 * no fusion, dense 6x6 algebra, Cholesky for 3x3 systems, one candidate at a time.
 */
#include "mkoracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846
#define TWO_PI (2.0 * PI)
#define C_LIGHT 0.00299792458     /* curvature [1/cm] = C_LIGHT * B[T] / pT[GeV] */
#define M_PION 0.13957039         /* GeV */
#define M_ELEC 0.51099895e-3      /* GeV */
#define SI_K 0.307075             /* MeV cm^2 / mol */
#define SI_ZA 0.49848
#define SI_RHO 2.329              /* g / cm^3 */
#define SI_X0 9.37                /* cm */
#define SI_I 173.0e-9             /* GeV */
#define INC_CAP 10.0              /* cap on the path-length factor 1/|cos(incidence)| */

static int ix(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

static void unpack6(const double c[21], double M[6][6]) {
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) M[i][j] = c[ix(i, j)];
}

static void pack6(double M[6][6], double c[21]) {
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) c[ix(i, j)] = M[i][j];
}

static double wrap_phi(double a) {
    while (a > PI) a -= TWO_PI;
    while (a <= -PI) a += TWO_PI;
    return a;
}

/* ------------------------------------------------------------------ helix (path-length form)
 * Transverse path s, signed curvature omega = -C_LIGHT*B*k, turning angle a = omega*s.
 * x' = x + s (cos(phi) S1(a) - sin(phi) C1(a)), y' = y + s (sin(phi) S1(a) + cos(phi) C1(a)),
 * z' = z + s cot(theta), phi' = phi + a, with S1 = sin(a)/a and C1 = (1 - cos a)/a.
 */
static void s1c1(double a, double* S1, double* C1) {
    if (fabs(a) < 1e-8) {
        *S1 = 1.0 - a * a / 6.0;
        *C1 = 0.5 * a - a * a * a / 24.0;
    } else {
        double h = sin(0.5 * a);
        *S1 = sin(a) / a;
        *C1 = 2.0 * h * h / a;
    }
}

static void s1c1_deriv(double a, double* dS1, double* dC1) {
    if (fabs(a) < 0.05) {
        double a2 = a * a;
        *dS1 = a * (-1.0 / 3.0 + a2 * (1.0 / 30.0 + a2 * (-1.0 / 840.0 + a2 * (1.0 / 45360.0 - a2 / 3991680.0))));
        *dC1 = 0.5 + a2 * (-1.0 / 8.0 + a2 * (1.0 / 144.0 + a2 * (-1.0 / 5760.0 + a2 / 403200.0)));
    } else {
        double S1, C1;
        s1c1(a, &S1, &C1);
        *dS1 = (cos(a) - S1) / a;
        *dC1 = (sin(a) - C1) / a;
    }
}

void orc_helix(double bz, const double p[6], double s, double out[6]) {
    double om = -C_LIGHT * bz * p[3];
    double a = om * s, S1, C1;
    s1c1(a, &S1, &C1);
    double cf = cos(p[4]), sf = sin(p[4]);
    out[0] = p[0] + s * (cf * S1 - sf * C1);
    out[1] = p[1] + s * (sf * S1 + cf * C1);
    out[2] = p[2] + s * cos(p[5]) / sin(p[5]);
    out[3] = p[3];
    out[4] = p[4] + a;
    out[5] = p[5];
}

/* Smallest s > 0 at which the helix meets the layer surface, and whether the
 * crossing lies inside the layer's extent.  Barrel: Newton on
 * g(s) = x'(s)^2 + y'(s)^2 - R^2 from the straight-line root, kept inside the
 * bracket [0, s_far] (s_far = path to the point of largest radius, where
 * g >= 0) by bisection.  Disk: s = (z_d - z) tan(theta).
 * edge_margin: smallest relative distance of a yes/no geometric decision from
 * its threshold (layer edges; reach of a curling track). */
int orc_path(const orc_geom* g, int layer, const double p[6], double* s_out, double* edge_margin) {
    const orc_layer* L = &g->layers[layer];
    double om = -C_LIGHT * g->bz * p[3];
    double s;
    double margin = INFINITY;
    if (L->kind == ORC_DISK) {
        double ct = cos(p[5]), st = sin(p[5]);
        if (fabs(ct) < 1e-15) { *edge_margin = margin; return 0; }
        s = (L->pos - p[2]) * st / ct;
        if (!(s > 0)) { *edge_margin = margin; return 0; }
        /* loopers are followed on the outgoing part of their current turn only: the disk must
           be reached before the next point of largest radius, moving outward in r */
        if (fabs(om) >= 1e-14) {
            double sf = sin(p[4]), cf = cos(p[4]);
            double cx = p[0] - sf / om, cy = p[1] + cf / om, d = hypot(cx, cy);
            double sg = om > 0 ? 1.0 : -1.0;
            double turn = fmod((atan2(sg * cx / d, -sg * cy / d) - p[4]) * sg, TWO_PI);
            if (turn < 0) turn += TWO_PI;
            double s_far = turn / fabs(om);
            double q[6];
            orc_helix(g->bz, p, s, q);
            double vr = (q[0] * cos(q[4]) + q[1] * sin(q[4])) / fmax(hypot(q[0], q[1]), 1e-300);
            margin = fmin(fabs(s - s_far) / s_far, fabs(vr));
            if (s > s_far || vr < 0) { *edge_margin = margin; return 0; }
        }
    } else {
        double R = L->pos, x = p[0], y = p[1], cf = cos(p[4]), sf = sin(p[4]);
        if (x * x + y * y >= R * R) { *edge_margin = margin; return 0; }
        double b = x * cf + y * sf, c = x * sf - y * cf;
        double s0 = -b + sqrt(R * R - c * c);
        if (fabs(om) < 1e-14) {
            s = s0;
        } else {
            double rho = 1.0 / fabs(om);
            double cx = x - sf / om, cy = y + cf / om, d = hypot(cx, cy);
            double reach = d + rho - R;
            margin = fabs(reach) / R;
            if (reach < 0) { *edge_margin = margin; return 0; }
            double sg = om > 0 ? 1.0 : -1.0;
            double psi_far = atan2(sg * cx / d, -sg * cy / d);
            double turn = fmod((psi_far - p[4]) * sg, TWO_PI);
            if (turn < 0) turn += TWO_PI;
            double lo = 0.0, hi = turn * rho;
            s = (s0 > lo && s0 < hi) ? s0 : 0.5 * (lo + hi);
            for (int it = 0; it < 300; ++it) {
                double q[6];
                orc_helix(g->bz, p, s, q);
                double gv = q[0] * q[0] + q[1] * q[1] - R * R;
                if (gv < 0) lo = s; else hi = s;
                double dg = 2.0 * (q[0] * cos(q[4]) + q[1] * sin(q[4]));
                double sn = dg > 0 ? s - gv / dg : 0.5 * (lo + hi);
                if (!(sn > lo && sn < hi)) sn = 0.5 * (lo + hi);
                double ds = sn - s;
                s = sn;
                if (fabs(ds) < 1e-12 * R || hi - lo < 1e-13 * R) break;
            }
        }
    }
    double q[6];
    orc_helix(g->bz, p, s, q);
    double v = (L->kind == ORC_BARREL) ? q[2] : hypot(q[0], q[1]);
    double m_lo = fabs(v - L->lo) / fmax(fabs(L->lo), 1.0);
    double m_hi = fabs(v - L->hi) / fmax(fabs(L->hi), 1.0);
    margin = fmin(margin, fmin(m_lo, m_hi));
    *edge_margin = margin;
    *s_out = s;
    return (v >= L->lo && v <= L->hi) ? 1 : 0;
}

/* Inward crossing of a state whose direction of motion points inward (the reversed state of
 * the backward fit): smallest s > 0 at which the helix meets the layer surface while its
 * transverse radius decreases, before the point of smallest radius of the current turn.
 * Barrel: the start lies outside the cylinder and moves inward; g(s) = x'^2 + y'^2 - R^2
 * decreases from g(0) > 0 over [0, s_near] (s_near = path to the point of smallest radius,
 * where g < 0 if the helix reaches R); Newton on g from the straight-line root, kept inside
 * the bracket by bisection.  Disk: s = (z_d - z) tan(theta) > 0, reached before s_near and
 * moving inward in r.  Then the extent check.  edge_margin as in orc_path. */
int orc_path_inward(const orc_geom* g, int layer, const double p[6], double* s_out, double* edge_margin) {
    const orc_layer* L = &g->layers[layer];
    double om = -C_LIGHT * g->bz * p[3];
    double cf = cos(p[4]), sf = sin(p[4]);
    double margin = INFINITY;
    double s;
    /* path to the point of smallest transverse radius (infinite for a straight line) */
    double s_near = INFINITY, r_near = 0.0;
    if (fabs(om) >= 1e-14) {
        double rho = 1.0 / fabs(om);
        double cx = p[0] - sf / om, cy = p[1] + cf / om, d = hypot(cx, cy);
        double sg = om > 0 ? 1.0 : -1.0;
        double psi_near = atan2(sg * cx / d, -sg * cy / d) + PI;
        double turn = fmod((psi_near - p[4]) * sg, TWO_PI);
        if (turn < 0) turn += TWO_PI;
        s_near = turn * rho;
        r_near = fabs(d - rho);
    } else {
        r_near = fabs(p[0] * sf - p[1] * cf);
    }
    if (L->kind == ORC_DISK) {
        double ct = cos(p[5]), st = sin(p[5]);
        if (fabs(ct) < 1e-15) { *edge_margin = margin; return 0; }
        s = (L->pos - p[2]) * st / ct;
        if (!(s > 0)) { *edge_margin = margin; return 0; }
        if (isfinite(s_near)) {
            double q[6];
            orc_helix(g->bz, p, s, q);
            double vr = (q[0] * cos(q[4]) + q[1] * sin(q[4])) / fmax(hypot(q[0], q[1]), 1e-300);
            margin = fmin(fabs(s - s_near) / s_near, fabs(vr));
            if (s > s_near || vr > 0) { *edge_margin = margin; return 0; }
        }
    } else {
        double R = L->pos, x = p[0], y = p[1];
        double b = x * cf + y * sf;
        if (x * x + y * y <= R * R || !(b < 0)) { *edge_margin = margin; return 0; }
        double reach = R - r_near;
        margin = fabs(reach) / R;
        if (reach < 0) { *edge_margin = margin; return 0; }
        double c = x * sf - y * cf;
        double s0 = -b - sqrt(fmax(R * R - c * c, 0.0));
        if (!isfinite(s_near)) {
            s = s0;
        } else {
            double lo = 0.0, hi = s_near;
            s = (s0 > lo && s0 < hi) ? s0 : 0.5 * (lo + hi);
            for (int it = 0; it < 300; ++it) {
                double q[6];
                orc_helix(g->bz, p, s, q);
                double gv = q[0] * q[0] + q[1] * q[1] - R * R;
                if (gv > 0) lo = s; else hi = s;
                double dg = 2.0 * (q[0] * cos(q[4]) + q[1] * sin(q[4]));
                double sn = dg < 0 ? s - gv / dg : 0.5 * (lo + hi);
                if (!(sn > lo && sn < hi)) sn = 0.5 * (lo + hi);
                double ds = sn - s;
                s = sn;
                if (fabs(ds) < 1e-12 * R || hi - lo < 1e-13 * R) break;
            }
        }
    }
    double q[6];
    orc_helix(g->bz, p, s, q);
    double v = (L->kind == ORC_BARREL) ? q[2] : hypot(q[0], q[1]);
    double m_lo = fabs(v - L->lo) / fmax(fabs(L->lo), 1.0);
    double m_hi = fabs(v - L->hi) / fmax(fabs(L->hi), 1.0);
    margin = fmin(margin, fmin(m_lo, m_hi));
    *edge_margin = margin;
    *s_out = s;
    return (v >= L->lo && v <= L->hi) ? 1 : 0;
}

/* d f(p, s) / d p at fixed s (rows and columns in state order x, y, z, k, phi, theta). */
void orc_jacobian_fixed_s(double bz, const double p[6], double s, double A[36]) {
    double cB = C_LIGHT * bz;
    double a = -cB * p[3] * s;
    double S1, C1, dS1, dC1;
    s1c1(a, &S1, &C1);
    s1c1_deriv(a, &dS1, &dC1);
    double cf = cos(p[4]), sf = sin(p[4]), st = sin(p[5]);
    memset(A, 0, 36 * sizeof(double));
    for (int i = 0; i < 6; ++i) A[i * 6 + i] = 1.0;
    double dx = s * (cf * S1 - sf * C1), dy = s * (sf * S1 + cf * C1);
    A[0 * 6 + 3] = s * (cf * dS1 - sf * dC1) * (-cB * s);
    A[0 * 6 + 4] = -dy;
    A[1 * 6 + 3] = s * (sf * dS1 + cf * dC1) * (-cB * s);
    A[1 * 6 + 4] = dx;
    A[2 * 6 + 5] = -s / (st * st);
    A[4 * 6 + 3] = -cB * s;
}

/* Full Jacobian of the surface-to-surface map: J = A + (df/ds)(ds/dp), with
 * ds/dp = -(dgamma/dp)/(dgamma/ds) from the surface equation gamma(f(p, s)) = 0. */
void orc_jacobian(const orc_geom* g, int layer, const double p[6], double s, double J[36]) {
    const orc_layer* L = &g->layers[layer];
    double A[36], q[6];
    orc_jacobian_fixed_s(g->bz, p, s, A);
    orc_helix(g->bz, p, s, q);
    double om = -C_LIGHT * g->bz * p[3];
    double dfds[6] = {cos(q[4]), sin(q[4]), cos(q[5]) / sin(q[5]), 0.0, om, 0.0};
    double grad[6] = {0, 0, 0, 0, 0, 0};
    if (L->kind == ORC_BARREL) {
        grad[0] = 2.0 * q[0];
        grad[1] = 2.0 * q[1];
    } else {
        grad[2] = 1.0;
    }
    double gs = 0.0;
    for (int i = 0; i < 6; ++i) gs += grad[i] * dfds[i];
    for (int j = 0; j < 6; ++j) {
        double gp = 0.0;
        for (int i = 0; i < 6; ++i) gp += grad[i] * A[i * 6 + j];
        for (int i = 0; i < 6; ++i) J[i * 6 + j] = A[i * 6 + j] - dfds[i] * gp / gs;
    }
}

/* C' = J C J^T, dense. */
void orc_transport(const double J[36], const double C[21], double Cout[21]) {
    double M[6][6], T[6][6], R[6][6];
    unpack6(C, M);
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double acc = 0.0;
            for (int l = 0; l < 6; ++l) acc += J[i * 6 + l] * M[l][j];
            T[i][j] = acc;
        }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double acc = 0.0;
            for (int l = 0; l < 6; ++l) acc += T[i][l] * J[j * 6 + l];
            R[i][j] = acc;
        }
    pack6(R, Cout);
}

/* PDG Highland formula (unit charge): theta0 = 13.6 MeV/(beta c p) sqrt(t) (1 + 0.038 ln(t/beta^2)). */
void orc_ms_theta0(double pmag, double t, double* theta0) {
    double beta = pmag / sqrt(pmag * pmag + M_PION * M_PION);
    *theta0 = 0.0136 / (beta * pmag) * sqrt(t) * (1.0 + 0.038 * log(t / (beta * beta)));
}

/* PDG Bethe-Bloch mean energy loss in silicon (no density-effect term), for a
 * path of t radiation lengths: dE/dx = K (Z/A) / beta^2 [ln(2 me b^2 g^2 Tmax / I^2)/2 - beta^2]. */
double orc_eloss(double pmag, double t) {
    double m = M_PION;
    double e = sqrt(pmag * pmag + m * m);
    double bg2 = (pmag / m) * (pmag / m);
    double b2 = bg2 / (1.0 + bg2);
    double gam = e / m;
    double tmax = 2.0 * M_ELEC * bg2 / (1.0 + 2.0 * gam * M_ELEC / m + (M_ELEC / m) * (M_ELEC / m));
    double dedx = SI_K * SI_ZA / b2 * (0.5 * log(2.0 * M_ELEC * bg2 * tmax / (SI_I * SI_I)) - b2);
    return dedx * SI_RHO * (t * SI_X0) * 1e-3;
}

/* Material of one layer at the crossing: thickness t = x/X0 * min(1/|n.u|, cap);
 * Highland kicks (delta theta and delta phi * sin(theta), each of variance theta0^2,
 * at fixed |p|) add Q to the (k, phi, theta) block, with dk/dtheta = -k cot(theta);
 * then the mean energy loss (direction +1 removes energy, -1 adds it back) scales
 * k and row/column k of C by p/p'.  Returns 0 if the particle stops. */
int orc_material(const orc_layer* L, double p[6], double C[21], double direction) {
    double st = sin(p[5]), ct = cos(p[5]);
    double ux = st * cos(p[4]), uy = st * sin(p[4]), uz = ct;
    double cosi;
    if (L->kind == ORC_BARREL) {
        double r = hypot(p[0], p[1]);
        cosi = fabs((p[0] * ux + p[1] * uy) / r);
    } else {
        cosi = fabs(uz);
    }
    double fac = (cosi * INC_CAP > 1.0) ? 1.0 / cosi : INC_CAP;
    double t = L->x_over_x0 * fac;
    double k = p[3];
    if (!(t > 0) || k == 0.0) return 1;
    double pm = 1.0 / (fabs(k) * st);
    double th0;
    orc_ms_theta0(pm, t, &th0);
    double th02 = th0 * th0, cot = ct / st;
    C[ix(4, 4)] += th02 / (st * st);
    C[ix(5, 5)] += th02;
    C[ix(3, 3)] += k * k * cot * cot * th02;
    C[ix(5, 3)] += -k * cot * th02;
    double e = sqrt(pm * pm + M_PION * M_PION);
    double e2 = e - direction * orc_eloss(pm, t);
    if (!(e2 > M_PION)) return 0;
    double p2 = sqrt(e2 * e2 - M_PION * M_PION);
    double a = pm / p2;
    p[3] = k * a;
    for (int j = 0; j < 6; ++j)
        if (j != 3) C[ix(3, j)] *= a;
    C[ix(3, 3)] *= a * a;
    return 1;
}

/* Propagation step: crossing, new parameters, J C J^T, then material (Sec. 3.1:
 * propagation to the next layer of the plan).  1 crossed, 0 not crossed, -1 stopped. */
int orc_propagate(const orc_geom* g, int layer, const double p[6], const double C[21],
                  int material, double pout[6], double Cout[21], double* s_out) {
    double s, em, J[36];
    if (!orc_path(g, layer, p, &s, &em)) return 0;
    orc_jacobian(g, layer, p, s, J);
    orc_helix(g->bz, p, s, pout);
    orc_transport(J, C, Cout);
    if (material && !orc_material(&g->layers[layer], pout, Cout, +1.0)) return -1;
    pout[4] = wrap_phi(pout[4]);
    *s_out = s;
    return 1;
}

/* The same trajectory traversed in the opposite direction: position unchanged, direction
 * reversed (phi + pi, pi - theta) and charge sign flipped (k -> -k) so that the reversed
 * particle follows the same circle.  C -> D C D with D = diag(1, 1, 1, -1, 1, -1). */
void orc_reverse(const double p[6], const double C[21], double pr[6], double Cr[21]) {
    static const double d[6] = {1, 1, 1, -1, 1, -1};
    pr[0] = p[0]; pr[1] = p[1]; pr[2] = p[2];
    pr[3] = -p[3];
    pr[4] = wrap_phi(p[4] + PI);
    pr[5] = PI - p[5];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) Cr[ix(i, j)] = d[i] * d[j] * C[ix(i, j)];
}

/* Propagation step of the backward fit (Sec. 2.2: the found track re-traversed inwards):
 * reverse the state, cross the (inner) layer along the reversed helix (orc_path_inward), the
 * new parameters and J C J^T as in orc_propagate, the material with the energy loss added back
 * (direction -1; the Highland variance is added as always), then reverse back.
 * 1 crossed, 0 not crossed, -1 stopped. */
int orc_propagate_backward(const orc_geom* g, int layer, const double p[6], const double C[21],
                           int material, double pout[6], double Cout[21], double* s_out) {
    double pr[6], Cr[21], qr[6], Cq[21], s, em, J[36];
    orc_reverse(p, C, pr, Cr);
    if (!orc_path_inward(g, layer, pr, &s, &em)) return 0;
    orc_jacobian(g, layer, pr, s, J);
    orc_helix(g->bz, pr, s, qr);
    orc_transport(J, Cr, Cq);
    if (material && !orc_material(&g->layers[layer], qr, Cq, -1.0)) return -1;
    qr[4] = wrap_phi(qr[4]);
    orc_reverse(qr, Cq, pout, Cout);
    *s_out = s;
    return 1;
}

/* ------------------------------------------------------------------ module planes (Sec. 3.1)
 * The Phase-2 modules are flat and some are tilted: a hit on a module is measured on the plane
 * through the module's position c with unit normal n.  The state is taken from the layer's
 * reference surface (cylinder or disk: window, material and binning) to that plane by the
 * helix, with the Jacobian of the plane-to-plane map; the step is a few millimetres long and
 * crosses no material. */

#define PLANE_SMAX 10.0      /* cm: largest |s| of the step from the reference surface to a module */
#define PLANE_MIN_COS 1e-3   /* smallest |n . dx/ds| (dx/ds per transverse path) of an accepted crossing */

/* g(s) = n . (x(s) - c) along the helix from p, and dg/ds = n . (cos phi', sin phi', cot theta). */
static double plane_gap(double bz, const double p[6], const double c[3], const double n[3], double s, double* dg) {
    double q[6];
    orc_helix(bz, p, s, q);
    *dg = n[0] * cos(q[4]) + n[1] * sin(q[4]) + n[2] * cos(q[5]) / sin(q[5]);
    return n[0] * (q[0] - c[0]) + n[1] * (q[1] - c[1]) + n[2] * (q[2] - c[2]);
}

/* Crossing of the helix with the plane n.(x - c) = 0 nearest to the state: Newton on g(s) from
 * the tangent-line root, to |ds| < 1e-13 (1 + |s|).  Returns 1 with s, or 0 if Newton does not
 * converge in 50 iterations, |s| > PLANE_SMAX or the crossing is grazing (|dg/ds| < PLANE_MIN_COS).
 * margin: relative distance of the last two decisions from their thresholds. */
int orc_path_plane(double bz, const double p[6], const double c[3], const double n[3], double* s_out,
                   double* margin) {
    double dg, g0 = plane_gap(bz, p, c, n, 0.0, &dg);
    *margin = INFINITY;
    if (dg == 0.0) return 0;
    double s = -g0 / dg;
    int ok = 0;
    for (int it = 0; it < 50 && !ok; ++it) {
        double gv = plane_gap(bz, p, c, n, s, &dg);
        if (dg == 0.0 || !isfinite(s)) return 0;
        double ds = -gv / dg;
        s += ds;
        ok = fabs(ds) < 1e-13 * (1.0 + fabs(s));
    }
    if (!ok) return 0;
    plane_gap(bz, p, c, n, s, &dg);
    *margin = fmin(fabs(fabs(s) - PLANE_SMAX) / PLANE_SMAX, fabs(fabs(dg) - PLANE_MIN_COS) / PLANE_MIN_COS);
    *s_out = s;
    return fabs(s) <= PLANE_SMAX && fabs(dg) >= PLANE_MIN_COS;
}

/* Jacobian of the map to the plane: J = A + (df/ds)(ds/dp), ds/dp = -(n . A_pos) / (n . df/ds). */
void orc_jacobian_plane(double bz, const double p[6], double s, const double n[3], double J[36]) {
    double A[36], q[6];
    orc_jacobian_fixed_s(bz, p, s, A);
    orc_helix(bz, p, s, q);
    double om = -C_LIGHT * bz * p[3];
    double dfds[6] = {cos(q[4]), sin(q[4]), cos(q[5]) / sin(q[5]), 0.0, om, 0.0};
    double gs = n[0] * dfds[0] + n[1] * dfds[1] + n[2] * dfds[2];
    for (int j = 0; j < 6; ++j) {
        double gp = n[0] * A[0 * 6 + j] + n[1] * A[1 * 6 + j] + n[2] * A[2 * 6 + j];
        for (int i = 0; i < 6; ++i) J[i * 6 + j] = A[i * 6 + j] - dfds[i] * gp / gs;
    }
}

/* Step to a module plane: crossing, new parameters, J C J^T (no material).  1 reached, 0 not. */
int orc_propagate_plane(double bz, const double p[6], const double C[21], const double c[3],
                        const double n[3], double pout[6], double Cout[21], double* s_out) {
    double s, m, J[36];
    if (!orc_path_plane(bz, p, c, n, &s, &m)) return 0;
    orc_jacobian_plane(bz, p, s, n, J);
    orc_helix(bz, p, s, pout);
    orc_transport(J, C, Cout);
    pout[4] = wrap_phi(pout[4]);
    *s_out = s;
    return 1;
}

/* Module of a global hit id (-1: the layer's own surface, or no module table). */
static int hit_module(const orc_geom* g, long long id) {
    return g->mods ? g->mods->hit_mod[id] : -1;
}

/* The state on the surface where hit id is measured: its module's plane, or the reference
 * surface's state itself for a hit without a module.  0 if the plane is not reached.
 * margin (may be NULL) as orc_path_plane. */
static int at_hit_surface(const orc_geom* g, long long id, const double p[6], const double C[21], double q[6],
                          double Cq[21], double* margin) {
    int m = hit_module(g, id);
    if (margin) *margin = INFINITY;
    if (m < 0) {
        memcpy(q, p, 6 * sizeof(double));
        memcpy(Cq, C, 21 * sizeof(double));
        return 1;
    }
    const double* c = &g->mods->c[3 * m];
    const double* n = &g->mods->nrm[3 * m];
    double s, mg;
    int r = orc_path_plane(g->bz, p, c, n, &s, &mg);
    if (margin) *margin = mg;
    if (!r) return 0;
    return orc_propagate_plane(g->bz, p, C, c, n, q, Cq, &s);
}

/* ------------------------------------------------------------------ hit selection */

static void local_cov(const orc_layer* L, double phi, double V[6]) {
    double c = cos(phi), s = sin(phi);
    double sr2 = L->sig[0] * L->sig[0], sp2 = L->sig[1] * L->sig[1], sz2 = L->sig[2] * L->sig[2];
    V[0] = sr2 * c * c + sp2 * s * s;
    V[1] = (sr2 - sp2) * c * s;
    V[2] = sr2 * s * s + sp2 * c * c;
    V[3] = 0.0;
    V[4] = 0.0;
    V[5] = sz2;
}

void orc_hit_eta_phi(const double m[3], double* eta, double* phi) {
    double r = hypot(m[0], m[1]);
    *eta = asinh(m[2] / r);
    *phi = atan2(m[1], m[0]);
}

/* Window (Sec. 2.2 hit selection; Sec. 3.2 per-layer search parameters):
 * predicted eta, phi; sigma^2 = grad^T (C_pos + V_layer) grad for eta and phi;
 * half-widths n_sigma * sigma clamped to [min, max].  out = (eta, phi, deta, dphi). */
void orc_window(const orc_layer* L, const orc_params* P, const double p[6], const double C[21],
                double out[4]) {
    double x = p[0], y = p[1], z = p[2];
    double rt2 = x * x + y * y, rt = sqrt(rt2), r3 = sqrt(rt2 + z * z);
    double eta = asinh(z / rt), phi = atan2(y, x);
    double ge[3] = {-z * x / (rt2 * r3), -z * y / (rt2 * r3), 1.0 / r3};
    double gp[3] = {-y / rt2, x / rt2, 0.0};
    double V[6], M[3][3];
    local_cov(L, phi, V);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] = C[ix(i, j)] + V[ix(i, j)];
    double ve = 0.0, vp = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            ve += ge[i] * M[i][j] * ge[j];
            vp += gp[i] * M[i][j] * gp[j];
        }
    double de = P->win_nsigma * sqrt(ve), dp = P->win_nsigma * sqrt(vp);
    de = fmin(fmax(de, P->deta_min), P->deta_max);
    dp = fmin(fmax(dp, P->dphi_min), P->dphi_max);
    out[0] = eta;
    out[1] = phi;
    out[2] = de;
    out[3] = dp;
}

/* ------------------------------------------------------------------ chi2 and update */

static int chol3(const double S[6], double Lc[6]) {
    if (!(S[0] > 0)) return 0;
    double l00 = sqrt(S[0]);
    double l10 = S[1] / l00, l20 = S[3] / l00;
    double d1 = S[2] - l10 * l10;
    if (!(d1 > 0)) return 0;
    double l11 = sqrt(d1);
    double l21 = (S[4] - l20 * l10) / l11;
    double d2 = S[5] - l20 * l20 - l21 * l21;
    if (!(d2 > 0)) return 0;
    Lc[0] = l00; Lc[1] = l10; Lc[2] = l11; Lc[3] = l20; Lc[4] = l21; Lc[5] = sqrt(d2);
    return 1;
}

static void inv3_from_chol(const double Lc[6], double Si[3][3]) {
    double i00 = 1.0 / Lc[0], i11 = 1.0 / Lc[2], i22 = 1.0 / Lc[5];
    double i10 = -Lc[1] * i00 * i11;
    double i21 = -Lc[4] * i11 * i22;
    double i20 = -(Lc[3] * i00 + Lc[4] * i10) * i22;
    double M[3][3] = {{i00, 0, 0}, {i10, i11, 0}, {i20, i21, i22}};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (int l = 0; l < 3; ++l) acc += M[l][a] * M[l][b];
            Si[a][b] = acc;
        }
}

/* Predicted-residual chi2 = r^T S^-1 r with r = m - H p, S = H C H^T + V. */
int orc_chi2(const double p[6], const double C[21], const double m[3], const double V[6], double* chi2) {
    double S[6], Lc[6];
    for (int i = 0; i < 6; ++i) S[i] = C[i] + V[i];  /* first 6 packed entries = position block */
    if (!chol3(S, Lc)) return 0;
    double r[3] = {m[0] - p[0], m[1] - p[1], m[2] - p[2]};
    double y0 = r[0] / Lc[0];
    double y1 = (r[1] - Lc[1] * y0) / Lc[2];
    double y2 = (r[2] - Lc[3] * y0 - Lc[4] * y1) / Lc[5];
    *chi2 = y0 * y0 + y1 * y1 + y2 * y2;
    return 1;
}

/* Kalman update: K = C H^T S^-1, p+ = p + K r, and either C+ = C - K S K^T (standard)
 * or C+ = (I - K H) C (I - K H)^T + K V K^T (Joseph).  Both are the same posterior; the
 * oracle's searches, seeds and fits use the Joseph form, whose result is first-order
 * insensitive to errors in K: when S is ill-conditioned (a grazing crossing with a prior
 * spread of ~10 cm against 30 um hits, condition ~1e7) the standard form loses ~1e-2 of the
 * posterior even in FP64.  phi is wrapped to (-pi, pi]; returns 0 if S is not positive
 * definite or theta leaves (0, pi). */
int orc_update(const double p[6], const double C[21], const double m[3], const double V[6],
               int joseph, double pout[6], double Cout[21], double* chi2) {
    double S[6], Lc[6], Si[3][3];
    for (int i = 0; i < 6; ++i) S[i] = C[i] + V[i];
    if (!chol3(S, Lc)) return 0;
    if (chi2 && !orc_chi2(p, C, m, V, chi2)) return 0;
    inv3_from_chol(Lc, Si);
    double B[6][3], K[6][3];
    for (int i = 0; i < 6; ++i)
        for (int a = 0; a < 3; ++a) B[i][a] = C[ix(i, a)];
    for (int i = 0; i < 6; ++i)
        for (int a = 0; a < 3; ++a) {
            double acc = 0.0;
            for (int b = 0; b < 3; ++b) acc += B[i][b] * Si[b][a];
            K[i][a] = acc;
        }
    double r[3] = {m[0] - p[0], m[1] - p[1], m[2] - p[2]};
    for (int i = 0; i < 6; ++i) pout[i] = p[i] + K[i][0] * r[0] + K[i][1] * r[1] + K[i][2] * r[2];
    if (!joseph) {
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j <= i; ++j) {
                double acc = 0.0;
                for (int a = 0; a < 3; ++a) acc += K[i][a] * B[j][a];
                Cout[ix(i, j)] = C[ix(i, j)] - acc;
            }
    } else {
        double A[6][6], M[6][6], T[6][6], Vf[3][3];
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) A[i][j] = (i == j) ? 1.0 : 0.0;
        for (int i = 0; i < 6; ++i)
            for (int a = 0; a < 3; ++a) A[i][a] -= K[i][a];
        unpack6(C, M);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Vf[i][j] = V[ix(i, j)];
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                double acc = 0.0;
                for (int l = 0; l < 6; ++l) acc += A[i][l] * M[l][j];
                T[i][j] = acc;
            }
        double R[6][6];
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                double acc = 0.0;
                for (int l = 0; l < 6; ++l) acc += T[i][l] * A[j][l];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) acc += K[i][a] * Vf[a][b] * K[j][b];
                R[i][j] = acc;
            }
        pack6(R, Cout);
    }
    pout[4] = wrap_phi(pout[4]);
    if (!(pout[5] > 0.0 && pout[5] < PI)) return 0;
    return 1;
}

/* ------------------------------------------------------------------ seeding */

int orc_select_region(const orc_geom* g, const double p[6]) {
    if (g->n_regions <= 1) return 0;
    double eta = -log(tan(0.5 * p[5]));
    if (fabs(eta) < g->barrel_eta_max) return 0;
    return eta > 0 ? 1 : 2;
}

/* Seed state (Sec. 2.2: seeds carry parameters at their outermost point): circle
 * through the transverse positions of the three hits gives |curvature|, the turning
 * sign gives the charge, the tangent at hit 1 gives phi, and dz over the arc length
 * from hit 1 to hit 3 gives cot(theta).  Starting from that estimate at hit 1 with a
 * diffuse diagonal covariance, a Kalman fit through hits 1, 2, 3 gives the state at hit 3. */
/* Seed fit (a1) of three hits; ids (may be NULL) names them so that a hit measured on a module
 * (Sec. 3.1) is used on its module's plane, reached from the layer's reference surface. */
static int seed_fit(const orc_geom* g, int material, const double h[9], const double V[18],
                    const int layers[3], const long long* ids, double p[6], double C[21], double pinit[6]) {
    double cB = C_LIGHT * g->bz;
    double ax = h[3] - h[0], ay = h[4] - h[1], bx = h[6] - h[0], by = h[7] - h[1];
    double cross = ax * by - ay * bx;
    double chord2 = bx * bx + by * by;
    double k, phi1, arc;
    if (fabs(cross) < 1e-12 * chord2) {
        k = 0.0;
        phi1 = atan2(by, bx);
        arc = sqrt(chord2);
    } else {
        double a2 = ax * ax + ay * ay;
        double ux = (by * a2 - ay * chord2) / (2.0 * cross);
        double uy = (ax * chord2 - bx * a2) / (2.0 * cross);
        double rho = hypot(ux, uy);
        double sg = cross > 0 ? 1.0 : -1.0;
        double om = sg / rho;
        k = -om / cB;
        phi1 = atan2(-sg * ux / rho, sg * uy / rho);
        double v1x = -ux, v1y = -uy, v3x = bx - ux, v3y = by - uy;
        double ang = atan2(v1x * v3y - v1y * v3x, v1x * v3x + v1y * v3y);
        arc = fabs(ang) * rho;
    }
    double cot = (h[8] - h[2]) / arc;
    double theta = atan2(1.0, cot);
    double q[6] = {h[0], h[1], h[2], k, phi1, theta};
    memcpy(pinit, q, sizeof(q));
    double Cq[21];
    memset(Cq, 0, sizeof(Cq));
    double sk = 0.5 * fabs(k) + 0.05;
    Cq[ix(0, 0)] = 0.01; Cq[ix(1, 1)] = 0.01; Cq[ix(2, 2)] = 0.01;
    Cq[ix(3, 3)] = sk * sk; Cq[ix(4, 4)] = 0.0025; Cq[ix(5, 5)] = 0.0025;
    double pu[6], Cu[21], pp[6], Cp[21], ph[6], Ch[21], s;
    /* hit 1 is the estimate's own position: on its module's plane as well */
    if (!orc_update(q, Cq, &h[0], &V[0], 1, pu, Cu, NULL)) return 0;
    for (int j = 1; j < 3; ++j) {
        if (orc_propagate(g, layers[j], pu, Cu, material, pp, Cp, &s) != 1) return 0;
        if (ids) {
            if (!at_hit_surface(g, ids[j], pp, Cp, ph, Ch, NULL)) return 0;
        } else {
            memcpy(ph, pp, sizeof(pp));
            memcpy(Ch, Cp, sizeof(Cp));
        }
        if (!orc_update(ph, Ch, &h[3 * j], &V[6 * j], 1, pu, Cu, NULL)) return 0;
    }
    memcpy(p, pu, sizeof(pu));
    memcpy(C, Cu, sizeof(Cu));
    return 1;
}

int orc_seed(const orc_geom* g, int material, const double h[9], const double V[18],
             const int layers[3], double p[6], double C[21], double pinit[6]) {
    return seed_fit(g, material, h, V, layers, NULL, p, C, pinit);
}

static int plan_start(const orc_geom* g, int region, int layer3) {
    for (int t = g->plan_off[region]; t < g->plan_off[region + 1]; ++t)
        if (g->plan[t] == layer3) return t - g->plan_off[region] + 1;
    return -1;
}

void orc_seed_batch(const orc_geom* g, int material, int n, const int* seed_hits,
                    const int* seed_layers, const double* xyz, const double* cov,
                    double* p, double* C, double* pinit, int* region, int* start, int* status) {
    for (int i = 0; i < n; ++i) {
        double h[9], V[18];
        long long ids[3];
        for (int j = 0; j < 3; ++j) {
            long long id = seed_hits[3 * i + j];
            ids[j] = id;
            memcpy(&h[3 * j], &xyz[3 * id], 3 * sizeof(double));
            memcpy(&V[6 * j], &cov[6 * id], 6 * sizeof(double));
        }
        int ok = seed_fit(g, material, h, V, &seed_layers[3 * i], ids, &p[6 * i], &C[21 * i], &pinit[6 * i]);
        region[i] = ok ? orc_select_region(g, &p[6 * i]) : -1;
        start[i] = ok ? plan_start(g, region[i], seed_layers[3 * i + 2]) : -1;
        status[i] = (ok && start[i] >= 0) ? 0 : 1;
    }
}

/* ------------------------------------------------------------------ fit over a known assignment */

void orc_fit_batch(const orc_geom* g, int material, int n, int max_steps, const int* layers,
                   const int* hits, const double* xyz, const double* cov, const double* p0,
                   const double* C0, double outlier_chi2, double* p, double* C, double* chi2, int* nupd,
                   int* status, int* near_cut, long long* counters) {
    for (int i = 0; i < n; ++i) {
        double q[6], Cq[21], pp[6], Cp[21], s;
        memcpy(q, &p0[6 * i], sizeof(q));
        memcpy(Cq, &C0[21 * i], sizeof(Cq));
        double sum = 0.0;
        int nu = 0, st = 0, near = 0;
        for (int j = 0; j < max_steps; ++j) {
            int L = layers[(long long)i * max_steps + j];
            if (L < 0) break;
            int r = orc_propagate(g, L, q, Cq, material, pp, Cp, &s);
            if (r != 1) { st = (r == 0) ? 1 : 2; break; }
            counters[0]++;
            memcpy(q, pp, sizeof(q));
            memcpy(Cq, Cp, sizeof(Cq));
            int h = hits[(long long)i * max_steps + j];
            if (h >= 0) {
                /* a module hit is used on its module's plane (not reached: status 1) */
                double x2, ph[6], Ch[21];
                if (!at_hit_surface(g, h, pp, Cp, ph, Ch, NULL)) { st = 1; break; }
                if (outlier_chi2 > 0.0) {   /* outlier rejection: a hit above the cut is not used */
                    if (!orc_chi2(ph, Ch, &xyz[3 * (long long)h], &cov[6 * (long long)h], &x2)) {
                        st = 3;
                        break;
                    }
                    if (fabs(x2 - outlier_chi2) < 1e-3 * outlier_chi2) near = 1;
                    if (x2 > outlier_chi2) continue;
                }
                if (!orc_update(ph, Ch, &xyz[3 * (long long)h], &cov[6 * (long long)h], 1, q, Cq, &x2)) {
                    st = 3;
                    break;
                }
                sum += x2;
                nu++;
                counters[1]++;
                counters[2]++;
            }
        }
        memcpy(&p[6 * i], q, sizeof(q));
        memcpy(&C[21 * i], Cq, sizeof(Cq));
        chi2[i] = sum;
        nupd[i] = nu;
        status[i] = st;
        if (near_cut) near_cut[i] = near;
    }
}

/* Backward fit (Sec. 2.2): each track re-traversed from its outermost listed layer to its
 * innermost.  layers/hits list the track's layers in the forward (outward) order as for
 * orc_fit_batch; p_start/C_start is its state on the last listed layer (the forward fit's
 * result there), whose covariance is scaled by cov_scale to release the forward fit's
 * information.  The hit on the last layer is used first (update), then for each earlier
 * listed layer: backward propagation and, with a hit, chi2 + update.  Outputs: the state at
 * the innermost listed layer, the summed predicted chi2, the number of updates and the status
 * (0 ok, 1 a listed layer not crossed, 2 stopped, 3 update failed). */
void orc_bkfit_batch(const orc_geom* g, int material, int n, int max_steps, const int* layers,
                     const int* hits, const double* xyz, const double* cov, const double* p_start,
                     const double* C_start, double cov_scale, double outlier_chi2, double* p, double* C,
                     double* chi2, int* nupd, int* status, int* near_cut, long long* counters) {
    for (int i = 0; i < n; ++i) {
        double q[6], Cq[21], pp[6], Cp[21], s;
        memcpy(q, &p_start[6 * i], sizeof(q));
        for (int k = 0; k < 21; ++k) Cq[k] = cov_scale * C_start[21 * i + k];
        int nl = 0;
        while (nl < max_steps && layers[(long long)i * max_steps + nl] >= 0) ++nl;
        double sum = 0.0;
        int nu = 0, st = 0, near = 0;
        if (nl > 0) {
            /* the start state lies on the last listed layer (on the plane of its hit's module
               for a module hit): its covariance is taken on that surface, without variance
               along the surface normal n (zero in exact arithmetic for a fitted state; the FP32
               rounding residue of an input is dropped): C -> Pi C Pi^T with Pi = I - n n^T on
               the position block */
            const orc_layer* Ls = &g->layers[layers[(long long)i * max_steps + nl - 1]];
            const int hl = hits[(long long)i * max_steps + nl - 1];
            const int ml = hl >= 0 ? hit_module(g, hl) : -1;
            double nv[3] = {0.0, 0.0, 1.0};
            if (ml >= 0) {
                memcpy(nv, &g->mods->nrm[3 * ml], sizeof(nv));
            } else if (Ls->kind == ORC_BARREL) {
                double r = hypot(q[0], q[1]);
                nv[0] = q[0] / r; nv[1] = q[1] / r; nv[2] = 0.0;
            }
            double M[6][6], Pi[6][6], T[6][6];
            unpack6(Cq, M);
            for (int a = 0; a < 6; ++a)
                for (int b = 0; b < 6; ++b) Pi[a][b] = (a == b) - (a < 3 && b < 3 ? nv[a] * nv[b] : 0.0);
            for (int a = 0; a < 6; ++a)
                for (int b = 0; b < 6; ++b) {
                    double acc = 0.0;
                    for (int l = 0; l < 6; ++l) acc += Pi[a][l] * M[l][b];
                    T[a][b] = acc;
                }
            for (int a = 0; a < 6; ++a)
                for (int b = 0; b < 6; ++b) {
                    double acc = 0.0;
                    for (int l = 0; l < 6; ++l) acc += T[a][l] * Pi[b][l];
                    M[a][b] = acc;
                }
            pack6(M, Cq);
        }
        for (int j = nl - 1; j >= 0; --j) {
            int L = layers[(long long)i * max_steps + j];
            if (j < nl - 1) {
                int r = orc_propagate_backward(g, L, q, Cq, material, pp, Cp, &s);
                if (r != 1) { st = (r == 0) ? 1 : 2; break; }
                counters[0]++;
                memcpy(q, pp, sizeof(q));
                memcpy(Cq, Cp, sizeof(Cq));
            }
            int h = hits[(long long)i * max_steps + j];
            if (h >= 0) {
                double x2;
                if (j < nl - 1) {   /* a module hit is used on its module's plane (not reached: 1) */
                    if (!at_hit_surface(g, h, q, Cq, pp, Cp, NULL)) { st = 1; break; }
                } else {            /* the start state already lies on its hit's surface */
                    memcpy(pp, q, sizeof(q));
                    memcpy(Cp, Cq, sizeof(Cq));
                }
                if (outlier_chi2 > 0.0) {   /* outlier rejection: a hit above the cut is not used */
                    if (!orc_chi2(pp, Cp, &xyz[3 * (long long)h], &cov[6 * (long long)h], &x2)) {
                        st = 3;
                        break;
                    }
                    if (fabs(x2 - outlier_chi2) < 1e-3 * outlier_chi2) near = 1;
                    if (x2 > outlier_chi2) continue;
                }
                if (!orc_update(pp, Cp, &xyz[3 * (long long)h], &cov[6 * (long long)h], 1, q, Cq, &x2)) {
                    st = 3;
                    break;
                }
                sum += x2;
                nu++;
                counters[1]++;
                counters[2]++;
            }
        }
        memcpy(&p[6 * i], q, sizeof(q));
        memcpy(&C[21 * i], Cq, sizeof(Cq));
        chi2[i] = sum;
        nupd[i] = nu;
        status[i] = st;
        if (near_cut) near_cut[i] = near;
    }
}

/* ------------------------------------------------------------------ combinatorial search */

typedef struct {
    double p[6], C[21];
    double score, chi2;
    int nfound, nholes, stopped;
    int hist[ORC_MAX_PLAN];
    int ovl[ORC_MAX_PLAN];   /* overlap hit id per plan step, -1 none */
} cand_t;

enum { K_HIT = 0, K_MISS = 1, K_SKIP = 2, K_STOP = 3, K_CARRY = 4 };

typedef struct {
    double score, chi2;
    int parent, kind;
    long long gid;
    long long ovl;   /* overlap hit picked up with the hit gid, -1 none */
} child_t;

/* Order of children: score descending, then parent slot ascending, then hit children
 * (by hit id ascending) before the parent's one non-hit child. */
static int child_cmp(const void* a, const void* b) {
    const child_t* x = (const child_t*)a;
    const child_t* y = (const child_t*)b;
    if (x->score != y->score) return x->score > y->score ? -1 : 1;
    if (x->parent != y->parent) return x->parent < y->parent ? -1 : 1;
    int xh = x->kind == K_HIT, yh = y->kind == K_HIT;
    if (xh != yh) return xh ? -1 : 1;
    if (xh && x->gid != y->gid) return x->gid < y->gid ? -1 : 1;
    return 0;
}

typedef struct {
    long long base;       /* first global hit id of the event */
    double* eta;          /* per hit of the event */
    double* phi;
    int* bin_start;       /* per layer: n_eta*n_phi + 1 offsets into bin_ids (absolute) */
    int* bin_ids;         /* global hit ids sorted by (layer, bin, id) */
    int* layer_bin_base;  /* n_layers: index of the layer's first offset in bin_start */
} evidx_t;

static int eta_bin(const orc_layer* L, double eta) {
    double f = (eta - L->eta_lo) / (L->eta_hi - L->eta_lo) * L->n_eta;
    if (!(f >= 0.0)) return 0;
    if (f >= L->n_eta) return L->n_eta - 1;
    return (int)floor(f);
}

static long long phi_cell(const orc_layer* L, double phi) {
    return (long long)floor((phi + PI) / TWO_PI * L->n_phi);
}

static int phi_bin(const orc_layer* L, double phi) {
    long long c = phi_cell(L, phi);
    if (c < 0) return 0;
    if (c >= L->n_phi) return L->n_phi - 1;
    return (int)c;
}

typedef struct {
    child_t* v;
    int n, cap;
} childvec;

static void push_child(childvec* cv, child_t c) {
    if (cv->n == cv->cap) {
        cv->cap = cv->cap ? 2 * cv->cap : 64;
        cv->v = (child_t*)realloc(cv->v, cv->cap * sizeof(child_t));
    }
    cv->v[cv->n++] = c;
}

typedef struct {
    long long* v;
    int n, cap;
} idvec;

static void push_id(idvec* iv, long long id) {
    if (iv->n == iv->cap) {
        iv->cap = iv->cap ? 2 * iv->cap : 256;
        iv->v = (long long*)realloc(iv->v, iv->cap * sizeof(long long));
    }
    iv->v[iv->n++] = id;
}

/* Hits to test for one window: all hits of the layer (brute force) or the hits in
 * the eta-phi bins overlapping the window widened by a small guard (binned).  The
 * window test itself decides membership, so both give the same children. */
static void window_hits(const orc_params* P, const orc_layer* L, int layer, const long long* layer_off,
                        const evidx_t* ev, const double w[4], idvec* out) {
    out->n = 0;
    if (!P->binned) {
        for (long long id = layer_off[layer]; id < layer_off[layer + 1]; ++id) push_id(out, id);
        return;
    }
    const double eps = 1e-9;
    int e0 = eta_bin(L, w[0] - w[2] - eps), e1 = eta_bin(L, w[0] + w[2] + eps);
    long long f0 = phi_cell(L, w[1] - w[3] - eps), f1 = phi_cell(L, w[1] + w[3] + eps);
    long long nf = f1 - f0 + 1;
    if (nf > L->n_phi) { f0 = 0; nf = L->n_phi; }
    const int* bs = &ev->bin_start[ev->layer_bin_base[layer]];
    for (int ie = e0; ie <= e1; ++ie)
        for (long long c = 0; c < nf; ++c) {
            int ip = (int)(((f0 + c) % L->n_phi + L->n_phi) % L->n_phi);
            int b = ie * L->n_phi + ip;
            for (int q = bs[b]; q < bs[b + 1]; ++q) push_id(out, ev->bin_ids[q]);
        }
}

static int cmp_ll(const void* a, const void* b) {
    long long x = *(const long long*)a, y = *(const long long*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static double gap_tol(const orc_tie* T, double s) { return fmax(T->score_abs, T->score_rel * fabs(s)); }

/* Frobenius condition number ||S||_F ||S^-1||_F of the innovation covariance S = C_pos + V. */
static double cond_frob(const double C[21], const double V[6]) {
    double S[6], Lc[6], Si[3][3];
    for (int i = 0; i < 6; ++i) S[i] = C[i] + V[i];
    if (!chol3(S, Lc)) return INFINITY;
    inv3_from_chol(Lc, Si);
    double a = 0.0, b = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double sij = S[ix(i, j)];
            a += sij * sij;
            b += Si[i][j] * Si[i][j];
        }
    return sqrt(a * b);
}

/* Per-event hit index: eta, phi and bins (Sec. 3.1: layers aggregate hits for uniform search). */
static void build_index(const orc_geom* g, const long long* layer_off, const double* xyz, evidx_t* ev) {
    const int NL = g->n_layers;
    ev->base = layer_off[0];
    long long nh = layer_off[NL] - layer_off[0];
    ev->eta = (double*)malloc((nh + 1) * sizeof(double));
    ev->phi = (double*)malloc((nh + 1) * sizeof(double));
    for (long long i = 0; i < nh; ++i) orc_hit_eta_phi(&xyz[3 * (ev->base + i)], &ev->eta[i], &ev->phi[i]);
    ev->layer_bin_base = (int*)malloc(NL * sizeof(int));
    long long tot = 0;
    for (int l = 0; l < NL; ++l) {
        ev->layer_bin_base[l] = (int)tot;
        tot += (long long)g->layers[l].n_eta * g->layers[l].n_phi + 1;
    }
    ev->bin_start = (int*)calloc(tot, sizeof(int));
    ev->bin_ids = (int*)malloc((nh + 1) * sizeof(int));
    for (int l = 0; l < NL; ++l) {
        const orc_layer* L = &g->layers[l];
        int nb = L->n_eta * L->n_phi;
        int* bs = &ev->bin_start[ev->layer_bin_base[l]];
        for (long long id = layer_off[l]; id < layer_off[l + 1]; ++id) {
            long long i = id - ev->base;
            bs[eta_bin(L, ev->eta[i]) * L->n_phi + phi_bin(L, ev->phi[i]) + 1]++;
        }
        bs[0] = (int)(layer_off[l] - ev->base);
        for (int b = 0; b < nb; ++b) bs[b + 1] += bs[b];
        int* fill = (int*)malloc((nb + 1) * sizeof(int));
        memcpy(fill, bs, (nb + 1) * sizeof(int));
        for (long long id = layer_off[l]; id < layer_off[l + 1]; ++id) {  /* ascending ids -> sorted within bin */
            long long i = id - ev->base;
            int b = eta_bin(L, ev->eta[i]) * L->n_phi + phi_bin(L, ev->phi[i]);
            ev->bin_ids[fill[b]++] = (int)id;
        }
        free(fill);
    }
}

static void free_index(evidx_t* ev) {
    free(ev->eta); free(ev->phi); free(ev->layer_bin_base); free(ev->bin_start); free(ev->bin_ids);
}

typedef struct {
    cand_t *cur, *nxt;
    double (*pp)[6];
    double (*CC)[21];
    childvec kids, amb, mh;
    idvec ids;
} search_ws;

static void ws_init(search_ws* w) {
    w->cur = (cand_t*)malloc(ORC_MAX_CANDS * sizeof(cand_t));
    w->nxt = (cand_t*)malloc(ORC_MAX_CANDS * sizeof(cand_t));
    w->pp = malloc(ORC_MAX_CANDS * sizeof(*w->pp));
    w->CC = malloc(ORC_MAX_CANDS * sizeof(*w->CC));
    w->kids = (childvec){0, 0, 0};
    w->amb = (childvec){0, 0, 0};
    w->mh = (childvec){0, 0, 0};
    w->ids = (idvec){0, 0, 0};
}

static void ws_free(search_ws* w) {
    free(w->cur); free(w->nxt); free(w->pp); free(w->CC);
    free(w->kids.v); free(w->amb.v); free(w->mh.v); free(w->ids.v);
}

/* Combinatorial search of one track (Sec. 2.2) from the state in w->cur[0] through plan steps
 * start .. plan_len - 1 of `plan`: per step every candidate is propagated to the layer (forwards,
 * or backwards for the backward search), the hits in its eta-phi window get a chi2, children
 * are ranked and the N best kept and updated; the best final candidate goes to slot si of out.
 * nfound0: hits the track already has (3 seed hits forwards, none backwards). */
static void search_track(const orc_geom* g, const orc_params* P, const orc_tie* T, const long long* layer_off,
                         const double* xyz, const double* cov, const evidx_t* evp, search_ws* w,
                         const int* plan, int plan_len, int start, int backward, int nfound0,
                         orc_build_out* out, int si) {
    const int N = P->max_cands;
    evidx_t ev = *evp;
    cand_t* cur = w->cur;
    cand_t* nxt = w->nxt;
    double (*pp)[6] = w->pp;
    double (*CC)[21] = w->CC;
    long long* ctr = out->counters;
    double* op = &out->params[6 * si];
    double* oC = &out->cov[21 * si];
    int* oh = &out->hits[(long long)si * out->max_plan];
    int ncur = 1;
    cur[0].score = 0.0;
    cur[0].chi2 = 0.0;
    cur[0].nfound = nfound0;
    cur[0].nholes = 0;
    cur[0].stopped = 0;
    for (int t = 0; t < ORC_MAX_PLAN; ++t) {
        cur[0].hist[t] = ORC_PRE;
        cur[0].ovl[t] = -1;
    }

    for (int t = start; t < plan_len; ++t) {
        const int layer = plan[t];
        const orc_layer* L = &g->layers[layer];
        int tie = 0;
        w->kids.n = 0;
        w->amb.n = 0;
        for (int c = 0; c < ncur; ++c) {
            cand_t* cd = &cur[c];
            child_t ch = {cd->score, 0.0, c, K_CARRY, -1, -1};
            if (cd->stopped) { push_child(&w->kids, ch); continue; }
            double s, em;
            int r;
            if (backward) {
                double pr[6], Cr[21];
                orc_reverse(cd->p, cd->C, pr, Cr);
                orc_path_inward(g, layer, pr, &s, &em);
                r = orc_propagate_backward(g, layer, cd->p, cd->C, P->material, pp[c], CC[c], &s);
            } else {
                orc_path(g, layer, cd->p, &s, &em);
                r = orc_propagate(g, layer, cd->p, cd->C, P->material, pp[c], CC[c], &s);
            }
            if (em < T->edge_rel) tie = 1;
            if (r < 0) continue;
            if (r == 0) { ch.kind = K_SKIP; push_child(&w->kids, ch); continue; }
            ctr[0]++;
            double wn[4];
            orc_window(L, P, pp[c], CC[c], wn);
            window_hits(P, L, layer, layer_off, &ev, wn, &w->ids);
            qsort(w->ids.v, w->ids.n, sizeof(long long), cmp_ll);
            double me = T->win_abs + T->win_rel * wn[2], mp = T->win_abs + T->win_rel * wn[3];
            const int k0 = w->kids.n, a0 = w->amb.n;
            int amb_mod = 0;
            w->mh.n = 0;
            for (int q = 0; q < w->ids.n; ++q) {
                long long id = w->ids.v[q];
                ctr[3]++;
                double de = fabs(ev.eta[id - ev.base] - wn[0]);
                double dp = fabs(wrap_phi(ev.phi[id - ev.base] - wn[1]));
                int in = de <= wn[2] && dp <= wn[3];
                int near_e = fabs(de - wn[2]) < me, near_p = fabs(dp - wn[3]) < mp;
                int near = (near_e && dp <= wn[3] + mp) || (near_p && de <= wn[2] + me);
                if (!in && !near) continue;
                /* a module hit is tested on its module's plane (Sec. 3.1 module vectors) */
                double x2, ph[6], Ch[21], hm;
                int on = at_hit_surface(g, id, pp[c], CC[c], ph, Ch, &hm);
                if (hm < T->edge_rel) tie = 1;
                if (!on) continue;
                if (!orc_chi2(ph, Ch, &xyz[3 * id], &cov[6 * id], &x2)) continue;
                if (in) ctr[1]++;
                child_t hc = {cd->score + P->score_hit - x2, x2, c, K_HIT, id, -1};
                if (in && x2 < P->chi2_cut) {
                    push_child(&w->kids, hc);
                    if (hit_module(g, id) >= 0) push_child(&w->mh, hc);
                }
                if ((near || fabs(x2 - P->chi2_cut) < T->chi2_rel * P->chi2_cut) &&
                    x2 < P->chi2_cut * (1.0 + T->chi2_rel)) {
                    push_child(&w->amb, hc);
                    if (hit_module(g, id) >= 0) amb_mod = 1;
                }
            }
            /* overlap hit (Sec. 2.2: a single additional detector-overlap hit per layer): a
               child taking module hit h also picks up the best accepted hit (chi2, then id) of
               the candidate's window that lies on another module, and scores score_overlap
               more.  With b1 the best accepted module hit and b2 the best one on a module other
               than b1's, that hit is b1 if h is not on b1's module, else b2; every module-hit
               child has one exactly when b2 exists (the accepted hits span two modules). */
            if (w->mh.n > 0) {
                childvec* mh = &w->mh;
                qsort(mh->v, mh->n, sizeof(child_t), child_cmp);   /* same parent: chi2 asc, id asc */
                long long b1 = mh->v[0].gid, b2 = -1;
                for (int q = 1; q < mh->n && b2 < 0; ++q)
                    if (hit_module(g, mh->v[q].gid) != hit_module(g, b1)) b2 = mh->v[q].gid;
                if (b2 >= 0) {
                    /* which hit is picked up is a chi2 comparison: near-equal chi2, or an
                       ambiguous hit at the window edge or the chi2 cut, may go either way */
                    for (int q = 1; q < mh->n; ++q)
                        if (mh->v[q].chi2 - mh->v[q - 1].chi2 < gap_tol(T, mh->v[q].chi2)) tie = 1;
                    for (childvec* cv = &w->kids; cv; cv = (cv == &w->kids) ? &w->amb : NULL)
                        for (int q = (cv == &w->kids) ? k0 : a0; q < cv->n; ++q) {
                            child_t* k = &cv->v[q];
                            if (k->kind != K_HIT || hit_module(g, k->gid) < 0) continue;
                            k->score += P->score_overlap;
                            k->ovl = hit_module(g, k->gid) != hit_module(g, b1) ? b1 : b2;
                        }
                }
                if (amb_mod) tie = 1;
            }
            if (cd->nholes < P->max_holes) {
                ch.kind = K_MISS;
                ch.score = cd->score - P->score_hole;
            } else {
                ch.kind = K_STOP;
            }
            push_child(&w->kids, ch);
        }
        childvec* kids = &w->kids;
        qsort(kids->v, kids->n, sizeof(child_t), child_cmp);
        int nkeep = kids->n < N ? kids->n : N;
        if (kids->n > N && kids->v[N - 1].score - kids->v[N].score < gap_tol(T, kids->v[N - 1].score)) tie = 1;
        for (int a = 0; a < w->amb.n; ++a) {
            double thr = kids->n >= N ? kids->v[N - 1].score : -INFINITY;
            if (w->amb.v[a].score >= thr - gap_tol(T, w->amb.v[a].score)) tie = 1;
        }
        if (tie && out->tie_step[si] < 0) out->tie_step[si] = t;

        /* precision limit: an update (or, for a non-hit child, a prediction measured with the
           layer's resolution) whose innovation covariance is too ill-conditioned for FP32 */
        for (int q = 0; q < nkeep && !tie; ++q) {
            child_t* k = &kids->v[q];
            if (k->kind == K_SKIP || k->kind == K_CARRY) continue;
            double Vc[6];
            const double* Cs = CC[k->parent];
            double ph[6], Ch[21];
            if (k->kind == K_HIT) {
                memcpy(Vc, &cov[6 * k->gid], sizeof(Vc));
                if (at_hit_surface(g, k->gid, pp[k->parent], CC[k->parent], ph, Ch, NULL)) Cs = Ch;
            } else {
                local_cov(L, atan2(pp[k->parent][1], pp[k->parent][0]), Vc);
            }
            if (cond_frob(Cs, Vc) > T->kappa) tie = 1;
        }
        if (tie && out->tie_step[si] < 0) out->tie_step[si] = t;

        int nn = 0;
        for (int q = 0; q < nkeep; ++q) {
            child_t* k = &kids->v[q];
            cand_t* par = &cur[k->parent];
            cand_t* nc = &nxt[nn];
            memcpy(nc->hist, par->hist, sizeof(nc->hist));
            memcpy(nc->ovl, par->ovl, sizeof(nc->ovl));
            nc->score = k->score;
            nc->chi2 = par->chi2;
            nc->nfound = par->nfound;
            nc->nholes = par->nholes;
            nc->stopped = par->stopped;
            if (k->kind == K_HIT) {
                double x2, ph[6], Ch[21];
                if (!at_hit_surface(g, k->gid, pp[k->parent], CC[k->parent], ph, Ch, NULL) ||
                    !orc_update(ph, Ch, &xyz[3 * k->gid], &cov[6 * k->gid], 1, nc->p, nc->C, &x2))
                    continue;
                ctr[2]++;
                nc->chi2 += x2;
                nc->nfound++;
                nc->hist[t] = (int)k->gid;
                nc->ovl[t] = (int)k->ovl;
            } else if (k->kind == K_MISS) {
                memcpy(nc->p, pp[k->parent], sizeof(nc->p));
                memcpy(nc->C, CC[k->parent], sizeof(nc->C));
                nc->nholes++;
                nc->hist[t] = ORC_MISS;
            } else if (k->kind == K_STOP) {
                memcpy(nc->p, pp[k->parent], sizeof(nc->p));
                memcpy(nc->C, CC[k->parent], sizeof(nc->C));
                nc->stopped = 1;
                nc->hist[t] = ORC_STOP;
            } else {
                memcpy(nc->p, par->p, sizeof(nc->p));
                memcpy(nc->C, par->C, sizeof(nc->C));
                nc->hist[t] = (k->kind == K_SKIP) ? ORC_SKIP : ORC_STOP;
            }
            nn++;
        }
        cand_t* tmp = cur;
        cur = nxt;
        nxt = tmp;
        ncur = nn;
        if (ncur == 0) break;
    }
    w->cur = cur;
    w->nxt = nxt;
    if (ncur == 0) return;
    if (ncur >= 2 && cur[0].score - cur[1].score < gap_tol(T, cur[0].score)) {
        int first = start;
        while (first < plan_len && cur[0].hist[first] == cur[1].hist[first]) ++first;
        if (out->tie_step[si] < 0 || first < out->tie_step[si]) out->tie_step[si] = first;
    }
    memcpy(op, cur[0].p, 6 * sizeof(double));
    memcpy(oC, cur[0].C, 21 * sizeof(double));
    out->score[si] = cur[0].score;
    out->chi2[si] = cur[0].chi2;
    out->nfound[si] = cur[0].nfound;
    out->nholes[si] = cur[0].nholes;
    for (int t = 0; t < plan_len && t < out->max_plan; ++t) oh[t] = cur[0].hist[t];
    if (out->ovl)
        for (int t = 0; t < plan_len && t < out->max_plan; ++t) out->ovl[(long long)si * out->max_plan + t] = cur[0].ovl[t];
}

static void clear_out(orc_build_out* out, int si) {
    int* oh = &out->hits[(long long)si * out->max_plan];
    for (int t = 0; t < out->max_plan; ++t) oh[t] = ORC_PRE;
    if (out->ovl)
        for (int t = 0; t < out->max_plan; ++t) out->ovl[(long long)si * out->max_plan + t] = -1;
    out->tie_step[si] = -1;
    out->score[si] = -INFINITY;
    out->chi2[si] = 0.0;
    out->nfound[si] = 0;
    out->nholes[si] = 0;
    memset(&out->params[6 * si], 0, 6 * sizeof(double));
    memset(&out->cov[21 * si], 0, 21 * sizeof(double));
}

int orc_build_event(const orc_geom* g, const orc_params* P, const orc_tie* T,
                    const long long* layer_off, const double* xyz, const double* cov,
                    int n_seeds, const int* seed_hits, const int* seed_layers,
                    orc_build_out* out) {
    if (P->max_cands < 1 || P->max_cands > ORC_MAX_CANDS) return -1;
    evidx_t ev;
    build_index(g, layer_off, xyz, &ev);
    search_ws w;
    ws_init(&w);
    for (int si = 0; si < n_seeds; ++si) {
        clear_out(out, si);
        double h[9], V[18], pinit[6];
        for (int j = 0; j < 3; ++j) {
            long long id = seed_hits[3 * si + j];
            memcpy(&h[3 * j], &xyz[3 * id], 3 * sizeof(double));
            memcpy(&V[6 * j], &cov[6 * id], 6 * sizeof(double));
        }
        out->region[si] = -1;
        out->start[si] = -1;
        /* a seed hit measured on a module is used on its module's plane (Sec. 3.1) */
        const long long ids[3] = {seed_hits[3 * si], seed_hits[3 * si + 1], seed_hits[3 * si + 2]};
        if (!seed_fit(g, P->material, h, V, &seed_layers[3 * si], ids, w.cur[0].p, w.cur[0].C, pinit)) continue;
        int region = orc_select_region(g, w.cur[0].p);
        int start = plan_start(g, region, seed_layers[3 * si + 2]);
        out->region[si] = region;
        out->start[si] = start;
        if (start < 0) continue;
        search_track(g, P, T, layer_off, xyz, cov, &ev, &w, &g->plan[g->plan_off[region]],
                     g->plan_off[region + 1] - g->plan_off[region], start, 0, 3, out, si);
    }
    ws_free(&w);
    free_index(&ev);
    return 0;
}

/* Combinatorial backward search (Sec. 2.2: going inwards from the first known hit).  For each
 * track: its state on its innermost found layer first_layer (the backward fit's output there);
 * the region from its eta as for a seed; the region's plan in reverse order (inner layers last);
 * the search runs through the reversed plan's steps after first_layer with backward
 * propagation, from score 0 and no hits.  out->hits is indexed by the reversed plan's steps;
 * out->start gets the first step searched (-1: first_layer not in the plan or no inner layer). */
int orc_build_backward_event(const orc_geom* g, const orc_params* P, const orc_tie* T,
                             const long long* layer_off, const double* xyz, const double* cov,
                             int n, const double* p_start, const double* C_start, const int* first_layer,
                             orc_build_out* out) {
    if (P->max_cands < 1 || P->max_cands > ORC_MAX_CANDS) return -1;
    evidx_t ev;
    build_index(g, layer_off, xyz, &ev);
    search_ws w;
    ws_init(&w);
    int rplan[ORC_MAX_PLAN];
    for (int si = 0; si < n; ++si) {
        clear_out(out, si);
        memcpy(w.cur[0].p, &p_start[6 * si], 6 * sizeof(double));
        memcpy(w.cur[0].C, &C_start[21 * si], 21 * sizeof(double));
        int region = orc_select_region(g, w.cur[0].p);
        const int* plan = &g->plan[g->plan_off[region]];
        int plan_len = g->plan_off[region + 1] - g->plan_off[region];
        int start = -1;
        for (int k = 0; k < plan_len; ++k) {
            rplan[k] = plan[plan_len - 1 - k];
            if (rplan[k] == first_layer[si]) start = k + 1;
        }
        if (start >= plan_len) start = -1;
        out->region[si] = region;
        out->start[si] = start;
        if (start < 0) continue;
        search_track(g, P, T, layer_off, xyz, cov, &ev, &w, rplan, plan_len, start, 1, 0, out, si);
    }
    ws_free(&w);
    free_index(&ev);
    return 0;
}

/* ------------------------------------------------------------------ seed cleaning, duplicate removal */

/* Number of hit ids two lists have in common (entries < 0 are not hits; a list holds no id twice). */
static int shared_hits(const int* a, int na, const int* b, int nb) {
    int s = 0;
    for (int i = 0; i < na; ++i) {
        if (a[i] < 0) continue;
        for (int j = 0; j < nb; ++j)
            if (b[j] == a[i]) { ++s; break; }
    }
    return s;
}

static int count_hits(const int* a, int na) {
    int c = 0;
    for (int i = 0; i < na; ++i) c += a[i] >= 0;
    return c;
}

/* Items (rows of `width` hit ids, < 0 = none) that share a hit, found through a list of the
 * items on each hit: calls visit(t, u) once per ordered pair t != u sharing at least one hit. */
typedef void (*pair_fn)(int t, int u, void* ctx);
static void for_sharing_pairs(int n, int width, const int* hits, long long n_hits, pair_fn visit, void* ctx) {
    long long* cnt = (long long*)calloc((size_t)n_hits + 1, sizeof(long long));
    for (long long q = 0; q < (long long)n * width; ++q)
        if (hits[q] >= 0) cnt[hits[q] + 1]++;
    for (long long h = 0; h < n_hits; ++h) cnt[h + 1] += cnt[h];
    int* items = (int*)malloc(((size_t)cnt[n_hits] + 1) * sizeof(int));
    long long* fill = (long long*)malloc(((size_t)n_hits + 1) * sizeof(long long));
    memcpy(fill, cnt, ((size_t)n_hits + 1) * sizeof(long long));
    for (int t = 0; t < n; ++t)
        for (int i = 0; i < width; ++i) {
            int h = hits[(long long)t * width + i];
            if (h >= 0) items[fill[h]++] = t;
        }
    int* seen = (int*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
    for (int t = 0; t < n; ++t) seen[t] = -1;
    for (int t = 0; t < n; ++t) {
        for (int i = 0; i < width; ++i) {
            int h = hits[(long long)t * width + i];
            if (h < 0) continue;
            for (long long q = cnt[h]; q < cnt[h + 1]; ++q) {
                int u = items[q];
                if (u == t || seen[u] == t) continue;
                seen[u] = t;
                visit(t, u, ctx);
            }
        }
    }
    free(cnt); free(items); free(fill); free(seen);
}

typedef struct { const int* hits; int* keep; } seed_ctx;

static void seed_visit(int t, int u, void* vc) {
    seed_ctx* c = (seed_ctx*)vc;
    if (u < t && shared_hits(&c->hits[3 * (long long)t], 3, &c->hits[3 * (long long)u], 3) >= 2) c->keep[t] = 0;
}

/* Seed cleaning (Sec. 2.2: seeds are processed in parallel, so hits consumed by earlier tracks
 * cannot be masked).  Reading: a seed that shares at least two of its three hits with a seed of
 * lower index is dropped (keep = 0), each seed judged against all others (not transitively). */
void orc_clean_seeds(int n, const int* seed_hits, long long n_hits, int* keep) {
    for (int t = 0; t < n; ++t) keep[t] = 1;
    seed_ctx c = {seed_hits, keep};
    for_sharing_pairs(n, 3, seed_hits, n_hits, seed_visit, &c);
}

typedef struct {
    const int* hits;
    const double* score;
    int width;
    double frac;
    int* keep;
} dup_ctx;

static void dup_visit(int t, int u, void* vc) {
    dup_ctx* c = (dup_ctx*)vc;
    int better = c->score[u] > c->score[t] || (c->score[u] == c->score[t] && u < t);
    if (!better) return;
    const int* a = &c->hits[(long long)t * c->width];
    const int* b = &c->hits[(long long)u * c->width];
    int na = count_hits(a, c->width), nb = count_hits(b, c->width);
    int s = shared_hits(a, c->width, b, c->width);
    if ((double)s >= c->frac * (double)(na < nb ? na : nb)) c->keep[t] = 0;
}

/* Quality filter and duplicate removal (Sec. 2.2, on the resulting tracks).  Reading: a track
 * with fewer than min_hits hits is dropped; a track is dropped if a better track (higher score,
 * or equal score and lower index) shares at least frac x (the smaller hit count) of its hits,
 * each track judged against all others (not transitively).  hits: n x width hit ids, < 0 none. */
void orc_remove_duplicates(int n, int width, const int* hits, const double* score, long long n_hits,
                           int min_hits, double frac, int* keep) {
    for (int t = 0; t < n; ++t) keep[t] = count_hits(&hits[(long long)t * width], width) >= min_hits;
    dup_ctx c = {hits, score, width, frac, keep};
    int* k2 = (int*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
    for (int t = 0; t < n; ++t) k2[t] = 1;
    c.keep = k2;
    for_sharing_pairs(n, width, hits, n_hits, dup_visit, &c);
    for (int t = 0; t < n; ++t) keep[t] = keep[t] && k2[t];
    free(k2);
}
