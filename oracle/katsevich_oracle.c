/*
 * FP64 CPU oracle of the Katsevich helical cone-beam reconstruction operator.
 * TEST INFRASTRUCTURE ONLY -- see katsevich_oracle.h for the conventions.
 *
 * Every routine is a plain loop over the definition it cites; the only
 * numerical devices are bisection (PI-line endpoints, the psi-hat root) and
 * direct sums (Hilbert quadrature, backprojection quadrature).
 */
#include "katsevich_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------- helpers */
static double dlam(const or_geom *g) { return 2.0 * M_PI / (double)g->views_per_turn; }
static double hrise(const or_geom *g) { return g->P / (2.0 * M_PI); }
static double col_alpha(const or_geom *g, double c)
{
    return (c - 0.5 * (double)(g->n_cols - 1)) * g->d_alpha + g->alpha_offset;
}
static double row_w(const or_geom *g, double r)
{
    return (r - 0.5 * (double)(g->n_rows - 1)) * g->d_w + g->w_offset;
}
static int64_t n_psi(const or_geom *g) { return g->n_psi > 0 ? g->n_psi : 2 * g->n_rows; }
static int64_t pitch_slices(const or_geom *g) { return (int64_t)llround(g->P / g->dz); }

/* Largest distance from the axis of a corner of the volume's xy extent. */
double or_r_fov(const or_geom *g)
{
    double xa = fabs(g->x0 - 0.5 * g->dx), xb = fabs(g->x0 + ((double)g->nx - 0.5) * g->dx);
    double ya = fabs(g->y0 - 0.5 * g->dy), yb = fabs(g->y0 + ((double)g->ny - 0.5) * g->dy);
    double xm = xa > xb ? xa : xb, ym = ya > yb ? ya : yb;
    return sqrt(xm * xm + ym * ym);
}

/* Half fan angle alpha_m = arcsin(r / R) (Sec. II, forward height rebinning). */
double or_alpha_m(const or_geom *g) { return asin(or_r_fov(g) / g->R); }

/*
 * Largest pitch whose Tam-Danielsson window fits the detector rows.  On the
 * curved detector the TD boundaries are w_top(a) = (D h / R)(pi/2 - a)/cos a
 * and w_bot(a) = -(D h / R)(pi/2 + a)/cos a (= w_kappa at psi = +-pi/2 - a);
 * over |a| <= alpha_m the largest |w| is (D h / R)(pi/2 + alpha_m)/cos alpha_m,
 * which must not exceed the outermost row centre (Nr - 1)/2 * d_w.
 */
double or_fit_pitch(double R, double D, int64_t n_rows, double d_w, double alpha_m)
{
    double wmax = 0.5 * (double)(n_rows - 1) * d_w;
    double h = wmax * R * cos(alpha_m) / (D * (0.5 * M_PI + alpha_m));
    return 2.0 * M_PI * h;
}

/* kappa-line height, Sec. II Eq. (w_k); psi / tan(psi) -> 1 at psi = 0. */
double or_w_kappa(const or_geom *g, double alpha, double psi)
{
    double q = (psi == 0.0) ? 1.0 : psi / tan(psi);
    return g->D * hrise(g) / g->R * (psi * cos(alpha) + q * sin(alpha));
}

double or_w_td_top(const or_geom *g, double alpha)
{
    return g->D * hrise(g) / g->R * (0.5 * M_PI - alpha) / cos(alpha);
}

double or_w_td_bottom(const or_geom *g, double alpha)
{
    return -g->D * hrise(g) / g->R * (0.5 * M_PI + alpha) / cos(alpha);
}

/* bisection for a sign change of f on [a, b], to full FP64 resolution */
typedef double (*fn1)(const or_geom *, double, double, double);

static double kap_res(const or_geom *g, double alpha, double w, double psi)
{
    return or_w_kappa(g, alpha, psi) - w;
}

/* d/dpsi of (psi cos a + psi cot psi sin a), up to the factor D h / R */
static double kap_slope(const or_geom *g, double alpha, double unused, double psi)
{
    (void)g;
    (void)unused;
    double s = sin(psi);
    double q = (cos(psi) * s - psi) / (s * s); /* cot psi - psi / sin^2 psi */
    return cos(alpha) + sin(alpha) * q;
}

static double bisect(const or_geom *g, fn1 f, double alpha, double w, double a, double b)
{
    double fa = f(g, alpha, w, a);
    for (int it = 0; it < 400; ++it) {
        double m = 0.5 * (a + b);
        if (m == a || m == b) break;
        double fm = f(g, alpha, w, m);
        if (fm == 0.0) return m;
        if ((fm < 0.0) == (fa < 0.0)) {
            a = m;
            fa = fm;
        } else {
            b = m;
        }
    }
    return 0.5 * (a + b);
}

/*
 * psi-hat(alpha, w): the root psi of w = w_kappa(alpha, psi) with the smallest
 * |psi| (Sec. II, backward height rebinning), searched over the rebinning range
 * [-psi_max, psi_max].  Returns 0 when there is no root there.
 *
 * Bracketing uses the shape of s(psi) = psi cos a + psi cot(psi) sin a: for
 * a >= 0 its slope cos a + sin a (cot psi - psi/sin^2 psi) is > cos a > 0 for
 * psi < 0 and strictly decreasing on (0, pi), so s is increasing on the
 * negative side and increasing-then-decreasing (one turning point psi_t) on
 * the positive side.  w_kappa(-a, -psi) = -w_kappa(a, psi) gives a < 0.
 */
int or_psi_hat(const or_geom *g, double alpha, double w, double *psi)
{
    if (alpha < 0.0) {
        double p;
        int ok = or_psi_hat(g, -alpha, -w, &p);
        *psi = ok ? -p : 0.0;
        return ok;
    }
    const double pm = 0.5 * M_PI + or_alpha_m(g);
    double f0 = kap_res(g, alpha, w, 0.0);
    if (f0 == 0.0) {
        *psi = 0.0;
        return 1;
    }
    /* turning point on the positive side */
    double pt = pm;
    if (kap_slope(g, alpha, 0.0, pm) < 0.0) pt = bisect(g, kap_slope, alpha, 0.0, 1e-9, pm);
    double best = 0.0;
    int found = 0;
    if (f0 < 0.0) {
        /* w above s(0): rising branch [0, pt] only (the negative side stays below) */
        if (kap_res(g, alpha, w, pt) >= 0.0) {
            best = bisect(g, kap_res, alpha, w, 0.0, pt);
            found = 1;
        }
    } else {
        /* w below s(0): negative side (rising) and the falling branch [pt, pm] */
        if (kap_res(g, alpha, w, -pm) <= 0.0) {
            best = bisect(g, kap_res, alpha, w, -pm, 0.0);
            found = 1;
        }
        if (kap_res(g, alpha, w, pm) <= 0.0) {
            double r = bisect(g, kap_res, alpha, w, pt, pm);
            if (!found || fabs(r) < fabs(best)) best = r;
            found = 1;
        }
    }
    *psi = found ? best : 0.0;
    return found;
}

/*
 * Extremities lam_i < lam_o of the PI-line through x (Sec. II, Eq. (e1) and
 * the pre-calculating step).  With chord midpoint b and half-width d, x lies on
 * the segment a(b-d) -- a(b+d) iff
 *     cos d = (x cos(b+l0) + y sin(b+l0)) / R        (in-plane)
 *     (z - z0)/h = b + d * t / (R sin d),  t = -x sin(b+l0) + y cos(b+l0)
 * The residual of the second equation changes sign on [zeta - pi, zeta + pi]
 * (|d t / (R sin d)| < pi inside the helix), and the PI-line is unique for
 * r < R, so bisection on the plain definition gives the endpoints.
 */
static double pi_residual(const or_geom *g, double x, double y, double zeta, double b, double *dout)
{
    double ph = b + g->lambda0;
    double cd = (x * cos(ph) + y * sin(ph)) / g->R;
    double d = acos(cd);
    double t = -x * sin(ph) + y * cos(ph);
    if (dout) *dout = d;
    return b + d * t / (g->R * sin(d)) - zeta;
}

void or_pi_endpoints(const or_geom *g, double x, double y, double z, double *lam_i, double *lam_o)
{
    double zeta = (z - g->z0) / hrise(g);
    double a = zeta - M_PI, b = zeta + M_PI;
    double fa = pi_residual(g, x, y, zeta, a, NULL);
    for (int it = 0; it < 400; ++it) {
        double m = 0.5 * (a + b);
        if (m == a || m == b) break;
        double fm = pi_residual(g, x, y, zeta, m, NULL);
        if (fm == 0.0) {
            a = b = m;
            break;
        }
        if ((fm < 0.0) == (fa < 0.0)) {
            a = m;
            fa = fm;
        } else {
            b = m;
        }
    }
    double beta = 0.5 * (a + b), d;
    pi_residual(g, x, y, zeta, beta, &d);
    *lam_i = beta - d;
    *lam_o = beta + d;
}

/* v*, alpha*, w* of Sec. II, backprojection step (paper's formulas). */
void or_project_point(const or_geom *g, double lam, double x, double y, double z,
                      double *alpha, double *w, double *v)
{
    double ph = lam + g->lambda0;
    double vs = g->R - x * cos(ph) - y * sin(ph);
    double as = atan((-x * sin(ph) + y * cos(ph)) / vs);
    *v = vs;
    *alpha = as;
    *w = g->D * cos(as) / vs * (z - g->z0 - hrise(g) * lam);
}

/* ---------------------------------------------------------------- tables */
/*
 * Forward-rebinning table (pre-calculating step 1): for psi line l and the
 * half-grid column c + 1/2 (where the derivative lives), the fractional row
 * u = (w_kappa(alpha_{c+1/2}, psi_l) - w_0) / d_w, stored as floor(u) and
 * u - floor(u).  Layout [n_psi][n_cols - 1].
 */
void or_kappa_table(const or_geom *g, int32_t *idx, double *frac)
{
    const int64_t np = n_psi(g), nc1 = g->n_cols - 1;
    const double pm = 0.5 * M_PI + or_alpha_m(g), dpsi = 2.0 * pm / (double)(np - 1);
    const double w0 = row_w(g, 0.0);
    for (int64_t l = 0; l < np; ++l)
        for (int64_t c = 0; c < nc1; ++c) {
            double psi = -pm + (double)l * dpsi;
            double u = (or_w_kappa(g, col_alpha(g, (double)c + 0.5), psi) - w0) / g->d_w;
            double f = floor(u);
            idx[l * nc1 + c] = (int32_t)f;
            frac[l * nc1 + c] = u - f;
        }
}

/*
 * Backward-rebinning table (pre-calculating step 1): for detector sample
 * (r, c) the fractional psi index u = (psi_hat(alpha_c, w_r) + psi_max) / dpsi,
 * stored as floor(u) and u - floor(u); no root -> index -2, weight 0 (both
 * taps outside the psi grid, so g5 = 0).  Layout [n_rows][n_cols].
 */
void or_psi_table(const or_geom *g, int32_t *idx, double *frac)
{
    const int64_t np = n_psi(g), nr = g->n_rows, nc = g->n_cols;
    const double pm = 0.5 * M_PI + or_alpha_m(g), dpsi = 2.0 * pm / (double)(np - 1);
#pragma omp parallel for collapse(2) schedule(dynamic, 16)
    for (int64_t r = 0; r < nr; ++r)
        for (int64_t c = 0; c < nc; ++c) {
            double psi;
            int ok = or_psi_hat(g, col_alpha(g, (double)c), row_w(g, (double)r), &psi);
            if (!ok) {
                idx[r * nc + c] = -2;
                frac[r * nc + c] = 0.0;
                continue;
            }
            double u = (psi + pm) / dpsi;
            double f = floor(u);
            idx[r * nc + c] = (int32_t)f;
            frac[r * nc + c] = u - f;
        }
}

/*
 * PI table for one pitch (pre-calculating step 2): slices j = 0..N-1 at
 * z_first + j dz.  Filtered view k covers [l_k, l_{k+1}] around l_{k+1/2};
 * the midpoint rule over [lam_i, lam_o] weights it by the covered fraction
 *   omega_k = clamp((l_{k+1} - lam_i)/dl, 0, 1) * clamp((lam_o - l_k)/dl, 0, 1)
 * (reading: the paper's integral has hard limits; this is its midpoint-rule
 * discretisation).  With u = (lam - lambda_first)/dl:
 *   k0 = floor(u_i), w0 = k0 + 1 - u_i;  k1 = ceil(u_o) - 1, w1 = u_o - k1.
 * Hard mode: views with l_{k+1/2} in [lam_i, lam_o], weight 1:
 *   k0 = ceil(u_i - 1/2), k1 = floor(u_o - 1/2).
 * Layout [N][ny][nx].
 */
void or_pi_table(const or_geom *g, int32_t *k0, int32_t *k1, double *w0, double *w1,
                 double *lam_i, double *lam_o)
{
    const int64_t N = pitch_slices(g), nx = g->nx, ny = g->ny;
    const double dl = dlam(g);
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int64_t j = 0; j < N; ++j)
        for (int64_t iy = 0; iy < ny; ++iy)
            for (int64_t ix = 0; ix < nx; ++ix) {
                double x = g->x0 + (double)ix * g->dx, y = g->y0 + (double)iy * g->dy;
                double z = g->z_first + (double)j * g->dz;
                double li, lo;
                or_pi_endpoints(g, x, y, z, &li, &lo);
                int64_t o = (j * ny + iy) * nx + ix;
                lam_i[o] = li;
                lam_o[o] = lo;
                double ui = (li - g->lambda_first) / dl, uo = (lo - g->lambda_first) / dl;
                if (g->endpoint_mode == 0) {
                    double a = floor(ui), b = ceil(uo) - 1.0;
                    k0[o] = (int32_t)a;
                    k1[o] = (int32_t)b;
                    w0[o] = a + 1.0 - ui;
                    w1[o] = uo - b;
                } else {
                    k0[o] = (int32_t)ceil(ui - 0.5);
                    k1[o] = (int32_t)floor(uo - 0.5);
                    w0[o] = 1.0;
                    w1[o] = 1.0;
                }
            }
}

/* ---------------------------------------------------------------- filter */
/*
 * Step 1, derivative at constant direction, Sec. II Eq. (Deriv):
 * g1 = dg/dq + dg/dalpha at fixed w, on the half grid (l_{k+1/2}, alpha_{c+1/2})
 * by centred differences over the 2 x 2 cell (reading; the paper is silent).
 * sino [nv_in][Nr][Nc] -> g1 [nv_in-1][Nr][Nc-1].
 */
void or_derivative(const or_geom *g, const double *sino, int64_t nv_in, double *g1)
{
    const int64_t nr = g->n_rows, nc = g->n_cols, nc1 = nc - 1;
    const double a = 1.0 / (2.0 * dlam(g)), b = 1.0 / (2.0 * g->d_alpha);
#pragma omp parallel for collapse(2)
    for (int64_t k = 0; k < nv_in - 1; ++k)
        for (int64_t r = 0; r < nr; ++r)
            for (int64_t c = 0; c < nc1; ++c) {
                const double *p = sino + (k * nr + r) * nc, *q = sino + ((k + 1) * nr + r) * nc;
                double d_lam = (q[c] - p[c]) + (q[c + 1] - p[c + 1]);
                double d_alp = (p[c + 1] - p[c]) + (q[c + 1] - q[c]);
                g1[(k * nr + r) * nc1 + c] = a * d_lam + b * d_alp;
            }
}

/* Step 2, length-correction weight D / sqrt(D^2 + w^2), Sec. II Eq. (LW). */
void or_length_weight(const or_geom *g, double *g1, int64_t nv)
{
    const int64_t nr = g->n_rows, nc1 = g->n_cols - 1;
    for (int64_t k = 0; k < nv; ++k)
        for (int64_t r = 0; r < nr; ++r) {
            double w = row_w(g, (double)r);
            double s = g->D / sqrt(g->D * g->D + w * w);
            for (int64_t c = 0; c < nc1; ++c) g1[(k * nr + r) * nc1 + c] *= s;
        }
}

/*
 * Step 3, forward height rebinning, Sec. II Eq. (FR): g3(psi_l, c+1/2) =
 * g2 at row position w_kappa, linear in the row index; rows outside the
 * detector read as zero (reading).  g2 [nv][Nr][Nc-1] -> g3 [nv][n_psi][Nc-1].
 */
void or_forward_rebin(const or_geom *g, const int32_t *kidx, const double *kfrac,
                      const double *g2, int64_t nv, double *g3)
{
    const int64_t nr = g->n_rows, nc1 = g->n_cols - 1, np = n_psi(g);
#pragma omp parallel for collapse(2)
    for (int64_t k = 0; k < nv; ++k)
        for (int64_t l = 0; l < np; ++l)
            for (int64_t c = 0; c < nc1; ++c) {
                int64_t r = kidx[l * nc1 + c];
                double f = kfrac[l * nc1 + c];
                double lo = (r >= 0 && r < nr) ? g2[(k * nr + r) * nc1 + c] : 0.0;
                double hi = (r + 1 >= 0 && r + 1 < nr) ? g2[(k * nr + r + 1) * nc1 + c] : 0.0;
                g3[(k * np + l) * nc1 + c] = (1.0 - f) * lo + f * hi;
            }
}

/*
 * Step 4, Hilbert transform in alpha at constant psi, Sec. II Eq. (HF) with
 * h_H(s) = 1/(pi s) (Eq. (e4)): midpoint quadrature over the half-grid
 * columns (reading),
 *   g4(alpha_c) = sum_{c'} d_alpha g3(alpha_{c'+1/2}) / (pi sin(alpha_c - alpha_{c'+1/2})),
 * alpha_c - alpha_{c'+1/2} = (c - c' - 1/2) d_alpha; never singular.
 * g3 [nv][n_psi][Nc-1] -> g4 [nv][n_psi][Nc].
 */
/* kernel value d_alpha / (pi sin((n - 1/2) d_alpha)) for n = c - c', stored at n + nc - 2 */
static double *hilbert_kernel(const or_geom *g)
{
    const int64_t nc = g->n_cols;
    double *hk = malloc(sizeof(double) * (size_t)(2 * nc - 2));
    for (int64_t n = -(nc - 2); n <= nc - 1; ++n)
        hk[n + nc - 2] = g->d_alpha / (M_PI * sin(((double)n - 0.5) * g->d_alpha));
    return hk;
}

void or_hilbert(const or_geom *g, const double *g3, int64_t nv, double *g4)
{
    const int64_t nc = g->n_cols, nc1 = nc - 1, np = n_psi(g);
    double *hk = hilbert_kernel(g);
#pragma omp parallel for collapse(2)
    for (int64_t k = 0; k < nv; ++k)
        for (int64_t l = 0; l < np; ++l) {
            const double *in = g3 + (k * np + l) * nc1;
            double *out = g4 + (k * np + l) * nc;
            for (int64_t c = 0; c < nc; ++c) {
                double acc = 0.0;
                for (int64_t cp = 0; cp < nc1; ++cp) acc += hk[c - cp + nc - 2] * in[cp];
                out[c] = acc;
            }
        }
    free(hk);
}

/*
 * Step 5, backward height rebinning, Sec. II Eq. (BR): g5(r, c) = g4 at
 * psi_hat(alpha_c, w_r), linear in the psi index, zero outside the psi grid.
 * g4 [nv][n_psi][Nc] -> g5 [nv][Nr][Nc].
 */
void or_backward_rebin(const or_geom *g, const int32_t *pidx, const double *pfrac,
                       const double *g4, int64_t nv, double *g5)
{
    const int64_t nr = g->n_rows, nc = g->n_cols, np = n_psi(g);
#pragma omp parallel for collapse(2)
    for (int64_t k = 0; k < nv; ++k)
        for (int64_t r = 0; r < nr; ++r)
            for (int64_t c = 0; c < nc; ++c) {
                int64_t l = pidx[r * nc + c];
                double f = pfrac[r * nc + c];
                double lo = (l >= 0 && l < np) ? g4[(k * np + l) * nc + c] : 0.0;
                double hi = (l + 1 >= 0 && l + 1 < np) ? g4[(k * np + l + 1) * nc + c] : 0.0;
                g5[(k * nr + r) * nc + c] = (1.0 - f) * lo + f * hi;
            }
}

/* Step 6, post-cosine weight, Sec. II Eq. (PW). */
void or_post_cosine(const or_geom *g, double *g5, int64_t nv)
{
    const int64_t nr = g->n_rows, nc = g->n_cols;
    for (int64_t k = 0; k < nv; ++k)
        for (int64_t r = 0; r < nr; ++r)
            for (int64_t c = 0; c < nc; ++c) g5[(k * nr + r) * nc + c] *= cos(col_alpha(g, (double)c));
}

/* Steps 1-6 in the paper's order: sino [nv_in][Nr][Nc] -> gF [nv_in-1][Nr][Nc]. */
void or_filter(const or_geom *g, const int32_t *kidx, const double *kfrac,
               const int32_t *pidx, const double *pfrac,
               const double *sino, int64_t nv_in, double *gF)
{
    const int64_t nv = nv_in - 1, nr = g->n_rows, nc = g->n_cols, np = n_psi(g);
    double *g1 = malloc(sizeof(double) * (size_t)(nv * nr * (nc - 1)));
    double *g3 = malloc(sizeof(double) * (size_t)(nv * np * (nc - 1)));
    double *g4 = malloc(sizeof(double) * (size_t)(nv * np * nc));
    or_derivative(g, sino, nv_in, g1);
    or_length_weight(g, g1, nv);
    or_forward_rebin(g, kidx, kfrac, g1, nv, g3);
    or_hilbert(g, g3, nv, g4);
    or_backward_rebin(g, pidx, pfrac, g4, nv, gF);
    or_post_cosine(g, gF, nv);
    free(g1);
    free(g3);
    free(g4);
}

/* ---------------------------------------------------------- backprojection */
/* bilinear sample of one filtered view at fractional (column, row), zero outside */
static double sample(const or_geom *g, const double *view, double uc, double ur)
{
    const int64_t nr = g->n_rows, nc = g->n_cols;
    double fc0 = floor(uc), fr0 = floor(ur);
    int64_t c = (int64_t)fc0, r = (int64_t)fr0;
    double fc = uc - fc0, fr = ur - fr0;
    double v00 = 0, v01 = 0, v10 = 0, v11 = 0;
    if (r >= 0 && r < nr && c >= 0 && c < nc) v00 = view[r * nc + c];
    if (r >= 0 && r < nr && c + 1 >= 0 && c + 1 < nc) v01 = view[r * nc + c + 1];
    if (r + 1 >= 0 && r + 1 < nr && c >= 0 && c < nc) v10 = view[(r + 1) * nc + c];
    if (r + 1 >= 0 && r + 1 < nr && c + 1 >= 0 && c + 1 < nc) v11 = view[(r + 1) * nc + c + 1];
    return (1.0 - fr) * ((1.0 - fc) * v00 + fc * v01) + fr * ((1.0 - fc) * v10 + fc * v11);
}

/* view window of voxel (ix, iy, s): table slice j = s mod N, shifted m pitches */
static void voxel_window(const or_geom *g, const int32_t *k0, const int32_t *k1,
                         const double *w0, const double *w1, int64_t ix, int64_t iy, int64_t s,
                         int64_t *ka, int64_t *kb, double *wa, double *wb)
{
    const int64_t N = pitch_slices(g);
    int64_t j = s % N, m = s / N;
    int64_t o = (j * g->ny + iy) * g->nx + ix;
    *ka = (int64_t)k0[o] + m * g->views_per_turn;
    *kb = (int64_t)k1[o] + m * g->views_per_turn;
    *wa = w0[o];
    *wb = w1[o];
}

/*
 * Step 7, backprojection (Sec. II, backprojection step and the pitch-by-pitch
 * reconstruction step): f(x) = (1/2pi) sum_k omega_k dl g^F(l_{k+1/2},
 * alpha*, w*) / v*, bilinear in (alpha, w) on the detector grid, over the
 * voxel's view window [ka, kb] with end weights wa, wb.
 */
static double bp_voxel(const or_geom *g, const double *gF, int64_t gf_v0, int64_t gf_nv,
                       int64_t ix, int64_t iy, int64_t s, int64_t ka, int64_t kb, double wa,
                       double wb, int *err)
{
    const int64_t nr = g->n_rows, nc = g->n_cols;
    const double dl = dlam(g), a0 = col_alpha(g, 0.0), wr0 = row_w(g, 0.0);
    if (ka < gf_v0 || kb >= gf_v0 + gf_nv) {
        *err = 1;
        return 0.0;
    }
    double x = g->x0 + (double)ix * g->dx, y = g->y0 + (double)iy * g->dy;
    double z = g->z_first + (double)s * g->dz;
    double acc = 0.0;
    for (int64_t k = ka; k <= kb; ++k) {
        double lam = g->lambda_first + ((double)k + 0.5) * dl;
        double alpha, w, v;
        or_project_point(g, lam, x, y, z, &alpha, &w, &v);
        double om = (k == ka ? wa : 1.0) * (k == kb ? wb : 1.0);
        double val = sample(g, gF + (k - gf_v0) * nr * nc, (alpha - a0) / g->d_alpha, (w - wr0) / g->d_w);
        acc += om * val / v;
    }
    return acc * dl / (2.0 * M_PI);
}

int or_backproject(const or_geom *g, const int32_t *k0, const int32_t *k1,
                   const double *w0, const double *w1,
                   const double *gF, int64_t gf_v0, int64_t gf_nv, double *vol)
{
    int err = 0;
    const int64_t nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for collapse(2) schedule(dynamic, 1) reduction(| : err)
    for (int64_t s = 0; s < nz; ++s)
        for (int64_t iy = 0; iy < ny; ++iy)
            for (int64_t ix = 0; ix < nx; ++ix) {
                int e = 0;
                int64_t ka, kb;
                double wa, wb;
                voxel_window(g, k0, k1, w0, w1, ix, iy, s, &ka, &kb, &wa, &wb);
                vol[(s * ny + iy) * nx + ix] = bp_voxel(g, gF, gf_v0, gf_nv, ix, iy, s, ka, kb, wa, wb, &e);
                err |= e;
            }
    return err ? -1 : 0;
}

/*
 * View windows of individual voxels ijk[n][3] = (ix, iy, s) from the PI-line
 * endpoints of their pitch-table point (x, y, z_first + (s mod N) dz), shifted
 * by (s div N) turns -- the same rule as or_pi_table, without the table.
 */
void or_pi_window_points(const or_geom *g, int64_t n, const int64_t *ijk,
                         int64_t *ka, int64_t *kb, double *wa, double *wb)
{
    const int64_t N = pitch_slices(g);
    const double dl = dlam(g);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < n; ++p) {
        int64_t ix = ijk[3 * p], iy = ijk[3 * p + 1], s = ijk[3 * p + 2];
        int64_t j = s % N, m = s / N;
        double li, lo;
        or_pi_endpoints(g, g->x0 + (double)ix * g->dx, g->y0 + (double)iy * g->dy,
                        g->z_first + (double)j * g->dz, &li, &lo);
        double ui = (li - g->lambda_first) / dl, uo = (lo - g->lambda_first) / dl;
        int64_t sh = m * g->views_per_turn;
        if (g->endpoint_mode == 0) {
            double a = floor(ui), b = ceil(uo) - 1.0;
            ka[p] = (int64_t)a + sh;
            kb[p] = (int64_t)b + sh;
            wa[p] = a + 1.0 - ui;
            wb[p] = uo - b;
        } else {
            ka[p] = (int64_t)ceil(ui - 0.5) + sh;
            kb[p] = (int64_t)floor(uo - 0.5) + sh;
            wa[p] = 1.0;
            wb[p] = 1.0;
        }
    }
}

int or_backproject_points(const or_geom *g, const double *gF, int64_t gf_v0, int64_t gf_nv,
                          int64_t n, const int64_t *ijk, const int64_t *ka, const int64_t *kb,
                          const double *wa, const double *wb, double *out)
{
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (int64_t p = 0; p < n; ++p) {
        int e = 0;
        out[p] = bp_voxel(g, gF, gf_v0, gf_nv, ijk[3 * p], ijk[3 * p + 1], ijk[3 * p + 2],
                          ka[p], kb[p], wa[p], wb[p], &e);
        err |= e;
    }
    return err ? -1 : 0;
}

/*
 * Transpose of step 7: every (voxel, view) term of the backprojection sum
 * sends its weight times the voxel value to the four bilinear taps.  Views are
 * distributed over threads so each thread owns its output view.
 */
int or_backproject_adjoint(const or_geom *g, const int32_t *k0, const int32_t *k1,
                           const double *w0, const double *w1,
                           const double *vol, double *gF, int64_t gf_v0, int64_t gf_nv)
{
    const int64_t nr = g->n_rows, nc = g->n_cols, nx = g->nx, ny = g->ny, nz = g->nz;
    const int64_t N = pitch_slices(g);
    const double dl = dlam(g), a0 = col_alpha(g, 0.0), wr0 = row_w(g, 0.0);
    int err = 0;
    /* per table slice: smallest first view and largest last view */
    int64_t *jlo = malloc(sizeof(int64_t) * (size_t)N), *jhi = malloc(sizeof(int64_t) * (size_t)N);
    for (int64_t j = 0; j < N; ++j) {
        int64_t lo = INT64_MAX, hi = INT64_MIN;
        for (int64_t o = j * nx * ny; o < (j + 1) * nx * ny; ++o) {
            if (k0[o] < lo) lo = k0[o];
            if (k1[o] > hi) hi = k1[o];
        }
        jlo[j] = lo;
        jhi[j] = hi;
    }
    for (int64_t s = 0; s < nz; ++s) {
        int64_t j = s % N, m = s / N;
        if (jlo[j] + m * g->views_per_turn < gf_v0 || jhi[j] + m * g->views_per_turn >= gf_v0 + gf_nv) err = 1;
    }
    memset(gF, 0, sizeof(double) * (size_t)(gf_nv * nr * nc));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t kv = 0; kv < gf_nv; ++kv) {
        int64_t k = kv + gf_v0;
        double *view = gF + kv * nr * nc;
        double lam = g->lambda_first + ((double)k + 0.5) * dl;
        for (int64_t s = 0; s < nz; ++s) {
            int64_t j = s % N, m = s / N;
            if (k < jlo[j] + m * g->views_per_turn || k > jhi[j] + m * g->views_per_turn) continue;
            for (int64_t iy = 0; iy < ny; ++iy)
                for (int64_t ix = 0; ix < nx; ++ix) {
                    int64_t ka, kb;
                    double wa, wb;
                    voxel_window(g, k0, k1, w0, w1, ix, iy, s, &ka, &kb, &wa, &wb);
                    if (k < ka || k > kb) continue;
                    double x = g->x0 + (double)ix * g->dx, y = g->y0 + (double)iy * g->dy;
                    double z = g->z_first + (double)s * g->dz;
                    double alpha, w, v;
                    or_project_point(g, lam, x, y, z, &alpha, &w, &v);
                    double om = (k == ka ? wa : 1.0) * (k == kb ? wb : 1.0);
                    double wt = om / v * dl / (2.0 * M_PI) * vol[(s * ny + iy) * nx + ix];
                    double uc = (alpha - a0) / g->d_alpha, ur = (w - wr0) / g->d_w;
                    double fc0 = floor(uc), fr0 = floor(ur);
                    int64_t c = (int64_t)fc0, r = (int64_t)fr0;
                    double fc = uc - fc0, fr = ur - fr0;
                    if (r >= 0 && r < nr && c >= 0 && c < nc) view[r * nc + c] += wt * (1 - fr) * (1 - fc);
                    if (r >= 0 && r < nr && c + 1 >= 0 && c + 1 < nc) view[r * nc + c + 1] += wt * (1 - fr) * fc;
                    if (r + 1 >= 0 && r + 1 < nr && c >= 0 && c < nc) view[(r + 1) * nc + c] += wt * fr * (1 - fc);
                    if (r + 1 >= 0 && r + 1 < nr && c + 1 >= 0 && c + 1 < nc)
                        view[(r + 1) * nc + c + 1] += wt * fr * fc;
                }
        }
    }
    free(jlo);
    free(jhi);
    return err ? -1 : 0;
}

/*
 * Transpose of steps 1-6, applied in reverse order:
 * gF [nv][Nr][Nc] -> sino [nv+1][Nr][Nc].
 */
void or_filter_adjoint(const or_geom *g, const int32_t *kidx, const double *kfrac,
                       const int32_t *pidx, const double *pfrac,
                       const double *gF, int64_t nv, double *sino)
{
    const int64_t nr = g->n_rows, nc = g->n_cols, nc1 = nc - 1, np = n_psi(g);
    const double da = g->d_alpha;
    double *hk = hilbert_kernel(g);
    double *g1 = calloc((size_t)(nv * nr * nc1), sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nv; ++k) {
        double *g4 = calloc((size_t)(np * nc), sizeof(double));
        double *g3 = calloc((size_t)(np * nc1), sizeof(double));
        /* step 6^T and 5^T: cosine, then scatter each (r, c) to psi lines l, l+1 */
        for (int64_t r = 0; r < nr; ++r)
            for (int64_t c = 0; c < nc; ++c) {
                double v = cos(col_alpha(g, (double)c)) * gF[(k * nr + r) * nc + c];
                int64_t l = pidx[r * nc + c];
                double f = pfrac[r * nc + c];
                if (l >= 0 && l < np) g4[l * nc + c] += (1.0 - f) * v;
                if (l + 1 >= 0 && l + 1 < np) g4[(l + 1) * nc + c] += f * v;
            }
        /* step 4^T: transposed Hilbert quadrature */
        for (int64_t l = 0; l < np; ++l)
            for (int64_t cp = 0; cp < nc1; ++cp) {
                double acc = 0.0;
                for (int64_t c = 0; c < nc; ++c) acc += hk[c - cp + nc - 2] * g4[l * nc + c];
                g3[l * nc1 + cp] = acc;
            }
        /* step 3^T: scatter psi lines back to detector rows */
        double *o = g1 + k * nr * nc1;
        for (int64_t l = 0; l < np; ++l)
            for (int64_t c = 0; c < nc1; ++c) {
                int64_t r = kidx[l * nc1 + c];
                double f = kfrac[l * nc1 + c], v = g3[l * nc1 + c];
                if (r >= 0 && r < nr) o[r * nc1 + c] += (1.0 - f) * v;
                if (r + 1 >= 0 && r + 1 < nr) o[(r + 1) * nc1 + c] += f * v;
            }
        /* step 2^T: diagonal */
        for (int64_t r = 0; r < nr; ++r) {
            double w = row_w(g, (double)r), s = g->D / sqrt(g->D * g->D + w * w);
            for (int64_t c = 0; c < nc1; ++c) o[r * nc1 + c] *= s;
        }
        free(g3);
        free(g4);
    }
    /* step 1^T: each sample gathers the 2 x 2 half-grid cells that used it */
    const double a = 1.0 / (2.0 * dlam(g)), b = 1.0 / (2.0 * da);
#pragma omp parallel for collapse(2)
    for (int64_t k = 0; k <= nv; ++k)
        for (int64_t r = 0; r < nr; ++r)
            for (int64_t c = 0; c < nc; ++c) {
                double acc = 0.0;
                /* cell (k', c') uses sample (k'+dk, c'+dc) with coefficient
                   (dk ? a : -a) + (dc ? b : -b) */
                for (int dk = 0; dk < 2; ++dk)
                    for (int dc = 0; dc < 2; ++dc) {
                        int64_t kp = k - dk, cp = c - dc;
                        if (kp < 0 || kp >= nv || cp < 0 || cp >= nc1) continue;
                        double coef = (dk ? a : -a) + (dc ? b : -b);
                        acc += coef * g1[(kp * nr + r) * nc1 + cp];
                    }
                sino[(k * nr + r) * nc + c] = acc;
            }
    free(g1);
    free(hk);
}

/* ---------------------------------------------------------------- extents */
/*
 * Sec. II Eq. (maxvalue): lam_min / lam_max over the PI endpoints of one
 * pitch, and alpha / w extremes of (alpha*, w*) over the views each voxel of
 * the pitch actually backprojects (reading: the voxel's own PI views, sampled
 * at the filtered view angles).  out = {lam_min, lam_max, a_min, a_max, w_min, w_max}.
 */
void or_extents(const or_geom *g, const int32_t *k0, const int32_t *k1,
                const double *lam_i, const double *lam_o, double out[6])
{
    const int64_t N = pitch_slices(g), nx = g->nx, ny = g->ny;
    const double dl = dlam(g);
    double lmin = INFINITY, lmax = -INFINITY, amin = INFINITY, amax = -INFINITY;
    double wmin = INFINITY, wmax = -INFINITY;
#pragma omp parallel for collapse(2) reduction(min : lmin, amin, wmin) reduction(max : lmax, amax, wmax)
    for (int64_t j = 0; j < N; ++j)
        for (int64_t iy = 0; iy < ny; ++iy)
            for (int64_t ix = 0; ix < nx; ++ix) {
                int64_t o = (j * ny + iy) * nx + ix;
                if (lam_i[o] < lmin) lmin = lam_i[o];
                if (lam_o[o] > lmax) lmax = lam_o[o];
                double x = g->x0 + (double)ix * g->dx, y = g->y0 + (double)iy * g->dy;
                double z = g->z_first + (double)j * g->dz;
                for (int64_t k = k0[o]; k <= k1[o]; ++k) {
                    double alpha, w, v;
                    or_project_point(g, g->lambda_first + ((double)k + 0.5) * dl, x, y, z, &alpha, &w, &v);
                    if (alpha < amin) amin = alpha;
                    if (alpha > amax) amax = alpha;
                    if (w < wmin) wmin = w;
                    if (w > wmax) wmax = w;
                }
            }
    out[0] = lmin;
    out[1] = lmax;
    out[2] = amin;
    out[3] = amax;
    out[4] = wmin;
    out[5] = wmax;
}

/* Number of (voxel, view) terms of the whole volume's backprojection. */
int64_t or_update_count(const or_geom *g, const int32_t *k0, const int32_t *k1)
{
    const int64_t N = pitch_slices(g), nxy = g->nx * g->ny;
    int64_t total = 0;
    for (int64_t j = 0; j < N; ++j) {
        int64_t reps = (j < g->nz) ? (g->nz - 1 - j) / N + 1 : 0;
        int64_t sum = 0;
        for (int64_t o = j * nxy; o < (j + 1) * nxy; ++o) sum += (int64_t)k1[o] - k0[o] + 1;
        total += reps * sum;
    }
    return total;
}
