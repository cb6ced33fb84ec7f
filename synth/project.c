/*
 * Seeded synthetic data for helical cone-beam CT: exact line integrals of
 * ellipsoid phantoms along the rays of a helical scan with a curved
 * (cylindrical) detector, in FP64.
 *
 * This file is the acquisition model only.  It holds none of the
 * reconstruction method's arithmetic and is shared, as an input generator,
 * by the oracle tests and the GPU tests/benchmark.
 *
 * Scan geometry (the paper's Section II, helix equation and the curved
 * detector of the backprojection step):
 *   source    a(l) = (R cos(l+l0), R sin(l+l0), z0 + P l / (2 pi))
 *   e_u(l)    = (-sin(l+l0),  cos(l+l0), 0)
 *   e_v(l)    = (-cos(l+l0), -sin(l+l0), 0)      (source -> axis)
 *   ray dir   ~ D sin(alpha) e_u + D cos(alpha) e_v + w e_z
 *   view k at l = lambda_first + k * dlam
 *   column c at alpha = (c - (Nc-1)/2) d_alpha + alpha_offset
 *   row r    at w     = (r - (Nr-1)/2) d_w     + w_offset
 *
 * Ellipsoid i is the set {p : (p - c_i)^T M_i (p - c_i) <= 1} with density
 * rho_i; each record holds 14 doubles:
 *   c (3), M row-major (9), rho (1), bounding radius (1).
 * The line integral of the indicator along the unit direction d from s is the
 * chord length 2 sqrt(B^2 - A C) / A, with A = d^T M d, B = d^T M (s - c),
 * C = (s - c)^T M (s - c) - 1.
 */
#include <math.h>
#include <stdint.h>

typedef struct synth_scan {
    double R, D, P, lambda0, z0, lambda_first, dlam;
    int64_t n_rows, n_cols;
    double d_alpha, alpha_offset, d_w, w_offset;
} synth_scan;

static double chord(const double *e, const double s[3], const double d[3])
{
    double p[3] = {s[0] - e[0], s[1] - e[1], s[2] - e[2]};
    /* quick reject: distance from the centre to the line vs bounding radius */
    double t = p[0] * d[0] + p[1] * d[1] + p[2] * d[2];
    double q0 = p[0] - t * d[0], q1 = p[1] - t * d[1], q2 = p[2] - t * d[2];
    double rb = e[13];
    if (q0 * q0 + q1 * q1 + q2 * q2 > rb * rb) return 0.0;
    const double *M = e + 3;
    double Md[3], Mp[3];
    for (int i = 0; i < 3; ++i) {
        Md[i] = M[3 * i] * d[0] + M[3 * i + 1] * d[1] + M[3 * i + 2] * d[2];
        Mp[i] = M[3 * i] * p[0] + M[3 * i + 1] * p[1] + M[3 * i + 2] * p[2];
    }
    double A = d[0] * Md[0] + d[1] * Md[1] + d[2] * Md[2];
    double B = d[0] * Mp[0] + d[1] * Mp[1] + d[2] * Mp[2];
    double C = p[0] * Mp[0] + p[1] * Mp[1] + p[2] * Mp[2] - 1.0;
    double disc = B * B - A * C;
    if (disc <= 0.0) return 0.0;
    return e[12] * 2.0 * sqrt(disc) / A;
}

/* One ray's direction for view angle l and detector position (alpha, w). */
void synth_ray(const synth_scan *g, double l, double alpha, double w,
               double src[3], double dir[3])
{
    double phi = l + g->lambda0;
    double cp = cos(phi), sp = sin(phi);
    src[0] = g->R * cp;
    src[1] = g->R * sp;
    src[2] = g->z0 + g->P * l / (2.0 * M_PI);
    double sa = sin(alpha), ca = cos(alpha);
    double du = g->D * sa, dv = g->D * ca;
    double d0 = -du * sp - dv * cp;
    double d1 = du * cp - dv * sp;
    double d2 = w;
    double n = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    dir[0] = d0 / n;
    dir[1] = d1 / n;
    dir[2] = d2 / n;
}

/* Sinogram for views [v_begin, v_begin + n_views): out[v][row][col]. */
void synth_project(const synth_scan *g, const double *ell, int64_t n_ell,
                   int64_t v_begin, int64_t n_views, double *out)
{
    const int64_t nr = g->n_rows, nc = g->n_cols;
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int64_t v = 0; v < n_views; ++v) {
        for (int64_t r = 0; r < nr; ++r) {
            double l = g->lambda_first + (double)(v_begin + v) * g->dlam;
            double w = ((double)r - 0.5 * (double)(nr - 1)) * g->d_w + g->w_offset;
            double *row = out + (v * nr + r) * nc;
            for (int64_t c = 0; c < nc; ++c) {
                double alpha = ((double)c - 0.5 * (double)(nc - 1)) * g->d_alpha + g->alpha_offset;
                double s[3], d[3];
                synth_ray(g, l, alpha, w, s, d);
                double acc = 0.0;
                for (int64_t i = 0; i < n_ell; ++i) acc += chord(ell + 14 * i, s, d);
                row[c] = acc;
            }
        }
    }
}

/* Line integrals along arbitrary rays (src, unit dir), n rays. */
void synth_project_rays(const double *ell, int64_t n_ell, int64_t n,
                        const double *src, const double *dir, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        double acc = 0.0;
        for (int64_t i = 0; i < n_ell; ++i) acc += chord(ell + 14 * i, src + 3 * k, dir + 3 * k);
        out[k] = acc;
    }
}

/* Phantom density at points (sum of rho over the ellipsoids containing p). */
void synth_density(const double *ell, int64_t n_ell, int64_t n, const double *pts, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        const double *q = pts + 3 * k;
        double acc = 0.0;
        for (int64_t i = 0; i < n_ell; ++i) {
            const double *e = ell + 14 * i;
            double p[3] = {q[0] - e[0], q[1] - e[1], q[2] - e[2]};
            const double *M = e + 3;
            double v = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) v += p[a] * M[3 * a + b] * p[b];
            if (v <= 1.0) acc += e[12];
        }
        out[k] = acc;
    }
}
