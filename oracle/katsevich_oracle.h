/*
 * FP64 CPU oracle of the Katsevich helical cone-beam reconstruction operator
 * (curved detector), computed pitch by pitch.
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path: only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no source, header, table or constant with the CUDA library.
 *
 * Conventions (the paper's Section II; readings of silent points noted):
 *   helix       a(l) = (R cos(l+l0), R sin(l+l0), z0 + h l),  h = P / (2 pi)
 *   views       l_k = lambda_first + k * dl,  dl = 2 pi / views_per_turn
 *   filtered    g^F lives on the half view grid l_{k+1/2} (reading: centred
 *               differences of the derivative step), k = 0 .. n_views-2
 *   columns     alpha_c = (c - (Nc-1)/2) d_alpha + alpha_offset
 *   rows        w_r     = (r - (Nr-1)/2) d_w     + w_offset
 *   voxels      (x0 + i dx, y0 + j dy, z_first + s dz), stored vol[s][j][i]
 *   psi grid    psi_l = -psi_max + l * 2 psi_max / (n_psi - 1),
 *               psi_max = pi/2 + alpha_m, alpha_m = asin(r_fov / R),
 *               r_fov = largest distance of a volume xy corner (voxel edges)
 *   pitch       N = P / dz slices per pitch (must be an integer); the PI table
 *               covers slices j = 0..N-1 and slice s = j + m N reuses table j
 *               with its view indices shifted by m * views_per_turn.
 */
#ifndef KATSEVICH_ORACLE_H
#define KATSEVICH_ORACLE_H
#include <stdint.h>

typedef struct or_geom {
    double R, D, P, lambda0, z0, lambda_first;
    int64_t views_per_turn, n_views;
    int64_t n_rows, n_cols;
    double d_alpha, alpha_offset, d_w, w_offset;
    int64_t nx, ny, nz;
    double dx, dy, dz, x0, y0, z_first;
    int64_t n_psi;
    int64_t endpoint_mode; /* 0 = fractional end weights, 1 = hard indicator */
} or_geom;

double or_r_fov(const or_geom *g);
double or_alpha_m(const or_geom *g);
double or_fit_pitch(double R, double D, int64_t n_rows, double d_w, double alpha_m);
double or_w_kappa(const or_geom *g, double alpha, double psi);
double or_w_td_top(const or_geom *g, double alpha);
double or_w_td_bottom(const or_geom *g, double alpha);
int or_psi_hat(const or_geom *g, double alpha, double w, double *psi);
void or_pi_endpoints(const or_geom *g, double x, double y, double z, double *lam_i, double *lam_o);
void or_project_point(const or_geom *g, double lam, double x, double y, double z,
                      double *alpha, double *w, double *v);

void or_kappa_table(const or_geom *g, int32_t *idx, double *frac);
void or_psi_table(const or_geom *g, int32_t *idx, double *frac);
void or_pi_table(const or_geom *g, int32_t *k0, int32_t *k1, double *w0, double *w1,
                 double *lam_i, double *lam_o);

void or_derivative(const or_geom *g, const double *sino, int64_t nv_in, double *g1);
void or_length_weight(const or_geom *g, double *g1, int64_t nv);
void or_forward_rebin(const or_geom *g, const int32_t *kidx, const double *kfrac,
                      const double *g2, int64_t nv, double *g3);
void or_hilbert(const or_geom *g, const double *g3, int64_t nv, double *g4);
void or_backward_rebin(const or_geom *g, const int32_t *pidx, const double *pfrac,
                       const double *g4, int64_t nv, double *g5);
void or_post_cosine(const or_geom *g, double *g5, int64_t nv);
void or_filter(const or_geom *g, const int32_t *kidx, const double *kfrac,
               const int32_t *pidx, const double *pfrac,
               const double *sino, int64_t nv_in, double *gF);

int or_backproject(const or_geom *g, const int32_t *k0, const int32_t *k1,
                   const double *w0, const double *w1,
                   const double *gF, int64_t gf_v0, int64_t gf_nv, double *vol);
void or_pi_window_points(const or_geom *g, int64_t n, const int64_t *ijk,
                         int64_t *ka, int64_t *kb, double *wa, double *wb);
int or_backproject_points(const or_geom *g, const double *gF, int64_t gf_v0, int64_t gf_nv,
                          int64_t n, const int64_t *ijk, const int64_t *ka, const int64_t *kb,
                          const double *wa, const double *wb, double *out);
int or_backproject_adjoint(const or_geom *g, const int32_t *k0, const int32_t *k1,
                           const double *w0, const double *w1,
                           const double *vol, double *gF, int64_t gf_v0, int64_t gf_nv);
void or_filter_adjoint(const or_geom *g, const int32_t *kidx, const double *kfrac,
                       const int32_t *pidx, const double *pfrac,
                       const double *gF, int64_t nv, double *sino);

void or_extents(const or_geom *g, const int32_t *k0, const int32_t *k1,
                const double *lam_i, const double *lam_o, double out[6]);
int64_t or_update_count(const or_geom *g, const int32_t *k0, const int32_t *k1);
/* data simulation (simulate_oracle.c): the paper's Sec. III-C data generation */
void or_ray(const or_geom *g, int64_t k, int64_t r, int64_t c, double *a, double *d);
void or_project(const or_geom *g, const double *vol, int64_t v0, int64_t nv, double *sino);
void or_sparse_upsample(const or_geom *g, const double *sino, int64_t nv, int64_t keep, double *out);
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
int64_t or_poisson(double lam, uint64_t seed, int64_t i);
double or_gaussian(uint64_t seed, int64_t i);
void or_add_noise(const double *g_up, int64_t n, double I0, double mean, double var, uint64_t seed,
                  double *g_in, int64_t *counts, double *M_out);

#endif
