/*
 * FP64 CPU oracle of the data-simulation steps that produce the network's
 * input sinograms (the paper's Sec. III-C "Data generation"):
 *   1. helical projection of a voxel volume: for every detector sample the
 *      line integral of the piecewise-constant voxel function along the ray
 *      from the source a(l) through the detector point (reading: voxels are
 *      cubes of constant value; the integral is exact for that function);
 *   2. sparse detector: keep every keep-th column, then linear interpolation
 *      back to the full column grid (reading: columns beyond the last kept
 *      one take its value);
 *   3. "Gaussian+Poisson" noise: counts I0 exp(-g/M), M = max g; a Poisson
 *      draw of the counts plus N(mean, var) (reading: the paper's
 *      "g + poisson(g)" is the Poisson draw of g, as in the noise model it
 *      cites), then log(I0 / counts) M (counts floored at 1).
 *
 * TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no source, header,
 * table or constant with the CUDA library.  Random numbers come from the
 * counter-based generator Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC 2011), written here from
 * its published definition; Poisson variates use the transformed rejection
 * method PTRS (Hormann, "The transformed rejection method for generating
 * Poisson random variables", 1993) for means >= 10 and multiplication of
 * uniforms below that.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include "katsevich_oracle.h"

static void ray_of(const or_geom *g, int64_t k, int64_t r, int64_t c, double a[3], double d[3])
{
    const double dl = 2.0 * M_PI / (double)g->views_per_turn;
    const double l = g->lambda_first + (double)k * dl;
    const double ph = l + g->lambda0;
    const double h = g->P / (2.0 * M_PI);
    const double alpha = ((double)c - 0.5 * (double)(g->n_cols - 1)) * g->d_alpha + g->alpha_offset;
    const double w = ((double)r - 0.5 * (double)(g->n_rows - 1)) * g->d_w + g->w_offset;
    const double eu[3] = {-sin(ph), cos(ph), 0.0};
    const double ev[3] = {-cos(ph), -sin(ph), 0.0};
    a[0] = g->R * cos(ph);
    a[1] = g->R * sin(ph);
    a[2] = g->z0 + h * l;
    for (int i = 0; i < 3; ++i) d[i] = g->D * sin(alpha) * eu[i] + g->D * cos(alpha) * ev[i];
    d[2] += w;
}

void or_ray(const or_geom *g, int64_t k, int64_t r, int64_t c, double *a, double *d) { ray_of(g, k, r, c, a, d); }

static int cmp_double(const void *p, const void *q)
{
    const double a = *(const double *)p, b = *(const double *)q;
    return (a > b) - (a < b);
}

/* Line integral of the voxel function along a + t d, t in R: every crossing of
 * a voxel face plane is listed, sorted, and each piece between neighbouring
 * crossings contributes (its length) x (the value of the voxel holding its
 * midpoint). */
static double ray_integral(const or_geom *g, const double *vol, const double a[3], const double d[3], double *ts)
{
    const int64_t n[3] = {g->nx, g->ny, g->nz};
    const double s[3] = {g->dx, g->dy, g->dz};
    const double o[3] = {g->x0, g->y0, g->z_first};
    int64_t m = 0;
    for (int ax = 0; ax < 3; ++ax) {
        if (d[ax] == 0.0) continue;
        for (int64_t i = 0; i <= n[ax]; ++i) ts[m++] = (o[ax] + ((double)i - 0.5) * s[ax] - a[ax]) / d[ax];
    }
    qsort(ts, (size_t)m, sizeof(double), cmp_double);
    const double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double sum = 0.0;
    for (int64_t q = 0; q + 1 < m; ++q) {
        const double t0 = ts[q], t1 = ts[q + 1];
        if (!(t1 > t0)) continue;
        const double tm = 0.5 * (t0 + t1);
        int64_t idx[3];
        int inside = 1;
        for (int ax = 0; ax < 3; ++ax) {
            const double u = (a[ax] + tm * d[ax] - o[ax]) / s[ax] + 0.5;
            const double f = floor(u);
            if (f < 0.0 || f >= (double)n[ax]) inside = 0;
            idx[ax] = (int64_t)f;
        }
        if (!inside) continue;
        sum += (t1 - t0) * len * vol[(idx[2] * g->ny + idx[1]) * g->nx + idx[0]];
    }
    return sum;
}

void or_project(const or_geom *g, const double *vol, int64_t v0, int64_t nv, double *sino)
{
    const int64_t per = g->n_rows * g->n_cols;
    const int64_t nplanes = g->nx + g->ny + g->nz + 3;
#pragma omp parallel
    {
        double *ts = (double *)malloc(sizeof(double) * (size_t)nplanes);
#pragma omp for schedule(dynamic, 4)
        for (int64_t t = 0; t < nv * per; ++t) {
            const int64_t k = v0 + t / per, r = (t % per) / g->n_cols, c = t % g->n_cols;
            double a[3], d[3];
            ray_of(g, k, r, c, a, d);
            sino[t] = ray_integral(g, vol, a, d, ts);
        }
        free(ts);
    }
}

void or_sparse_upsample(const or_geom *g, const double *sino, int64_t nv, int64_t keep, double *out)
{
    const int64_t nc = g->n_cols, ns = (nc - 1) / keep + 1; /* kept columns 0, keep, 2 keep, ... */
    for (int64_t v = 0; v < nv * g->n_rows; ++v) {
        const double *row = sino + v * nc;
        double *o = out + v * nc;
        for (int64_t c = 0; c < nc; ++c) {
            const int64_t j = c / keep;
            if (j + 1 >= ns) {
                o[c] = row[(ns - 1) * keep];
                continue;
            }
            const double f = (double)(c - j * keep) / (double)keep;
            o[c] = (1.0 - f) * row[j * keep] + f * row[(j + 1) * keep];
        }
    }
}

/* ---- Philox4x32-10: 10 rounds of a Feistel-like bijection on 4 x 32-bit words,
 * two 32 x 32 -> 64-bit multiplications per round, key bumped by the Weyl
 * constants between rounds. */
static void mulhilo(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo(0xD2511F53u, c[0], &hi0, &lo0);
        mulhilo(0xCD9E8D57u, c[2], &hi1, &lo1);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
        c[0] = n0;
        c[1] = n1;
        c[2] = n2;
        c[3] = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

/* Two uniforms in (0, 1) with 53 random bits each from one generator call:
 * counter (sample index low, high, draw index, stream), key (seed low, high). */
static void uniforms(uint64_t seed, int64_t i, uint32_t draw, uint32_t stream, double *u0, double *u1)
{
    const uint32_t ctr[4] = {(uint32_t)(uint64_t)i, (uint32_t)((uint64_t)i >> 32), draw, stream};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    const double scale = 1.0 / 9007199254740992.0; /* 2^-53 */
    *u0 = ((double)(w[0] >> 5) * 67108864.0 + (double)(w[1] >> 6) + 0.5) * scale;
    *u1 = ((double)(w[2] >> 5) * 67108864.0 + (double)(w[3] >> 6) + 0.5) * scale;
}

/* log(k!) : exact sum below 16, Stirling's series with four correction terms above. */
static double log_factorial(double k)
{
    if (k < 16.0) {
        double s = 0.0;
        for (double j = 2.0; j <= k; j += 1.0) s += log(j);
        return s;
    }
    const double x = k + 1.0, ix = 1.0 / x, ix2 = ix * ix;
    return (x - 0.5) * log(x) - x + 0.91893853320467274178 /* log(2 pi) / 2 */ +
           ix * (1.0 / 12.0 - ix2 * (1.0 / 360.0 - ix2 * (1.0 / 1260.0 - ix2 * (1.0 / 1680.0))));
}

int64_t or_poisson(double lam, uint64_t seed, int64_t i)
{
    if (!(lam > 0.0)) return 0;
    if (lam < 10.0) { /* multiply uniforms until the product drops below exp(-lam) */
        const double lim = exp(-lam);
        double prod = 1.0;
        int64_t k = 0;
        for (uint32_t draw = 0;; ++draw) {
            double u0, u1;
            uniforms(seed, i, draw, 0u, &u0, &u1);
            prod *= u0;
            if (prod < lim) return k;
            ++k;
            prod *= u1;
            if (prod < lim) return k;
            ++k;
        }
    }
    const double slam = sqrt(lam), loglam = log(lam);
    const double b = 0.931 + 2.53 * slam, a = -0.059 + 0.02483 * b;
    const double inv_alpha = 1.1239 + 1.1328 / (b - 3.4), vr = 0.9277 - 3.6224 / (b - 2.0);
    for (uint32_t draw = 0;; ++draw) {
        double u, v;
        uniforms(seed, i, draw, 0u, &u, &v);
        u -= 0.5;
        const double us = 0.5 - fabs(u);
        const double k = floor((2.0 * a / us + b) * u + lam + 0.43);
        if (us >= 0.07 && v <= vr) return (int64_t)k;
        if (k < 0.0 || (us < 0.013 && v > us)) continue;
        if (log(v) + log(inv_alpha) - log(a / (us * us) + b) <= -lam + k * loglam - log_factorial(k))
            return (int64_t)k;
    }
}

double or_gaussian(uint64_t seed, int64_t i)
{
    double u0, u1;
    uniforms(seed, i, 0u, 1u, &u0, &u1);
    return sqrt(-2.0 * log(u0)) * cos(2.0 * M_PI * u1);
}

void or_add_noise(const double *g_up, int64_t n, double I0, double mean, double var, uint64_t seed, double *g_in,
                  int64_t *counts, double *M_out)
{
    double M = 0.0;
    for (int64_t i = 0; i < n; ++i) M = g_up[i] > M ? g_up[i] : M;
    *M_out = M;
    const double sd = sqrt(var);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const double lam = M > 0.0 ? I0 * exp(-g_up[i] / M) : I0;
        const int64_t k = or_poisson(lam, seed, i);
        if (counts) counts[i] = k;
        double q = (double)k + mean + sd * or_gaussian(seed, i);
        if (q < 1.0) q = 1.0;
        g_in[i] = log(I0 / q) * M;
    }
}
