// Data simulation for training the reconstruction network (the paper's
// Sec. III-C "Data generation"): helical projection of a voxel volume, the
// sparse detector (every keep-th column) upsampled back by linear
// interpolation, and the "Gaussian+Poisson" noise model
//   counts = Poisson(I0 exp(-g / M)) + N(mean, var),  g_in = M log(I0 / counts),
// M = max g (counts floored at one photon; the paper's "g + poisson(g)" is read
// as the Poisson draw of g, as in the noise model it cites).
//
// Projection: the exact line integral of the piecewise-constant voxel function
// (voxels are cubes of constant value) along the ray from the source a(l)
// through the detector sample, by voxel traversal.  The ray set-up (source,
// direction, entry and exit of the volume box) is FP64; the traversal runs in
// FP32 in voxel units relative to the entry point, with every face crossing
// computed from its plane index (no accumulated step error).
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011) keyed by
// the seed with counter (sample index, draw, stream), two 53-bit uniforms per
// call; Poisson variates by transformed rejection (PTRS, Hormann 1993) for
// means >= 10 and multiplication of uniforms below; normal variates by
// Box-Muller.  Everything that decides a draw is FP64; the normal variate and
// the final log, which only perturb the float output, are FP32.
#include <cstdint>
#include <cstring>

#include "common.cuh"

namespace kats {

namespace {

// ------------------------------------------------------------- projection
struct ProjArgs {
    double R, D, h, lambda0, lambda_first, dl, z0;
    double alpha_c0, d_alpha, w_r0, d_w;
    double lo[3], vs[3];  // volume box corner (voxel edges) and voxel sizes
    int n[3];
    int n_rows, n_cols;
    int64_t v0, nv;
};

__global__ void __launch_bounds__(256) k_project(ProjArgs P, const float *__restrict__ vol, float *__restrict__ sino)
{
    const int64_t per = (int64_t)P.n_rows * P.n_cols;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= per * P.nv) return;
    const int64_t k = P.v0 + t / per;
    const int r = (int)((t % per) / P.n_cols), c = (int)(t % P.n_cols);
    const double l = P.lambda_first + (double)k * P.dl, ph = l + P.lambda0;
    double sp, cp, sa, ca;
    sincos(ph, &sp, &cp);
    sincos(P.alpha_c0 + (double)c * P.d_alpha, &sa, &ca);
    const double w = P.w_r0 + (double)r * P.d_w;
    // source and direction: a + d is the detector sample (e_u = (-sin, cos, 0), e_v = (-cos, -sin, 0))
    const double a[3] = {P.R * cp, P.R * sp, P.z0 + P.h * l};
    const double d[3] = {-P.D * sa * sp - P.D * ca * cp, P.D * sa * cp - P.D * ca * sp, w};
    // entry / exit of the volume box (slab method)
    double tin = -1e300, tout = 1e300;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const double hi = P.lo[ax] + P.n[ax] * P.vs[ax];
        if (d[ax] == 0.0) {
            if (a[ax] < P.lo[ax] || a[ax] > hi) tout = -1e300;
            continue;
        }
        const double t0 = (P.lo[ax] - a[ax]) / d[ax], t1 = (hi - a[ax]) / d[ax];
        tin = fmax(tin, fmin(t0, t1));
        tout = fmin(tout, fmax(t0, t1));
    }
    if (!(tout > tin)) {
        sino[t] = 0.0f;
        return;
    }
    const double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    // traversal in voxel units relative to the entry point, parameter s in [0, T] along d; one
    // scalar set per axis (no per-axis arrays: indexing them by the crossing axis would put them
    // in local memory)
    const float T = (float)(tout - tin);
    float ux, uy, uz, ivx, ivy, ivz, tx, ty, tz;
    int ixx, iyy, izz, sx, sy, sz;
    auto axis_setup = [&](int ax, float *uu, float *iv, float *tb, int *ii, int *st) {
        *uu = (float)((a[ax] + tin * d[ax] - P.lo[ax]) / P.vs[ax]);
        const float du = (float)(d[ax] / P.vs[ax]);
        *ii = min(max((int)floorf(*uu), 0), P.n[ax] - 1);
        if (du > 0.0f) {
            *st = 1;
            *iv = 1.0f / du;
            *tb = ((float)(*ii + 1) - *uu) * *iv;
        } else if (du < 0.0f) {
            *st = -1;
            *iv = 1.0f / du;
            *tb = ((float)*ii - *uu) * *iv;
        } else {
            *st = 0;
            *iv = 0.0f;
            *tb = INFINITY;
        }
    };
    axis_setup(0, &ux, &ivx, &tx, &ixx, &sx);
    axis_setup(1, &uy, &ivy, &ty, &iyy, &sy);
    axis_setup(2, &uz, &ivz, &tz, &izz, &sz);
    const int nx = P.n[0], nxy = P.n[0] * P.n[1];
    float acc = 0.0f, s = 0.0f;
    const int max_steps = P.n[0] + P.n[1] + P.n[2] + 3;
    // The next voxel follows from the face crossings alone, not from the loaded values: walk
    // UNROLL segments (ALU only), then load their voxels together so the loads overlap.
    constexpr int UNROLL = 4;
    bool done = false;
    int idx = izz * nxy + iyy * nx + ixx;
    for (int it = 0; it < max_steps && !done; it += UNROLL) {
        float seg[UNROLL];
        int vi[UNROLL];
#pragma unroll
        for (int q = 0; q < UNROLL; ++q) {
            vi[q] = idx;  // a finished ray repeats a valid voxel with zero length
            seg[q] = 0.0f;
            if (!done) {
                const bool mx = tx <= ty && tx <= tz, my = !mx && ty <= tz, mz = !mx && !my;
                const float sn = fminf(fminf(fminf(tx, ty), tz), T);
                seg[q] = sn - s;
                s = sn;
                if (sn >= T) {
                    done = true;
                } else {
                    // cross the nearest face; its axis's next face from the plane index
                    if (mx) {
                        ixx += sx;
                        tx = ((float)(sx > 0 ? ixx + 1 : ixx) - ux) * ivx;
                    } else if (my) {
                        iyy += sy;
                        ty = ((float)(sy > 0 ? iyy + 1 : iyy) - uy) * ivy;
                    } else {
                        izz += sz;
                        tz = ((float)(sz > 0 ? izz + 1 : izz) - uz) * ivz;
                    }
                    (void)mz;
                    if (ixx < 0 || ixx >= P.n[0] || iyy < 0 || iyy >= P.n[1] || izz < 0 || izz >= P.n[2])
                        done = true;
                    else
                        idx = izz * nxy + iyy * nx + ixx;
                }
            }
        }
        float v[UNROLL];
#pragma unroll
        for (int q = 0; q < UNROLL; ++q) v[q] = __ldg(vol + vi[q]);
#pragma unroll
        for (int q = 0; q < UNROLL; ++q) acc = fmaf(seg[q], v[q], acc);
    }
    sino[t] = (float)((double)acc * len);
}

// ---------------------------------------------------------- sparse detector
__global__ void k_sparse_upsample(const float *__restrict__ in, float *__restrict__ out, int64_t n_lines, int nc,
                                  int keep)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_lines * nc) return;
    const int64_t line = t / nc;
    const int c = (int)(t % nc);
    const int ns = (nc - 1) / keep + 1, j = c / keep;
    const float *row = in + line * nc;
    if (j + 1 >= ns) {
        out[t] = row[(ns - 1) * keep];
        return;
    }
    const float f = (float)(c - j * keep) / (float)keep;
    out[t] = (1.0f - f) * row[j * keep] + f * row[(j + 1) * keep];
}

// ------------------------------------------------------------------ noise
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1, uint32_t out[4])
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// two uniforms in (0, 1), 53 random bits each
__device__ __forceinline__ void uniforms(uint64_t seed, int64_t i, uint32_t draw, uint32_t stream, double *u0,
                                         double *u1)
{
    uint32_t w[4];
    philox4x32_10((uint32_t)(uint64_t)i, (uint32_t)((uint64_t)i >> 32), draw, stream, (uint32_t)seed,
                  (uint32_t)(seed >> 32), w);
    const double scale = 1.0 / 9007199254740992.0;  // 2^-53
    *u0 = ((double)(w[0] >> 5) * 67108864.0 + (double)(w[1] >> 6) + 0.5) * scale;
    *u1 = ((double)(w[2] >> 5) * 67108864.0 + (double)(w[3] >> 6) + 0.5) * scale;
}

// log(k!): exact sum below 16, Stirling's series with four correction terms above
__device__ double log_factorial(double k)
{
    if (k < 16.0) {
        double s = 0.0;
        for (double j = 2.0; j <= k; j += 1.0) s += log(j);
        return s;
    }
    const double x = k + 1.0, ix = 1.0 / x, ix2 = ix * ix;
    return (x - 0.5) * log(x) - x + 0.91893853320467274178 +
           ix * (1.0 / 12.0 - ix2 * (1.0 / 360.0 - ix2 * (1.0 / 1260.0 - ix2 * (1.0 / 1680.0))));
}

__device__ int64_t poisson_draw(double lam, uint64_t seed, int64_t i)
{
    if (!(lam > 0.0)) return 0;
    if (lam < 10.0) {
        const double lim = exp(-lam);
        double prod = 1.0;
        int64_t k = 0;
        for (uint32_t draw = 0; draw < (1u << 20); ++draw) {
            double u0, u1;
            uniforms(seed, i, draw, 0u, &u0, &u1);
            prod *= u0;
            if (prod < lim) return k;
            ++k;
            prod *= u1;
            if (prod < lim) return k;
            ++k;
        }
        return k;
    }
    const double slam = sqrt(lam);
    const double b = 0.931 + 2.53 * slam, a = -0.059 + 0.02483 * b;
    const double vr = 0.9277 - 3.6224 / (b - 2.0);
    for (uint32_t draw = 0; draw < (1u << 20); ++draw) {  // acceptance is > 85% per draw
        double u, v;
        uniforms(seed, i, draw, 0u, &u, &v);
        u -= 0.5;
        const double us = 0.5 - fabs(u);
        const double k = floor((2.0 * a / us + b) * u + lam + 0.43);
        if (us >= 0.07 && v <= vr) return (int64_t)k;
        if (k < 0.0 || (us < 0.013 && v > us)) continue;
        // the rare full test (its constants computed here, not on the common path)
        const double loglam = log(lam), inv_alpha = 1.1239 + 1.1328 / (b - 3.4);
        if (log(v) + log(inv_alpha) - log(a / (us * us) + b) <= -lam + k * loglam - log_factorial(k))
            return (int64_t)k;
    }
    return (int64_t)floor(lam);  // not reached in practice (2^20 rejections in a row)
}

__global__ void k_max(const float *__restrict__ x, int64_t n, unsigned int *out_bits)
{
    float m = 0.0f;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, x[t]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    // non-negative floats order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(out_bits, __float_as_uint(m));
}

__global__ void k_noise(const float *__restrict__ g_up, float *__restrict__ g_in, int64_t n, double I0, double mean,
                        double sd, uint64_t seed, const unsigned int *M_bits, int64_t *counts)
{
    const double M = (double)__uint_as_float(*M_bits);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double lam = M > 0.0 ? I0 * exp(-(double)g_up[i] / M) : I0;
        const int64_t k = poisson_draw(lam, seed, i);
        if (counts) counts[i] = k;
        // the normal variate and the log only perturb a float output: FP32 (their rounding moves
        // g_in by ~1e-7 M; the integer draw above is decided in FP64)
        double u0, u1;
        uniforms(seed, i, 0u, 1u, &u0, &u1);
        const float z = sqrtf(-2.0f * logf((float)u0)) * cospif(2.0f * (float)u1);
        const float q = fmaxf((float)k + (float)mean + (float)sd * z, 1.0f);
        g_in[i] = (float)M * logf((float)I0 / q);
    }
}

int check_geometry_sizes(const kats_geometry *g)
{
    if (!g || g->n_rows < 1 || g->n_cols < 1 || g->nx < 1 || g->ny < 1 || g->nz < 1 || g->views_per_turn < 1 ||
        !(g->dx > 0) || !(g->dy > 0) || !(g->dz > 0) || !(g->R > 0) || !(g->D > 0) || !(g->d_alpha > 0) ||
        !(g->d_w > 0) || g->nx * g->ny * g->nz > INT32_MAX) {
        set_error("geometry: need positive sizes, spacings, R and D (volume below 2^31 voxels)");
        return KATS_EGEOM;
    }
    return KATS_OK;
}

}  // namespace

}  // namespace kats

using namespace kats;

extern "C" {

int katsevich_project(const kats_geometry *g, const float *vol, float *sino, int64_t v0, int64_t nv, void *stream)
{
    kats::NvtxRange nvtx_range("katsevich: project");
    int rc = check_geometry_sizes(g);
    if (rc) return rc;
    if (!vol || !sino || v0 < 0 || nv < 1 || v0 + nv > g->n_views) {
        set_error("project: null buffer or views [%lld, %lld) outside [0, %lld)", (long long)v0,
                  (long long)(v0 + nv), (long long)g->n_views);
        return KATS_EINVAL;
    }
    ProjArgs P;
    P.R = g->R;
    P.D = g->D;
    P.h = g->P / (2.0 * kPi);
    P.lambda0 = g->lambda0;
    P.lambda_first = g->lambda_first;
    P.dl = 2.0 * kPi / (double)g->views_per_turn;
    P.z0 = g->z0;
    P.alpha_c0 = -0.5 * (double)(g->n_cols - 1) * g->d_alpha + g->alpha_offset;
    P.d_alpha = g->d_alpha;
    P.w_r0 = -0.5 * (double)(g->n_rows - 1) * g->d_w + g->w_offset;
    P.d_w = g->d_w;
    P.vs[0] = g->dx;
    P.vs[1] = g->dy;
    P.vs[2] = g->dz;
    P.lo[0] = g->x0 - 0.5 * g->dx;
    P.lo[1] = g->y0 - 0.5 * g->dy;
    P.lo[2] = g->z_first - 0.5 * g->dz;
    P.n[0] = (int)g->nx;
    P.n[1] = (int)g->ny;
    P.n[2] = (int)g->nz;
    P.n_rows = (int)g->n_rows;
    P.n_cols = (int)g->n_cols;
    P.v0 = v0;
    P.nv = nv;
    const int64_t rays = nv * g->n_rows * g->n_cols;
    k_project<<<(unsigned)ceil_div(rays, 256), 256, 0, (cudaStream_t)stream>>>(P, vol, sino);
    count_launches(1);
    KATS_CUDA(cudaGetLastError());
    return KATS_OK;
}

int katsevich_sparse_upsample(const kats_geometry *g, const float *sino, float *out, int64_t nv, int keep,
                              void *stream)
{
    kats::NvtxRange nvtx_range("katsevich: sparse upsample");
    if (!g || !sino || !out || nv < 1 || keep < 1 || g->n_rows < 1 || g->n_cols < 1) {
        set_error("sparse_upsample: null buffer or non-positive sizes");
        return KATS_EINVAL;
    }
    const int64_t n = nv * g->n_rows * g->n_cols;
    k_sparse_upsample<<<(unsigned)ceil_div(n, 256), 256, 0, (cudaStream_t)stream>>>(sino, out, nv * g->n_rows,
                                                                                   (int)g->n_cols, keep);
    count_launches(1);
    KATS_CUDA(cudaGetLastError());
    return KATS_OK;
}

int64_t katsevich_noise_workspace_bytes(void) { return 256; }

int katsevich_add_noise(const float *g_up, float *g_in, int64_t n, double I0, double mean, double var,
                        uint64_t seed, int64_t *counts, void *workspace, size_t workspace_bytes, double *host_M,
                        void *stream)
{
    kats::NvtxRange nvtx_range("katsevich: add noise");
    if (!g_up || !g_in || n < 1 || !(I0 > 0) || !(var >= 0) || !workspace) {
        set_error("add_noise: null buffer, n < 1, I0 <= 0 or var < 0");
        return KATS_EINVAL;
    }
    if (workspace_bytes < 256) {
        set_error("add_noise: workspace %zu < 256 bytes", workspace_bytes);
        return KATS_ESPACE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int *M_bits = (unsigned int *)workspace;
    KATS_CUDA(cudaMemsetAsync(M_bits, 0, sizeof(unsigned int), st));
    k_max<<<148 * 4, 256, 0, st>>>(g_up, n, M_bits);
    count_launches(1);
    KATS_CUDA(cudaGetLastError());
    k_noise<<<148 * 8, 256, 0, st>>>(g_up, g_in, n, I0, mean, sqrt(var), seed, M_bits, counts);
    count_launches(1);
    KATS_CUDA(cudaGetLastError());
    if (host_M) {
        unsigned int bits = 0;
        KATS_CUDA(cudaMemcpyAsync(&bits, M_bits, sizeof(bits), cudaMemcpyDeviceToHost, st));
        KATS_CUDA(cudaStreamSynchronize(st));
        float m;
        memcpy(&m, &bits, sizeof(m));
        *host_M = (double)m;
    }
    return KATS_OK;
}

}  // extern "C"
