// Pre-calculating step (Sec. II): geometry validation and the one-pitch
// tables, built on the device in FP64.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <vector>

#include <atomic>

#include "common.cuh"

namespace kats {

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what)
{
    set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
    return (e == cudaErrorMemoryAllocation) ? KATS_ENOMEM : KATS_ECUDA;
}

static std::atomic<int64_t> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

// Host-side fault injection for tests: the next g_fail_allocs device
// allocations made through dev_malloc / dev_malloc_async report
// cudaErrorMemoryAllocation without calling CUDA.
static std::atomic<int> g_fail_allocs{0};

static bool inject_alloc_failure()
{
    int n = g_fail_allocs.load();
    while (n > 0)
        if (g_fail_allocs.compare_exchange_weak(n, n - 1)) return true;
    return false;
}

cudaError_t dev_malloc(void **ptr, size_t bytes)
{
    if (inject_alloc_failure()) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(ptr, bytes);
}

cudaError_t dev_malloc_async(void **ptr, size_t bytes, cudaStream_t st)
{
    if (inject_alloc_failure()) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(ptr, bytes, st);
}

// ------------------------------------------------- host 16-bit conversions
// Round-to-nearest-even conversions of a double to bfloat16 (8-bit exponent,
// 7-bit fraction) and IEEE binary16 (5-bit exponent, 10-bit fraction) bit
// patterns, from the formats' definitions; finite inputs in range only.
static uint16_t host_to_bf16(double v)
{
    const float f = (float)v;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t rounding = 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)((u + rounding) >> 16);
}

static double host_from_bf16(uint16_t h)
{
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

static uint16_t host_to_fp16(double v)
{
    const double a = fabs(v);
    uint16_t sign = v < 0 ? 0x8000 : 0;
    if (a < 6.103515625e-05) {  // subnormal range: multiples of 2^-24
        const double q = nearbyint(a * 16777216.0);
        return (uint16_t)(sign | (uint16_t)q);
    }
    int e;
    const double m = frexp(a, &e);  // a = m 2^e, m in [0.5, 1)
    double frac = nearbyint((m * 2.0 - 1.0) * 1024.0);
    int exp = e - 1;
    if (frac >= 1024.0) {
        frac = 0.0;
        exp += 1;
    }
    return (uint16_t)(sign | (uint16_t)((exp + 15) << 10) | (uint16_t)frac);
}

static double host_from_fp16(uint16_t h)
{
    const int exp = (h >> 10) & 0x1F;
    const int frac = h & 0x3FF;
    const double s = (h & 0x8000) ? -1.0 : 1.0;
    if (exp == 0) return s * ldexp((double)frac, -24);
    return s * ldexp(1.0 + frac / 1024.0, exp - 15);
}

// ----------------------------------------------------------------- geometry
struct DevGeom {
    double R, D, P, lambda0, z0, lambda_first, dlam, h;
    double d_alpha, alpha0, d_w, w0;  // alpha0 / w0: centre of column 0 / row 0
    double x0, y0, z_first, dx, dy, dz;
    double psi_max, dpsi;
    int64_t nx, ny, N, n_rows, n_cols, n_psi, vpt;
    int endpoint_mode;
};

static double r_fov(const kats_geometry &g)
{
    double xa = fabs(g.x0 - 0.5 * g.dx), xb = fabs(g.x0 + ((double)g.nx - 0.5) * g.dx);
    double ya = fabs(g.y0 - 0.5 * g.dy), yb = fabs(g.y0 + ((double)g.ny - 0.5) * g.dy);
    double xm = xa > xb ? xa : xb, ym = ya > yb ? ya : yb;
    return sqrt(xm * xm + ym * ym);
}

static DevGeom dev_geom(const kats_geometry &g, int64_t N, int64_t n_psi, double alpha_m)
{
    DevGeom d;
    d.R = g.R;
    d.D = g.D;
    d.P = g.P;
    d.lambda0 = g.lambda0;
    d.z0 = g.z0;
    d.lambda_first = g.lambda_first;
    d.dlam = 2.0 * kPi / (double)g.views_per_turn;
    d.h = g.P / (2.0 * kPi);
    d.d_alpha = g.d_alpha;
    d.alpha0 = -0.5 * (double)(g.n_cols - 1) * g.d_alpha + g.alpha_offset;
    d.d_w = g.d_w;
    d.w0 = -0.5 * (double)(g.n_rows - 1) * g.d_w + g.w_offset;
    d.x0 = g.x0;
    d.y0 = g.y0;
    d.z_first = g.z_first;
    d.dx = g.dx;
    d.dy = g.dy;
    d.dz = g.dz;
    d.psi_max = 0.5 * kPi + alpha_m;
    d.dpsi = 2.0 * d.psi_max / (double)(n_psi - 1);
    d.nx = g.nx;
    d.ny = g.ny;
    d.N = N;
    d.n_rows = g.n_rows;
    d.n_cols = g.n_cols;
    d.n_psi = n_psi;
    d.vpt = g.views_per_turn;
    d.endpoint_mode = (int)g.endpoint_mode;
    return d;
}

// kappa-line height w_kappa(alpha, psi), Sec. II Eq. (w_k)
__device__ __forceinline__ double w_kappa(const DevGeom &G, double alpha, double psi)
{
    double q = (psi == 0.0) ? 1.0 : psi / tan(psi);
    return G.D * G.h / G.R * (psi * cos(alpha) + q * sin(alpha));
}

// d/dpsi (psi cos a + psi cot(psi) sin a)
__device__ __forceinline__ double kappa_slope(double alpha, double psi)
{
    double s = sin(psi), c = cos(psi);
    return cos(alpha) + sin(alpha) * (c * s - psi) / (s * s);
}

// Safeguarded Newton for a root of f on [a, b] with f(a), f(b) of opposite
// signs (or zero).  f(kind, x, &df).
template <class F>
__device__ double newton_bracket(F f, double a, double b)
{
    double df;
    double fa = f(a, df);
    double fb = f(b, df);
    if (fa == 0.0) return a;
    if (fb == 0.0) return b;
    if (fa > 0.0) {  // orient so that f(a) < 0 < f(b)
        double t = a;
        a = b;
        b = t;
    }
    double x = 0.5 * (a + b);
    for (int it = 0; it < 200; ++it) {
        double fx = f(x, df);
        if (fx == 0.0) return x;
        if (fx < 0.0) a = x; else b = x;
        double xn = x - fx / df;
        double lo = fmin(a, b), hi = fmax(a, b);
        if (!(xn > lo && xn < hi) || !isfinite(xn)) xn = 0.5 * (a + b);
        if (xn == x || fabs(xn - x) <= 4e-16 * fmax(1.0, fabs(x))) {
            // polish: one more bracketed bisection-free check of the neighbourhood
            return xn;
        }
        if (hi - lo <= 2e-16 * fmax(1.0, fabs(x))) return 0.5 * (a + b);
        x = xn;
    }
    return x;
}

// psi_hat(alpha, w): root of w = w_kappa(alpha, psi) with the smallest |psi|
// in [-psi_max, psi_max] (Sec. II step 5).  For alpha >= 0 the function is
// increasing on psi < 0 and increasing-then-decreasing on psi > 0 (its slope
// cos a + sin a (cot psi - psi / sin^2 psi) decreases strictly on (0, pi));
// alpha < 0 follows from w_kappa(-a, -psi) = -w_kappa(a, psi).
__device__ bool psi_hat(const DevGeom &G, double alpha, double w, double *out)
{
    double sgn = 1.0;
    if (alpha < 0.0) {
        alpha = -alpha;
        w = -w;
        sgn = -1.0;
    }
    const double pm = G.psi_max;
    const double K = G.D * G.h / G.R;
    auto res = [&](double p, double &d) {
        d = K * kappa_slope(alpha, p);
        return w_kappa(G, alpha, p) - w;
    };
    double dd;
    double f0 = res(0.0, dd);
    if (f0 == 0.0) {
        *out = 0.0;
        return true;
    }
    double pt = pm;
    if (kappa_slope(alpha, pm) < 0.0) {
        auto slope = [&](double p, double &d) {
            double s = sin(p), c = cos(p);
            // derivative of the slope: 2 sin a (p cos p - sin p) / sin^3 p
            d = 2.0 * sin(alpha) * (p * c - s) / (s * s * s);
            return kappa_slope(alpha, p);
        };
        pt = newton_bracket(slope, 1e-9, pm);
    }
    bool found = false;
    double best = 0.0;
    if (f0 < 0.0) {
        if (res(pt, dd) >= 0.0) {
            best = newton_bracket(res, 0.0, pt);
            found = true;
        }
    } else {
        if (res(-pm, dd) <= 0.0) {
            best = newton_bracket(res, -pm, 0.0);
            found = true;
        }
        if (res(pm, dd) <= 0.0) {
            double r = newton_bracket(res, pt, pm);
            if (!found || fabs(r) < fabs(best)) best = r;
            found = true;
        }
    }
    *out = sgn * best;
    return found;
}

// PI-line endpoints (Sec. II, Eq. (e1)): chord midpoint b and half-width d
// with cos d = (x cos(b+l0) + y sin(b+l0)) / R and
// (z - z0)/h = b + d t / (R sin d), t = -x sin(b+l0) + y cos(b+l0).
__device__ void pi_endpoints(const DevGeom &G, double x, double y, double z, double *li, double *lo)
{
    const double zeta = (z - G.z0) / G.h;
    auto F = [&](double b, double &dF) {
        double sp, cp;
        sincos(b + G.lambda0, &sp, &cp);
        double cd = (x * cp + y * sp) / G.R;
        double d = acos(cd);
        double sd = sqrt(fmax(0.0, (1.0 - cd) * (1.0 + cd)));
        double t = -x * sp + y * cp;
        double Gt = t / (G.R * sd);
        dF = 1.0 - Gt * Gt + d * cd * (t * Gt - G.R * sd) / (G.R * sd * sd);
        return b + d * Gt - zeta;
    };
    double b = newton_bracket(F, zeta - kPi, zeta + kPi);
    double sp, cp;
    sincos(b + G.lambda0, &sp, &cp);
    double d = acos((x * cp + y * sp) / G.R);
    *li = b - d;
    *lo = b + d;
}

__global__ void k_plan_kappa(DevGeom G, int32_t *idx, float *frac)
{
    int64_t n = G.n_psi * (G.n_cols - 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t l = t / (G.n_cols - 1), c = t % (G.n_cols - 1);
        double psi = -G.psi_max + (double)l * G.dpsi;
        double alpha = G.alpha0 + ((double)c + 0.5) * G.d_alpha;
        double u = (w_kappa(G, alpha, psi) - G.w0) / G.d_w;
        double f = floor(u);
        idx[t] = (int32_t)f;
        frac[t] = (float)(u - f);
    }
}

__global__ void k_plan_psi(DevGeom G, int32_t *idx, float *frac)
{
    int64_t n = G.n_rows * G.n_cols;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = t / G.n_cols, c = t % G.n_cols;
        double psi;
        bool ok = psi_hat(G, G.alpha0 + (double)c * G.d_alpha, G.w0 + (double)r * G.d_w, &psi);
        if (!ok) {
            idx[t] = -2;
            frac[t] = 0.0f;
            continue;
        }
        double u = (psi + G.psi_max) / G.dpsi;
        double f = floor(u);
        idx[t] = (int32_t)f;
        frac[t] = (float)(u - f);
    }
}

// Tile-relative projection table (layout and meaning in Plan::geo): one thread per (tile, view of a
// turn), FP64.  The window start is the lowest column any of the tile's corner columns (clamped to
// the volume) reaches in that view, minus one, aligned down to 4 floats (16-byte TMA start).
__global__ void k_plan_geo(DevGeom G, int ntx, int nty, float4 *geo)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)ntx * nty * G.vpt) return;
    const int t = (int)(i / G.vpt), k = (int)(i % G.vpt);
    const int tx = t % ntx, ty = t / ntx;
    const double ph = G.lambda_first + ((double)k + 0.5) * G.dlam + G.lambda0;
    const double cs = cos(ph), sn = sin(ph);
    double cmin = 1e300;
    for (int q = 0; q < 4; ++q) {
        const int64_t ix = (q & 1) ? min((int64_t)tx * kTileX + kTileX - 1, G.nx - 1) : (int64_t)tx * kTileX;
        const int64_t iy = (q & 2) ? min((int64_t)ty * kTileY + kTileY - 1, G.ny - 1) : (int64_t)ty * kTileY;
        const double x = G.x0 + (double)ix * G.dx, y = G.y0 + (double)iy * G.dy;
        cmin = fmin(cmin, (atan2(-x * sn + y * cs, G.R - x * cs - y * sn) - G.alpha0) / G.d_alpha);
    }
    const int clo = ((int)floor(cmin) - 1) & ~3;
    const double xc = G.x0 + ((double)tx * kTileX + 0.5 * (kTileX - 1)) * G.dx;
    const double yc = G.y0 + ((double)ty * kTileY + 0.5 * (kTileY - 1)) * G.dy;
    const double uc = -xc * sn + yc * cs, vc = G.R - xc * cs - yc * sn;
    const float ur = (float)uc, vr = (float)vc;
    const double cref = (atan2((double)ur, (double)vr) - G.alpha0) / G.d_alpha - (double)clo;
    const float chi = (float)cref;
    geo[2 * i] = make_float4(ur, vr, (float)(uc - (double)ur), (float)(vc - (double)vr));
    geo[2 * i + 1] = make_float4((float)((double)ur * ur + (double)vr * vr), chi, (float)(cref - (double)chi),
                                 __int_as_float(clo));
}

// One-pitch PI table: first/last filtered view and their covered fractions
// (midpoint rule over [lam_i, lam_o]; hard mode: indicator at l_{k+1/2}).
__global__ void k_plan_pi(DevGeom G, int32_t *k0, int32_t *k1, float *w0, float *w1, double *lam_i,
                          double *lam_o)
{
    int64_t n = G.N * G.ny * G.nx;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t ix = t % G.nx, iy = (t / G.nx) % G.ny, j = t / (G.nx * G.ny);
        double li, lo;
        pi_endpoints(G, G.x0 + (double)ix * G.dx, G.y0 + (double)iy * G.dy, G.z_first + (double)j * G.dz, &li, &lo);
        lam_i[t] = li;
        lam_o[t] = lo;
        double ui = (li - G.lambda_first) / G.dlam, uo = (lo - G.lambda_first) / G.dlam;
        if (G.endpoint_mode == 0) {
            double a = floor(ui), b = ceil(uo) - 1.0;
            k0[t] = (int32_t)a;
            k1[t] = (int32_t)b;
            w0[t] = (float)(a + 1.0 - ui);
            w1[t] = (float)(uo - b);
        } else {
            k0[t] = (int32_t)ceil(ui - 0.5);
            k1[t] = (int32_t)floor(uo - 0.5);
            w0[t] = 1.0f;
            w1[t] = 1.0f;
        }
    }
}

__global__ void k_pi_points(DevGeom G, int64_t n, const double *xyz, double *li, double *lo)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        pi_endpoints(G, xyz[3 * t], xyz[3 * t + 1], xyz[3 * t + 2], &li[t], &lo[t]);
}

// Per table slice: min k0, max k1, sum of window lengths; and global lambda extents.
// Clears *flag when some voxel column's window start k0 - w0 or end k1 + w1 (in
// view units, exact in FP64) decreases from one slice to the next; slice N-1 is
// followed by slice 0 of the next pitch, one turn (vpt views) later.  The PI
// window of a point moves monotonically with z along the helix (Sec. II), so the
// flag stays set up to the tables' rounding; the backprojection then walks only
// the slices a view reaches.
__global__ void k_pi_monotone(DevGeom G, const int32_t *k0, const int32_t *k1, const float *w0, const float *w1,
                              int *flag)
{
    const int64_t nxy = G.nx * G.ny, n = G.N * nxy;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / nxy, xy = t % nxy;
        const bool wrap = j + 1 == G.N;
        const int64_t tn = wrap ? xy : t + nxy;
        const double shift = wrap ? (double)G.vpt : 0.0;
        const double s0 = (double)k0[t] - (double)w0[t], s1 = (double)k0[tn] + shift - (double)w0[tn];
        const double e0 = (double)k1[t] + (double)w1[t], e1 = (double)k1[tn] + shift + (double)w1[tn];
        if (s1 < s0 || e1 < e0) *flag = 0;
    }
}

__global__ void k_slice_reduce(int64_t nxy, const int32_t *k0, const int32_t *k1, const double *li,
                               const double *lo, int32_t *kmin, int32_t *kmax, unsigned long long *sum,
                               double *lmin_part, double *lmax_part)
{
    const int j = blockIdx.x;
    int mn = INT32_MAX, mx = INT32_MIN;
    unsigned long long s = 0;
    double a = INFINITY, b = -INFINITY;
    for (int64_t o = threadIdx.x; o < nxy; o += blockDim.x) {
        int64_t q = j * nxy + o;
        mn = min(mn, k0[q]);
        mx = max(mx, k1[q]);
        s += (unsigned long long)(k1[q] - k0[q] + 1);
        a = fmin(a, li[q]);
        b = fmax(b, lo[q]);
    }
    __shared__ int smn[256], smx[256];
    __shared__ unsigned long long ss[256];
    __shared__ double sa[256], sb[256];
    smn[threadIdx.x] = mn;
    smx[threadIdx.x] = mx;
    ss[threadIdx.x] = s;
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            smn[threadIdx.x] = min(smn[threadIdx.x], smn[threadIdx.x + w]);
            smx[threadIdx.x] = max(smx[threadIdx.x], smx[threadIdx.x + w]);
            ss[threadIdx.x] += ss[threadIdx.x + w];
            sa[threadIdx.x] = fmin(sa[threadIdx.x], sa[threadIdx.x + w]);
            sb[threadIdx.x] = fmax(sb[threadIdx.x], sb[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        kmin[j] = smn[0];
        kmax[j] = smx[0];
        sum[j] = ss[0];
        lmin_part[j] = sa[0];
        lmax_part[j] = sb[0];
    }
}

// alpha*/w* extremes over each table voxel's own PI views, FP32 (Eq. (maxvalue)).
__global__ void k_extents(DevGeom G, const int32_t *k0, const int32_t *k1, const float2 *trig, float *part)
{
    float amin = INFINITY, amax = -INFINITY, wmin = INFINITY, wmax = -INFINITY;
    const int64_t n = G.N * G.ny * G.nx;
    const float R = (float)G.R, D = (float)G.D;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t ix = t % G.nx, iy = (t / G.nx) % G.ny, j = t / (G.nx * G.ny);
        float x = (float)(G.x0 + (double)ix * G.dx), y = (float)(G.y0 + (double)iy * G.dy);
        int ka = k0[t], kb = k1[t];
        // z - z_src(k) = zb - hdl * (k - ka), zb in FP64 once per voxel
        double zb = G.z_first + (double)j * G.dz - G.z0 - G.h * (G.lambda_first + ((double)ka + 0.5) * G.dlam);
        float hdl = (float)(G.h * G.dlam);
        int64_t km = ((ka % G.vpt) + G.vpt) % G.vpt;
        for (int k = ka; k <= kb; ++k) {
            float2 cs = trig[km];
            km = (km + 1 == G.vpt) ? 0 : km + 1;
            float v = R - x * cs.x - y * cs.y;
            float u = -x * cs.y + y * cs.x;
            float a = atanf(u / v);
            float w = D * rsqrtf(u * u + v * v) * ((float)zb - hdl * (float)(k - ka));
            amin = fminf(amin, a);
            amax = fmaxf(amax, a);
            wmin = fminf(wmin, w);
            wmax = fmaxf(wmax, w);
        }
    }
    __shared__ float s[4][256];
    s[0][threadIdx.x] = amin;
    s[1][threadIdx.x] = amax;
    s[2][threadIdx.x] = wmin;
    s[3][threadIdx.x] = wmax;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s[0][threadIdx.x] = fminf(s[0][threadIdx.x], s[0][threadIdx.x + w]);
            s[1][threadIdx.x] = fmaxf(s[1][threadIdx.x], s[1][threadIdx.x + w]);
            s[2][threadIdx.x] = fminf(s[2][threadIdx.x], s[2][threadIdx.x + w]);
            s[3][threadIdx.x] = fmaxf(s[3][threadIdx.x], s[3][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) part[4 * blockIdx.x + q] = s[q][0];
}

// ------------------------------------------------------------- validation
static int validate(const kats_geometry *g, int64_t *N_out)
{
    if (!g) {
        set_error("null geometry");
        return KATS_EINVAL;
    }
    if (!(g->R > 0) || !(g->D > 0) || !(g->P > 0)) {
        set_error("R, D and P must be positive (R=%g D=%g P=%g)", g->R, g->D, g->P);
        return KATS_EGEOM;
    }
    if (g->views_per_turn < 2 || g->n_views < 3 || g->n_rows < 2 || g->n_cols < 3 || g->nx < 1 || g->ny < 1 ||
        g->nz < 1) {
        set_error("sizes out of range (views_per_turn>=2, n_views>=3, n_rows>=2, n_cols>=3, volume>=1)");
        return KATS_EGEOM;
    }
    if (g->n_rows > 1024 || g->n_cols > 16384 || g->n_psi > 1024 || g->n_views > (int64_t)1 << 30 ||
        g->nx * g->ny > ((int64_t)1 << 28)) {
        set_error("sizes above the supported maximum (n_rows<=1024, n_cols<=16384, n_psi<=1024)");
        return KATS_EGEOM;
    }
    if (!(g->d_alpha > 0) || !(g->d_w > 0) || !(g->dx > 0) || !(g->dy > 0) || !(g->dz > 0)) {
        set_error("detector and voxel spacings must be positive");
        return KATS_EGEOM;
    }
    if (g->n_psi != 0 && g->n_psi < 2) {
        set_error("n_psi must be 0 (default) or >= 2");
        return KATS_EGEOM;
    }
    if (g->endpoint_mode != 0 && g->endpoint_mode != 1) {
        set_error("endpoint_mode must be 0 or 1");
        return KATS_EGEOM;
    }
    if (g->flags != 0) {
        set_error("flags must be 0");
        return KATS_EGEOM;
    }
    double rf = r_fov(*g);
    if (!(rf < g->R)) {
        set_error("volume corner radius %g must be inside the helix radius %g", rf, g->R);
        return KATS_EGEOM;
    }
    double q = g->P / g->dz;
    double N = std::round(q);
    if (N < 1 || fabs(q - N) > 1e-9 * fmax(1.0, q)) {
        set_error("pitch %g is not a whole number of slices of %g", g->P, g->dz);
        return KATS_EGEOM;
    }
    double cols_alpha = 0.5 * (double)(g->n_cols - 1) * g->d_alpha;
    if (cols_alpha + fabs(g->alpha_offset) >= 0.5 * kPi) {
        set_error("detector fan exceeds pi/2");
        return KATS_EGEOM;
    }
    *N_out = (int64_t)N;
    return KATS_OK;
}

static void free_plan(Plan *p)
{
    if (!p) return;
    void *ptrs[] = {p->kap_idx, p->kap_frac, p->psi_idx, p->psi_frac, p->pi_k0, p->pi_k1, p->pi_w0,
                    p->pi_w1, p->slice_kmin, p->slice_kmax, p->hk, p->lw, p->cosa, p->trig, p->dev_status,
                    p->bt_hi, p->bt_lo, p->btT_hi, p->btT_lo, p->trig_lo, p->bt16_hi[0], p->bt16_lo[0], p->bt16_hi[1],
                    p->bt16_lo[1], p->geo};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete p;
}

template <class T>
static int dalloc(Plan *p, T **ptr, size_t count)
{
    cudaError_t e = dev_malloc((void **)ptr, sizeof(T) * (count ? count : 1));
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return cuda_fail(e, "cudaMalloc(plan table)");
    }
    p->plan_bytes += sizeof(T) * count;
    return KATS_OK;
}

static int build(Plan *p)
{
    const kats_geometry &g = p->g;
    const int64_t nr = g.n_rows, nc = g.n_cols, nxy = g.nx * g.ny, N = p->N;
    DevGeom G = dev_geom(g, N, p->n_psi, p->alpha_m);
    int rc;
    if ((rc = dalloc(p, &p->kap_idx, p->n_psi * p->nc1)) || (rc = dalloc(p, &p->kap_frac, p->n_psi * p->nc1)) ||
        (rc = dalloc(p, &p->psi_idx, nr * nc)) || (rc = dalloc(p, &p->psi_frac, nr * nc)) ||
        (rc = dalloc(p, &p->pi_k0, N * nxy)) || (rc = dalloc(p, &p->pi_k1, N * nxy)) ||
        (rc = dalloc(p, &p->pi_w0, N * nxy)) || (rc = dalloc(p, &p->pi_w1, N * nxy)) ||
        (rc = dalloc(p, &p->slice_kmin, N)) || (rc = dalloc(p, &p->slice_kmax, N)) ||
        (rc = dalloc(p, &p->hk, 2 * nc - 2)) || (rc = dalloc(p, &p->lw, nr)) || (rc = dalloc(p, &p->cosa, nc)) ||
        (rc = dalloc(p, &p->trig, g.views_per_turn)) || (rc = dalloc(p, &p->trig_lo, g.views_per_turn)) ||
        (rc = dalloc(p, &p->dev_status, 1)) ||
        (rc = dalloc(p, &p->bt_hi, p->tc_n * p->tc_k)) || (rc = dalloc(p, &p->bt_lo, p->tc_n * p->tc_k)) ||
        (rc = dalloc(p, &p->btT_hi, p->tct_n * p->tct_k)) || (rc = dalloc(p, &p->btT_lo, p->tct_n * p->tct_k)) ||
        (rc = dalloc(p, &p->bt16_hi[0], p->tc_n * p->tc_k16)) || (rc = dalloc(p, &p->bt16_lo[0], p->tc_n * p->tc_k16)) ||
        (rc = dalloc(p, &p->bt16_hi[1], p->tc_n * p->tc_k16)) || (rc = dalloc(p, &p->bt16_lo[1], p->tc_n * p->tc_k16)) ||
        (rc = dalloc(p, &p->geo, 2 * (size_t)p->geo_ntx * p->geo_nty * g.views_per_turn)))
        return rc;
    // Everything below runs on a private non-blocking stream (host tables are
    // copied with stream-ordered copies, scratch is stream-ordered), so
    // building a plan waits only for its own work: requests running on other
    // streams, e.g. in the serving loop, keep going.
    struct StreamGuard {
        cudaStream_t s = nullptr;
        ~StreamGuard()
        {
            if (s) {
                cudaStreamSynchronize(s);
                cudaStreamDestroy(s);
            }
        }
    } guard;
    KATS_CUDA(cudaStreamCreateWithFlags(&guard.s, cudaStreamNonBlocking));
    cudaStream_t st = guard.s;
    KATS_CUDA(cudaMemsetAsync(p->dev_status, 0, sizeof(int), st));

    // small 1-D tables in FP64 on the host, stored FP32
    {
        std::vector<float> hk(2 * nc - 2), lw(nr), cosa(nc);
        std::vector<float2> trig(g.views_per_turn), trig_lo(g.views_per_turn);
        for (int64_t n = -(nc - 2); n <= nc - 1; ++n)
            hk[n + nc - 2] = (float)(g.d_alpha / (kPi * sin(((double)n - 0.5) * g.d_alpha)));
        for (int64_t r = 0; r < nr; ++r) {
            double w = G.w0 + (double)r * g.d_w;
            lw[r] = (float)(g.D / sqrt(g.D * g.D + w * w));
        }
        for (int64_t c = 0; c < nc; ++c) cosa[c] = (float)cos(G.alpha0 + (double)c * g.d_alpha);
        for (int64_t k = 0; k < g.views_per_turn; ++k) {
            double ph = g.lambda_first + ((double)k + 0.5) * G.dlam + g.lambda0;
            const double c = cos(ph), s = sin(ph);
            trig[k] = make_float2((float)c, (float)s);
            trig_lo[k] = make_float2((float)(c - (double)(float)c), (float)(s - (double)(float)s));
        }
        KATS_CUDA(cudaMemcpyAsync(p->hk, hk.data(), hk.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        KATS_CUDA(cudaMemcpyAsync(p->lw, lw.data(), lw.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        KATS_CUDA(cudaMemcpyAsync(p->cosa, cosa.data(), cosa.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        KATS_CUDA(cudaMemcpyAsync(p->trig, trig.data(), trig.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
        KATS_CUDA(cudaMemcpyAsync(p->trig_lo, trig_lo.data(), trig_lo.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
        std::vector<float> bhi((size_t)(p->tc_n * p->tc_k), 0.0f), blo((size_t)(p->tc_n * p->tc_k), 0.0f);
        for (int64_t c = 0; c < nc; ++c)
            for (int64_t cp = 0; cp < p->nc1; ++cp) {
                const float v = hk[c - cp + nc - 2];
                uint32_t bits;
                std::memcpy(&bits, &v, 4);
                bits &= 0xFFFFE000u;
                float hi;
                std::memcpy(&hi, &bits, 4);
                bhi[(size_t)(c * p->tc_k + cp)] = hi;
                blo[(size_t)(c * p->tc_k + cp)] = v - hi;
            }
        KATS_CUDA(cudaMemcpyAsync(p->bt_hi, bhi.data(), bhi.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        KATS_CUDA(cudaMemcpyAsync(p->bt_lo, blo.data(), blo.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        // the transpose's operand, the same values with the roles of c and c' swapped
        std::vector<float> thi((size_t)(p->tct_n * p->tct_k), 0.0f), tlo((size_t)(p->tct_n * p->tct_k), 0.0f);
        for (int64_t cp = 0; cp < p->nc1; ++cp)
            for (int64_t c = 0; c < nc; ++c) {
                thi[(size_t)(cp * p->tct_k + c)] = bhi[(size_t)(c * p->tc_k + cp)];
                tlo[(size_t)(cp * p->tct_k + c)] = blo[(size_t)(c * p->tc_k + cp)];
            }
        KATS_CUDA(cudaMemcpyAsync(p->btT_hi, thi.data(), thi.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        KATS_CUDA(cudaMemcpyAsync(p->btT_lo, tlo.data(), tlo.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        // 16-bit pairs: hi = value rounded to the type, lo = remainder rounded to the type
        const size_t n16 = (size_t)(p->tc_n * p->tc_k16);
        std::vector<uint16_t> h16(n16, 0), l16(n16, 0);
        for (int kind = 0; kind < 2; ++kind) {
            std::fill(h16.begin(), h16.end(), 0);
            std::fill(l16.begin(), l16.end(), 0);
            for (int64_t c = 0; c < nc; ++c)
                for (int64_t cp = 0; cp < p->nc1; ++cp) {
                    const double v = g.d_alpha / (kPi * sin(((double)(c - cp) - 0.5) * g.d_alpha));
                    const size_t o = (size_t)(c * p->tc_k16 + cp);
                    if (kind == 0) {
                        const uint16_t hb = host_to_bf16(v);
                        h16[o] = hb;
                        l16[o] = host_to_bf16(v - host_from_bf16(hb));
                    } else {
                        const uint16_t hb = host_to_fp16(v);
                        h16[o] = hb;
                        l16[o] = host_to_fp16(v - host_from_fp16(hb));
                    }
                }
            KATS_CUDA(cudaMemcpyAsync(p->bt16_hi[kind], h16.data(), n16 * 2, cudaMemcpyHostToDevice, st));
            KATS_CUDA(cudaMemcpyAsync(p->bt16_lo[kind], l16.data(), n16 * 2, cudaMemcpyHostToDevice, st));
        }
    }

    double *lam_i = nullptr, *lam_o = nullptr, *lmin_part = nullptr, *lmax_part = nullptr;
    unsigned long long *sums = nullptr;
    float *ext_part = nullptr;
    int *mono_flag = nullptr;
    const int ext_blocks = 148 * 8;
    auto cleanup = [&]() {
        for (void *q : {(void *)lam_i, (void *)lam_o, (void *)lmin_part, (void *)lmax_part, (void *)sums,
                        (void *)ext_part, (void *)mono_flag})
            if (q) cudaFreeAsync(q, st);
    };
    k_plan_kappa<<<(unsigned)ceil_div(p->n_psi * p->nc1, 256), 256, 0, st>>>(G, p->kap_idx, p->kap_frac);
    count_launches(1);
    k_plan_geo<<<(unsigned)ceil_div((int64_t)p->geo_ntx * p->geo_nty * g.views_per_turn, 128), 128, 0, st>>>(
        G, p->geo_ntx, p->geo_nty, p->geo);
    count_launches(1);
    k_plan_psi<<<(unsigned)ceil_div(nr * nc, 128), 128, 0, st>>>(G, p->psi_idx, p->psi_frac);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = dev_malloc_async((void **)&lam_i, sizeof(double) * N * nxy, st);
    if (e == cudaSuccess) e = dev_malloc_async((void **)&lam_o, sizeof(double) * N * nxy, st);
    if (e == cudaSuccess) e = dev_malloc_async((void **)&lmin_part, sizeof(double) * N, st);
    if (e == cudaSuccess) e = dev_malloc_async((void **)&lmax_part, sizeof(double) * N, st);
    if (e == cudaSuccess) e = dev_malloc_async((void **)&sums, sizeof(unsigned long long) * N, st);
    if (e == cudaSuccess) e = dev_malloc_async((void **)&ext_part, sizeof(float) * 4 * ext_blocks, st);
    if (e == cudaSuccess) e = dev_malloc_async((void **)&mono_flag, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(mono_flag, 0xFF, sizeof(int), st);  // nonzero: monotone
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "plan scratch allocation");
    }
    k_plan_pi<<<(unsigned)ceil_div(N * nxy, 128), 128, 0, st>>>(G, p->pi_k0, p->pi_k1, p->pi_w0, p->pi_w1, lam_i,
                                                                 lam_o);
    count_launches(1);
    k_slice_reduce<<<(unsigned)N, 256, 0, st>>>(nxy, p->pi_k0, p->pi_k1, lam_i, lam_o, p->slice_kmin,
                                               p->slice_kmax, sums, lmin_part, lmax_part);
    count_launches(1);
    k_extents<<<ext_blocks, 256, 0, st>>>(G, p->pi_k0, p->pi_k1, p->trig, ext_part);
    count_launches(1);
    k_pi_monotone<<<(unsigned)std::min<int64_t>(ceil_div(N * nxy, 256), 148 * 16), 256, 0, st>>>(
        G, p->pi_k0, p->pi_k1, p->pi_w0, p->pi_w1, mono_flag);
    count_launches(1);
    e = cudaGetLastError();
    int mono = 0;
    std::vector<int32_t> kmin(N), kmax(N);
    std::vector<unsigned long long> hs(N);
    std::vector<double> lmin(N), lmax(N);
    std::vector<float> ext(4 * ext_blocks);
    if (e == cudaSuccess) e = cudaMemcpyAsync(kmin.data(), p->slice_kmin, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(kmax.data(), p->slice_kmax, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), sums, sizeof(unsigned long long) * N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(lmin.data(), lmin_part, sizeof(double) * N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(lmax.data(), lmax_part, sizeof(double) * N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ext.data(), ext_part, sizeof(float) * 4 * ext_blocks, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&mono, mono_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "plan kernels and reductions");

    p->pi_monotone = mono != 0;
    p->h_slice_kmin = kmin;
    p->h_slice_kmax = kmax;
    // views the whole volume needs; slice s uses table slice s mod N shifted by (s div N) turns
    int64_t vmin = INT64_MAX, vmax = INT64_MIN, count = 0;
    for (int64_t j = 0; j < N && j < g.nz; ++j) {
        int64_t reps = (g.nz - 1 - j) / N + 1;
        vmin = std::min<int64_t>(vmin, kmin[j]);
        vmax = std::max<int64_t>(vmax, kmax[j] + (reps - 1) * g.views_per_turn);
        count += reps * (int64_t)hs[j];
    }
    p->first_view = vmin;
    p->n_fviews = vmax - vmin + 1;
    p->update_count = count;
    p->ext[0] = INFINITY;
    p->ext[1] = -INFINITY;
    for (int64_t j = 0; j < N; ++j) {
        p->ext[0] = fmin(p->ext[0], lmin[j]);
        p->ext[1] = fmax(p->ext[1], lmax[j]);
    }
    p->ext[2] = p->ext[4] = INFINITY;
    p->ext[3] = p->ext[5] = -INFINITY;
    for (int b = 0; b < ext_blocks; ++b) {
        p->ext[2] = fmin(p->ext[2], (double)ext[4 * b]);
        p->ext[3] = fmax(p->ext[3], (double)ext[4 * b + 1]);
        p->ext[4] = fmin(p->ext[4], (double)ext[4 * b + 2]);
        p->ext[5] = fmax(p->ext[5], (double)ext[4 * b + 3]);
    }
    if (vmin < 0 || vmax > g.n_views - 2) {
        set_error("the volume needs filtered views [%lld, %lld] but the sinogram gives [0, %lld]",
                  (long long)vmin, (long long)vmax, (long long)(g.n_views - 2));
        return KATS_EGEOM;
    }
    return KATS_OK;
}

}  // namespace kats

using namespace kats;

extern "C" {

const char *katsevich_last_error(void) { return g_err; }

int64_t katsevich_launch_count(void) { return kats::launches_so_far(); }

void katsevich_debug_fail_allocs(int n) { g_fail_allocs.store(n > 0 ? n : 0); }

int katsevich_fit_pitch(const kats_geometry *g, double factor, double *pitch_out)
{
    if (!g || !pitch_out || !(factor > 0) || !(g->dz > 0) || !(g->R > 0) || !(g->D > 0) || g->n_rows < 2 ||
        !(g->d_w > 0)) {
        set_error("katsevich_fit_pitch: bad argument");
        return KATS_EINVAL;
    }
    double rf = r_fov(*g);
    if (!(rf < g->R)) {
        set_error("volume corner radius %g must be inside the helix radius %g", rf, g->R);
        return KATS_EGEOM;
    }
    double am = asin(rf / g->R);
    double top = 0.5 * (double)(g->n_rows - 1) * g->d_w;
    double h = top * g->R * cos(am) / (g->D * (0.5 * kPi + am));
    *pitch_out = floor(factor * 2.0 * kPi * h / g->dz) * g->dz;
    return KATS_OK;
}

int katsevich_plan(const kats_geometry *g, kats_plan **out)
{
    kats::NvtxRange nvtx_range("katsevich: plan");
    if (!out) {
        set_error("null output pointer");
        return KATS_EINVAL;
    }
    *out = nullptr;
    int64_t N = 0;
    int rc = validate(g, &N);
    if (rc) return rc;
    Plan *p = new Plan();
    p->g = *g;
    cudaError_t de = cudaGetDevice(&p->device);
    if (de == cudaSuccess) de = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
    if (de != cudaSuccess) {
        delete p;
        return cuda_fail(de, "cudaGetDevice");
    }
    p->N = N;
    p->n_psi = g->n_psi > 0 ? g->n_psi : 2 * g->n_rows;
    p->nc1 = g->n_cols - 1;
    p->r_fov = r_fov(*g);
    p->alpha_m = asin(p->r_fov / g->R);
    p->psi_max = 0.5 * kPi + p->alpha_m;
    p->geo_ntx = (int)ceil_div(g->nx, kTileX);
    p->geo_nty = (int)ceil_div(g->ny, kTileY);
    // a voxel's offset from its tile centre over the nearest source distance bounds the tangent of
    // its angle from the centre's ray
    p->geo_tmax = (float)(std::hypot(0.5 * (kTileX - 1) * g->dx, 0.5 * (kTileY - 1) * g->dy) / (g->R - p->r_fov));
    p->dpsi = 2.0 * p->psi_max / (double)(p->n_psi - 1);
    p->h = g->P / (2.0 * kPi);
    p->dlam = 2.0 * kPi / (double)g->views_per_turn;
    p->gf_cols = (g->n_cols + 3) / 4 * 4;
    p->tc_k = (p->nc1 + 31) / 32 * 32;
    p->tc_n = (g->n_cols + 255) / 256 * 256;
    p->tct_k = (g->n_cols + 31) / 32 * 32;
    p->tct_n = (p->nc1 + 255) / 256 * 256;
    p->tc_k16 = (p->nc1 + 63) / 64 * 64;
    rc = build(p);
    if (rc) {
        free_plan(p);
        return rc;
    }
    *out = reinterpret_cast<kats_plan *>(p);
    return KATS_OK;
}

int katsevich_plan_info(const kats_plan *plan, kats_plan_info *info)
{
    if (!plan || !info) {
        set_error("null argument");
        return KATS_EINVAL;
    }
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    info->lambda_min = p->ext[0];
    info->lambda_max = p->ext[1];
    info->alpha_min = p->ext[2];
    info->alpha_max = p->ext[3];
    info->w_min = p->ext[4];
    info->w_max = p->ext[5];
    info->alpha_m = p->alpha_m;
    info->psi_max = p->psi_max;
    info->slices_per_pitch = p->N;
    info->n_psi = p->n_psi;
    info->first_view = p->first_view;
    info->n_filtered_views = p->n_fviews;
    info->update_count = p->update_count;
    info->gf_cols = p->gf_cols;
    info->workspace_bytes = katsevich_workspace_bytes(plan, KATS_PREC_FP32);
    info->plan_bytes = (int64_t)p->plan_bytes;
    info->pi_monotone = p->pi_monotone ? 1 : 0;
    return KATS_OK;
}

int katsevich_plan_table(const kats_plan *plan, int which, void *host_dst, size_t bytes)
{
    if (!plan || !host_dst) {
        set_error("null argument");
        return KATS_EINVAL;
    }
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    const void *src = nullptr;
    size_t n = 0;
    const size_t nk = (size_t)(p->n_psi * p->nc1), np = (size_t)(p->g.n_rows * p->g.n_cols),
                 nt = (size_t)(p->N * p->g.nx * p->g.ny);
    switch (which) {
        case 0: src = p->kap_idx; n = nk * 4; break;
        case 1: src = p->kap_frac; n = nk * 4; break;
        case 2: src = p->psi_idx; n = np * 4; break;
        case 3: src = p->psi_frac; n = np * 4; break;
        case 4: src = p->pi_k0; n = nt * 4; break;
        case 5: src = p->pi_k1; n = nt * 4; break;
        case 6: src = p->pi_w0; n = nt * 4; break;
        case 7: src = p->pi_w1; n = nt * 4; break;
        default: set_error("unknown table %d", which); return KATS_EINVAL;
    }
    if (bytes != n) {
        set_error("table %d has %zu bytes, caller gave %zu", which, n, bytes);
        return KATS_EINVAL;
    }
    KATS_CUDA(cudaMemcpy(host_dst, src, n, cudaMemcpyDeviceToHost));
    return KATS_OK;
}

int katsevich_pi_endpoints(const kats_geometry *g, int64_t n, const double *host_xyz, double *host_lam_i,
                           double *host_lam_o)
{
    if (!g || n < 0 || (n > 0 && (!host_xyz || !host_lam_i || !host_lam_o))) {
        set_error("bad argument");
        return KATS_EINVAL;
    }
    if (n == 0) return KATS_OK;
    if (!(g->R > 0) || !(g->P > 0)) {
        set_error("R and P must be positive");
        return KATS_EGEOM;
    }
    DevGeom G = dev_geom(*g, 1, 2, 0.0);
    double *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(double) * 5 * n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    e = cudaMemcpy(d, host_xyz, sizeof(double) * 3 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_pi_points<<<(unsigned)ceil_div(n, 128), 128>>>(G, n, d, d + 3 * n, d + 4 * n);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(host_lam_i, d + 3 * n, sizeof(double) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(host_lam_o, d + 4 * n, sizeof(double) * n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "katsevich_pi_endpoints");
    return KATS_OK;
}

void katsevich_plan_destroy(kats_plan *plan) { free_plan(reinterpret_cast<Plan *>(plan)); }

int katsevich_device_status(const kats_plan *plan, int *status)
{
    if (!plan || !status) {
        set_error("null argument");
        return KATS_EINVAL;
    }
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    KATS_CUDA(cudaDeviceSynchronize());
    KATS_CUDA(cudaMemcpy(status, p->dev_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (*status != 0) KATS_CUDA(cudaMemset(p->dev_status, 0, sizeof(int)));
    return KATS_OK;
}

}  // extern "C"
