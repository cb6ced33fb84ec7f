// Step 7 of the reconstruction step (Sec. II): backprojection of g^F over
// each voxel's PI interval,
//   f(x) = (1 / 2pi) sum_k omega_k dl g^F(l_{k+1/2}, alpha*, w*) / v*,
// with the one-pitch PI table reused for every pitch (Sec. II periodicity:
// slice s reads table slice s mod N and shifts its views by (s div N) turns).
//
// Thread mapping: one thread owns one (x, y) column and BP_T consecutive
// slices held in registers.  alpha* and v* do not depend on z and w* is affine
// in z, so the per-view geometry (trig, atan, rsqrt) is computed once per view
// and reused by the thread's BP_T slices.
#include <algorithm>

#include "common.cuh"

namespace kats {

constexpr int BP_T = 8;  // slices per thread
constexpr int BP_BX = 16, BP_BY = 8;

struct BPArgs {
    const float *gF;  // [n_fviews][n_rows][n_cols], view 0 = half-view first_view
    float *vol;       // [nz][ny][nx]
    const int32_t *k0, *k1;
    const float *w0, *w1;
    const float2 *trig;
    int nx, ny, nz, N, vpt, n_rows, n_cols;
    int64_t first_view;
    float R, D, x0, y0, dx, dy;
    float alpha0, inv_da, w0row, inv_dw, dz_over_dw, scale;
    // FP64 terms for z - z_src: z_first + s dz - z0 - h (lambda_first + (k + 1/2) dl)
    double z_first, dz, z0, h, lambda_first, dlam;
};

__device__ __forceinline__ float tap(const float *view, int r, int c, int n_rows, int n_cols)
{
    return (r >= 0 && r < n_rows && c >= 0 && c < n_cols) ? __ldg(view + r * n_cols + c) : 0.0f;
}

__global__ void __launch_bounds__(BP_BX *BP_BY) k_backproject(BPArgs a)
{
    const int ix = blockIdx.x * BP_BX + threadIdx.x;
    const int iy = blockIdx.y * BP_BY + threadIdx.y;
    const int s0 = blockIdx.z * BP_T;
    if (ix >= a.nx || iy >= a.ny) return;
    int ka[BP_T], kb[BP_T];
    float wa[BP_T], wb[BP_T], acc[BP_T];
    int kmin = INT32_MAX, kmax = INT32_MIN;
#pragma unroll
    for (int t = 0; t < BP_T; ++t) {
        acc[t] = 0.0f;
        const int s = s0 + t;
        if (s < a.nz) {
            const int j = s % a.N, m = s / a.N;
            const int64_t o = ((int64_t)j * a.ny + iy) * a.nx + ix;
            ka[t] = a.k0[o] + m * a.vpt;
            kb[t] = a.k1[o] + m * a.vpt;
            wa[t] = a.w0[o];
            wb[t] = a.w1[o];
            kmin = min(kmin, ka[t]);
            kmax = max(kmax, kb[t]);
        } else {
            ka[t] = INT32_MAX;
            kb[t] = INT32_MIN;
            wa[t] = wb[t] = 0.0f;
        }
    }
    const float x = a.x0 + (float)ix * a.dx, y = a.y0 + (float)iy * a.dy;
    // z_{s0} - z_src(kmin) in FP64 once; later views subtract h dl (k - kmin)
    const float zb = (float)(a.z_first + (double)s0 * a.dz - a.z0 - a.h * (a.lambda_first + ((double)kmin + 0.5) * a.dlam));
    const float hdl = (float)(a.h * a.dlam);
    int km = ((kmin % a.vpt) + a.vpt) % a.vpt;
    const int64_t per_view = (int64_t)a.n_rows * a.n_cols;
    for (int k = kmin; k <= kmax; ++k) {
        const float2 cs = __ldg(a.trig + km);
        km = (km + 1 == a.vpt) ? 0 : km + 1;
        const float v = a.R - x * cs.x - y * cs.y;
        const float u = -x * cs.y + y * cs.x;
        const float inv_v = 1.0f / v;
        const float alpha = atanf(u * inv_v);
        const float uc = (alpha - a.alpha0) * a.inv_da;
        const float M = a.D * rsqrtf(u * u + v * v);  // D cos(alpha*) / v*
        const float zr = zb - hdl * (float)(k - kmin);
        const float ur0 = (M * zr - a.w0row) * a.inv_dw;
        const float dur = M * a.dz_over_dw;
        const float cf = floorf(uc);
        const int ci = (int)cf;
        const float fc = uc - cf;
        const float *view = a.gF + (int64_t)(k - a.first_view) * per_view;
#pragma unroll
        for (int t = 0; t < BP_T; ++t) {
            if (k < ka[t] || k > kb[t]) continue;
            const float om = (k == ka[t] ? wa[t] : 1.0f) * (k == kb[t] ? wb[t] : 1.0f);
            const float ur = ur0 + (float)t * dur;
            const float rf = floorf(ur);
            const int ri = (int)rf;
            const float fr = ur - rf;
            const float v00 = tap(view, ri, ci, a.n_rows, a.n_cols);
            const float v01 = tap(view, ri, ci + 1, a.n_rows, a.n_cols);
            const float v10 = tap(view, ri + 1, ci, a.n_rows, a.n_cols);
            const float v11 = tap(view, ri + 1, ci + 1, a.n_rows, a.n_cols);
            const float top = v00 + fc * (v01 - v00);
            const float bot = v10 + fc * (v11 - v10);
            acc[t] = fmaf(om * inv_v, top + fr * (bot - top), acc[t]);
        }
    }
#pragma unroll
    for (int t = 0; t < BP_T; ++t) {
        const int s = s0 + t;
        if (s < a.nz) a.vol[((int64_t)s * a.ny + iy) * a.nx + ix] = acc[t] * a.scale;
    }
}

static BPArgs bp_args(const Plan &p)
{
    const kats_geometry &g = p.g;
    BPArgs a;
    a.k0 = p.pi_k0;
    a.k1 = p.pi_k1;
    a.w0 = p.pi_w0;
    a.w1 = p.pi_w1;
    a.trig = p.trig;
    a.nx = (int)g.nx;
    a.ny = (int)g.ny;
    a.nz = (int)g.nz;
    a.N = (int)p.N;
    a.vpt = (int)g.views_per_turn;
    a.n_rows = (int)g.n_rows;
    a.n_cols = (int)g.n_cols;
    a.first_view = p.first_view;
    a.R = (float)g.R;
    a.D = (float)g.D;
    a.x0 = (float)g.x0;
    a.y0 = (float)g.y0;
    a.dx = (float)g.dx;
    a.dy = (float)g.dy;
    a.alpha0 = (float)(-0.5 * (double)(g.n_cols - 1) * g.d_alpha + g.alpha_offset);
    a.inv_da = (float)(1.0 / g.d_alpha);
    a.w0row = (float)(-0.5 * (double)(g.n_rows - 1) * g.d_w + g.w_offset);
    a.inv_dw = (float)(1.0 / g.d_w);
    a.dz_over_dw = (float)(g.dz / g.d_w);
    a.scale = (float)(p.dlam / (2.0 * kPi));
    a.z_first = g.z_first;
    a.dz = g.dz;
    a.z0 = g.z0;
    a.h = p.h;
    a.lambda_first = g.lambda_first;
    a.dlam = p.dlam;
    return a;
}

int launch_backproject(const Plan &p, const float *gF, float *vol, cudaStream_t st)
{
    BPArgs a = bp_args(p);
    a.gF = gF;
    a.vol = vol;
    dim3 grid((unsigned)ceil_div(p.g.nx, BP_BX), (unsigned)ceil_div(p.g.ny, BP_BY), (unsigned)ceil_div(p.g.nz, BP_T));
    k_backproject<<<grid, dim3(BP_BX, BP_BY), 0, st>>>(a);
    KATS_CUDA(cudaGetLastError());
    return KATS_OK;
}

// Transpose of step 7: each (voxel, view) term sends its weight times the
// voxel value to the four bilinear taps of that view (FP32 atomics).
__device__ __forceinline__ void splat(float *view, int r, int c, int n_rows, int n_cols, float val)
{
    if (r >= 0 && r < n_rows && c >= 0 && c < n_cols) atomicAdd(view + r * n_cols + c, val);
}

__global__ void __launch_bounds__(BP_BX *BP_BY) k_backproject_T(BPArgs a, const float *__restrict__ vol, float *gF)
{
    const int ix = blockIdx.x * BP_BX + threadIdx.x;
    const int iy = blockIdx.y * BP_BY + threadIdx.y;
    const int s0 = blockIdx.z * BP_T;
    if (ix >= a.nx || iy >= a.ny) return;
    int ka[BP_T], kb[BP_T];
    float wa[BP_T], wb[BP_T], f[BP_T];
    int kmin = INT32_MAX, kmax = INT32_MIN;
#pragma unroll
    for (int t = 0; t < BP_T; ++t) {
        const int s = s0 + t;
        if (s < a.nz) {
            const int j = s % a.N, m = s / a.N;
            const int64_t o = ((int64_t)j * a.ny + iy) * a.nx + ix;
            ka[t] = a.k0[o] + m * a.vpt;
            kb[t] = a.k1[o] + m * a.vpt;
            wa[t] = a.w0[o];
            wb[t] = a.w1[o];
            f[t] = vol[((int64_t)s * a.ny + iy) * a.nx + ix] * a.scale;
            kmin = min(kmin, ka[t]);
            kmax = max(kmax, kb[t]);
        } else {
            ka[t] = INT32_MAX;
            kb[t] = INT32_MIN;
            wa[t] = wb[t] = f[t] = 0.0f;
        }
    }
    const float x = a.x0 + (float)ix * a.dx, y = a.y0 + (float)iy * a.dy;
    const float zb = (float)(a.z_first + (double)s0 * a.dz - a.z0 - a.h * (a.lambda_first + ((double)kmin + 0.5) * a.dlam));
    const float hdl = (float)(a.h * a.dlam);
    int km = ((kmin % a.vpt) + a.vpt) % a.vpt;
    const int64_t per_view = (int64_t)a.n_rows * a.n_cols;
    for (int k = kmin; k <= kmax; ++k) {
        const float2 cs = __ldg(a.trig + km);
        km = (km + 1 == a.vpt) ? 0 : km + 1;
        const float v = a.R - x * cs.x - y * cs.y;
        const float u = -x * cs.y + y * cs.x;
        const float inv_v = 1.0f / v;
        const float alpha = atanf(u * inv_v);
        const float uc = (alpha - a.alpha0) * a.inv_da;
        const float M = a.D * rsqrtf(u * u + v * v);
        const float zr = zb - hdl * (float)(k - kmin);
        const float ur0 = (M * zr - a.w0row) * a.inv_dw;
        const float dur = M * a.dz_over_dw;
        const float cf = floorf(uc);
        const int ci = (int)cf;
        const float fc = uc - cf;
        float *view = gF + (int64_t)(k - a.first_view) * per_view;
#pragma unroll
        for (int t = 0; t < BP_T; ++t) {
            if (k < ka[t] || k > kb[t]) continue;
            const float om = (k == ka[t] ? wa[t] : 1.0f) * (k == kb[t] ? wb[t] : 1.0f);
            const float ur = ur0 + (float)t * dur;
            const float rf = floorf(ur);
            const int ri = (int)rf;
            const float fr = ur - rf;
            const float wv = om * inv_v * f[t];
            splat(view, ri, ci, a.n_rows, a.n_cols, wv * (1.0f - fr) * (1.0f - fc));
            splat(view, ri, ci + 1, a.n_rows, a.n_cols, wv * (1.0f - fr) * fc);
            splat(view, ri + 1, ci, a.n_rows, a.n_cols, wv * fr * (1.0f - fc));
            splat(view, ri + 1, ci + 1, a.n_rows, a.n_cols, wv * fr * fc);
        }
    }
}

int launch_backproject_adjoint(const Plan &p, const float *vol, float *gF, cudaStream_t st)
{
    BPArgs a = bp_args(p);
    a.gF = gF;
    a.vol = nullptr;
    KATS_CUDA(cudaMemsetAsync(gF, 0, sizeof(float) * (size_t)(p.n_fviews * p.g.n_rows * p.g.n_cols), st));
    dim3 grid((unsigned)ceil_div(p.g.nx, BP_BX), (unsigned)ceil_div(p.g.ny, BP_BY), (unsigned)ceil_div(p.g.nz, BP_T));
    k_backproject_T<<<grid, dim3(BP_BX, BP_BY), 0, st>>>(a, vol, gF);
    KATS_CUDA(cudaGetLastError());
    return KATS_OK;
}

}  // namespace kats
