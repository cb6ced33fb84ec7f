// Device helpers of the staged backprojection kernels (k_backproject_tma in backproject.cu,
// k_backproject_multi in backproject_multi.cu): the kernel arguments, the mbarrier / TMA
// primitives, the per-view geometry from the tile reference rays and the bilinear taps.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"

namespace kats {

// Invariant checks of the staged-window kernels, compiled in with KATS_DEBUG_CHECKS (the
// bounds-checked build that stands in for a memory checker): bit 1 a backprojection tap column
// outside the CTA's staged columns, bit 2 an unclamped backprojection tap row outside the staged
// rows, bit 4 / 8 the same for the adjoint's window.  A violation is recorded and the access is
// clamped into the window, so the checked build never touches shared memory outside it.  Each
// translation unit holds its own copy (internal linkage); the host hooks read and set every copy.
static __device__ int g_debug_flags = 0;

#ifdef KATS_DEBUG_CHECKS
#define KATS_DCHECK(ok, bit)                                  \
    do {                                                      \
        if (!(ok)) atomicOr(&::kats::g_debug_flags, (bit));   \
    } while (0)
#else
#define KATS_DCHECK(ok, bit) \
    do {                     \
    } while (0)
#endif

struct BPArgs {
    const float *gF;  // [n_fviews][n_rows][gcols], view 0 = half-view first_view
    float *vol;       // [nz][ny][nx]
    const int32_t *k0, *k1;
    const float *w0, *w1;
    const float2 *trig, *trig_lo;
    int nx, ny, nz, N, vpt, n_rows, n_cols, gcols;
    int s_begin, s_end;  // slices [s_begin, s_end) of this launch (z tiles start at s_begin)
    // views [k_lo, k_hi] of this launch (backprojection only).  acc_in: the volume holds the raw
    // sums of the views below k_lo and the launch continues them; acc_final: scale and store the
    // result, else store raw sums for a later launch.  A split run adds every view in the order
    // of one launch, so its result is bit for bit that of one launch.
    int k_lo, k_hi, acc_in, acc_final;
    int64_t first_view;
    float R, D, x0, y0, dx, dy;
    float alpha0, inv_da, w0row, inv_dw, dz_over_dw, scale;
    // FP64 terms for z - z_src: z_first + s dz - z0 - h (lambda_first + (k + 1/2) dl)
    double z_first, dz, z0, h, lambda_first, dlam;
    float hdl, hdl_lo;  // h dl as float plus its rounding residual
    float K_hi, K_lo;   // alpha0 / d_alpha as float plus its rounding residual
};

// Detector column of angle alpha, given p = alpha / d_alpha, as integer ci and
// fraction fc.  Keeping the large constant alpha0 / d_alpha (hi + lo) out of
// the rounded fraction bounds the error by about 2 ulp(p) instead of
// ulp(n_cols / 2): this matters for the transpose, whose splat weights carry
// the coordinate error times the value itself.
__device__ __forceinline__ void column_split(const BPArgs &a, float p, int *ci, float *fc)
{
    const float cf = floorf((p - a.K_hi) - a.K_lo);
    *ci = (int)cf;
    *fc = (p - (cf + a.K_hi)) - a.K_lo;
}

// Per-view source geometry with the trig table carried as float hi + lo, so
// u* and v* keep FP32 precision relative to themselves (the table's own
// rounding would otherwise add ~1e-7 x radius of absolute error).
__device__ __forceinline__ void view_uv(const BPArgs &a, float2 cs, float2 cl, float x, float y, float *u, float *v)
{
    *u = fmaf(-x, cs.y, fmaf(y, cs.x, fmaf(-x, cl.y, y * cl.x)));
    *v = fmaf(-x, cs.x, fmaf(-y, cs.y, fmaf(-x, cl.x, fmaf(-y, cl.y, a.R))));
}

// z_s - z_src(kbase + kf) for a thread whose slice offset at kbase is zb + zb_lo.
__device__ __forceinline__ float z_rel(const BPArgs &a, float zb, float zb_lo, float kf)
{
    return fmaf(-a.hdl, kf, zb) + fmaf(-a.hdl_lo, kf, zb_lo);
}

// zb (float) and its residual for slice s0 and view kbase.
__device__ __forceinline__ void z_base(const BPArgs &a, int s0, int kbase, float *zb, float *zb_lo)
{
    const double z = a.z_first + (double)s0 * a.dz - a.z0 - a.h * (a.lambda_first + ((double)kbase + 0.5) * a.dlam);
    *zb = (float)z;
    *zb_lo = (float)(z - (double)*zb);
}

// ---------------------------------------------------------------- TMA kernel
// CTA = B2_TX x B2_TY columns x B2_T slices: B2_CW consumer warps (one thread
// per column) plus one producer warp that stages each view's detector window
// into a ring of shared-memory slots.  Consumers take two views per
// iteration, so the slots go in pairs, each pair with one full / empty
// mbarrier: one wait and one release per two views.  The ring holds RP
// pairs, 3 or 2 (chosen at launch from the slot size).
constexpr int B2_TX = kTileX, B2_TY = kTileY, B2_T = 16;
constexpr int B2_CW = B2_TX * B2_TY / 32;       // consumer warps
constexpr int B2_THREADS = (B2_CW + 1) * 32;    // + producer warp
constexpr int kWaitLimit = 1 << 22;  // try_wait polls before a wait gives up

#ifdef KATS_DEBUG_CHECKS
// Checked build only, for the test of the timeout path: a lower poll limit, and a producer that
// stops issuing after this many view pairs (-1: never), so that the consumers' waits run out
// without any copy in flight.  Set by katsevich_debug_wait_limit / katsevich_debug_stall_producer.
static __device__ int g_debug_wait_limit = kWaitLimit;
static __device__ int g_debug_stall_pairs = -1;
#define KATS_BP_WAIT_LIMIT ::kats::g_debug_wait_limit
#else
#define KATS_BP_WAIT_LIMIT kWaitLimit
#endif

// The staged kernels measure a voxel's detector column from its tile centre's ray: with the
// centre's (u_r, v_r) from the plan's table and the voxel's offset (du, dv) from it, the angle
// between the two rays is atan(cross / dot), cross = du v_r - dv u_r, dot = r2 + du u_r + dv v_r,
// small (|cross / dot| <= kTileTanMax) and formed without cancellation.  Its arctan is the Taylor
// series to t^11 (truncation below t^13 / 13 <= 6e-10 at the bound).
constexpr float kTileTanMax = 0.25f;

struct BP2Args {
    BPArgs a;
    int W;            // columns of the staged box any voxel of the tile can touch (<= PITCH)
    int srows;        // staged rows: n_rows + 3 (row 0 and rows n_rows+1.. are zero fill)
    int slot_floats;  // floats per staged view, multiple of 32 (128-byte slots)
    int *status;
    float out_scale;  // dl / 2pi, divided by d_alpha for the scaled 16-bit storage
    int mono;         // window starts and ends nondecreasing in the slice (plan check)
    const float4 *geo;  // the plan's tile-relative projection table [tile][view of a turn][2]
    int geo_ntx;        // tiles per row of the table
    // k_backproject_multi only: rows of its staged box (<= srows), whether the box is a band of
    // rows placed per view (else rows 0 .. srows - 1), and the largest distance of a tile's voxel
    // centre from the tile centre
    int box_rows, band;
    float hd;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// A consumer thread's voxel column in its 16 x 16 tile: a warp covers 8 x 4 columns (two warps side
// by side per four rows of the tile) rather than 16 x 2, so that fewer of a warp's voxels lie on one
// ray and meet in one detector column at different rows, which are shared-memory bank conflicts
// (clinical backprojection 26.2 -> 25.55 ms, bit-identical; 4 x 8: 25.6 ms).
static_assert(B2_TX == 16 && B2_TY == 16, "the warp shape assumes 16 x 16 tiles");
__device__ __forceinline__ void consumer_column(int tid, int *tx, int *ty)
{
    *tx = (tid & 7) + 8 * ((tid >> 5) & 1);
    *ty = ((tid >> 3) & 3) + 4 * (tid >> 6);
}

// The staged kernels' column tile of a CTA.  Launch order walks the tile grid in strips of
// kStripTiles tile columns, row by row within a strip (the last strip narrower when the grid's
// width is not a multiple), so that the CTAs resident at one time cover a compact patch of the
// volume: their views' detector columns and rows overlap, and the staged windows are re-read from
// L2 rather than DRAM (clinical backprojection: DRAM reads 24.5 -> 7.0 GB per reconstruction
// against row-by-row order; strips of 4, 6 and 16 tiles: 9.2, 8.2 and 9.0 GB).
constexpr int kStripTiles = 8;
__device__ __forceinline__ void cta_tile(int *bx, int *by)
{
    const int gx = (int)gridDim.x, gy = (int)gridDim.y;
    const int l = (int)blockIdx.x + gx * (int)blockIdx.y;
    const int x0 = l / (kStripTiles * gy) * kStripTiles, w = min(kStripTiles, gx - x0);
    const int r = l - x0 * gy;
    *bx = x0 + r % w;
    *by = r / w;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (int i = 0; i < KATS_BP_WAIT_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}

// arctan(t) for |t| <= kTileTanMax: t (1 - t^2 / 3 + t^4 / 5 - t^6 / 7 + t^8 / 9 - t^10 / 11)
__device__ __forceinline__ float atan_small(float t)
{
    const float s = t * t;
    float p = fmaf(s, -1.0f / 11.0f, 1.0f / 9.0f);
    p = fmaf(s, p, -1.0f / 7.0f);
    p = fmaf(s, p, 1.0f / 5.0f);
    p = fmaf(s, p, -1.0f / 3.0f);
    return fmaf(t * s, p, t);
}

// Two slices' taps: bilinear samples at column colx + fc and rows ur2.x,
// ur2.y of the staged window, smem[colx + (row << log2 PITCH)] (colx carries
// the -2^23 row-bias of the floor trick and the window's first staged row, in
// modulo-2^32 arithmetic), in packed FP32x2 arithmetic: every component is
// rounded exactly as the scalar tap rounds it (a - b is formed as fma(b, -1, a)),
// at half the instruction count.  CLAMP: rows clamped into [rmin, rmax], the
// staged rows whose taps stay inside the window.  The 16-bit forms read
// row-pair words (g[r-1][c] low, g[r][c] high): fp16 lerps the column pair in
// half2 as the scalar tap does, bf16 unpacks exactly to FP32 first.
template <int PITCH, int MODE, bool CLAMP>
__device__ __forceinline__ void bp_tap2(const float *smem, uint32_t colx, float2 fc2, __half2 fch, float2 ur2,
                                        float rmin, float rmax, float2 w2, float2 &acc2)
{
    constexpr int SH = PITCH == 32 ? 5 : (PITCH == 64 ? 6 : 7);
    if (CLAMP) {
        ur2.x = fminf(fmaxf(ur2.x, rmin), rmax);
        ur2.y = fminf(fmaxf(ur2.y, rmin), rmax);
    } else {
#ifdef KATS_DEBUG_CHECKS
        if (!(ur2.x >= rmin && ur2.x <= rmax && ur2.y >= rmin && ur2.y <= rmax)) {
            atomicOr(&g_debug_flags, 2);
            ur2.x = fminf(fmaxf(ur2.x, rmin), rmax);
            ur2.y = fminf(fmaxf(ur2.y, rmin), rmax);
        }
#endif
    }
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 yv = __fadd2_rd(ur2, make_float2(8388608.0f, 8388608.0f));  // 2^23 + floor(ur)
    const uint32_t q0 = colx + ((uint32_t)__float_as_int(yv.x) << SH);
    const uint32_t q1 = colx + ((uint32_t)__float_as_int(yv.y) << SH);
    const float2 fr = __ffma2_rn(__fadd2_rn(yv, make_float2(-8388608.0f, -8388608.0f)), m1, ur2);
    float2 top, bot;
    if (MODE == 0) {
        const float2 v00 = make_float2(smem[q0], smem[q1]);
        const float2 v01 = make_float2(smem[q0 + 1], smem[q1 + 1]);
        const float2 v10 = make_float2(smem[q0 + PITCH], smem[q1 + PITCH]);
        const float2 v11 = make_float2(smem[q0 + PITCH + 1], smem[q1 + PITCH + 1]);
        top = __ffma2_rn(fc2, __ffma2_rn(v00, m1, v01), v00);
        bot = __ffma2_rn(fc2, __ffma2_rn(v10, m1, v11), v10);
    } else if (MODE == 2) {
        const __half2 *h = reinterpret_cast<const __half2 *>(smem);
        const __half2 c0 = __hfma2(fch, __hsub2(h[q0 + 1], h[q0]), h[q0]);
        const __half2 c1 = __hfma2(fch, __hsub2(h[q1 + 1], h[q1]), h[q1]);
        top = make_float2(__low2float(c0), __low2float(c1));
        bot = make_float2(__high2float(c0), __high2float(c1));
    } else {
        const uint32_t *w = reinterpret_cast<const uint32_t *>(smem);
        const uint32_t a0 = w[q0], b0 = w[q0 + 1], a1 = w[q1], b1 = w[q1 + 1];
        const float2 ta = make_float2(__uint_as_float(a0 << 16), __uint_as_float(a1 << 16));
        const float2 tb = make_float2(__uint_as_float(b0 << 16), __uint_as_float(b1 << 16));
        const float2 ba = make_float2(__uint_as_float(a0 & 0xFFFF0000u), __uint_as_float(a1 & 0xFFFF0000u));
        const float2 bb = make_float2(__uint_as_float(b0 & 0xFFFF0000u), __uint_as_float(b1 & 0xFFFF0000u));
        top = __ffma2_rn(fc2, __ffma2_rn(ta, m1, tb), ta);
        bot = __ffma2_rn(fc2, __ffma2_rn(ba, m1, bb), ba);
    }
    acc2 = __ffma2_rn(w2, __ffma2_rn(fr, __ffma2_rn(top, m1, bot), top), acc2);
}

// One view's contribution to a thread's slices, in slice pairs: G groups of T slices (T / 2 pairs
// each), group m's window GOFF * m floats after group 0's.  Every group takes the same rows,
// column, weights and 1/v* (by the periodicity of Sec. II a slice m pitches up sees the view m
// turns later exactly as group 0's slice sees this one, and the producer stages that view at
// group m's offset); GOFF is a compile-time constant, so the groups' loads reuse group 0's
// addresses.  WEIGHTED: the view ends some slice's PI window (end weights, zero outside it; a
// pair with neither slice in its window is skipped, one with a single such slice still loads its
// taps, so weighted pairs always clamp); otherwise every slice takes the view with weight 1.
template <int PITCH, int MODE, bool WEIGHTED, bool CLAMP, int T, int G = 1, int GOFF = 0>
__device__ __forceinline__ void bp_view(const float *smem, uint32_t colx, float fc, float ur0, float dur, float rmin,
                                        float rmax, float inv_v, float kf, const float *lo, const float *hi,
                                        float2 (&acc)[G][T / 2])
{
    const float2 fc2 = make_float2(fc, fc), dur2 = make_float2(dur, dur), ur02 = make_float2(ur0, ur0);
    const __half2 fch = __float2half2_rn(fc);
#pragma unroll
    for (int pr = 0; pr < T / 2; ++pr) {
        const float2 ur2 = __ffma2_rn(make_float2(2 * pr, 2 * pr + 1), dur2, ur02);
        if (WEIGHTED) {
            const float2 om = __fmul2_rn(make_float2(__saturatef(kf - lo[2 * pr]), __saturatef(kf - lo[2 * pr + 1])),
                                         make_float2(__saturatef(hi[2 * pr] - kf), __saturatef(hi[2 * pr + 1] - kf)));
            if (om.x == 0.0f && om.y == 0.0f) continue;
            const float2 w2 = __fmul2_rn(om, make_float2(inv_v, inv_v));
#pragma unroll
            for (int m = 0; m < G; ++m)
                bp_tap2<PITCH, MODE, true>(smem + m * GOFF, colx, fc2, fch, ur2, rmin, rmax, w2, acc[m][pr]);
        } else {
#pragma unroll
            for (int m = 0; m < G; ++m)
                bp_tap2<PITCH, MODE, CLAMP>(smem + m * GOFF, colx, fc2, fch, ur2, rmin, rmax,
                                            make_float2(inv_v, inv_v), acc[m][pr]);
        }
    }
}

// One view in a ramp of the thread's slice windows, the windows nondecreasing in
// the slice.  IN: no slice has ended and some have not started, so the slices
// the view reaches are a prefix with weights sat(k - lo); otherwise every slice
// has started, the open ones are a suffix with weights sat(hi - k).  The pair
// loop stops at the first pair outside; in a boundary pair the closed slice reads
// its partner's rows (its weight is 0), so the rows stay inside the staged window
// without clamping.  The weights and taps equal the general weighted path's.
// Groups as in bp_view.
template <int PITCH, int MODE, bool IN, bool CLAMP, int T, int G = 1, int GOFF = 0>
__device__ __forceinline__ void bp_view_ramp(const float *smem, uint32_t colx, float fc, float ur0, float dur,
                                             float rmin, float rmax, float inv_v, float kf, const float *lo,
                                             const float *hi, float2 (&acc)[G][T / 2])
{
    const float2 fc2 = make_float2(fc, fc), dur2 = make_float2(dur, dur), ur02 = make_float2(ur0, ur0);
    const float2 iv2 = make_float2(inv_v, inv_v);
    const __half2 fch = __float2half2_rn(fc);
#pragma unroll
    for (int i = 0; i < T / 2; ++i) {
        const int pr = IN ? i : T / 2 - 1 - i;
        if (IN ? !(kf > lo[2 * pr]) : !(kf < hi[2 * pr + 1])) break;
        float2 ur2 = __ffma2_rn(make_float2(2 * pr, 2 * pr + 1), dur2, ur02);
        const float2 om = IN ? make_float2(__saturatef(kf - lo[2 * pr]), __saturatef(kf - lo[2 * pr + 1]))
                             : make_float2(__saturatef(hi[2 * pr] - kf), __saturatef(hi[2 * pr + 1] - kf));
        if (!CLAMP) {
            if (IN && om.y == 0.0f) ur2.y = ur2.x;
            if (!IN && om.x == 0.0f) ur2.x = ur2.y;
        }
        const float2 w2 = __fmul2_rn(om, iv2);
#pragma unroll
        for (int m = 0; m < G; ++m)
            bp_tap2<PITCH, MODE, CLAMP>(smem + m * GOFF, colx, fc2, fch, ur2, rmin, rmax, w2, acc[m][pr]);
    }
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Geometry of two consecutive views for one voxel column, in FP32x2, from the tile's reference
// rays (table rows gA0 gA1 / gB0 gB1 of the two views, cs = (cos, sin) of both): the column index
// relative to the staged window's first column and its fraction (the floor taken as 1.5 * 2^23 +
// floor(c) rounded down), first staged row of slice 0, row step per slice, and 1/v*.  (ox, oy): the
// voxel's offset from its tile centre.
struct ViewGeo2 {
    float2 fc, ur0, dur, inv_v;
    int ci0, ci1;
};

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

__device__ __forceinline__ void view_geo2(const BPArgs &a, float ox, float oy, float4 cs, float4 gA0, float4 gA1,
                                          float4 gB0, float4 gB1, float zb, float zb_lo, float kfA, ViewGeo2 &g)
{
    const float2 m1 = f2(-1.0f);
    const float2 c = make_float2(cs.x, cs.z), sn = make_float2(cs.y, cs.w);
    const float2 ur = make_float2(gA0.x, gB0.x), vr = make_float2(gA0.y, gB0.y);
    const float2 du = __ffma2_rn(f2(-ox), sn, __ffma2_rn(f2(oy), c, make_float2(gA0.z, gB0.z)));
    const float2 dv = __ffma2_rn(f2(-ox), c, __ffma2_rn(f2(-oy), sn, make_float2(gA0.w, gB0.w)));
    const float2 cross = __ffma2_rn(du, vr, __fmul2_rn(dv, __fmul2_rn(ur, m1)));
    const float2 dot = __ffma2_rn(ur, du, __ffma2_rn(vr, dv, make_float2(gA1.x, gB1.x)));
    const float2 t = __fmul2_rn(cross, make_float2(rcp_approx(dot.x), rcp_approx(dot.y)));
    const float2 s2 = __fmul2_rn(t, t);
    float2 p = __ffma2_rn(s2, f2(-1.0f / 11.0f), f2(1.0f / 9.0f));
    p = __ffma2_rn(s2, p, f2(-1.0f / 7.0f));
    p = __ffma2_rn(s2, p, f2(1.0f / 5.0f));
    p = __ffma2_rn(s2, p, f2(-1.0f / 3.0f));
    const float2 at = __ffma2_rn(__fmul2_rn(t, s2), p, t);
    const float2 cr = __fadd2_rn(__ffma2_rn(at, f2(a.inv_da), make_float2(gA1.z, gB1.z)), make_float2(gA1.y, gB1.y));
    const float2 yv = __fadd2_rd(cr, f2(12582912.0f));  // 1.5 * 2^23 + floor(cr), |cr| < 2^22
    g.ci0 = __float_as_int(yv.x) - 0x4B400000;
    g.ci1 = __float_as_int(yv.y) - 0x4B400000;
    g.fc = __ffma2_rn(__fadd2_rn(yv, f2(-12582912.0f)), m1, cr);
    const float2 v = __fadd2_rn(vr, dv), u = __fadd2_rn(ur, du);
    g.inv_v = make_float2(rcp_approx(v.x), rcp_approx(v.y));
    const float2 M = __fmul2_rn(f2(a.D), make_float2(rsqrtf(fmaf(u.x, u.x, v.x * v.x)), rsqrtf(fmaf(u.y, u.y, v.y * v.y))));
    const float2 kf = make_float2(kfA, kfA + 1.0f);
    const float2 zr = __fadd2_rn(__ffma2_rn(f2(-a.hdl), kf, f2(zb)), __ffma2_rn(f2(-a.hdl_lo), kf, f2(zb_lo)));
    g.ur0 = __ffma2_rn(__ffma2_rn(M, zr, f2(-a.w0row)), f2(a.inv_dw), f2(1.0f));  // staged row 0 = detector row -1
    g.dur = __fmul2_rn(M, f2(a.dz_over_dw));
}

// Geometry of one view for one voxel column (the scalar form of view_geo2).
struct ViewGeo1 {
    float fc, ur0, dur, inv_v;
    int ci;
};

__device__ __forceinline__ void view_geo1(const BPArgs &a, float ox, float oy, float2 cs, float4 g0, float4 g1,
                                          float zb, float zb_lo, float kf, ViewGeo1 &g)
{
    const float du = fmaf(-ox, cs.y, fmaf(oy, cs.x, g0.z));
    const float dv = fmaf(-ox, cs.x, fmaf(-oy, cs.y, g0.w));
    const float cross = fmaf(du, g0.y, dv * -g0.x);
    const float dot = fmaf(g0.x, du, fmaf(g0.y, dv, g1.x));
    const float cr = fmaf(atan_small(cross * rcp_approx(dot)), a.inv_da, g1.z) + g1.y;
    const float yv = __fadd_rd(cr, 12582912.0f);  // 1.5 * 2^23 + floor(cr)
    g.ci = __float_as_int(yv) - 0x4B400000;
    g.fc = cr - (yv - 12582912.0f);
    const float v = g0.y + dv, u = g0.x + du;
    g.inv_v = rcp_approx(v);
    const float M = a.D * rsqrtf(fmaf(u, u, v * v));
    const float zr = fmaf(-a.hdl, kf, zb) + fmaf(-a.hdl_lo, kf, zb_lo);
    g.ur0 = fmaf(fmaf(M, zr, -a.w0row), a.inv_dw, 1.0f);  // staged row 0 = detector row -1
    g.dur = M * a.dz_over_dw;
}

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver (null when unavailable).
inline EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)ptr;
    });
    return fn;
}

// Slices [s_begin, s_end) of one launch of k_backproject_multi (backproject_multi.cu); rows_ok:
// every contributing tap lies within half a row of the detector (plan extents).
struct MultiLaunch {
    int s_begin, s_end;
    bool rows_ok;
    int lead_end;  // leading slices [s_begin, min(s_begin + N, lead_end)) only (BPRange::lead_end)
};


// Launches the multi-pitch kernel over the slices of ml that have a partner one or more pitches up
// (each launch after the first of a call with programmatic dependent launch when *n_launched > 0;
// *n_launched counts them); *rest: the slice ranges left for k_backproject_tma.  *used false: the
// plan cannot take it (nothing launched).  b0: the single kernel's arguments (W, srows, status, ...).
template <int MODE>
int launch_multi(const Plan &p, const BP2Args &b0, const void *gF, const MultiLaunch &ml, cudaStream_t st,
                 int *n_launched, std::vector<std::pair<int, int>> *rest, bool *used);

// Checked-build hooks for backproject_multi.cu's kernels: the wait limit (0: unchanged) and the
// producer stall (INT32_MIN: unchanged); the invariant flags, read and cleared.
int multi_debug_set(int wait_limit, int stall_pairs);
int multi_debug_take_flags(int *flags);

}  // namespace kats
