// Step 7 of the reconstruction step (Sec. II): backprojection of g^F over
// each voxel's PI interval,
//   f(x) = (1 / 2pi) sum_k omega_k dl g^F(l_{k+1/2}, alpha*, w*) / v*,
// with the one-pitch PI table reused for every pitch (Sec. II periodicity:
// slice s reads table slice s mod N and shifts its views by (s div N) turns).
//
// Thread mapping (both kernels): one thread owns one (x, y) column and T
// consecutive slices held in registers.  alpha* and v* do not depend on z and
// w* is affine in z, so the per-view geometry (trig, atan, rsqrt) is computed
// once per view and reused by the thread's T slices.
//
// k_backproject_tma (main path): a CTA owns a 16 x 16 column tile and 16
// slices.  For each view a producer warp copies its detector window (all rows
// plus zero rows above and below, a column range covering the tile's
// projection) into a ring of shared-memory slots by TMA; eight consumer warps
// read every bilinear tap as a plain shared-memory load with no bounds test.
// Where a thread's slice windows are opening or closing it visits only the
// slices the view reaches (the windows move monotonically with z), and a
// launch may take a range of the views and continue raw sums of earlier ones.
// k_backproject (fallback for windows TMA cannot stage): the same arithmetic
// with bounds-tested loads from global memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <utility>
#include <vector>

#include "bp_staged.cuh"

namespace kats {


constexpr int BP_T = 8;  // slices per thread
constexpr int BP_BX = 16, BP_BY = 8;


__device__ __forceinline__ float tap(const float *view, int r, int c, int n_rows, int n_cols, int gcols)
{
    return (r >= 0 && r < n_rows && c >= 0 && c < n_cols) ? __ldg(view + r * gcols + c) : 0.0f;
}

// ------------------------------------------------------------ fallback kernel
__global__ void __launch_bounds__(BP_BX *BP_BY) k_backproject(BPArgs a)
{
    const int ix = blockIdx.x * BP_BX + threadIdx.x;
    const int iy = blockIdx.y * BP_BY + threadIdx.y;
    const int s0 = a.s_begin + blockIdx.z * BP_T;
    if (ix >= a.nx || iy >= a.ny) return;
    int ka[BP_T], kb[BP_T];
    float wa[BP_T], wb[BP_T], acc[BP_T];
    int kmin = INT32_MAX, kmax = INT32_MIN;
#pragma unroll
    for (int t = 0; t < BP_T; ++t) {
        acc[t] = 0.0f;
        const int s = s0 + t;
        if (s < a.s_end) {
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
    float zb, zb_lo;
    z_base(a, s0, kmin, &zb, &zb_lo);
    if (a.acc_in) {
#pragma unroll
        for (int t = 0; t < BP_T; ++t)
            if (s0 + t < a.s_end) acc[t] = a.vol[((int64_t)(s0 + t) * a.ny + iy) * a.nx + ix];
    }
    const int kv0 = max(kmin, a.k_lo), kv1 = min(kmax, a.k_hi);
    int km = ((kv0 % a.vpt) + a.vpt) % a.vpt;
    const int64_t per_view = (int64_t)a.n_rows * a.gcols;
    for (int k = kv0; k <= kv1; ++k) {
        float u, v;
        view_uv(a, __ldg(a.trig + km), __ldg(a.trig_lo + km), x, y, &u, &v);
        km = (km + 1 == a.vpt) ? 0 : km + 1;
        const float inv_v = 1.0f / v;
        int ci;
        float fc;
        column_split(a, atanf(u * inv_v) * a.inv_da, &ci, &fc);
        const float M = a.D * rsqrtf(u * u + v * v);  // D cos(alpha*) / v*
        const float zr = z_rel(a, zb, zb_lo, (float)(k - kmin));
        const float ur0 = (M * zr - a.w0row) * a.inv_dw;
        const float dur = M * a.dz_over_dw;
        const float *view = a.gF + (int64_t)(k - a.first_view) * per_view;
#pragma unroll
        for (int t = 0; t < BP_T; ++t) {
            if (k < ka[t] || k > kb[t]) continue;
            const float om = (k == ka[t] ? wa[t] : 1.0f) * (k == kb[t] ? wb[t] : 1.0f);
            const float ur = ur0 + (float)t * dur;
            const float rf = floorf(ur);
            const int ri = (int)rf;
            const float fr = ur - rf;
            const float v00 = tap(view, ri, ci, a.n_rows, a.n_cols, a.gcols);
            const float v01 = tap(view, ri, ci + 1, a.n_rows, a.n_cols, a.gcols);
            const float v10 = tap(view, ri + 1, ci, a.n_rows, a.n_cols, a.gcols);
            const float v11 = tap(view, ri + 1, ci + 1, a.n_rows, a.n_cols, a.gcols);
            const float top = v00 + fc * (v01 - v00);
            const float bot = v10 + fc * (v11 - v10);
            acc[t] = fmaf(om * inv_v, top + fr * (bot - top), acc[t]);
        }
    }
#pragma unroll
    for (int t = 0; t < BP_T; ++t) {
        const int s = s0 + t;
        if (s < a.s_end) a.vol[((int64_t)s * a.ny + iy) * a.nx + ix] = a.acc_final ? acc[t] * a.scale : acc[t];
    }
}

// RANGED: the launch takes a share of the views (BPArgs k_lo .. acc_final); the plain form
// compiles without that bookkeeping.
// PARTIAL: the launch's last z tile holds fewer than B2_T slices.  Its missing slices take every view
// with clamped rows (nothing of them is stored), so the tile keeps the full and ramp paths instead
// of weighing every view; launched with ROWS_OK false.
template <int PITCH, int MODE, bool ROWS_OK, bool RANGED, int RP, bool PARTIAL = false>
__global__ void __launch_bounds__(B2_THREADS, 2)
    k_backproject_tma(const __grid_constant__ CUtensorMap gmap, BP2Args p)
{
    static_assert(!PARTIAL || !ROWS_OK, "a partial tile's missing slices read clamped rows");
    extern __shared__ __align__(128) float smem[];
    // a backprojection launch that follows this one on the stream (other slices, same inputs) may
    // start its CTAs while this grid's last wave drains
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __shared__ __align__(8) uint64_t s_full[RP], s_empty[RP];
    __shared__ float4 s_geo[RP][4];  // the pair's two views' table rows (tile reference rays, window start)
    __shared__ float4 s_cs[RP];      // (cos, sin) of the pair's two views
    __shared__ int s_K0, s_K1;
    const BPArgs &a = p.a;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const bool producer = warp == B2_CW;
    int tx, ty;  // consumers only
    consumer_column(tid, &tx, &ty);
    int bx, by;
    cta_tile(&bx, &by);
    const int ix = bx * B2_TX + tx, iy = by * B2_TY + ty;
    const int s0 = a.s_begin + blockIdx.z * B2_T;
    const bool active = !producer && ix < a.nx && iy < a.ny;
    // slots start at the first 128-byte boundary of the dynamic shared memory (TMA destinations)
    const int base = (int)(((128u - (smem_addr(smem) & 127u)) & 127u) >> 2);

    // per-slice view windows; weights omega(k) = sat(k - lo_t) * sat(hi_t - k) relative to kbase
    int kmin = INT32_MAX, kmax = INT32_MIN, kfull_lo = INT32_MIN, kfull_hi = INT32_MAX;
    float lo[B2_T], hi[B2_T];
    float2 acc2[1][B2_T / 2];
    {
        int ka[B2_T], kb[B2_T];
        float wa[B2_T], wb[B2_T];
#pragma unroll
        for (int t = 0; t < B2_T; ++t) {
            const int s = s0 + t;
            ka[t] = INT32_MAX;
            kb[t] = INT32_MIN;
            wa[t] = wb[t] = 0.0f;
            if (active && s < a.s_end) {
                const int j = s % a.N, m = s / a.N;
                const int64_t o = ((int64_t)j * a.ny + iy) * a.nx + ix;
                ka[t] = a.k0[o] + m * a.vpt;
                kb[t] = a.k1[o] + m * a.vpt;
                wa[t] = a.w0[o];
                wb[t] = a.w1[o];
                kmin = min(kmin, ka[t]);
                kmax = max(kmax, kb[t]);
            }
            if (!(PARTIAL && active && s >= a.s_end)) {
                kfull_lo = max(kfull_lo, ka[t]);
                kfull_hi = min(kfull_hi, kb[t]);
            }
        }
        if (!p.mono) {  // windows not monotone in the slice: no full range and no ramp walk
            kfull_lo = INT32_MAX;
            kfull_hi = INT32_MIN;
        }
        const int kbase = active ? kmin : 0;
#pragma unroll
        for (int t = 0; t < B2_T / 2; ++t) acc2[0][t] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int t = 0; t < B2_T; ++t) {
            if (ka[t] <= kb[t]) {
                lo[t] = (float)(ka[t] - kbase) - wa[t];
                hi[t] = (float)(kb[t] - kbase) + wb[t];
            } else if (PARTIAL && active) {  // a missing slice of a partial tile: open in every view
                lo[t] = -3.0e9f;
                hi[t] = 3.0e9f;
            } else {
                lo[t] = 3.0e9f;
                hi[t] = -3.0e9f;
            }
        }
    }

    if (tid == 0) {
        s_K0 = INT32_MAX;
        s_K1 = INT32_MIN;
        for (int r = 0; r < RP; ++r) {
            mbar_init(&s_full[r], 1);
            mbar_init(&s_empty[r], B2_CW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // views this launch adds (kmin / kmax stay the windows' ends: weights and geometry use them)
    const int kvmin = RANGED ? max(kmin, a.k_lo) : kmin, kvmax = RANGED ? min(kmax, a.k_hi) : kmax;
    if (active && kvmin <= kvmax) {
        atomicMin(&s_K0, kvmin);
        atomicMax(&s_K1, kvmax);
    }
    __syncthreads();
    const int K0 = s_K0, K1 = s_K1;
    // no view in range: raw sums that stay raw need no store (uniform exit); otherwise the
    // store below still writes zeros (first launch) or scales the sums (last launch)
    if (K0 > K1 && (!RANGED || (a.acc_in && !a.acc_final))) return;
    const int nviews = K0 <= K1 ? K1 - K0 + 1 : 0;
    if (RANGED && a.acc_in && active && !producer) {
#pragma unroll
        for (int t = 0; t < B2_T; ++t) {
            const int s = s0 + t;
            if (s < a.s_end) {
                const float v = a.vol[((int64_t)s * a.ny + iy) * a.nx + ix];
                if (t & 1) acc2[0][t >> 1].y = v; else acc2[0][t >> 1].x = v;
            }
        }
    }

    if (producer) {
        // ---------------- producer warp: the views' table rows (window start in them) + TMA
        const float4 *geo_t = p.geo + (size_t)(by * p.geo_ntx + bx) * a.vpt * 2;
        const uint32_t box_bytes = (uint32_t)(PITCH * p.srows * 4);
        const uint32_t dst0 = smem_addr(smem) + 4u * (uint32_t)base;
        int ps = 0, issued = 0;  // pair slot; view pairs issued
        uint32_t phase = 0;
        int kmod = ((K0 % a.vpt) + a.vpt) % a.vpt;
        bool ok = true;
        // the next pair's table rows (tile reference rays, window start) and (cos, sin), loaded a pair
        // ahead of their use so that their latency overlaps the wait for a free slot
        float4 gA0, gA1, gB0, gB1;
        float2 csA, csB;
        auto load_rows = [&](int km) {
            const int km1 = km + 1 == a.vpt ? 0 : km + 1;
            gA0 = __ldg(geo_t + 2 * km);
            gA1 = __ldg(geo_t + 2 * km + 1);
            gB0 = __ldg(geo_t + 2 * km1);
            gB1 = __ldg(geo_t + 2 * km1 + 1);
            csA = __ldg(a.trig + km);
            csB = __ldg(a.trig + km1);
        };
        if (lane == 0) load_rows(kmod);
        for (int j = 0; j < nviews; j += 2) {
#ifdef KATS_DEBUG_CHECKS
            if (g_debug_stall_pairs >= 0 && j / 2 >= g_debug_stall_pairs) break;  // test hook: stop issuing
#endif
            const int kmod1 = kmod + 1 == a.vpt ? 0 : kmod + 1;
            if (j >= 2 * RP && !mbar_wait(&s_empty[ps], phase ^ 1u)) {
                ok = false;
                break;
            }
            const int nv2 = min(2, nviews - j);
            if (lane == 0) {
                s_geo[ps][0] = gA0;
                s_geo[ps][1] = gA1;
                s_geo[ps][2] = gB0;
                s_geo[ps][3] = gB1;
                s_cs[ps] = make_float4(csA.x, csA.y, csB.x, csB.y);
                mbar_arrive_expect_tx(&s_full[ps], box_bytes * (uint32_t)nv2);
                // fp32 windows start one zero row above the detector; row-pair windows at pair-row 0
                for (int h = 0; h < nv2; ++h)
                    tma_load_3d(dst0 + 4u * (uint32_t)((2 * ps + h) * p.slot_floats), &gmap, &s_full[ps],
                                __float_as_int(h ? gB1.w : gA1.w), MODE == 0 ? -1 : 0, K0 + j + h - (int)a.first_view);
                if (j + 2 < nviews) load_rows(kmod1 + 1 == a.vpt ? 0 : kmod1 + 1);
            }
            __syncwarp();
            issued = j / 2 + 1;
            if (++ps == RP) {
                ps = 0;
                phase ^= 1u;
            }
            kmod = kmod1 + 1 == a.vpt ? 0 : kmod1 + 1;
        }
        if (lane == 0) {
            // Every copy this CTA issued lands before the producer warp retires, on every exit
            // path: consumers that give up on a wait return early, and the CTA (and its shared
            // memory) must not retire under a bulk copy still in flight.  Pairs before the last
            // RP were released by the consumers (so landed) or the empty wait above gave up.
            bool landed = true;
            for (int i = max(0, issued - RP); i < issued; ++i)
                landed = mbar_wait(&s_full[i % RP], (uint32_t)((i / RP) & 1)) && landed;
            if (!ok || !landed) atomicExch(p.status, kDevStatusTimeout);
        }
        return;
    }

    // ---------------- consumer warps: two views per iteration, their per-view
    // geometry computed together in FP32x2 (offset from the tile centre, exact)
    const float ox = ((float)tx - 0.5f * (B2_TX - 1)) * a.dx, oy = ((float)ty - 0.5f * (B2_TY - 1)) * a.dy;
    const int kbase = active ? kmin : 0;
    float zb, zb_lo;
    z_base(a, s0, kbase, &zb, &zb_lo);
    const float rmax = (float)(a.n_rows + 1);
    constexpr int SH = PITCH == 32 ? 5 : (PITCH == 64 ? 6 : 7);
    int ps = 0;  // pair slot: views kA and kB in slots 2 ps and 2 ps + 1
    uint32_t phase = 0;
    for (int j = 0; j < nviews; j += 2) {
        const int kA = K0 + j, kB = kA + 1;
        const bool hasB = j + 1 < nviews;
        // warp-uniform: a wait that ends at the limit for some lanes only still stops the warp
        if (!__all_sync(0xffffffffu, mbar_wait(&s_full[ps], phase))) {
            if (lane == 0) atomicExch(p.status, kDevStatusTimeout);
            return;  // the producer retires only after its issued copies have landed
        }
        const bool onA = active && kA >= kvmin && kA <= kvmax;
        const bool onB = hasB && active && kB >= kvmin && kB <= kvmax;
        if (onA || onB) {
            const float kfA = (float)(kA - kbase);
            ViewGeo2 g;
            view_geo2(a, ox, oy, s_cs[ps], s_geo[ps][0], s_geo[ps][1], s_geo[ps][2], s_geo[ps][3], zb, zb_lo, kfA, g);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!(h ? onB : onA)) continue;
                const int k = kA + h, sl = 2 * ps + h;
                const float fc = h ? g.fc.y : g.fc.x, ur0 = h ? g.ur0.y : g.ur0.x, dur = h ? g.dur.y : g.dur.x;
                const float inv_v = h ? g.inv_v.y : g.inv_v.x, kf = kfA + (float)h;
                KATS_DCHECK((h ? g.ci1 : g.ci0) >= 0 && (h ? g.ci1 : g.ci0) <= p.W - 2, 1);
                const uint32_t colx = (uint32_t)(base + sl * p.slot_floats + min(max(h ? g.ci1 : g.ci0, 0), p.W - 2)) -
                                      (0x4B000000u << SH);
                // full: every slice inside its window with weight 1; ramps: windows
                // still opening (no slice ended) or closing (every slice started); a plan
                // without monotone windows has an empty full range (every view general)
                if (k > kfull_lo && k < kfull_hi)
                    bp_view<PITCH, MODE, false, !ROWS_OK, B2_T>(smem, colx, fc, ur0, dur, 0.0f, rmax, inv_v, kf, lo,
                                                                hi, acc2);
                else if (k < kfull_hi)
                    bp_view_ramp<PITCH, MODE, true, !ROWS_OK, B2_T>(smem, colx, fc, ur0, dur, 0.0f, rmax, inv_v, kf,
                                                                    lo, hi, acc2);
                else if (k > kfull_lo)
                    bp_view_ramp<PITCH, MODE, false, !ROWS_OK, B2_T>(smem, colx, fc, ur0, dur, 0.0f, rmax, inv_v, kf,
                                                                     lo, hi, acc2);
                else
                    bp_view<PITCH, MODE, true, !ROWS_OK, B2_T>(smem, colx, fc, ur0, dur, 0.0f, rmax, inv_v, kf, lo,
                                                               hi, acc2);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&s_empty[ps]);
        if (++ps == RP) {
            ps = 0;
            phase ^= 1u;
        }
    }
    if (!active) return;
#pragma unroll
    for (int t = 0; t < B2_T; ++t) {
        const int s = s0 + t;
        if (s < a.s_end) {
            const float v = (t & 1) ? acc2[0][t >> 1].y : acc2[0][t >> 1].x;
            a.vol[((int64_t)s * a.ny + iy) * a.nx + ix] = (!RANGED || a.acc_final) ? v * p.out_scale : v;
        }
    }
}

// ----------------------------------------------------------------- launch
static BPArgs bp_args(const Plan &p)
{
    const kats_geometry &g = p.g;
    BPArgs a;
    a.k0 = p.pi_k0;
    a.k1 = p.pi_k1;
    a.w0 = p.pi_w0;
    a.w1 = p.pi_w1;
    a.trig = p.trig;
    a.trig_lo = p.trig_lo;
    a.nx = (int)g.nx;
    a.ny = (int)g.ny;
    a.nz = (int)g.nz;
    a.s_begin = 0;
    a.s_end = (int)g.nz;
    a.k_lo = INT32_MIN;
    a.k_hi = INT32_MAX;
    a.acc_in = 0;
    a.acc_final = 1;
    a.N = (int)p.N;
    a.vpt = (int)g.views_per_turn;
    a.n_rows = (int)g.n_rows;
    a.n_cols = (int)g.n_cols;
    a.gcols = (int)p.gf_cols;
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
    const double hdl = p.h * p.dlam;
    a.hdl = (float)hdl;
    a.hdl_lo = (float)(hdl - (double)a.hdl);
    const double K = (-0.5 * (double)(g.n_cols - 1) * g.d_alpha + g.alpha_offset) / g.d_alpha;
    a.K_hi = (float)K;
    a.K_lo = (float)(K - (double)a.K_hi);
    return a;
}


// Checked build only: columns taken off every staged window, so that a test can see the column
// check fire (the taps stay clamped inside the window, the result is wrong, nothing faults).
static std::atomic<int> g_debug_narrow{0};
// Checked build only: launch as if the plan's PI windows were not monotone in z (every view takes
// the general end-weight path), so that a test can compare that path with the ramp walk.
static std::atomic<int> g_debug_nonmono{0};

// Staged window width: the tile's columns (B2_TX x B2_TY voxel centres) subtend at
// most 2 atan(L / 2 d) with L the tile diagonal and d = R - r_fov the nearest
// source distance; add floor and alignment slack.
static int window_cols(const Plan &p)
{
    const kats_geometry &g = p.g;
    const double L = std::hypot((B2_TX - 1) * g.dx, (B2_TY - 1) * g.dy);
    const double xa = fabs(g.x0 - 0.5 * g.dx), xb = fabs(g.x0 + ((double)g.nx - 0.5) * g.dx);
    const double ya = fabs(g.y0 - 0.5 * g.dy), yb = fabs(g.y0 + ((double)g.ny - 0.5) * g.dy);
    const double rf = std::hypot(std::max(xa, xb), std::max(ya, yb));
    const double span = 2.0 * atan(L / (2.0 * (g.R - rf))) / g.d_alpha;
    return ((int)ceil(span) + 8 + 3) / 4 * 4;
}

template <int PITCH, int MODE, int RP>
static auto select_tma(bool ranged, bool rows_ok)
{
    return ranged ? (rows_ok ? k_backproject_tma<PITCH, MODE, true, true, RP> : k_backproject_tma<PITCH, MODE, false, true, RP>)
                  : (rows_ok ? k_backproject_tma<PITCH, MODE, true, false, RP>
                             : k_backproject_tma<PITCH, MODE, false, false, RP>);
}

template <int PITCH, int MODE>
static int launch_tma(const Plan &p, const BPArgs &a, const void *gF, int W, cudaStream_t st, bool *launched,
                      int lead_end)
{
    *launched = false;
    // staged rows: fp32 -> detector rows -1 .. n_rows + 1; row pairs -> pair-rows 0 .. n_rows + 1
    const int srows = (int)p.g.n_rows + (MODE == 0 ? 3 : 2);
    const int slot = (PITCH * srows + 31) / 32 * 32;
    // 3 slot pairs where two CTAs still fit on an SM (228 KB less 1 KB per CTA and the static shared
    // memory), else 2 pairs; + 128 bytes of base alignment slack
    auto ring_bytes = [&](int rp) { return sizeof(float) * (size_t)slot * 2 * rp + 128; };
    constexpr size_t kTwoPerSm = 112 * 1024, kMax = 200 * 1024;
    const int rp = ring_bytes(3) <= kTwoPerSm || ring_bytes(2) > kTwoPerSm ? (ring_bytes(3) <= kMax ? 3 : 2) : 2;
    const size_t smem = ring_bytes(rp);
    EncodeTiledFn enc = encode_fn();
    if (!enc || W > PITCH || PITCH > p.gf_cols || srows > 256 || smem > kMax ||
        (reinterpret_cast<uintptr_t>(gF) % 16) != 0 || p.n_fviews >= INT32_MAX || !(p.geo_tmax <= kTileTanMax))
        return KATS_OK;
    const int64_t drows = p.g.n_rows + (MODE == 0 ? 0 : 1);
    CUtensorMap map;
    cuuint64_t dims[3] = {(cuuint64_t)p.gf_cols, (cuuint64_t)drows, (cuuint64_t)p.n_fviews};
    cuuint64_t strides[2] = {(cuuint64_t)p.gf_cols * 4, (cuuint64_t)(p.gf_cols * drows) * 4};
    cuuint32_t box[3] = {(cuuint32_t)PITCH, (cuuint32_t)srows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)gF, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return KATS_OK;
    BP2Args b{a, W, srows, slot, p.dev_status, (float)(p.dlam / (2.0 * kPi) / (MODE == 0 ? 1.0 : p.g.d_alpha)),
              p.pi_monotone && !g_debug_nonmono.load() ? 1 : 0, p.geo, p.geo_ntx};
    // every contributing row within half a row of the detector (plan extents, FP32 on device)
    const double w_first = -0.5 * (double)(p.g.n_rows - 1) * p.g.d_w + p.g.w_offset;
    const double w_last = w_first + (double)(p.g.n_rows - 1) * p.g.d_w;
    const bool rows_ok = p.ext[4] >= w_first - 0.5 * p.g.d_w && p.ext[5] <= w_last + 0.5 * p.g.d_w;
    const bool ranged = a.k_lo != INT32_MIN || a.k_hi != INT32_MAX || a.acc_in || !a.acc_final;
    auto kern = rp == 3 ? select_tma<PITCH, MODE, 3>(ranged, rows_ok) : select_tma<PITCH, MODE, 2>(ranged, rows_ok);
    KATS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned gx = (unsigned)ceil_div(p.g.nx, B2_TX), gy = (unsigned)ceil_div(p.g.ny, B2_TY);
    // slices [s, e) in 16-slice z tiles
    // The launches of one call write disjoint slices from inputs complete before the first starts, so
    // each launch after the first may begin while the previous one's last wave drains (programmatic
    // dependent launch; measured 33.5 -> 33.0 ms at config 2).  Launches over a share of the views
    // continue each other's sums and stay fully ordered.
    int n_launched = 0;
    auto launch = [&](auto kernel, dim3 grid, size_t shm, auto... args) -> cudaError_t {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = dim3(B2_THREADS);
        cfg.dynamicSmemBytes = shm;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = (!ranged && n_launched > 0) ? 1 : 0;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        ++n_launched;
        return cudaLaunchKernelEx(&cfg, kernel, args...);
    };
    // slices [s, e) in 16-slice z tiles; without view ranges a last partial tile of at least half a
    // tile goes to the PARTIAL form (a smaller one costs less on the weighted path, which skips the
    // missing slices' pairs)
    auto single = [&](int s, int e) -> int {
        if (e <= s) return KATS_OK;
        const int rem = (e - s) % B2_T;
        const int e_full = ranged || rem < B2_T / 2 ? e : e - rem;
        BP2Args bs = b;
        if (e_full > s) {
            bs.a.s_begin = s;
            bs.a.s_end = e_full;
            KATS_CUDA(launch(kern, dim3(gx, gy, (unsigned)ceil_div(e_full - s, B2_T)), smem, map, bs));
            count_launches(1);
            KATS_CUDA(cudaGetLastError());
        }
        if (e_full < e) {
            auto kp = rp == 3 ? k_backproject_tma<PITCH, MODE, false, false, 3, true>
                              : k_backproject_tma<PITCH, MODE, false, false, 2, true>;
            KATS_CUDA(cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            bs.a.s_begin = e_full;
            bs.a.s_end = e;
            KATS_CUDA(launch(kp, dim3(gx, gy, 1), smem, map, bs));
            count_launches(1);
            KATS_CUDA(cudaGetLastError());
        }
        return KATS_OK;
    };
    // Slices one or more pitches apart share their views' geometry (Sec. II periodicity): where a
    // launch holds such slices and takes every view, k_backproject_multi reconstructs them together
    // and the rest go through the single kernel.
    bool multi = false;
    std::vector<std::pair<int, int>> rest;
    if (!ranged) {
        BP2Args bm = b;
        bm.srows = srows;
        int rc = launch_multi<MODE>(p, bm, gF, MultiLaunch{a.s_begin, a.s_end, rows_ok, lead_end}, st, &n_launched,
                                    &rest, &multi);
        if (rc) return rc;
    }
    if (multi) {
        for (const auto &r : rest) {
            int rc = single(r.first, r.second);
            if (rc) return rc;
        }
    } else {
        for (const auto &r : lead_ranges(a.s_begin, a.s_end, (int)p.N, lead_end)) {
            int rc = single(r.first, r.second);
            if (rc) return rc;
        }
    }
    *launched = true;
    return KATS_OK;
}

template <int MODE>
static int launch_tma_any(const Plan &p, const BPArgs &a, const void *gF, int W, cudaStream_t st, bool *launched,
                          int lead_end)
{
    if (W <= 32) return launch_tma<32, MODE>(p, a, gF, W, st, launched, lead_end);
    if (W <= 64) return launch_tma<64, MODE>(p, a, gF, W, st, launched, lead_end);
    if (W <= 128) return launch_tma<128, MODE>(p, a, gF, W, st, launched, lead_end);
    *launched = false;
    return KATS_OK;
}

int launch_backproject16(const Plan &p, int prec, const uint32_t *gFp, float *vol, cudaStream_t st, int s_begin,
                         int s_count, const BPRange &range)
{
    kats::NvtxRange nvtx_range("backprojection16 (step 7)");
    BPArgs a = bp_args(p);
    if (s_count >= 0) {
        a.s_begin = s_begin;
        a.s_end = std::min(s_begin + s_count, (int)p.g.nz);
    }
    a.k_lo = range.k_lo;
    a.k_hi = range.k_hi;
    a.acc_in = range.acc_in;
    a.acc_final = range.acc_final;
    a.gF = nullptr;
    a.vol = vol;
    bool launched = false;
    const int W = std::max(4, window_cols(p) - g_debug_narrow.load());
    if (range.lead_end != INT32_MAX && (range.k_lo != INT32_MIN || range.k_hi != INT32_MAX || range.acc_in ||
                                        !range.acc_final)) {
        set_error("a launch restricted to leading slices takes every view");
        return KATS_EINVAL;
    }
    int rc = prec == KATS_PREC_FP16 ? launch_tma_any<2>(p, a, gFp, W, st, &launched, range.lead_end)
                                    : launch_tma_any<1>(p, a, gFp, W, st, &launched, range.lead_end);
    if (rc) return rc;
    if (!launched) {
        set_error("reduced-precision backprojection needs the staged (TMA) kernel; this detector is narrower than "
                  "its column window");
        return KATS_EINVAL;
    }
    return KATS_OK;
}

int launch_backproject(const Plan &p, const float *gF, float *vol, cudaStream_t st, int s_begin, int s_count,
                       const BPRange &range)
{
    kats::NvtxRange nvtx_range("backprojection (step 7)");
    BPArgs a = bp_args(p);
    if (s_count >= 0) {
        a.s_begin = s_begin;
        a.s_end = std::min(s_begin + s_count, (int)p.g.nz);
    }
    a.k_lo = range.k_lo;
    a.k_hi = range.k_hi;
    a.acc_in = range.acc_in;
    a.acc_final = range.acc_final;
    a.gF = gF;
    a.vol = vol;
    const int W = std::max(4, window_cols(p) - g_debug_narrow.load());
    bool launched = false;
    if (range.lead_end != INT32_MAX && (range.k_lo != INT32_MIN || range.k_hi != INT32_MAX || range.acc_in ||
                                        !range.acc_final)) {
        set_error("a launch restricted to leading slices takes every view");
        return KATS_EINVAL;
    }
    int rc = launch_tma_any<0>(p, a, gF, W, st, &launched, range.lead_end);
    if (rc || launched) return rc;
    for (const auto &r : lead_ranges(a.s_begin, a.s_end, (int)p.N, range.lead_end)) {
        BPArgs ar = a;
        ar.s_begin = r.first;
        ar.s_end = r.second;
        dim3 grid((unsigned)ceil_div(p.g.nx, BP_BX), (unsigned)ceil_div(p.g.ny, BP_BY),
                  (unsigned)ceil_div(ar.s_end - ar.s_begin, BP_T));
        k_backproject<<<grid, dim3(BP_BX, BP_BY), 0, st>>>(ar);
        count_launches(1);
        KATS_CUDA(cudaGetLastError());
    }
    return KATS_OK;
}

// Transpose of step 7: each (voxel, view) term sends its weight times the
// voxel value to the four bilinear taps of that view (FP32 atomics).
__device__ __forceinline__ void splat(float *view, int r, int c, int n_rows, int n_cols, int gcols, float val)
{
    if (r >= 0 && r < n_rows && c >= 0 && c < n_cols) atomicAdd(view + r * gcols + c, val);
}

__global__ void __launch_bounds__(BP_BX *BP_BY) k_backproject_T(BPArgs a, const float *__restrict__ vol, float *gF)
{
    const int ix = blockIdx.x * BP_BX + threadIdx.x;
    const int iy = blockIdx.y * BP_BY + threadIdx.y;
    const int s0 = a.s_begin + blockIdx.z * BP_T;
    if (ix >= a.nx || iy >= a.ny) return;
    int ka[BP_T], kb[BP_T];
    float wa[BP_T], wb[BP_T], f[BP_T];
    int kmin = INT32_MAX, kmax = INT32_MIN;
#pragma unroll
    for (int t = 0; t < BP_T; ++t) {
        const int s = s0 + t;
        if (s < a.s_end) {
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
    float zb, zb_lo;
    z_base(a, s0, kmin, &zb, &zb_lo);
    int km = ((kmin % a.vpt) + a.vpt) % a.vpt;
    const int64_t per_view = (int64_t)a.n_rows * a.gcols;
    for (int k = kmin; k <= kmax; ++k) {
        float u, v;
        view_uv(a, __ldg(a.trig + km), __ldg(a.trig_lo + km), x, y, &u, &v);
        km = (km + 1 == a.vpt) ? 0 : km + 1;
        const float inv_v = 1.0f / v;
        int ci;
        float fc;
        column_split(a, atanf(u * inv_v) * a.inv_da, &ci, &fc);
        const float M = a.D * rsqrtf(u * u + v * v);
        const float zr = z_rel(a, zb, zb_lo, (float)(k - kmin));
        const float ur0 = (M * zr - a.w0row) * a.inv_dw;
        const float dur = M * a.dz_over_dw;
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
            splat(view, ri, ci, a.n_rows, a.n_cols, a.gcols, wv * (1.0f - fr) * (1.0f - fc));
            splat(view, ri, ci + 1, a.n_rows, a.n_cols, a.gcols, wv * (1.0f - fr) * fc);
            splat(view, ri + 1, ci, a.n_rows, a.n_cols, a.gcols, wv * fr * (1.0f - fc));
            splat(view, ri + 1, ci + 1, a.n_rows, a.n_cols, a.gcols, wv * fr * fc);
        }
    }
}

// Transpose of step 7 with a shared-memory window per view: a CTA of 16 x 16
// voxel columns x 16 slices adds its four bilinear taps per (voxel, view) into
// the view's detector window in shared memory (the window the forward kernel
// stages), then adds the window's non-zero entries to g^F with one global
// atomic each.  The window holds 32-bit fixed point (native integer shared
// atomics; float and 64-bit ones are compare-and-swap loops, 8-10 times slower
// here).  A thread first sums its slices' taps per detector row in registers
// (the rows rise with z), so it deposits into a window entry at most once per
// view, at most K taps per deposit (K from the smallest row step per slice,
// two per slice sharing the row).  The CTA's warps form G groups, each with
// its own copy of the window, so a copy's entry takes at most 256 / G
// deposits per view; with 2^hb >= (256 / G) K and the CTA's largest possible
// tap c_max < 2^e, the CTA scales by 2^s, s = 30 - hb - e, and a copy's entry
// stays below 2^30.  The drain adds the G copies in 64-bit integers.  Taps on
// clamped (off-detector) rows may wrap; those entries are never added to g^F.
// The quantum is 2^(hb-30) c_max (2^-22 c_max for the clinical scanners at
// G = 4).  Two windows alternate (one filling, one draining), one CTA barrier
// per view; the window's first column per view is computed at the tile
// corners one view ahead.
constexpr int BT_THREADS = B2_TX * B2_TY;

// x (already scaled: at most K taps of magnitude below 2^(30 - hb)) into the window at p.
__device__ __forceinline__ void deposit(int *p, float x) { atomicAdd(p, __float2int_rn(x)); }

template <int PITCH, bool ROWS_OK>
__global__ void __launch_bounds__(BT_THREADS, 2)
    k_backproject_T_win(BPArgs a, int W, int srows, int slot_floats, float out_scale, float inv_v_max, int hb,
                        int G, const float4 *__restrict__ geo, int geo_ntx, const float *__restrict__ vol, float *gF)
{
    constexpr int SH = PITCH == 32 ? 5 : (PITCH == 64 ? 6 : 7);
    extern __shared__ int win[];  // [2 windows][G copies][slot_floats] fixed-point sums
    __shared__ int s_col[3];
    // staged rows [s_rlo, s_rhi] touched in view j, slot j % 3 (reset two views ahead of its use)
    __shared__ int s_rlo[3], s_rhi[3];
    __shared__ int s_K0, s_K1;
    __shared__ float s_fmax[BT_THREADS / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tx = tid % B2_TX, ty = tid / B2_TX;
    int bx, by;
    cta_tile(&bx, &by);
    const int ix = bx * B2_TX + tx, iy = by * B2_TY + ty;
    const int s0 = a.s_begin + blockIdx.z * B2_T;
    const bool active = ix < a.nx && iy < a.ny;

    int kmin = INT32_MAX, kmax = INT32_MIN, kfull_lo = INT32_MIN, kfull_hi = INT32_MAX;
    float lo[B2_T], hi[B2_T], f[B2_T];
    {
        int ka[B2_T], kb[B2_T];
        float wa[B2_T], wb[B2_T];
#pragma unroll
        for (int t = 0; t < B2_T; ++t) {
            const int s = s0 + t;
            ka[t] = INT32_MAX;
            kb[t] = INT32_MIN;
            wa[t] = wb[t] = f[t] = 0.0f;
            if (active && s < a.s_end) {
                const int j = s % a.N, m = s / a.N;
                const int64_t o = ((int64_t)j * a.ny + iy) * a.nx + ix;
                ka[t] = a.k0[o] + m * a.vpt;
                kb[t] = a.k1[o] + m * a.vpt;
                wa[t] = a.w0[o];
                wb[t] = a.w1[o];
                f[t] = vol[((int64_t)s * a.ny + iy) * a.nx + ix] * out_scale;
                if (ka[t] <= kb[t]) {
                    kmin = min(kmin, ka[t]);
                    kmax = max(kmax, kb[t]);
                }
            }
            kfull_lo = max(kfull_lo, ka[t]);
            kfull_hi = min(kfull_hi, kb[t]);
        }
        const int kbase = kmin <= kmax ? kmin : 0;
#pragma unroll
        for (int t = 0; t < B2_T; ++t) {
            if (ka[t] <= kb[t]) {
                lo[t] = (float)(ka[t] - kbase) - wa[t];
                hi[t] = (float)(kb[t] - kbase) + wb[t];
            } else {
                lo[t] = 3.0e9f;
                hi[t] = -3.0e9f;
            }
        }
    }
    if (tid == 0) {
        s_K0 = INT32_MAX;
        s_K1 = INT32_MIN;
        for (int q = 0; q < 3; ++q) {
            s_rlo[q] = INT32_MAX;
            s_rhi[q] = -1;
        }
    }
    float fm = 0.0f;
#pragma unroll
    for (int t = 0; t < B2_T; ++t) fm = fmaxf(fm, fabsf(f[t]));
    for (int o = 16; o > 0; o >>= 1) fm = fmaxf(fm, __shfl_xor_sync(0xffffffffu, fm, o));
    if (lane == 0) s_fmax[warp] = fm;
    for (int e = tid; e < 2 * G * slot_floats; e += BT_THREADS) win[e] = 0;
    __syncthreads();
    // fixed-point scale: 2^(30 - hb - e) with the largest tap below 2^e
    fm = 0.0f;
    for (int w8 = 0; w8 < BT_THREADS / 32; ++w8) fm = fmaxf(fm, s_fmax[w8]);
    int ex = 0;
    frexpf(fm * inv_v_max, &ex);
    const float scale = fm > 0.0f ? exp2f((float)min(30 - hb - ex, 126)) : 0.0f;
    const float inv_scale = fm > 0.0f ? exp2f(-(float)min(30 - hb - ex, 126)) : 0.0f;
    if (kmin <= kmax) {
        atomicMin(&s_K0, kmin);
        atomicMax(&s_K1, kmax);
    }
    __syncthreads();
    const int K0 = s_K0, K1 = s_K1;
    if (K0 > K1) return;  // uniform: no voxel of the tile has a PI view
    const int nviews = K1 - K0 + 1;

    // first window column of view k: the plan's table (lowest column touched at the tile corners,
    // one column of slack, 16-byte aligned)
    const float4 *geo_t = geo + (size_t)(by * geo_ntx + bx) * a.vpt * 2;
    auto window_col = [&](int k) {
        const int km = ((k % a.vpt) + a.vpt) % a.vpt;
        return __float_as_int(__ldg(geo_t + 2 * km + 1).w);
    };
    if (warp == 0) {
        const int c = window_col(K0);
        if (lane == 0) s_col[0] = c;
    }
    __syncthreads();

    const float ox = ((float)tx - 0.5f * (B2_TX - 1)) * a.dx, oy = ((float)ty - 0.5f * (B2_TY - 1)) * a.dy;
    const int kbase = kmin <= kmax ? kmin : 0;
    float zb, zb_lo;
    z_base(a, s0, kbase, &zb, &zb_lo);
    const float rmax = (float)(a.n_rows + 1);
    const int64_t per_view = (int64_t)a.n_rows * a.gcols;
    const int wsize = srows * PITCH;
    int km = ((K0 % a.vpt) + a.vpt) % a.vpt;
    for (int j = 0; j < nviews; ++j) {
        const int k = K0 + j;
        const int b = j & 1;
        if (warp == 0 && j + 1 < nviews) {
            const int c = window_col(k + 1);
            if (lane == 0) {
                s_col[(j + 1) % 3] = c;
                // the band of view j + 1 is filled after this iteration's barrier; its slot was last
                // read by the drain of view j - 2, which every thread finished before view j - 1's barrier
                s_rlo[(j + 1) % 3] = INT32_MAX;
                s_rhi[(j + 1) % 3] = -1;
            }
        }
        int r_first = INT32_MAX, r_last = -1;  // staged rows this thread deposits into in view k
        if (active && k >= kmin && k <= kmax) {
            // the voxel's ray against its tile centre's (the forward kernel's tile-relative geometry)
            const float2 cs = __ldg(a.trig + km);
            const float4 g0 = __ldg(geo_t + 2 * km), g1 = __ldg(geo_t + 2 * km + 1);
            const float du = fmaf(-ox, cs.y, fmaf(oy, cs.x, g0.z));
            const float dv = fmaf(-ox, cs.x, fmaf(-oy, cs.y, g0.w));
            const float cross = fmaf(du, g0.y, dv * -g0.x);
            const float dot = fmaf(g0.x, du, fmaf(g0.y, dv, g1.x));
            const float cr = fmaf(atan_small(cross * rcp_approx(dot)), a.inv_da, g1.z) + g1.y;
            const float yv = __fadd_rd(cr, 12582912.0f);  // 1.5 * 2^23 + floor(cr)
            const int ci = __float_as_int(yv) - 0x4B400000;
            const float fc = cr - (yv - 12582912.0f);
            const float v = g0.y + dv, u = g0.x + du;
            const float inv_v = rcp_approx(v);
            KATS_DCHECK(ci >= 0 && ci <= W - 2, 4);
            const uint32_t colx = (uint32_t)((b * G + (warp & (G - 1))) * slot_floats + min(max(ci, 0), W - 2)) -
                                  (0x4B000000u << SH);
            const float M = a.D * rsqrtf(fmaf(u, u, v * v));
            const float kf = (float)(k - kbase);
            const float ur0 = (M * z_rel(a, zb, zb_lo, kf) - a.w0row) * a.inv_dw + 1.0f;
            const float dur = M * a.dz_over_dw;
            const bool full = k > kfull_lo && k < kfull_hi;
            // The slices' rows rise with t (dur > 0), so a thread's taps of one view fall
            // on a run of rows of two columns: sum them per row in registers (rows qa and
            // qa + PITCH pending) and deposit a row once the run has moved past it.
            constexpr uint32_t kNone = 0xFFFFFFFFu;
            uint32_t qa = kNone;  // window offset of the pending top row
            uint32_t q_first = kNone;
            float a0 = 0.0f, a1 = 0.0f, b0 = 0.0f, b1 = 0.0f;  // pending rows, columns ci and ci + 1
#pragma unroll
            for (int t = 0; t < B2_T; ++t) {
                const float om = full ? 1.0f : __saturatef(kf - lo[t]) * __saturatef(hi[t] - kf);
                const float wv = om * inv_v * f[t];
                if (wv == 0.0f) continue;
                float ur = fmaf((float)t, dur, ur0);
                if (!ROWS_OK) ur = fminf(fmaxf(ur, 0.0f), rmax);
#ifdef KATS_DEBUG_CHECKS
                else if (!(ur >= 0.0f && ur <= rmax)) {
                    atomicOr(&g_debug_flags, 8);
                    ur = fminf(fmaxf(ur, 0.0f), rmax);
                }
#endif
                const float yv = __fadd_rd(ur, 8388608.0f);
                const uint32_t q = colx + ((uint32_t)__float_as_int(yv) << SH);
                const float fr = ur - (yv - 8388608.0f);
                const float top = wv * scale * (1.0f - fr), bot = wv * scale * fr;
                if (q != qa) {
                    if (qa == kNone) q_first = q;
                    if (qa != kNone) {
                        deposit(win + qa, a0);
                        deposit(win + qa + 1, a1);
                    }
                    if (qa != kNone && q == qa + PITCH) {  // down one row: the old bottom row becomes the top
                        a0 = b0;
                        a1 = b1;
                    } else {
                        if (qa != kNone) {
                            deposit(win + qa + PITCH, b0);
                            deposit(win + qa + PITCH + 1, b1);
                        }
                        a0 = a1 = 0.0f;
                    }
                    b0 = b1 = 0.0f;
                    qa = q;
                }
                a0 = fmaf(top, 1.0f - fc, a0);
                a1 = fmaf(top, fc, a1);
                b0 = fmaf(bot, 1.0f - fc, b0);
                b1 = fmaf(bot, fc, b1);
            }
            if (qa != kNone) {
                deposit(win + qa, a0);
                deposit(win + qa + 1, a1);
                deposit(win + qa + PITCH, b0);
                deposit(win + qa + PITCH + 1, b1);
                const uint32_t base = colx + (0x4B000000u << SH);  // window offset of staged row 0
                r_first = (int)((q_first - base) >> SH);
                r_last = (int)((qa - base) >> SH) + 1;
            }
        }
        r_first = __reduce_min_sync(0xffffffffu, r_first);
        r_last = __reduce_max_sync(0xffffffffu, r_last);
        if (lane == 0 && r_last >= 0) {
            atomicMin(&s_rlo[j % 3], r_first);
            atomicMax(&s_rhi[j % 3], r_last);
        }
        if (++km == a.vpt) km = 0;
        __syncthreads();  // window b of view k is complete; window b^1 (view k-1) has been drained
        // drain window b into g^F: staged row 0 is detector row -1, columns from s_col
        const int col0 = s_col[j % 3];
        int *w = win + b * G * slot_floats;
        float *view = gF + (int64_t)(k - a.first_view) * per_view;
        // only the staged rows some thread deposited into can be nonzero
        const int rlo = s_rlo[j % 3], rhi = s_rhi[j % 3];
        const int e_end = rhi >= 0 ? min((rhi + 1) * PITCH, wsize) : 0;
        for (int e = (rhi >= 0 ? rlo * PITCH : 0) + tid; e < e_end; e += BT_THREADS) {
            long long q = 0;
            for (int gi = 0; gi < G; ++gi) {
                int *we = w + gi * slot_floats + e;
                q += *we;
                *we = 0;
            }
            if (q == 0) continue;
            const int r = e / PITCH - 1, c = col0 + e % PITCH;
            if (r >= 0 && r < a.n_rows && c >= 0 && c < a.n_cols)
                atomicAdd(view + r * a.gcols + c, (float)q * inv_scale);
        }
    }
}

template <int PITCH>
static int launch_adjoint_win(const Plan &p, const BPArgs &a, const float *vol, float *gF, int W, cudaStream_t st,
                              bool *launched)
{
    *launched = false;
    const int srows = (int)p.g.n_rows + 3;
    const int slot = (PITCH * srows + 31) / 32 * 32;
    // window copies: 4 where two CTAs per SM still fit, else 2, else 1
    auto ring_bytes = [&](int copies) { return sizeof(int) * (size_t)slot * 2 * copies; };
    const int G = ring_bytes(4) <= 100 * 1024 ? 4 : (ring_bytes(2) <= 100 * 1024 ? 2 : 1);
    const size_t smem = ring_bytes(G);
    if (W > PITCH || smem > 100 * 1024 || p.n_fviews >= INT32_MAX || !(p.g.R > p.r_fov)) return KATS_OK;
    // headroom: a row step per slice of at least dur_min = D / (R + r_max) dz / d_w puts at most
    // floor(1 / dur_min) + 1 of a thread's slices on one row, two taps each (that row as top or bottom)
    const kats_geometry &g = p.g;
    const double xa = fabs(g.x0 - 0.5 * g.dx), xb = fabs(g.x0 + ((double)g.nx - 0.5) * g.dx);
    const double ya = fabs(g.y0 - 0.5 * g.dy), yb = fabs(g.y0 + ((double)g.ny - 0.5) * g.dy);
    const double r_max = std::hypot(std::max(xa, xb), std::max(ya, yb));
    const double dur_min = g.D / (g.R + r_max) * g.dz / g.d_w;
    if (!(dur_min > 0.0)) return KATS_OK;
    const double taps = 2.0 * (std::floor(1.0 / dur_min) + 1.0);
    const int hb = (int)std::ceil(std::log2((double)(BT_THREADS / G) * taps));
    if (hb > 24) return KATS_OK;  // quantum coarser than 2^-6 c_max: leave it to the global-atomic kernel
    if (!(p.geo_tmax <= kTileTanMax)) return KATS_OK;
    const double w_first = -0.5 * (double)(p.g.n_rows - 1) * p.g.d_w + p.g.w_offset;
    const double w_last = w_first + (double)(p.g.n_rows - 1) * p.g.d_w;
    const bool rows_ok = p.ext[4] >= w_first - 0.5 * p.g.d_w && p.ext[5] <= w_last + 0.5 * p.g.d_w;
    auto kern = rows_ok ? k_backproject_T_win<PITCH, true> : k_backproject_T_win<PITCH, false>;
    KATS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((unsigned)ceil_div(p.g.nx, B2_TX), (unsigned)ceil_div(p.g.ny, B2_TY),
              (unsigned)ceil_div(a.s_end - a.s_begin, B2_T));
    // 1/v* <= 1/(R - r_fov) for every voxel column, rounded up
    const float inv_v_max = (float)(1.0 / (p.g.R - p.r_fov)) * 1.0001f;
    kern<<<grid, BT_THREADS, smem, st>>>(a, W, srows, slot, (float)(p.dlam / (2.0 * kPi)), inv_v_max, hb, G, p.geo,
                                         p.geo_ntx, vol, gF);
    count_launches(1);
    KATS_CUDA(cudaGetLastError());
    *launched = true;
    return KATS_OK;
}

int launch_backproject_adjoint(const Plan &p, const float *vol, float *gF, cudaStream_t st)
{
    BPArgs a = bp_args(p);
    a.gF = gF;
    a.vol = nullptr;
    KATS_CUDA(cudaMemsetAsync(gF, 0, sizeof(float) * (size_t)(p.n_fviews * p.g.n_rows * p.gf_cols), st));
    const int W = std::max(4, window_cols(p) - g_debug_narrow.load());
    bool launched = false;
    int rc = KATS_OK;
    if (W <= 32)
        rc = launch_adjoint_win<32>(p, a, vol, gF, W, st, &launched);
    else if (W <= 64)
        rc = launch_adjoint_win<64>(p, a, vol, gF, W, st, &launched);
    else if (W <= 128)
        rc = launch_adjoint_win<128>(p, a, vol, gF, W, st, &launched);
    if (rc || launched) return rc;
    dim3 grid((unsigned)ceil_div(p.g.nx, BP_BX), (unsigned)ceil_div(p.g.ny, BP_BY),
              (unsigned)ceil_div(a.s_end - a.s_begin, BP_T));
    k_backproject_T<<<grid, dim3(BP_BX, BP_BY), 0, st>>>(a, vol, gF);
    count_launches(1);
    KATS_CUDA(cudaGetLastError());
    return KATS_OK;
}

}  // namespace kats

extern "C" {

int katsevich_debug_checks_enabled(void)
{
#ifdef KATS_DEBUG_CHECKS
    return 1;
#else
    return 0;
#endif
}

void katsevich_debug_narrow_window(int cols)
{
#ifdef KATS_DEBUG_CHECKS
    kats::g_debug_narrow.store(cols > 0 ? cols : 0);
#else
    (void)cols;
#endif
}

void katsevich_debug_nonmonotone(int on)
{
#ifdef KATS_DEBUG_CHECKS
    kats::g_debug_nonmono.store(on ? 1 : 0);
#else
    (void)on;
#endif
}

int katsevich_debug_wait_limit(int polls)
{
#ifdef KATS_DEBUG_CHECKS
    const int v = polls > 0 ? polls : kats::kWaitLimit;
    KATS_CUDA(cudaMemcpyToSymbol(kats::g_debug_wait_limit, &v, sizeof(int)));
    int rc = kats::multi_debug_set(v, INT32_MIN);
    if (rc) return rc;
#else
    (void)polls;
#endif
    return KATS_OK;
}

int katsevich_debug_stall_producer(int pairs)
{
#ifdef KATS_DEBUG_CHECKS
    const int v = pairs >= 0 ? pairs : -1;
    KATS_CUDA(cudaMemcpyToSymbol(kats::g_debug_stall_pairs, &v, sizeof(int)));
    int rc = kats::multi_debug_set(0, v);
    if (rc) return rc;
#else
    (void)pairs;
#endif
    return KATS_OK;
}

int katsevich_debug_check_flags(int *flags)
{
    if (!flags) {
        kats::set_error("bad argument");
        return KATS_EINVAL;
    }
    KATS_CUDA(cudaDeviceSynchronize());
    int v = 0;
    KATS_CUDA(cudaMemcpyFromSymbol(&v, kats::g_debug_flags, sizeof(int)));
    const int zero = 0;
    KATS_CUDA(cudaMemcpyToSymbol(kats::g_debug_flags, &zero, sizeof(int)));
    int vm = 0;
    int rc = kats::multi_debug_take_flags(&vm);
    if (rc) return rc;
    *flags = v | vm;
    return KATS_OK;
}

}  // extern "C"
