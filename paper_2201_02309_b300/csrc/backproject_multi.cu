// Step 7 (Sec. II backprojection) for slices one or more pitches apart: k_backproject_multi.
//
// By the periodicity of Sec. II a slice m pitches above slice s has s's PI window shifted by m
// turns, and at view k + m * views_per_turn it sees the same alpha*, v* and w* as slice s at view
// k.  A CTA owns B2_TX x B2_TY columns and G groups of T slices, group m at s0 + m N; a thread
// computes each view's geometry, window classification and end weights once for all G groups,
// and only the taps differ: for every step the producer warp stages view k for group 0 and views
// k + m * views_per_turn for the others, with the same columns and rows, into G slots of a ring
// entry.  One view per consumer iteration; ring of RP entries with one full / empty mbarrier
// each.
//
// Band staging: a view's taps from T consecutive slices of a 16 x 16 column tile fall in a band of
// detector rows far narrower than the detector when T is small.  Where every contributing tap lies
// within half a row of the detector (the plan's row extents), the producer stages only a band of
// box_rows rows per view, starting at the lowest row any group-0 slice can read there: with the
// tile centre's distance rho from the source (its table row) and the tile's largest voxel offset
// hd, a voxel's magnification D / rho' has rho' in [rho - hd, rho + hd], and the lowest row is the
// smaller of the two magnifications times the lowest slice's z offset.  box_rows bounds the band's
// height over every tile and view (band_rows below); the consumers subtract the band's first row
// from their tap addresses, so the taps and their rounding equal the whole-window form's.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "bp_staged.cuh"

namespace kats {

namespace {

constexpr int kMaxMultiItems = 64;
struct MultiItems {
    int n;
    int s0[kMaxMultiItems];   // group 0's first slice; group m starts N m slices higher
    int cnt[kMaxMultiItems];  // slices per group, <= T (< T only in a PARTIAL launch)
};

constexpr int kFullRows = 72;              // slot rows of the whole-window form (n_rows + 3 <= 72)
constexpr int kRingFloats = 111 * 256;     // one CTA's ring: 111 KB, two CTAs per SM
constexpr int kGuardRows = 8;              // rows of slack before and after a band ring

// Ring geometry of one instantiation: slots of PITCH x HS floats, G per entry, RP entries, and
// kGuardRows rows of slack on both sides of a band ring.
template <int G, int HS, int PITCH>
struct MultiRing {
    static constexpr int SLOT = PITCH * HS;
    static constexpr int GUARD = HS >= kFullRows ? 0 : kGuardRows * PITCH;
    static constexpr int RP0 = (kRingFloats - 2 * GUARD) / (G * SLOT);
    static constexpr int RP = RP0 > 5 ? 5 : RP0;
    static constexpr size_t BYTES = sizeof(float) * (size_t)(2 * GUARD + RP * G * SLOT) + 128;
};

// PARTIAL: items with fewer than T slices per group; the missing slices take every view with
// clamped rows and are not stored (as in k_backproject_tma's PARTIAL form); launched with ROWS_OK
// false.
template <int PITCH, int MODE, bool ROWS_OK, int G, int T, int HS, bool PARTIAL>
__global__ void __launch_bounds__(B2_THREADS, 2)
    k_backproject_multi(const __grid_constant__ CUtensorMap gmap, BP2Args p, const __grid_constant__ MultiItems it)
{
    using Ring = MultiRing<G, HS, PITCH>;
    constexpr int SLOT = Ring::SLOT, RP = Ring::RP;
    static_assert(SLOT % 32 == 0, "slots start on 128-byte boundaries (TMA destinations)");
    static_assert(Ring::GUARD % 32 == 0, "the guard keeps the slots on 128-byte boundaries");
    static_assert(RP >= 2, "a ring of at least two entries");
    static_assert(!PARTIAL || !ROWS_OK, "missing slices read clamped rows");
    static_assert(T % 2 == 0, "slices go in pairs");
    extern __shared__ __align__(128) float smem[];
    // a backprojection launch that follows this one on the stream (other slices, same inputs) may
    // start its CTAs while this grid's last wave drains
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __shared__ __align__(8) uint64_t s_full[RP], s_empty[RP];
    __shared__ float4 s_geo[RP][2];  // the view's table rows (tile reference ray, window start)
    __shared__ float2 s_cs[RP];      // its (cos, sin)
    __shared__ int s_row[RP];        // the entry's first staged row
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
    const int s0 = it.s0[blockIdx.z], cnt = PARTIAL ? it.cnt[blockIdx.z] : T;
    const bool active = !producer && ix < a.nx && iy < a.ny;
    // slots start at the first 128-byte boundary of the dynamic shared memory after the guard
    const int base = (int)(((128u - (smem_addr(smem) & 127u)) & 127u) >> 2) + Ring::GUARD;

    // per-slice view windows of group 0 (group m's are m turns later)
    int kmin = INT32_MAX, kmax = INT32_MIN, kfull_lo = INT32_MIN, kfull_hi = INT32_MAX;
    float lo[T], hi[T];
    float2 acc[G][T / 2];
    {
        int ka[T], kb[T];
        float wa[T], wb[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int s = s0 + t;
            ka[t] = INT32_MAX;
            kb[t] = INT32_MIN;
            wa[t] = wb[t] = 0.0f;
            if (active && t < cnt) {
                const int j = s % a.N, m = s / a.N;
                const int64_t o = ((int64_t)j * a.ny + iy) * a.nx + ix;
                ka[t] = a.k0[o] + m * a.vpt;
                kb[t] = a.k1[o] + m * a.vpt;
                wa[t] = a.w0[o];
                wb[t] = a.w1[o];
                kmin = min(kmin, ka[t]);
                kmax = max(kmax, kb[t]);
            }
            if (!(PARTIAL && active && t >= cnt)) {
                kfull_lo = max(kfull_lo, ka[t]);
                kfull_hi = min(kfull_hi, kb[t]);
            }
        }
        if (!p.mono) {
            kfull_lo = INT32_MAX;
            kfull_hi = INT32_MIN;
        }
        const int kbase = active ? kmin : 0;
#pragma unroll
        for (int m = 0; m < G; ++m)
#pragma unroll
            for (int t = 0; t < T / 2; ++t) acc[m][t] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const bool missing = PARTIAL && t >= cnt;  // open in every view, not stored
            lo[t] = missing ? -3.0e9f : (float)(ka[t] - kbase) - wa[t];
            hi[t] = missing ? 3.0e9f : (float)(kb[t] - kbase) + wb[t];
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
    if (active) {
        atomicMin(&s_K0, kmin);
        atomicMax(&s_K1, kmax);
    }
    __syncthreads();
    const int K0 = s_K0, K1 = s_K1;
    if (K0 > K1) return;  // uniform: no column of the tile in the volume
    const int nviews = K1 - K0 + 1;

    if (producer) {
        const float4 *geo_t = p.geo + (size_t)(by * p.geo_ntx + bx) * a.vpt * 2;
        const uint32_t box_bytes = (uint32_t)(PITCH * p.box_rows * 4);
        const uint32_t dst0 = smem_addr(smem) + 4u * (uint32_t)base;
        // group 0's lowest slice relative to the source at view K0 + j: z_rel(zb, zb_lo, j)
        float zb, zb_lo;
        z_base(a, s0, K0, &zb, &zb_lo);
        const int row_hi = p.srows - p.box_rows;
        int ps = 0, issued = 0;
        uint32_t phase = 0;
        int kmod = ((K0 % a.vpt) + a.vpt) % a.vpt;
        bool ok = true;
        float4 g0, g1;
        float2 cs;
        if (lane == 0) {
            g0 = __ldg(geo_t + 2 * kmod);
            g1 = __ldg(geo_t + 2 * kmod + 1);
            cs = __ldg(a.trig + kmod);
        }
        for (int j = 0; j < nviews; ++j) {
#ifdef KATS_DEBUG_CHECKS
            if (g_debug_stall_pairs >= 0 && j >= g_debug_stall_pairs) break;  // test hook: stop issuing
#endif
            if (j >= RP && !mbar_wait(&s_empty[ps], phase ^ 1u)) {
                ok = false;
                break;
            }
            if (lane == 0) {
                int row0 = 0;
                if (p.band) {
                    // lowest staged row (detector row + 1) a tap of the groups' slices in their
                    // windows can read: the lowest slice's offset zr times the magnification that
                    // makes it lowest, at least half a row inside the detector
                    const float rho = sqrtf(g1.x);
                    const float zr = z_rel(a, zb, zb_lo, (float)j);
                    const float M = a.D / (zr >= 0.0f ? rho + p.hd : rho - p.hd);
                    const float u = fmaxf(fmaf(fmaf(M, zr, -a.w0row), a.inv_dw, 1.0f), 0.5f);
                    row0 = min(max((int)floorf(u - 0.5f), 0), row_hi);
                }
                s_row[ps] = row0;
                s_geo[ps][0] = g0;
                s_geo[ps][1] = g1;
                s_cs[ps] = cs;
                mbar_arrive_expect_tx(&s_full[ps], G * box_bytes);
                const int clo = __float_as_int(g1.w), kv = K0 + j - (int)a.first_view;
                // fp32 windows: staged row 0 is detector row -1; row-pair windows: pair-row 0
#pragma unroll
                for (int m = 0; m < G; ++m)
                    tma_load_3d(dst0 + 4u * (uint32_t)((ps * G + m) * SLOT), &gmap, &s_full[ps], clo,
                                row0 + (MODE == 0 ? -1 : 0), kv + m * a.vpt);
                kmod = kmod + 1 == a.vpt ? 0 : kmod + 1;
                if (j + 1 < nviews) {
                    g0 = __ldg(geo_t + 2 * kmod);
                    g1 = __ldg(geo_t + 2 * kmod + 1);
                    cs = __ldg(a.trig + kmod);
                }
            }
            __syncwarp();
            issued = j + 1;
            if (++ps == RP) {
                ps = 0;
                phase ^= 1u;
            }
        }
        if (lane == 0) {
            // every copy issued lands before the producer retires (see k_backproject_tma)
            bool landed = true;
            for (int i = max(0, issued - RP); i < issued; ++i)
                landed = mbar_wait(&s_full[i % RP], (uint32_t)((i / RP) & 1)) && landed;
            if (!ok || !landed) atomicExch(p.status, kDevStatusTimeout);
        }
        return;
    }

    const float ox = ((float)tx - 0.5f * (B2_TX - 1)) * a.dx, oy = ((float)ty - 0.5f * (B2_TY - 1)) * a.dy;
    const int kbase = active ? kmin : 0;
    float zb, zb_lo;
    z_base(a, s0, kbase, &zb, &zb_lo);
    // rows whose taps stay inside a slot: fp32 reads rows r and r + 1, row pairs the word at r
    const float rspan = (float)(p.box_rows - (MODE == 0 ? 2 : 1));
    constexpr int SH = PITCH == 32 ? 5 : (PITCH == 64 ? 6 : 7);
    int ps = 0;
    uint32_t phase = 0;
    for (int j = 0; j < nviews; ++j) {
        const int k = K0 + j;
        if (!__all_sync(0xffffffffu, mbar_wait(&s_full[ps], phase))) {
            if (lane == 0) atomicExch(p.status, kDevStatusTimeout);
            return;
        }
        if (active && k >= kmin && k <= kmax) {
            const float kf = (float)(k - kbase);
            ViewGeo1 g;
            view_geo1(a, ox, oy, s_cs[ps], s_geo[ps][0], s_geo[ps][1], zb, zb_lo, kf, g);
            KATS_DCHECK(g.ci >= 0 && g.ci <= p.W - 2, 1);
            const int row0 = s_row[ps];
            const float rmin = (float)row0, rmax = rmin + rspan;
            // staged row r of the entry's slots holds row r of the window from row0 on
            const uint32_t colx = (uint32_t)(base + ps * G * SLOT + min(max(g.ci, 0), p.W - 2)) -
                                  (0x4B000000u << SH) - ((uint32_t)row0 << SH);
            if (k > kfull_lo && k < kfull_hi)
                bp_view<PITCH, MODE, false, !ROWS_OK, T, G, SLOT>(smem, colx, g.fc, g.ur0, g.dur, rmin, rmax, g.inv_v,
                                                                  kf, lo, hi, acc);
            else if (k < kfull_hi)
                bp_view_ramp<PITCH, MODE, true, !ROWS_OK, T, G, SLOT>(smem, colx, g.fc, g.ur0, g.dur, rmin, rmax,
                                                                      g.inv_v, kf, lo, hi, acc);
            else if (k > kfull_lo)
                bp_view_ramp<PITCH, MODE, false, !ROWS_OK, T, G, SLOT>(smem, colx, g.fc, g.ur0, g.dur, rmin, rmax,
                                                                       g.inv_v, kf, lo, hi, acc);
            else
                bp_view<PITCH, MODE, true, !ROWS_OK, T, G, SLOT>(smem, colx, g.fc, g.ur0, g.dur, rmin, rmax, g.inv_v,
                                                                 kf, lo, hi, acc);
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
    for (int m = 0; m < G; ++m)
#pragma unroll
        for (int t = 0; t < T; ++t) {
            if (PARTIAL && t >= cnt) break;
            const float v = (t & 1) ? acc[m][t >> 1].y : acc[m][t >> 1].x;
            a.vol[((int64_t)(s0 + m * a.N + t) * a.ny + iy) * a.nx + ix] = v * p.out_scale;
        }
}

// The instantiated (G, T, HS) forms.  Band rings hold HS rows per slot; every form also exists
// with whole windows (HS = kFullRows) for G = 2.
struct Form {
    int G, T, HS;
};
constexpr Form kBandForms[] = {{4, 8, 24}, {4, 6, 24}, {3, 10, 32}, {3, 8, 24}, {2, 14, 40}, {2, 12, 40}};
constexpr Form kFullForms[] = {{2, 14, kFullRows}, {2, 12, kFullRows}};

// Height in rows of the band that holds every tap of T consecutive slices of one tile at one view,
// plus the margins of the band's placement: with rho the tile centre's distance from the source,
// hd the largest voxel offset, M+ = D / (rho - hd), M- = D / (rho + hd), L = (T - 1) dz and the
// rows taken within half a row of the detector (|w| <= Wd), the taps' w span at most
// max(M+ L, Wd (1 - M- / M+) + M- L): the first when the slices straddle the source's height, the
// second when the band is cut by the detector's edge.  Both shrink as rho grows, so the bound is
// taken at the nearest a tile centre comes to the source, R - r_max.  The band's first row is
// floor(u_min - 1/2), u_min at least 1/2 row inside the detector: floor effects, the half-row
// margin and the second tap row add 4.
static int band_rows(const Plan &p, int T)
{
    const kats_geometry &g = p.g;
    const double hd = 0.5 * std::hypot((B2_TX - 1) * g.dx, (B2_TY - 1) * g.dy);
    const int ntx = (int)ceil_div(g.nx, B2_TX), nty = (int)ceil_div(g.ny, B2_TY);
    const double xc = std::max(std::fabs(g.x0 + 0.5 * (B2_TX - 1) * g.dx),
                               std::fabs(g.x0 + ((double)(ntx - 1) * B2_TX + 0.5 * (B2_TX - 1)) * g.dx));
    const double yc = std::max(std::fabs(g.y0 + 0.5 * (B2_TY - 1) * g.dy),
                               std::fabs(g.y0 + ((double)(nty - 1) * B2_TY + 0.5 * (B2_TY - 1)) * g.dy));
    const double rho = g.R - std::hypot(xc, yc);
    if (!(rho - hd > 0.0)) return INT32_MAX;
    const double mp = g.D / (rho - hd), mm = g.D / (rho + hd), L = (T - 1) * g.dz;
    const double w0 = -0.5 * (double)(g.n_rows - 1) * g.d_w + g.w_offset;
    const double wd = std::max(std::fabs(w0 - 0.5 * g.d_w), std::fabs(w0 + ((double)g.n_rows - 0.5) * g.d_w));
    const double span = std::max(mp * L, wd * (1.0 - mm / mp) + mm * L);
    return (int)std::ceil(span / g.d_w) + 4;
}

struct MultiItem {
    int G, T, s0, cnt;
};

// Decomposition of slices [S0, S1): slice S0 + i (i < N) leads the groups S0 + i + m N below S1.
// Runs of leading slices with the same number of groups g split into parts of at most gmax groups
// (as even as possible); a part of two or more groups goes into items of T slices (of the forms
// available for its group count, the T that leaves the least work, the larger on a tie), the
// run's remainder into one item of the smallest form that holds it (partial when it is larger), a
// part of one group into the single kernel's ranges.
static void multi_plan(int S0, int S1, int N, int gmax, const std::vector<std::vector<int>> &Ts,
                       std::vector<MultiItem> *items, std::vector<std::pair<int, int>> *rest,
                       int lead_limit = INT32_MAX)
{
    auto groups = [&](int s) { return (S1 - 1 - s) / N + 1; };
    const int lead_end = std::min(std::min(S0 + N, S1), lead_limit);
    for (int sa = S0; sa < lead_end;) {
        const int g = groups(sa);
        int sb = sa + 1;
        while (sb < lead_end && groups(sb) == g) ++sb;
        const int L = sb - sa;
        const int parts = (g + gmax - 1) / gmax;
        for (int q = 0, m0 = 0; q < parts; ++q) {
            const int gc = g / parts + (q < g % parts ? 1 : 0);
            const int a0 = sa + m0 * N;
            if (gc >= 2 && !Ts[gc].empty()) {
                // the form for a remainder of r slices, and the slices the items of T hold
                auto tail_of = [&](int r) {
                    int t = 0;
                    for (int T : Ts[gc])
                        if (T >= r && (!t || T < t)) t = T;
                    return r ? t : 0;
                };
                auto work = [&](int T) { return L / T * T + tail_of(L % T); };
                int best = Ts[gc][0];
                for (int T : Ts[gc])
                    if (work(T) < work(best) || (work(T) == work(best) && T > best)) best = T;
                for (int i = 0; i + best <= L; i += best) items->push_back({gc, best, a0 + i, best});
                if (L % best) items->push_back({gc, tail_of(L % best), a0 + L - L % best, L % best});
            } else {
                for (int m = 0; m < gc; ++m) rest->push_back({a0 + m * N, a0 + m * N + L});
            }
            m0 += gc;
        }
        sa = sb;
    }
    // merge adjacent single-kernel ranges
    std::sort(rest->begin(), rest->end());
    std::vector<std::pair<int, int>> merged;
    for (const auto &r : *rest) {
        if (!merged.empty() && merged.back().second == r.first)
            merged.back().second = r.second;
        else
            merged.push_back(r);
    }
    *rest = merged;
}

typedef void (*MultiKernel)(CUtensorMap, BP2Args, MultiItems);

// Band forms run only for plans whose taps lie within half a row of the detector; whole-window
// forms for any plan.
template <int MODE, int G, int T, int HS>
static MultiKernel pick(bool rows_ok, bool partial)
{
    if (partial) return k_backproject_multi<64, MODE, false, G, T, HS, true>;
    if (HS < kFullRows || rows_ok) return k_backproject_multi<64, MODE, true, G, T, HS, false>;
    if constexpr (HS >= kFullRows) return k_backproject_multi<64, MODE, false, G, T, HS, false>;
    return nullptr;
}

template <int MODE>
static MultiKernel select_multi(const Form &f, bool rows_ok, bool partial, size_t *smem)
{
#define KATS_MULTI_FORM(g, t, hs)                                  \
    if (f.G == g && f.T == t && f.HS == hs) {                      \
        *smem = MultiRing<g, hs, 64>::BYTES;                       \
        return pick<MODE, g, t, hs>(rows_ok, partial);             \
    }
    KATS_MULTI_FORM(4, 8, 24)
    KATS_MULTI_FORM(4, 6, 24)
    KATS_MULTI_FORM(3, 10, 32)
    KATS_MULTI_FORM(3, 8, 24)
    KATS_MULTI_FORM(2, 14, 40)
    KATS_MULTI_FORM(2, 12, 40)
    KATS_MULTI_FORM(2, 14, kFullRows)
    KATS_MULTI_FORM(2, 12, kFullRows)
#undef KATS_MULTI_FORM
    return nullptr;
}

// The T values per group count of a set of forms (index G).
std::vector<std::vector<int>> forms_T(const std::vector<Form> &forms, int *gmax)
{
    std::vector<std::vector<int>> Ts(5);
    *gmax = 1;
    for (const Form &f : forms) {
        Ts[f.G].push_back(f.T);
        *gmax = std::max(*gmax, f.G);
    }
    return Ts;
}

}  // namespace

template <int MODE>
int launch_multi(const Plan &p, const BP2Args &b0, const void *gF, const MultiLaunch &ml, cudaStream_t st,
                 int *n_launched, std::vector<std::pair<int, int>> *rest, bool *used)
{
    *used = false;
    EncodeTiledFn enc = encode_fn();
    const int srows = b0.srows;
    if (!enc || b0.W > 64 || p.gf_cols < 64 || srows > kFullRows) return KATS_OK;
    // the forms this plan can take: band forms where every tap lies within half a row of the
    // detector and the band fits the form's slots, whole-window forms otherwise
    std::vector<Form> forms;
    if (ml.rows_ok && p.g.dz > 0.0)
        for (const Form &f : kBandForms)
            if (band_rows(p, f.T) <= std::min(f.HS, srows) || f.HS >= srows) forms.push_back(f);
    bool have2 = false;
    for (const Form &f : forms) have2 |= f.G == 2;
    if (!have2)
        for (const Form &f : kFullForms) forms.push_back(f);
    int gmax = 1;
    const std::vector<std::vector<int>> Ts = forms_T(forms, &gmax);
    std::vector<MultiItem> items;
    std::vector<std::pair<int, int>> rst;
    multi_plan(ml.s_begin, ml.s_end, (int)p.N, gmax, Ts, &items, &rst, ml.lead_end);
    if (items.empty()) return KATS_OK;

    const dim3 block(B2_THREADS);
    const unsigned gx = (unsigned)ceil_div(p.g.nx, B2_TX), gy = (unsigned)ceil_div(p.g.ny, B2_TY);
    const int64_t drows = p.g.n_rows + (MODE == 0 ? 0 : 1);
    for (const Form &f : forms)
        for (int partial = 0; partial < 2; ++partial) {
            std::vector<MultiItem> grp;
            for (const MultiItem &i : items)
                if (i.G == f.G && i.T == f.T && (i.cnt < f.T) == (partial != 0)) grp.push_back(i);
            if (grp.empty()) continue;
            BP2Args b = b0;
            b.band = f.HS < kFullRows && f.HS < srows ? 1 : 0;
            b.box_rows = b.band ? f.HS : srows;
            b.hd = (float)(0.5 * std::hypot((B2_TX - 1) * p.g.dx, (B2_TY - 1) * p.g.dy));
            CUtensorMap map;
            cuuint64_t dims[3] = {(cuuint64_t)p.gf_cols, (cuuint64_t)drows, (cuuint64_t)p.n_fviews};
            cuuint64_t strides[2] = {(cuuint64_t)p.gf_cols * 4, (cuuint64_t)(p.gf_cols * drows) * 4};
            cuuint32_t box[3] = {64u, (cuuint32_t)b.box_rows, 1};
            cuuint32_t estr[3] = {1, 1, 1};
            CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(gF), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                set_error("tensor map of the multi-pitch backprojection");
                return KATS_ECUDA;
            }
            size_t smem = 0;
            MultiKernel kern = select_multi<MODE>(f, ml.rows_ok, partial != 0, &smem);
            if (!kern) {  // every form in kBandForms / kFullForms is instantiated
                set_error("multi-pitch backprojection form (%d groups of %d, %d rows) not built", f.G, f.T, f.HS);
                return KATS_EINVAL;
            }
            KATS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            for (size_t i0 = 0; i0 < grp.size(); i0 += kMaxMultiItems) {
                MultiItems it;
                it.n = (int)std::min<size_t>(kMaxMultiItems, grp.size() - i0);
                for (int i = 0; i < it.n; ++i) {
                    it.s0[i] = grp[i0 + (size_t)i].s0;
                    it.cnt[i] = grp[i0 + (size_t)i].cnt;
                }
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(gx, gy, (unsigned)it.n);
                cfg.blockDim = block;
                cfg.dynamicSmemBytes = smem;
                cfg.stream = st;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
                attr[0].val.programmaticStreamSerializationAllowed = *n_launched > 0 ? 1 : 0;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                ++*n_launched;
                KATS_CUDA(cudaLaunchKernelEx(&cfg, kern, map, b, it));
                count_launches(1);
                KATS_CUDA(cudaGetLastError());
            }
        }
    *rest = rst;
    *used = true;
    return KATS_OK;
}

template int launch_multi<0>(const Plan &, const BP2Args &, const void *, const MultiLaunch &, cudaStream_t, int *,
                             std::vector<std::pair<int, int>> *, bool *);
template int launch_multi<1>(const Plan &, const BP2Args &, const void *, const MultiLaunch &, cudaStream_t, int *,
                             std::vector<std::pair<int, int>> *, bool *);
template int launch_multi<2>(const Plan &, const BP2Args &, const void *, const MultiLaunch &, cudaStream_t, int *,
                             std::vector<std::pair<int, int>> *, bool *);

// checked-build hooks of this translation unit's kernels
int multi_debug_set(int wait_limit, int stall_pairs)
{
#ifdef KATS_DEBUG_CHECKS
    if (wait_limit) KATS_CUDA(cudaMemcpyToSymbol(g_debug_wait_limit, &wait_limit, sizeof(int)));
    if (stall_pairs != INT32_MIN) KATS_CUDA(cudaMemcpyToSymbol(g_debug_stall_pairs, &stall_pairs, sizeof(int)));
#else
    (void)wait_limit;
    (void)stall_pairs;
#endif
    return KATS_OK;
}

int multi_debug_take_flags(int *flags)
{
    int v = 0;
    KATS_CUDA(cudaMemcpyFromSymbol(&v, g_debug_flags, sizeof(int)));
    const int zero = 0;
    KATS_CUDA(cudaMemcpyToSymbol(g_debug_flags, &zero, sizeof(int)));
    *flags = v;
    return KATS_OK;
}

}  // namespace kats

extern "C" int katsevich_slice_groups(int64_t s_begin, int64_t s_end, int64_t slices_per_pitch, int max_groups,
                                      int64_t lead_end, int32_t *groups, int32_t *t, int32_t *s0, int32_t *cnt,
                                      int max_items, int *n_items, int32_t *rest, int max_rest, int *n_rest)
{
    using namespace kats;
    if (!groups || !t || !s0 || !cnt || !n_items || !rest || !n_rest || s_begin < 0 || s_end < s_begin ||
        s_end > INT32_MAX || slices_per_pitch < 1 || slices_per_pitch > INT32_MAX || max_groups < 2 ||
        max_groups > 4 || max_items < 0 || max_rest < 0) {
        set_error("bad argument");
        return KATS_EINVAL;
    }
    std::vector<Form> forms;
    for (const Form &f : kBandForms)
        if (f.G <= max_groups) forms.push_back(f);
    int gmax = 1;
    const std::vector<std::vector<int>> Ts = forms_T(forms, &gmax);
    std::vector<MultiItem> items;
    std::vector<std::pair<int, int>> rst;
    multi_plan((int)s_begin, (int)s_end, (int)slices_per_pitch, gmax, Ts, &items, &rst,
               (int)std::min<int64_t>(std::max<int64_t>(lead_end, INT32_MIN), INT32_MAX));
    *n_items = (int)items.size();
    *n_rest = (int)rst.size();
    if ((int)items.size() > max_items || (int)rst.size() > max_rest) {
        set_error("%zu items and %zu ranges do not fit %d / %d", items.size(), rst.size(), max_items, max_rest);
        return KATS_ESPACE;
    }
    for (size_t i = 0; i < items.size(); ++i) {
        groups[i] = items[i].G;
        t[i] = items[i].T;
        s0[i] = items[i].s0;
        cnt[i] = items[i].cnt;
    }
    for (size_t j = 0; j < rst.size(); ++j) {
        rest[2 * j] = rst[j].first;
        rest[2 * j + 1] = rst[j].second;
    }
    return KATS_OK;
}
