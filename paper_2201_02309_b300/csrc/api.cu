// C-ABI entry points of the reconstruction step (Sec. II): steps 1-6 then 7,
// their transposes, and the host-buffer variant.
#include <algorithm>
#include <vector>

#include "common.cuh"

using namespace kats;

namespace {

size_t gf_bytes(const Plan &p) { return sizeof(float) * (size_t)(p.n_fviews * p.g.n_rows * p.gf_cols); }
size_t gf_item(const Plan &p) { return (size_t)(p.n_fviews * p.g.n_rows * p.gf_cols); }
size_t sino_item(const Plan &p) { return (size_t)(p.g.n_views * p.g.n_rows * p.g.n_cols); }
size_t vol_item(const Plan &p) { return (size_t)(p.g.nx * p.g.ny * p.g.nz); }
size_t view_elems(const Plan &p) { return (size_t)(p.g.n_rows * p.g.n_cols); }

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

int check_common(const kats_plan *plan, const void *in, const void *out, int batch, int precision, const void *ws,
                 bool allow16 = false)
{
    if (!plan || !in || !out) {
        set_error("null plan or buffer");
        return KATS_EINVAL;
    }
    if (batch < 1) {
        set_error("batch must be >= 1 (got %d)", batch);
        return KATS_EINVAL;
    }
    const bool is16 = precision == KATS_PREC_BF16 || precision == KATS_PREC_FP16;
    if (precision != KATS_PREC_FP32 && !(allow16 && is16)) {
        set_error(is16 ? "reduced precision is available for katsevich_recon / katsevich_recon_host only"
                       : "unknown precision %d",
                  precision);
        return KATS_EINVAL;
    }
    if (!ws) {
        set_error("null workspace");
        return KATS_EINVAL;
    }
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device) {
        set_error("plan was built on device %d, current device is %d", p->device, dev);
        return KATS_EINVAL;
    }
    return KATS_OK;
}

size_t recon_ws(const Plan &p) { return align256(gf_bytes(p)) + filter_workspace_bytes(p); }
// reduced precision: row-pair filtered data [n_fviews][n_rows + 1][gf_cols] words + 16-bit filter scratch
size_t gfp_bytes(const Plan &p) { return 4 * (size_t)(p.n_fviews * (p.g.n_rows + 1) * p.gf_cols); }
size_t recon16_ws(const Plan &p) { return align256(gfp_bytes(p)) + filter16_workspace_bytes(p); }
size_t recon_ws_for(const Plan &p, int precision) { return precision == KATS_PREC_FP32 ? recon_ws(p) : recon16_ws(p); }

// One item of steps 1-7 with the workspace layout of the given precision.
int recon_item(const Plan &p, int precision, const float *sino_first, float *vol, void *ws, size_t ws_bytes,
               cudaStream_t st)
{
    if (precision == KATS_PREC_FP32) {
        float *gF = (float *)ws;
        char *fws = (char *)ws + align256(gf_bytes(p));
        int rc = launch_filter(p, sino_first, gF, fws, ws_bytes - align256(gf_bytes(p)), st);
        return rc ? rc : launch_backproject(p, gF, vol, st);
    }
    uint32_t *gFp = (uint32_t *)ws;
    char *fws = (char *)ws + align256(gfp_bytes(p));
    int rc = launch_filter16(p, precision, sino_first, gFp, fws, ws_bytes - align256(gfp_bytes(p)), st);
    return rc ? rc : launch_backproject16(p, precision, gFp, vol, st);
}
size_t adjoint_ws(const Plan &p) { return align256(gf_bytes(p)) + filter_adjoint_workspace_bytes(p); }

}  // namespace

namespace kats {

size_t host_item_bytes(const Plan &p, int precision)
{
    const size_t win = sizeof(float) * (size_t)(p.n_fviews + 1) * view_elems(p);
    return align256(win) + align256(sizeof(float) * vol_item(p)) + recon_ws_for(p, precision);
}

// Filtered views [lo, hi] (relative to first_view) that slices [s0, s1) read.
static void slab_views(const Plan &p, int64_t s0, int64_t s1, int64_t *lo, int64_t *hi)
{
    int64_t a = INT64_MAX, b = INT64_MIN;
    for (int64_t s = s0; s < s1; ++s) {
        const int64_t j = s % p.N, shift = (s / p.N) * p.g.views_per_turn;
        if (p.h_slice_kmin[(size_t)j] > p.h_slice_kmax[(size_t)j]) continue;  // no voxel of the slice has a window
        a = std::min<int64_t>(a, p.h_slice_kmin[(size_t)j] + shift);
        b = std::max<int64_t>(b, p.h_slice_kmax[(size_t)j] + shift);
    }
    *lo = a == INT64_MAX ? 0 : a - p.first_view;
    *hi = b == INT64_MIN ? -1 : b - p.first_view;
}

// One item from host buffers, stream-ordered and asynchronous: copy the view
// window the volume needs, steps 1-7, copy the volume back.  ws holds
// host_item_bytes(p, precision) bytes.  For windows of 128 MiB and more the
// copies overlap the kernels: the window arrives in chunks on a copy stream and
// each chunk is filtered on a filter stream as it lands; a slab of slices is
// backprojected on st once the chunks holding its views are filtered (the PI
// windows rise with z), the first slab chunk by chunk from partial sums, while
// later chunks are still arriving; each slab of the volume is copied back
// while later slabs are backprojected.  Work issued on st after this call
// waits for all of it.
// Groups of leading slices [la, lb) for the host pipeline's last slab [s0, s1), in launch order:
// leads s in [s0, s0 + N) head the slices s + mN below s1; runs of leads with the same number of
// groups in increasing s (the most groups first), the first run split in two halves, so that the
// last group launched (the fewest groups) has few slices to copy back.  Empty when the slab spans
// no more than a pitch (no slice has a partner).
constexpr int kMaxLeadChunks = 8;
static std::vector<std::pair<int, int>> lead_chunks(int s0, int s1, int N)
{
    std::vector<std::pair<int, int>> out;
    if (s1 - s0 <= N) return out;
    const int le = std::min(s0 + N, s1);
    auto groups = [&](int s) { return (s1 - 1 - s) / N + 1; };
    for (int a = s0; a < le && (int)out.size() < kMaxLeadChunks - 1;) {
        int b = a + 1;
        while (b < le && groups(b) == groups(a)) ++b;
        if (out.empty() && b - a > 1) {
            out.push_back({a, a + (b - a) / 2});
            out.push_back({a + (b - a) / 2, b});
        } else {
            out.push_back({a, b});
        }
        a = b;
    }
    out.back().second = le;  // any runs beyond the limit go with the last group
    return out;
}

int recon_one_host(const Plan &p, int precision, const float *host_sino, float *host_vol, void *ws, cudaStream_t st)
{
    kats::NvtxRange nvtx_range("katsevich: host item");
    const size_t view = view_elems(p);
    const size_t win = sizeof(float) * (size_t)(p.n_fviews + 1) * view;
    float *d_win = (float *)ws;
    float *d_vol = (float *)((char *)ws + align256(win));
    char *rws = (char *)d_vol + align256(sizeof(float) * vol_item(p));
    const bool fp32 = precision == KATS_PREC_FP32;
    const size_t gfb = fp32 ? align256(gf_bytes(p)) : align256(gfp_bytes(p));
    char *fws = rws + gfb;
    const size_t fws_bytes = recon_ws_for(p, precision) - gfb;
    const int64_t nf = p.n_fviews, nz = p.g.nz, nxy = p.g.nx * p.g.ny;
    if (win < ((size_t)128 << 20)) {
        // small items: copies are short, a second stream and events would cost more than they hide
        KATS_CUDA(cudaMemcpyAsync(d_win, host_sino + p.first_view * view, win, cudaMemcpyHostToDevice, st));
        int rc = recon_item(p, precision, d_win, d_vol, rws, recon_ws_for(p, precision), st);
        if (rc) return rc;
        KATS_CUDA(cudaMemcpyAsync(host_vol, d_vol, sizeof(float) * vol_item(p), cudaMemcpyDeviceToHost, st));
        return KATS_OK;
    }
    const int n_chunks = (int)std::max<int64_t>(1, std::min<int64_t>(16, nf / 256));
    // slabs of whole 16-slice z tiles.  The first four are small: the first starts backprojecting
    // after a few chunks, and each further 16 slices need only about a chunk more of views, which
    // arrive faster than a small slab is backprojected, so the GPU is not left waiting for the
    // copies.  Five of them fill the GPU until the last views have arrived.  Then, where more than
    // a pitch is left, the rest in one slab whose slices one and more pitches apart the multi-pitch
    // kernel reconstructs together, launched in groups of leading slices (lead_chunks) so that
    // each group is copied back while the next one runs; otherwise one slab up to 32 slices below
    // the top and the last 32.  Measured on the clinical workload (timelines from CUDA events):
    // 16 x 5 and 176 in leads 80-97, 98-115 (three groups), 116-149 (two) in 42.4 ms; the same
    // with 80-115 whole in 42.9, with the two-group leads first in 43.6, in one launch in 44.6;
    // 16 x 4 and 192 in leads 64-115, 116-133 in 43.2, with 116-133 first in 45.4 (36 slices of
    // two groups, two small launches: 6 ms); 16 x 4, 160, 32 in 43.2.
    std::vector<int> slab_lo{0};
    while (slab_lo.back() < nz) {
        const int64_t s0 = slab_lo.back(), left = nz - s0;
        const int64_t n = s0 < 80 ? 16 : (left > p.N ? left : (left > 64 ? (left - 32) / 16 * 16 : left));
        slab_lo.push_back((int)std::min<int64_t>(nz, s0 + n));
    }
    const int n_slabs = (int)slab_lo.size() - 1;
    auto chunk_lo = [&](int i) { return nf * i / n_chunks; };

    // copies on cs, filter chunks on fs, backprojection slabs on st: a filter chunk can run
    // while a slab's last wave of CTAs leaves SMs idle
    cudaStream_t cs = nullptr, fs = nullptr;
    // events: [0] start, [1, n_chunks] copies, then slabs, then [.. + n_chunks] filter chunks, last: copies done
    std::vector<cudaEvent_t> ev((size_t)(2 * n_chunks + n_slabs + 2), nullptr);
    std::vector<cudaEvent_t> lev(kMaxLeadChunks, nullptr);  // the last slab's groups of leading slices
    const size_t ev_filt = (size_t)(1 + n_chunks + n_slabs);
    auto cleanup = [&]() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);  // released once recorded work completes
        for (cudaEvent_t e : lev)
            if (e) cudaEventDestroy(e);
        if (cs) cudaStreamDestroy(cs);   // likewise
        if (fs) cudaStreamDestroy(fs);
    };
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&fs, cudaStreamNonBlocking);
    for (size_t i = 0; e == cudaSuccess && i < ev.size(); ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    for (size_t i = 0; e == cudaSuccess && i < lev.size(); ++i)
        e = cudaEventCreateWithFlags(&lev[i], cudaEventDisableTiming);
    int rc = KATS_OK;
    if (e != cudaSuccess) rc = cuda_fail(e, "copy / filter streams and events");
    // both side streams start after the work already issued on st (e.g. a previous item using ws)
    if (!rc && (e = cudaEventRecord(ev[0], st)) == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[0], 0);
    if (!rc && e == cudaSuccess) e = cudaStreamWaitEvent(fs, ev[0], 0);
    for (int i = 0; !rc && e == cudaSuccess && i < n_chunks; ++i) {
        const int64_t v0 = chunk_lo(i), v1 = chunk_lo(i + 1);  // filtered views [v0, v1) need [v0, v1]
        e = cudaMemcpyAsync(d_win + v0 * view, host_sino + (p.first_view + v0) * view,
                            sizeof(float) * (size_t)(v1 - v0 + 1) * view, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1 + i], cs);
    }
    int filtered = 0;  // chunks already filtered on st
    for (int j = 0; !rc && e == cudaSuccess && j < n_slabs; ++j) {
        const int s0 = slab_lo[(size_t)j], n = slab_lo[(size_t)j + 1] - s0;
        int64_t lo, hi;
        slab_views(p, s0, s0 + n, &lo, &hi);
        // filter every chunk up to the one holding the slab's last view
        auto more = [&]() { return filtered < n_chunks && (j == n_slabs - 1 || chunk_lo(filtered) <= hi); };
        while (!rc && e == cudaSuccess && more()) {
            const int i = filtered++;
            const int64_t v0 = chunk_lo(i), v1 = chunk_lo(i + 1);
            e = cudaStreamWaitEvent(fs, ev[1 + i], 0);
            if (e != cudaSuccess) break;
            if (fp32)
                rc = launch_filter(p, d_win + v0 * view, (float *)rws + v0 * p.g.n_rows * p.gf_cols, fws, fws_bytes,
                                   fs, v1 - v0);
            else
                rc = launch_filter16(p, precision, d_win + v0 * view,
                                     (uint32_t *)rws + v0 * (p.g.n_rows + 1) * p.gf_cols, fws, fws_bytes, fs,
                                     v1 - v0);
            if (!rc) e = cudaEventRecord(ev[ev_filt + (size_t)i], fs);
            if (rc || e != cudaSuccess || j > 0) continue;
            // the first slab takes each chunk's views as soon as they are filtered (partial sums in
            // the volume, the same order of additions as one launch), so the GPU does not sit idle
            // while the rest of the slab's views arrive
            const bool last = !more();
            BPRange r;
            r.k_lo = i == 0 ? INT32_MIN : (int)(p.first_view + v0);
            r.k_hi = last ? INT32_MAX : (int)(p.first_view + v1 - 1);
            r.acc_in = i > 0;
            r.acc_final = last;
            e = cudaStreamWaitEvent(st, ev[ev_filt + (size_t)i], 0);
            if (e != cudaSuccess) break;
            rc = fp32 ? launch_backproject(p, (const float *)rws, d_vol, st, s0, n, r)
                      : launch_backproject16(p, precision, (const uint32_t *)rws, d_vol, st, s0, n, r);
        }
        if (rc || e != cudaSuccess) break;
        if (j > 0) {
            // the slab needs every chunk filtered so far (chunks complete in order on fs)
            e = cudaStreamWaitEvent(st, ev[ev_filt + (size_t)(filtered - 1)], 0);
            if (e != cudaSuccess) break;
            const std::vector<std::pair<int, int>> leads =
                j == n_slabs - 1 ? lead_chunks(s0, s0 + n, (int)p.N) : std::vector<std::pair<int, int>>();
            if (!leads.empty()) {
                // groups of leading slices, each copied back while the next one is backprojected
                for (size_t q = 0; !rc && e == cudaSuccess && q < leads.size(); ++q) {
                    BPRange r;
                    r.lead_end = leads[q].second;
                    const int la = leads[q].first;
                    rc = fp32 ? launch_backproject(p, (const float *)rws, d_vol, st, la, s0 + n - la, r)
                              : launch_backproject16(p, precision, (const uint32_t *)rws, d_vol, st, la, s0 + n - la,
                                                     r);
                    if (rc) break;
                    e = cudaEventRecord(lev[q], st);
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, lev[q], 0);
                    for (const auto &sr : lead_ranges(la, s0 + n, (int)p.N, leads[q].second))
                        if (e == cudaSuccess)
                            e = cudaMemcpyAsync(host_vol + sr.first * nxy, d_vol + sr.first * nxy,
                                                sizeof(float) * (size_t)((sr.second - sr.first) * nxy),
                                                cudaMemcpyDeviceToHost, cs);
                }
                continue;
            }
            rc = fp32 ? launch_backproject(p, (const float *)rws, d_vol, st, s0, n)
                      : launch_backproject16(p, precision, (const uint32_t *)rws, d_vol, st, s0, n);
            if (rc) break;
        }
        e = cudaEventRecord(ev[1 + n_chunks + j], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[1 + n_chunks + j], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host_vol + s0 * nxy, d_vol + s0 * nxy, sizeof(float) * (size_t)(n * nxy),
                                cudaMemcpyDeviceToHost, cs);
    }
    if (!rc && e == cudaSuccess && (e = cudaEventRecord(ev[ev.size() - 1], cs)) == cudaSuccess)
        e = cudaStreamWaitEvent(st, ev[ev.size() - 1], 0);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "pipelined host item");
    cleanup();
    return rc;
}

}  // namespace kats

extern "C" {

int64_t katsevich_workspace_bytes(const kats_plan *plan, int precision)
{
    if (!plan) return -1;
    const Plan &p = *reinterpret_cast<const Plan *>(plan);
    if (precision == KATS_PREC_FP32) return (int64_t)std::max(recon_ws(p), adjoint_ws(p));
    if (precision == KATS_PREC_BF16 || precision == KATS_PREC_FP16) return (int64_t)recon16_ws(p);
    return -1;
}

int katsevich_filter(const kats_plan *plan, const float *sino, float *gF, int batch, int precision, void *workspace,
                     size_t workspace_bytes, void *stream)
{
    kats::NvtxRange nvtx_range("katsevich: filter");
    int rc = check_common(plan, sino, gF, batch, precision, workspace);
    if (rc) return rc;
    const Plan &p = *reinterpret_cast<const Plan *>(plan);
    if (workspace_bytes < filter_workspace_bytes(p)) {
        set_error("workspace %zu < %zu bytes", workspace_bytes, filter_workspace_bytes(p));
        return KATS_ESPACE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    for (int b = 0; b < batch; ++b) {
        rc = launch_filter(p, sino + b * sino_item(p) + p.first_view * view_elems(p), gF + b * gf_item(p), workspace,
                           workspace_bytes, st);
        if (rc) return rc;
    }
    return KATS_OK;
}

int katsevich_backproject(const kats_plan *plan, const float *gF, float *vol, int batch, void *stream)
{
    kats::NvtxRange nvtx_range("katsevich: backproject");
    if (!plan || !gF || !vol || batch < 1) {
        set_error("bad argument");
        return KATS_EINVAL;
    }
    const Plan &p = *reinterpret_cast<const Plan *>(plan);
    cudaStream_t st = (cudaStream_t)stream;
    for (int b = 0; b < batch; ++b) {
        int rc = launch_backproject(p, gF + b * gf_item(p), vol + b * vol_item(p), st);
        if (rc) return rc;
    }
    return KATS_OK;
}

int katsevich_recon(const kats_plan *plan, const float *sino, float *vol, int batch, int precision, void *workspace,
                    size_t workspace_bytes, void *stream)
{
    kats::NvtxRange nvtx_range("katsevich: recon");
    int rc = check_common(plan, sino, vol, batch, precision, workspace, true);
    if (rc) return rc;
    const Plan &p = *reinterpret_cast<const Plan *>(plan);
    const size_t need = recon_ws_for(p, precision);
    if (workspace_bytes < need) {
        set_error("workspace %zu < %zu bytes", workspace_bytes, need);
        return KATS_ESPACE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    for (int b = 0; b < batch; ++b) {
        rc = recon_item(p, precision, sino + b * sino_item(p) + p.first_view * view_elems(p), vol + b * vol_item(p),
                        workspace, workspace_bytes, st);
        if (rc) return rc;
    }
    return KATS_OK;
}

int katsevich_adjoint(const kats_plan *plan, const float *vol_grad, float *sino_grad, int batch, int precision,
                      void *workspace, size_t workspace_bytes, void *stream)
{
    kats::NvtxRange nvtx_range("katsevich: adjoint");
    int rc = check_common(plan, vol_grad, sino_grad, batch, precision, workspace);
    if (rc) return rc;
    const Plan &p = *reinterpret_cast<const Plan *>(plan);
    if (workspace_bytes < adjoint_ws(p)) {
        set_error("workspace %zu < %zu bytes", workspace_bytes, adjoint_ws(p));
        return KATS_ESPACE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    float *gF = (float *)workspace;
    char *fws = (char *)workspace + align256(gf_bytes(p));
    const size_t fws_bytes = workspace_bytes - align256(gf_bytes(p));
    for (int b = 0; b < batch; ++b) {
        rc = launch_backproject_adjoint(p, vol_grad + b * vol_item(p), gF, st);
        if (rc) return rc;
        rc = launch_filter_adjoint(p, gF, sino_grad + b * sino_item(p), fws, fws_bytes, st);
        if (rc) return rc;
    }
    return KATS_OK;
}

int katsevich_backproject_adjoint(const kats_plan *plan, const float *vol, float *gF, int batch, void *stream)
{
    kats::NvtxRange nvtx_range("katsevich: backproject adjoint");
    if (!plan || !vol || !gF || batch < 1) {
        set_error("bad argument");
        return KATS_EINVAL;
    }
    const Plan &p = *reinterpret_cast<const Plan *>(plan);
    cudaStream_t st = (cudaStream_t)stream;
    for (int b = 0; b < batch; ++b) {
        int rc = launch_backproject_adjoint(p, vol + b * vol_item(p), gF + b * gf_item(p), st);
        if (rc) return rc;
    }
    return KATS_OK;
}

int katsevich_filter_adjoint(const kats_plan *plan, const float *gF, float *sino, int batch, int precision,
                             void *workspace, size_t workspace_bytes, void *stream)
{
    kats::NvtxRange nvtx_range("katsevich: filter adjoint");
    int rc = check_common(plan, gF, sino, batch, precision, workspace);
    if (rc) return rc;
    const Plan &p = *reinterpret_cast<const Plan *>(plan);
    if (workspace_bytes < filter_adjoint_workspace_bytes(p)) {
        set_error("workspace %zu < %zu bytes", workspace_bytes, filter_adjoint_workspace_bytes(p));
        return KATS_ESPACE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    for (int b = 0; b < batch; ++b) {
        rc = launch_filter_adjoint(p, gF + b * gf_item(p), sino + b * sino_item(p), workspace, workspace_bytes, st);
        if (rc) return rc;
    }
    return KATS_OK;
}

int katsevich_slab_views(const kats_plan *plan, int64_t s_begin, int64_t s_end, int64_t *view_begin,
                         int64_t *view_count)
{
    if (!plan || !view_begin || !view_count) {
        set_error("null plan or output");
        return KATS_EINVAL;
    }
    const Plan &p = *reinterpret_cast<const Plan *>(plan);
    if (s_begin < 0 || s_end <= s_begin || s_end > p.g.nz) {
        set_error("slices [%lld, %lld) not a non-empty range of [0, %lld)", (long long)s_begin, (long long)s_end,
                  (long long)p.g.nz);
        return KATS_EINVAL;
    }
    int64_t lo, hi;
    slab_views(p, s_begin, s_end, &lo, &hi);
    // filtered half-views [lo, hi] (relative to first_view) are formed from sinogram views [lo, hi + 1]
    *view_begin = hi >= lo ? p.first_view + lo : p.first_view;
    *view_count = hi >= lo ? hi - lo + 2 : 0;
    return KATS_OK;
}

int katsevich_recon_slab(const kats_plan *plan, const float *sino_views, int64_t view_begin, int64_t view_count,
                         int64_t s_begin, int64_t s_end, float *vol_slab, int precision, void *workspace,
                         size_t workspace_bytes, void *stream)
{
    kats::NvtxRange nvtx_range("katsevich: recon slab");
    int rc = check_common(plan, sino_views, vol_slab, 1, precision, workspace, true);
    if (rc) return rc;
    const Plan &p = *reinterpret_cast<const Plan *>(plan);
    int64_t need_begin = 0, need_count = 0;
    rc = katsevich_slab_views(plan, s_begin, s_end, &need_begin, &need_count);
    if (rc) return rc;
    if (s_begin % 16 != 0) {
        set_error("slab start %lld is not a multiple of 16 slices", (long long)s_begin);
        return KATS_EINVAL;
    }
    if (need_count > 0 && (view_begin > need_begin || view_begin + view_count < need_begin + need_count)) {
        set_error("sinogram views [%lld, %lld) do not cover the slab's views [%lld, %lld)", (long long)view_begin,
                  (long long)(view_begin + view_count), (long long)need_begin, (long long)(need_begin + need_count));
        return KATS_EINVAL;
    }
    const size_t need = recon_ws_for(p, precision);
    if (workspace_bytes < need) {
        set_error("workspace %zu < %zu bytes", workspace_bytes, need);
        return KATS_ESPACE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const bool fp32 = precision == KATS_PREC_FP32;
    const size_t gfb = fp32 ? align256(gf_bytes(p)) : align256(gfp_bytes(p));
    char *fws = (char *)workspace + gfb;
    const int64_t lo = need_begin - p.first_view, nv = std::max<int64_t>(need_count - 1, 0);
    const float *first = sino_views + (need_begin - view_begin) * (int64_t)view_elems(p);
    // the filtered views land at their places in the full-size g^F layout, so the backprojection
    // indexes them as in katsevich_recon; its slice tiles start at s_begin, a multiple of 16 as in
    // the full volume, so every slice is added in the same order and equals katsevich_recon's
    if (nv > 0) {
        rc = fp32 ? launch_filter(p, first, (float *)workspace + lo * p.g.n_rows * p.gf_cols, fws, need - gfb, st, nv)
                  : launch_filter16(p, precision, first, (uint32_t *)workspace + lo * (p.g.n_rows + 1) * p.gf_cols,
                                    fws, need - gfb, st, nv);
        if (rc) return rc;
    }
    // vol_slab holds slices [s_begin, s_end); the kernels address slice s at base + s * nx * ny
    float *base = reinterpret_cast<float *>(reinterpret_cast<uintptr_t>(vol_slab) -
                                            sizeof(float) * (uintptr_t)(s_begin * p.g.nx * p.g.ny));
    const int n = (int)(s_end - s_begin);
    return fp32 ? launch_backproject(p, (const float *)workspace, base, st, (int)s_begin, n)
                : launch_backproject16(p, precision, (const uint32_t *)workspace, base, st, (int)s_begin, n);
}

int64_t katsevich_host_workspace_bytes(const kats_plan *plan, int batch, int precision)
{
    if (!plan || batch < 1 || (precision != KATS_PREC_FP32 && precision != KATS_PREC_BF16 &&
                               precision != KATS_PREC_FP16))
        return -1;
    return (int64_t)host_item_bytes(*reinterpret_cast<const Plan *>(plan), precision);
}

int katsevich_recon_host(const kats_plan *plan, const float *host_sino, float *host_vol, int batch, int precision,
                         void *workspace, size_t workspace_bytes, void *stream)
{
    kats::NvtxRange nvtx_range("katsevich: recon host");
    int rc = check_common(plan, host_sino, host_vol, batch, precision, workspace, true);
    if (rc) return rc;
    const Plan &p = *reinterpret_cast<const Plan *>(plan);
    const int64_t need = katsevich_host_workspace_bytes(plan, batch, precision);
    if ((int64_t)workspace_bytes < need) {
        set_error("workspace %zu < %lld bytes", workspace_bytes, (long long)need);
        return KATS_ESPACE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    for (int b = 0; b < batch; ++b) {
        rc = recon_one_host(p, precision, host_sino + b * sino_item(p), host_vol + b * vol_item(p), workspace, st);
        if (rc) return rc;
    }
    KATS_CUDA(cudaStreamSynchronize(st));
    return KATS_OK;
}

}  // extern "C"
