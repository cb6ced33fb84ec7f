// Steps 1-6 of the reconstruction step (Sec. II) with reduced-precision
// storage (KATS_PREC_BF16 / KATS_PREC_FP16): the derivative data after
// rebinning (g3) and the filtered data (g^F) are stored as 16-bit values,
// scaled by d_alpha so that FP16's range holds them (a derivative in
// per-column units is bounded by the largest sinogram difference between
// neighbouring samples).  Arithmetic and accumulation stay in FP32; the
// Hilbert contraction runs on the tensor cores with a 16-bit A and the
// Toeplitz operand split hi + lo (hilbert_tc.cu).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "common.cuh"

namespace kats {

template <bool FP16>
__device__ __forceinline__ uint16_t to16(float v)
{
    if (FP16) return __half_as_ushort(__float2half_rn(v));
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// chunk by chunk like the FP32 filter: g3 16-bit [chunk][n_psi][tc_k16], then g4 fp32 [chunk][n_psi][tc_n]
static size_t chunk16_bytes_per_view(const Plan &p) { return (size_t)p.n_psi * ((size_t)p.tc_k16 * 2 + (size_t)p.tc_n * 4); }
static int64_t chunk16_views(const Plan &p) { return filter_chunk_views(p, chunk16_bytes_per_view(p)); }
static size_t g3_chunk16_bytes(const Plan &p)
{
    return ((size_t)(chunk16_views(p) * p.n_psi) * (size_t)p.tc_k16 * 2 + 255) / 256 * 256;
}

size_t filter16_workspace_bytes(const Plan &p)
{
    return g3_chunk16_bytes(p) + (size_t)(chunk16_views(p) * p.n_psi) * (size_t)p.tc_n * 4;
}

// Steps 1-3 as k_deriv_rebin, output g3 * d_alpha in 16 bits, rows of tc_k16 (zero tail).
// grid (ceil(tc_k16 / 32), ceil(n_fviews / views_per_block)); block 256; dynamic smem n_rows * 32
// floats, plus with CACHED the block's n_psi * 32 (int, float) kappa-table entries.
template <bool FP16, bool CACHED>
__global__ void __launch_bounds__(256) k_deriv_rebin16(const float *__restrict__ sino, uint16_t *__restrict__ g3,
                                                       const int32_t *__restrict__ kap_idx,
                                                       const float *__restrict__ kap_frac,
                                                       const float *__restrict__ lw, int nv, int n_rows, int n_cols,
                                                       int n_psi, int Kp, float a_lam, float a_alp, float scale,
                                                       int views_per_block)
{
    extern __shared__ float s_g2[];  // [n_rows][32]
    int *s_ki = reinterpret_cast<int *>(s_g2 + n_rows * 32);  // [n_psi][32]
    float *s_kf = reinterpret_cast<float *>(s_ki + n_psi * 32);
    const int nc1 = n_cols - 1;
    const int cc = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + cc;
    if (CACHED)
        for (int l = warp; l < n_psi; l += 8) {
            s_ki[l * 32 + cc] = c < nc1 ? kap_idx[l * nc1 + c] : -2;  // -2: no tap
            s_kf[l * 32 + cc] = c < nc1 ? kap_frac[l * nc1 + c] : 0.0f;
        }
    const int vb = blockIdx.y * views_per_block, ve = min(vb + views_per_block, nv);
    for (int v = vb; v < ve; ++v) {
        const float *p0 = sino + (int64_t)v * n_rows * n_cols;
        const float *p1 = p0 + (int64_t)n_rows * n_cols;
        __syncthreads();
#pragma unroll 4
        for (int r = warp; r < n_rows; r += 8) {
            float val = 0.0f;
            if (c < nc1) {
                const float a = p0[r * n_cols + c], b = p0[r * n_cols + c + 1];
                const float d = p1[r * n_cols + c], e = p1[r * n_cols + c + 1];
                val = lw[r] * (a_lam * ((d - a) + (e - b)) + a_alp * ((b - a) + (e - d)));
            }
            s_g2[r * 32 + cc] = val;
        }
        __syncthreads();
        if (c < Kp) {
            uint16_t *out = g3 + (int64_t)v * n_psi * Kp + c;
#pragma unroll 4
            for (int l = warp; l < n_psi; l += 8) {
                const int r = CACHED ? s_ki[l * 32 + cc] : (c < nc1 ? kap_idx[l * nc1 + c] : -2);
                const float f = CACHED ? s_kf[l * 32 + cc] : (c < nc1 ? kap_frac[l * nc1 + c] : 0.0f);
                const float lo = (r >= 0 && r < n_rows) ? s_g2[r * 32 + cc] : 0.0f;
                const float hi = (r + 1 >= 0 && r + 1 < n_rows) ? s_g2[(r + 1) * 32 + cc] : 0.0f;
                out[(int64_t)l * Kp] = to16<FP16>(((1.0f - f) * lo + f * hi) * scale);
            }
        }
    }
}

// Steps 5-6 into the row-pair layout: word (pair-row pr, column c) holds
// (g^F[pr-1][c], g^F[pr][c]) in its low / high 16 bits, zero outside the
// detector.  A thread walks one column of one view down the rows, so each
// row's value is computed once and lands in two words.  grid (ceil(gcols / 32),
// ceil(n_fviews / (8 * views_per_warp))); block 256: warp w of a block takes views
// w, w + 8, ... of the block's range for the block's 32 columns; with CACHED the
// columns' psi-table entries (n_rows * 32 (int, float)) sit in shared memory.
template <bool FP16, bool CACHED>
__global__ void __launch_bounds__(256) k_unrebin_cos16(const float *__restrict__ g4, uint32_t *__restrict__ gFp,
                                                       const int32_t *__restrict__ psi_idx,
                                                       const float *__restrict__ psi_frac,
                                                       const float *__restrict__ cosa, int64_t nv, int n_rows,
                                                       int n_cols, int n_psi, int gcols, int ld4, int views_per_warp)
{
    extern __shared__ int s_li[];  // [n_rows][32]
    float *s_lf = reinterpret_cast<float *>(s_li + n_rows * 32);
    const int cc = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + cc;
    if (CACHED)
        for (int r = warp; r < n_rows; r += 8) {
            s_li[r * 32 + cc] = c < n_cols ? psi_idx[r * n_cols + c] : -2;  // -2: no tap
            s_lf[r * 32 + cc] = c < n_cols ? psi_frac[r * n_cols + c] : 0.0f;
        }
    const float w = c < n_cols ? cosa[c] : 0.0f;
    __syncthreads();
    if (c >= gcols) return;
    const int64_t vb = (int64_t)blockIdx.y * 8 * views_per_warp, ve = min(vb + 8 * views_per_warp, nv);
    for (int64_t v = vb + warp; v < ve; v += 8) {
        uint32_t *out = gFp + v * (int64_t)(n_rows + 1) * gcols + c;
        uint32_t prev = 0;  // 16-bit value of row pr - 1
        const float *col = g4 + v * n_psi * ld4 + c;
#pragma unroll 4
        for (int r = 0; r < n_rows; ++r) {
            const int l = CACHED ? s_li[r * 32 + cc] : (c < n_cols ? psi_idx[r * n_cols + c] : -2);
            const float f = CACHED ? s_lf[r * 32 + cc] : (c < n_cols ? psi_frac[r * n_cols + c] : 0.0f);
            const float lo = (l >= 0 && l < n_psi) ? col[(int64_t)l * ld4] : 0.0f;
            const float hi = (l + 1 >= 0 && l + 1 < n_psi) ? col[(int64_t)(l + 1) * ld4] : 0.0f;
            const uint32_t cur = to16<FP16>(w * ((1.0f - f) * lo + f * hi));  // pad columns: w = 0, no taps
            out[(int64_t)r * gcols] = prev | (cur << 16);
            prev = cur;
        }
        out[(int64_t)n_rows * gcols] = prev;
    }
}

// Steps 1-6 of views [0, nv) of the given pointers in one pass (nv at most one chunk).
static int filter16_pass(const Plan &p, int prec, const float *sino, uint32_t *gFp, uint16_t *g3, float *g4,
                         int64_t nv, cudaStream_t st)
{
    const int64_t nc = p.g.n_cols, nr = p.g.n_rows, np = p.n_psi, M = nv * np;
    const bool fp16 = prec == KATS_PREC_FP16;
    const float a_lam = (float)(1.0 / (2.0 * p.dlam)), a_alp = (float)(1.0 / (2.0 * p.g.d_alpha));
    const float scale = (float)p.g.d_alpha;
    constexpr size_t kCacheMax = 64 * 1024;  // table entries in shared memory up to this size
    const size_t smem1 = sizeof(float) * 32 * (size_t)nr, tab1 = 8 * 32 * (size_t)np;
    const bool cache1 = tab1 <= kCacheMax;
    auto kd = fp16 ? (cache1 ? k_deriv_rebin16<true, true> : k_deriv_rebin16<true, false>)
                   : (cache1 ? k_deriv_rebin16<false, true> : k_deriv_rebin16<false, false>);
    const size_t sm1 = smem1 + (cache1 ? tab1 : 0);
    if (sm1 > 48 * 1024) KATS_CUDA(cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
    const int vpb = (int)std::max<int64_t>(8, ceil_div(nv, 65535));  // views per block
    dim3 g1((unsigned)ceil_div(p.tc_k16, 32), (unsigned)ceil_div(nv, vpb));
    kd<<<g1, 256, sm1, st>>>(sino, g3, p.kap_idx, p.kap_frac, p.lw, (int)nv, (int)nr, (int)nc, (int)np,
                             (int)p.tc_k16, a_lam, a_alp, scale, vpb);
    count_launches(1);
    KATS_CUDA(cudaGetLastError());
    bool tc = false;
    int rc = launch_hilbert_tc16(p, prec, g3, g4, M, (int)p.tc_n, st, &tc);
    if (rc) return rc;
    if (!tc) {
        set_error("the 16-bit Hilbert step needs the tensor-core path (TMA encoder or alignment unavailable)");
        return KATS_EINVAL;
    }
    const size_t tab3 = 8 * 32 * (size_t)nr;
    const bool cache3 = tab3 <= kCacheMax;
    auto ku = fp16 ? (cache3 ? k_unrebin_cos16<true, true> : k_unrebin_cos16<true, false>)
                   : (cache3 ? k_unrebin_cos16<false, true> : k_unrebin_cos16<false, false>);
    if (cache3 && tab3 > 48 * 1024)
        KATS_CUDA(cudaFuncSetAttribute(ku, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tab3));
    const int vpw = (int)std::max<int64_t>(2, ceil_div(nv, 8 * 65535));  // views per warp
    dim3 g3d((unsigned)ceil_div(p.gf_cols, 32), (unsigned)ceil_div(nv, 8 * vpw));
    ku<<<g3d, 256, cache3 ? tab3 : 0, st>>>(g4, gFp, p.psi_idx, p.psi_frac, p.cosa, nv, (int)nr, (int)nc, (int)np,
                                         (int)p.gf_cols, (int)p.tc_n, vpw);
    count_launches(1);
    KATS_CUDA(cudaGetLastError());
    return KATS_OK;
}

int launch_filter16(const Plan &p, int prec, const float *sino, uint32_t *gFp, void *ws, size_t ws_bytes,
                    cudaStream_t st, int64_t nv_chunk)
{
    kats::NvtxRange nvtx_range("filter16 (steps 1-6)");
    const int64_t nv = nv_chunk < 0 ? p.n_fviews : std::min<int64_t>(nv_chunk, p.n_fviews);
    if (ws_bytes < filter16_workspace_bytes(p)) {
        set_error("filter workspace too small: %zu < %zu", ws_bytes, filter16_workspace_bytes(p));
        return KATS_ESPACE;
    }
    const int64_t chunk = chunk16_views(p);
    uint16_t *g3 = (uint16_t *)ws;
    float *g4 = (float *)((char *)ws + g3_chunk16_bytes(p));
    const size_t view_in = (size_t)(p.g.n_rows * p.g.n_cols), view_out = (size_t)((p.g.n_rows + 1) * p.gf_cols);
    for (int64_t v0 = 0; v0 < nv; v0 += chunk) {
        int rc = filter16_pass(p, prec, sino + v0 * view_in, gFp + v0 * view_out, g3, g4, std::min(chunk, nv - v0), st);
        if (rc) return rc;
    }
    return KATS_OK;
}

}  // namespace kats
