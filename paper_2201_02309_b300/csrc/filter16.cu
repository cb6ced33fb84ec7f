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

size_t filter16_workspace_bytes(const Plan &p)
{
    const int64_t M = p.n_fviews * p.n_psi;
    return (size_t)M * (size_t)p.tc_k16 * 2 + 256 + (size_t)M * (size_t)p.tc_n * 4;  // g3 16-bit, g4 fp32
}

// Steps 1-3 as k_deriv_rebin, output g3 * d_alpha in 16 bits, rows of tc_k16 (zero tail).
template <bool FP16>
__global__ void k_deriv_rebin16(const float *__restrict__ sino, uint16_t *__restrict__ g3,
                                const int32_t *__restrict__ kap_idx, const float *__restrict__ kap_frac,
                                const float *__restrict__ lw, int nv, int n_rows, int n_cols, int n_psi, int Kp,
                                float a_lam, float a_alp, float scale)
{
    extern __shared__ float s_g2[];  // [n_rows][32]
    const int nc1 = n_cols - 1;
    const int c0 = blockIdx.x * 32;
    const int cc = threadIdx.x & 31;
    const int c = c0 + cc;
    for (int v = blockIdx.y; v < nv; v += gridDim.y) {
        const float *p0 = sino + (int64_t)v * n_rows * n_cols;
        const float *p1 = p0 + (int64_t)n_rows * n_cols;
        __syncthreads();
        for (int r = threadIdx.x >> 5; r < n_rows; r += blockDim.x >> 5) {
            float val = 0.0f;
            if (c < nc1) {
                const float a = p0[r * n_cols + c], b = p0[r * n_cols + c + 1];
                const float d = p1[r * n_cols + c], e = p1[r * n_cols + c + 1];
                val = lw[r] * (a_lam * ((d - a) + (e - b)) + a_alp * ((b - a) + (e - d)));
            }
            s_g2[r * 32 + cc] = val;
        }
        __syncthreads();
        uint16_t *out = g3 + (int64_t)v * n_psi * Kp;
        for (int l = threadIdx.x >> 5; l < n_psi; l += blockDim.x >> 5) {
            float val = 0.0f;
            if (c < nc1) {
                const int r = kap_idx[l * nc1 + c];
                const float f = kap_frac[l * nc1 + c];
                const float lo = (r >= 0 && r < n_rows) ? s_g2[r * 32 + cc] : 0.0f;
                const float hi = (r + 1 >= 0 && r + 1 < n_rows) ? s_g2[(r + 1) * 32 + cc] : 0.0f;
                val = (1.0f - f) * lo + f * hi;
            }
            if (c < Kp) out[(int64_t)l * Kp + c] = to16<FP16>(val * scale);
        }
    }
}

// Steps 5-6 into the row-pair layout: word (pair-row pr, column c) holds
// (g^F[pr-1][c], g^F[pr][c]) in its low / high 16 bits, zero outside the
// detector.  A thread walks one column of one view down the rows, so each
// row's value is computed once and lands in two words.
template <bool FP16>
__global__ void k_unrebin_cos16(const float *__restrict__ g4, uint32_t *__restrict__ gFp,
                                const int32_t *__restrict__ psi_idx, const float *__restrict__ psi_frac,
                                const float *__restrict__ cosa, int64_t nv, int n_rows, int n_cols, int n_psi,
                                int gcols, int ld4)
{
    const int64_t total = nv * gcols;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = t / gcols;
        const int c = (int)(t % gcols);
        uint32_t *out = gFp + v * (int64_t)(n_rows + 1) * gcols + c;
        uint32_t prev = 0;  // 16-bit value of row pr - 1
        const float *col = g4 + v * n_psi * ld4 + c;
        for (int r = 0; r <= n_rows; ++r) {
            uint32_t cur = 0;
            if (r < n_rows && c < n_cols) {
                const int rc = r * n_cols + c;
                const int l = psi_idx[rc];
                const float f = psi_frac[rc];
                const float lo = (l >= 0 && l < n_psi) ? col[(int64_t)l * ld4] : 0.0f;
                const float hi = (l + 1 >= 0 && l + 1 < n_psi) ? col[(int64_t)(l + 1) * ld4] : 0.0f;
                cur = to16<FP16>(cosa[c] * ((1.0f - f) * lo + f * hi));
            }
            out[(int64_t)r * gcols] = prev | (cur << 16);
            prev = cur;
        }
    }
}

int launch_filter16(const Plan &p, int prec, const float *sino, uint32_t *gFp, void *ws, size_t ws_bytes,
                    cudaStream_t st, int64_t nv_chunk)
{
    const int64_t nv = nv_chunk < 0 ? p.n_fviews : std::min<int64_t>(nv_chunk, p.n_fviews);
    const int64_t nc = p.g.n_cols, nr = p.g.n_rows, np = p.n_psi, M = nv * np;
    if (ws_bytes < filter16_workspace_bytes(p)) {
        set_error("filter workspace too small: %zu < %zu", ws_bytes, filter16_workspace_bytes(p));
        return KATS_ESPACE;
    }
    const bool fp16 = prec == KATS_PREC_FP16;
    uint16_t *g3 = (uint16_t *)ws;
    // workspace laid out for every view; a chunk uses the front of each part
    float *g4 = (float *)((char *)ws + ((size_t)(p.n_fviews * np) * (size_t)p.tc_k16 * 2 + 255) / 256 * 256);
    const float a_lam = (float)(1.0 / (2.0 * p.dlam)), a_alp = (float)(1.0 / (2.0 * p.g.d_alpha));
    const float scale = (float)p.g.d_alpha;
    const size_t smem = sizeof(float) * 32 * (size_t)nr;
    auto kd = fp16 ? k_deriv_rebin16<true> : k_deriv_rebin16<false>;
    if (smem > 48 * 1024) KATS_CUDA(cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 g1((unsigned)ceil_div(p.tc_k16, 32), (unsigned)std::min<int64_t>(nv, 65535));
    kd<<<g1, 256, smem, st>>>(sino, g3, p.kap_idx, p.kap_frac, p.lw, (int)nv, (int)nr, (int)nc, (int)np,
                              (int)p.tc_k16, a_lam, a_alp, scale);
    KATS_CUDA(cudaGetLastError());
    bool tc = false;
    int rc = launch_hilbert_tc16(p, prec, g3, g4, M, (int)p.tc_n, st, &tc);
    if (rc) return rc;
    if (!tc) {
        set_error("the 16-bit Hilbert step needs the tensor-core path (TMA encoder or alignment unavailable)");
        return KATS_EINVAL;
    }
    const int64_t total = nv * p.gf_cols;
    auto ku = fp16 ? k_unrebin_cos16<true> : k_unrebin_cos16<false>;
    ku<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 148 * 64), 256, 0, st>>>(
        g4, gFp, p.psi_idx, p.psi_frac, p.cosa, nv, (int)nr, (int)nc, (int)np, (int)p.gf_cols, (int)p.tc_n);
    KATS_CUDA(cudaGetLastError());
    return KATS_OK;
}

}  // namespace kats
