// Steps 1-6 of the reconstruction step (Sec. II): sinogram -> filtered data g^F.
//
//   k_deriv_rebin   steps 1-3: derivative at constant direction (Eq. (Deriv)) on
//                   the half grid, length weight (Eq. (LW)), forward height
//                   rebinning onto kappa-lines (Eq. (FR)) -> g3 [v][psi][Kp]
//   k_toeplitz_gemm step 4: Hilbert transform in alpha at constant psi
//                   (Eq. (HF)) as a Toeplitz contraction g4 = g3 . T,
//                   T[c'][c] = d_alpha / (pi sin((c - c' - 1/2) d_alpha))
//   k_unrebin_cos   steps 5-6: backward height rebinning (Eq. (BR)) and the
//                   post-cosine weight (Eq. (PW)) -> g^F [v][row][col]
#include <algorithm>

#include "common.cuh"

namespace kats {

// Padded K extent of the g3 rows (multiple of 32 floats = one 128-byte
// tensor-core K block, zero tail).
static inline int64_t kpad(const Plan &p) { return p.tc_k; }

// Steps 1-6 run chunk by chunk over the filtered views through one reused buffer of a chunk's
// rebinned data (g3) and Hilbert output (g4), so the workspace holds one chunk of them rather than
// every view's.  A chunk's g3 + g4 take at most kChunkBudget bytes (about 600 views of the clinical
// detector: 9 chunks per volume; 128 MiB chunks, 36 per volume, measured 1.3 ms slower per volume
// from the extra kernel boundaries), and among the lengths that fit, the chunk is the one whose
// tensor-core tiles best fill whole waves of the SMs.
int64_t filter_chunk_views(const Plan &p, size_t bytes_per_view)
{
    constexpr size_t kChunkBudget = (size_t)480 << 20;
    const int64_t vmax = std::max<int64_t>(1, std::min<int64_t>(p.n_fviews, (int64_t)(kChunkBudget / bytes_per_view)));
    const int64_t n_nt = std::max<int64_t>(1, p.tc_n / 256), sms = std::max(1, p.sm_count);
    int64_t best = vmax;
    double best_eff = 0.0;
    for (int64_t v = vmax; v >= std::max<int64_t>(1, vmax / 2); --v) {
        const int64_t tiles = ceil_div(v * p.n_psi, 128) * n_nt;
        const double eff = (double)tiles / (double)(ceil_div(tiles, sms) * sms);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = v;
        }
    }
    return best;
}

static size_t chunk_bytes_per_view(const Plan &p) { return sizeof(float) * (size_t)(p.n_psi * (kpad(p) + p.tc_n)); }

// g3 [chunk][n_psi][Kp] then g4 [chunk][n_psi][tc_n] (rows padded to tensor-core K and N tiles)
size_t filter_workspace_bytes(const Plan &p)
{
    return chunk_bytes_per_view(p) * (size_t)filter_chunk_views(p, chunk_bytes_per_view(p));
}

// ---------------------------------------------------------------- steps 1-3
// grid (ceil(Kp / 32), ceil(n_fviews / views_per_block)); block 256 (8 warps); dynamic smem
// n_rows * 32 floats (g2 of one view), plus with CACHED n_psi * 32 (int, float) kappa-table
// entries.  A block handles 32 columns of consecutive views; CACHED reads its columns' table
// entries once instead of once per view.
// RT > 0 (n_rows <= 8 RT): a thread keeps its RT rows of views v and v + 1 in registers, carries view
// v + 1 into the next iteration and loads view v + 2 while the block writes view v's lines, so
// every sinogram value is read once per block and the loads overlap the stores.
template <bool CACHED, int RT>
__global__ void __launch_bounds__(256) k_deriv_rebin(const float *__restrict__ sino, float *__restrict__ g3,
                                                     const int32_t *__restrict__ kap_idx,
                                                     const float *__restrict__ kap_frac, const float *__restrict__ lw,
                                                     int nv, int n_rows, int n_cols, int n_psi, int Kp, float a_lam,
                                                     float a_alp, int views_per_block)
{
    extern __shared__ float s_g2[];  // [n_rows][32]
    int *s_ki = reinterpret_cast<int *>(s_g2 + n_rows * 32);  // [n_psi][32]
    float *s_kf = reinterpret_cast<float *>(s_ki + n_psi * 32);
    const int nc1 = n_cols - 1;
    const int c0 = blockIdx.x * 32;
    const int cc = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = c0 + cc;
    if (CACHED)
        for (int l = warp; l < n_psi; l += 8) {
            s_ki[l * 32 + cc] = c < nc1 ? kap_idx[l * nc1 + c] : -2;  // -2: no tap, both rows out of range
            s_kf[l * 32 + cc] = c < nc1 ? kap_frac[l * nc1 + c] : 0.0f;
        }
    const int vb = blockIdx.y * views_per_block, ve = min(vb + views_per_block, nv);
    const int64_t vstride = (int64_t)n_rows * n_cols;  // sino points at sinogram view first_view
    constexpr int RA = RT > 0 ? RT : 1;
    float ra[RA], rb[RA], rd[RA], re[RA], rl[RA];  // rows warp + 8 i: views v (a, b), v + 1 (d, e); lw
    if (RT > 0) {
        const float *p0 = sino + vb * vstride, *p1 = p0 + vstride;
#pragma unroll
        for (int i = 0; i < RA; ++i) {
            const int r = warp + 8 * i;
            const bool ok = c < nc1 && r < n_rows;
            ra[i] = ok ? p0[r * n_cols + c] : 0.0f;
            rb[i] = ok ? p0[r * n_cols + c + 1] : 0.0f;
            rd[i] = ok ? p1[r * n_cols + c] : 0.0f;
            re[i] = ok ? p1[r * n_cols + c + 1] : 0.0f;
            rl[i] = r < n_rows ? lw[r] : 0.0f;
        }
    }
    for (int v = vb; v < ve; ++v) {
        const float *p0 = sino + v * vstride;
        const float *p1 = p0 + vstride;
        __syncthreads();  // s_g2 of the previous view consumed (first pass: tables written)
        if (RT > 0) {
#pragma unroll
            for (int i = 0; i < RA; ++i) {
                const int r = warp + 8 * i;
                // (dg/dlambda + dg/dalpha) at the cell centre, times D / sqrt(D^2 + w^2)
                if (r < n_rows)
                    s_g2[r * 32 + cc] = c < nc1 ? rl[i] * (a_lam * ((rd[i] - ra[i]) + (re[i] - rb[i])) +
                                                           a_alp * ((rb[i] - ra[i]) + (re[i] - rd[i])))
                                                : 0.0f;
            }
            if (v + 1 < ve) {
                const float *p2 = p1 + vstride;  // view v + 2 <= ve <= nv
#pragma unroll
                for (int i = 0; i < RA; ++i) {
                    const int r = warp + 8 * i;
                    const bool ok = c < nc1 && r < n_rows;
                    ra[i] = rd[i];
                    rb[i] = re[i];
                    rd[i] = ok ? p2[r * n_cols + c] : 0.0f;
                    re[i] = ok ? p2[r * n_cols + c + 1] : 0.0f;
                }
            }
        } else {
#pragma unroll 4
            for (int r = warp; r < n_rows; r += 8) {
                float val = 0.0f;
                if (c < nc1) {
                    const float a = p0[r * n_cols + c], b = p0[r * n_cols + c + 1];
                    const float d = p1[r * n_cols + c], e = p1[r * n_cols + c + 1];
                    // (dg/dlambda + dg/dalpha) at the cell centre, times D / sqrt(D^2 + w^2)
                    val = lw[r] * (a_lam * ((d - a) + (e - b)) + a_alp * ((b - a) + (e - d)));
                }
                s_g2[r * 32 + cc] = val;
            }
        }
        __syncthreads();
        if (c < Kp) {
            float *out = g3 + (int64_t)v * n_psi * Kp + c;
#pragma unroll 4
            for (int l = warp; l < n_psi; l += 8) {
                const int r = CACHED ? s_ki[l * 32 + cc] : (c < nc1 ? kap_idx[l * nc1 + c] : -2);
                const float f = CACHED ? s_kf[l * 32 + cc] : (c < nc1 ? kap_frac[l * nc1 + c] : 0.0f);
                const float lo = (r >= 0 && r < n_rows) ? s_g2[r * 32 + cc] : 0.0f;
                const float hi = (r + 1 >= 0 && r + 1 < n_rows) ? s_g2[(r + 1) * 32 + cc] : 0.0f;
                out[(int64_t)l * Kp] = (1.0f - f) * lo + f * hi;
            }
        }
    }
}

// ---------------------------------------------------------------- step 4
// C[m][n] = sum_k A[m][k] * T(k, n), T from the 1-D kernel hk:
//   forward   (transpose = 0): k = c' < nc1, n = c < nc, T = hk[n - k + nc - 2]
//   transpose (transpose = 1): k = c < nc,   n = c' < nc1, T = hk[k - n + nc - 2]
// A is [M][lda] (row-major, zero beyond the valid K), C is [M][ldc].
constexpr int GBM = 128, GBN = 128, GBK = 16;

__global__ void __launch_bounds__(256) k_toeplitz_gemm(const float *__restrict__ A, float *__restrict__ C,
                                                       const float *__restrict__ hk, int64_t M, int K, int Nn,
                                                       int lda, int ldc, int nc, int transpose)
{
    __shared__ float As[GBK][GBM + 4];
    __shared__ float Bs[GBK][GBN + 4];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * GBM;
    const int n0 = blockIdx.x * GBN;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

    for (int k0 = 0; k0 < K; k0 += GBK) {
        // A tile: 128 rows x 16 k -> As[k][m]
        for (int e = tid; e < GBM * GBK; e += 256) {
            const int mm = e / GBK, kk = e % GBK;
            const int64_t m = m0 + mm;
            const int k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? A[m * lda + k] : 0.0f;
        }
        // B tile generated from the Toeplitz kernel
        for (int e = tid; e < GBN * GBK; e += 256) {
            const int kk = e / GBN, nn = e % GBN;
            const int k = k0 + kk, n = n0 + nn;
            float t = 0.0f;
            if (k < K && n < Nn) t = transpose ? hk[k - n + nc - 2] : hk[n - k + nc - 2];
            Bs[kk][nn] = t;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            float a[8], b[8];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][ty * 4 + i];
                a[i + 4] = As[kk][64 + ty * 4 + i];
                b[i] = Bs[kk][tx * 4 + i];
                b[i + 4] = Bs[kk][64 + tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
            if (n < ldc) C[m * ldc + n] = (n < Nn) ? acc[i][j] : 0.0f;
        }
    }
}

// ---------------------------------------------------------------- steps 5-6
// gF rows have pitch gcols >= n_cols; the pad columns are written as zeros.
// grid (ceil(gcols / 32), ceil(n_fviews / views_per_block)); block 256 (8 warps); dynamic smem
// n_rows * 32 (int, float) psi-table entries with CACHED, read once per block for its 32 columns
// instead of once per view.
template <bool CACHED>
__global__ void __launch_bounds__(256) k_unrebin_cos(const float *__restrict__ g4, float *__restrict__ gF,
                                                     const int32_t *__restrict__ psi_idx,
                                                     const float *__restrict__ psi_frac,
                                                     const float *__restrict__ cosa, int64_t nv, int n_rows,
                                                     int n_cols, int n_psi, int gcols, int ld4, int views_per_block)
{
    extern __shared__ int s_li[];  // [n_rows][32]
    float *s_lf = reinterpret_cast<float *>(s_li + n_rows * 32);
    const int cc = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + cc;
    if (CACHED)
        for (int r = warp; r < n_rows; r += 8) {
            s_li[r * 32 + cc] = c < n_cols ? psi_idx[r * n_cols + c] : -2;  // -2: no tap, both lines out of range
            s_lf[r * 32 + cc] = c < n_cols ? psi_frac[r * n_cols + c] : 0.0f;
        }
    const float w = c < n_cols ? cosa[c] : 0.0f;  // pad columns get 0
    __syncthreads();
    if (c >= gcols) return;
    const int64_t vb = (int64_t)blockIdx.y * views_per_block, ve = min(vb + views_per_block, nv);
    for (int64_t v = vb; v < ve; ++v) {
        const float *col = g4 + v * n_psi * ld4 + c;
        float *out = gF + v * (int64_t)n_rows * gcols + c;
#pragma unroll 4
        for (int r = warp; r < n_rows; r += 8) {
            const int l = CACHED ? s_li[r * 32 + cc] : (c < n_cols ? psi_idx[r * n_cols + c] : -2);
            const float f = CACHED ? s_lf[r * 32 + cc] : (c < n_cols ? psi_frac[r * n_cols + c] : 0.0f);
            const float lo = (l >= 0 && l < n_psi) ? col[(int64_t)l * ld4] : 0.0f;
            const float hi = (l + 1 >= 0 && l + 1 < n_psi) ? col[(int64_t)(l + 1) * ld4] : 0.0f;
            out[(int64_t)r * gcols] = w * ((1.0f - f) * lo + f * hi);
        }
    }
}

// Steps 1-6 of views [0, nv) of the given pointers, in one pass (nv at most one chunk).
static int filter_pass(const Plan &p, const float *sino, float *gF, float *g3, float *g4, int64_t nv, cudaStream_t st)
{
    const int64_t Kp = kpad(p), nc = p.g.n_cols, nr = p.g.n_rows, np = p.n_psi;
    const float a_lam = (float)(1.0 / (2.0 * p.dlam)), a_alp = (float)(1.0 / (2.0 * p.g.d_alpha));
    // Table entries stay in shared memory while that leaves room for several blocks per SM.
    constexpr size_t kCacheMax = 64 * 1024;
    const size_t smem1 = sizeof(float) * 32 * (size_t)nr, tab1 = 8 * 32 * (size_t)np;
    const bool cache1 = tab1 <= kCacheMax;
    const int vpb = (int)std::max<int64_t>(8, ceil_div(nv, 65535));  // views per block
    dim3 g1((unsigned)ceil_div(Kp, 32), (unsigned)ceil_div(nv, vpb));
    auto kd = nr <= 64 ? (cache1 ? k_deriv_rebin<true, 8> : k_deriv_rebin<false, 8>)
                       : (cache1 ? k_deriv_rebin<true, 0> : k_deriv_rebin<false, 0>);
    const size_t sm1 = smem1 + (cache1 ? tab1 : 0);
    if (sm1 > 48 * 1024) KATS_CUDA(cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
    kd<<<g1, 256, sm1, st>>>(sino, g3, p.kap_idx, p.kap_frac, p.lw, (int)nv, (int)nr, (int)nc, (int)np, (int)Kp,
                             a_lam, a_alp, vpb);
    count_launches(1);
    KATS_CUDA(cudaGetLastError());
    const int64_t M = nv * np;
    const int ld4 = (int)p.tc_n;
    bool tc = false;
    int rc = launch_hilbert_tc(p, g3, g4, M, ld4, st, &tc);
    if (rc) return rc;
    if (!tc) {
        if (ceil_div(M, GBM) > 65535) {
            set_error("too many filtered views for one launch (%lld)", (long long)nv);
            return KATS_EINVAL;
        }
        dim3 g2((unsigned)ceil_div(nc, GBN), (unsigned)ceil_div(M, GBM));
        k_toeplitz_gemm<<<g2, 256, 0, st>>>(g3, g4, p.hk, M, (int)p.nc1, (int)nc, (int)Kp, ld4, (int)nc, 0);
        count_launches(1);
        KATS_CUDA(cudaGetLastError());
    }
    dim3 g3d((unsigned)ceil_div(p.gf_cols, 32), (unsigned)ceil_div(nv, vpb));
    const size_t tab3 = 8 * 32 * (size_t)nr;
    const bool cache3 = tab3 <= kCacheMax;
    auto ku = cache3 ? k_unrebin_cos<true> : k_unrebin_cos<false>;
    if (cache3 && tab3 > 48 * 1024)
        KATS_CUDA(cudaFuncSetAttribute(ku, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tab3));
    ku<<<g3d, 256, cache3 ? tab3 : 0, st>>>(g4, gF, p.psi_idx, p.psi_frac, p.cosa, nv, (int)nr, (int)nc, (int)np,
                                         (int)p.gf_cols, ld4, vpb);
    count_launches(1);
    KATS_CUDA(cudaGetLastError());
    return KATS_OK;
}

int launch_filter(const Plan &p, const float *sino, float *gF, void *ws, size_t ws_bytes, cudaStream_t st,
                  int64_t nv_chunk)
{
    kats::NvtxRange nvtx_range("filter (steps 1-6)");
    const int64_t nv = nv_chunk < 0 ? p.n_fviews : std::min<int64_t>(nv_chunk, p.n_fviews);
    if (ws_bytes < filter_workspace_bytes(p)) {
        set_error("filter workspace too small: %zu < %zu", ws_bytes, filter_workspace_bytes(p));
        return KATS_ESPACE;
    }
    const int64_t chunk = filter_chunk_views(p, chunk_bytes_per_view(p));
    float *g3 = (float *)ws;
    float *g4 = g3 + chunk * p.n_psi * kpad(p);
    const size_t view_in = (size_t)(p.g.n_rows * p.g.n_cols), view_out = (size_t)(p.g.n_rows * p.gf_cols);
    for (int64_t v0 = 0; v0 < nv; v0 += chunk) {
        int rc = filter_pass(p, sino + v0 * view_in, gF + v0 * view_out, g3, g4, std::min(chunk, nv - v0), st);
        if (rc) return rc;
    }
    return KATS_OK;
}

// ------------------------------------------------------------ transposes
// Chunk by chunk like the forward filter: per view, region 1 holds g4^T [psi][tct_k] and later g1^T
// [row][nc1]; region 2 g3^T [psi][tct_n] (rows padded to the tensor-core transpose's K and N); plus
// one view of g1^T carried from the previous chunk for the derivative's transpose, which couples
// each sinogram view to the half-grid views on both sides of it.
static int64_t adj_region1(const Plan &p) { return std::max<int64_t>(p.n_psi * p.tct_k, p.g.n_rows * p.nc1); }
static size_t adj_bytes_per_view(const Plan &p) { return sizeof(float) * (size_t)(adj_region1(p) + p.n_psi * p.tct_n); }

size_t filter_adjoint_workspace_bytes(const Plan &p)
{
    return adj_bytes_per_view(p) * (size_t)filter_chunk_views(p, adj_bytes_per_view(p)) +
           sizeof(float) * (size_t)(p.g.n_rows * p.nc1);
}

// 6^T then 5^T: g4a[v][l][c] = sum_r cos(alpha_c) gF[v][r][c] * (tap weight of l)
// grid (ceil(nc / 32), nv); block 256; smem n_psi * 32 floats.
__global__ void k_unrebin_cos_T(const float *__restrict__ gF, float *__restrict__ g4a, const int32_t *__restrict__ psi_idx,
                                const float *__restrict__ psi_frac, const float *__restrict__ cosa, int nv,
                                int n_rows, int n_cols, int n_psi, int ld4, int gcols)
{
    extern __shared__ float s[];  // [n_psi][32]
    const int c0 = blockIdx.x * 32, cc = threadIdx.x & 31, c = c0 + cc;
    for (int v = blockIdx.y; v < nv; v += gridDim.y) {
    __syncthreads();  // previous view's results written out
    for (int e = threadIdx.x; e < n_psi * 32; e += blockDim.x) s[e] = 0.0f;
    __syncthreads();
    if (c < n_cols) {
        const float *in = gF + (int64_t)v * n_rows * gcols;
        for (int r = threadIdx.x >> 5; r < n_rows; r += blockDim.x >> 5) {
            const int rc = r * n_cols + c;
            const float val = cosa[c] * in[r * gcols + c];
            const int l = psi_idx[rc];
            const float f = psi_frac[rc];
            if (l >= 0 && l < n_psi) atomicAdd(&s[l * 32 + cc], (1.0f - f) * val);
            if (l + 1 >= 0 && l + 1 < n_psi) atomicAdd(&s[(l + 1) * 32 + cc], f * val);
        }
    }
    __syncthreads();
    float *out = g4a + (int64_t)v * n_psi * ld4;
    for (int l = threadIdx.x >> 5; l < n_psi; l += blockDim.x >> 5)
        if (c < ld4) out[(int64_t)l * ld4 + c] = (c < n_cols) ? s[l * 32 + cc] : 0.0f;
    }
}

// 3^T then 2^T: g1a[v][r][c'] = lw[r] * sum_l (tap weight of r) g3a[v][l][c']
__global__ void k_rebin_T(const float *__restrict__ g3a, float *__restrict__ g1a, const int32_t *__restrict__ kap_idx,
                          const float *__restrict__ kap_frac, const float *__restrict__ lw, int nv, int n_rows,
                          int n_cols, int n_psi, int Kp)
{
    extern __shared__ float s[];  // [n_rows][32]
    const int nc1 = n_cols - 1;
    const int c0 = blockIdx.x * 32, cc = threadIdx.x & 31, c = c0 + cc;
    for (int v = blockIdx.y; v < nv; v += gridDim.y) {
    __syncthreads();  // previous view's results written out
    for (int e = threadIdx.x; e < n_rows * 32; e += blockDim.x) s[e] = 0.0f;
    __syncthreads();
    if (c < nc1) {
        const float *in = g3a + (int64_t)v * n_psi * Kp;
        for (int l = threadIdx.x >> 5; l < n_psi; l += blockDim.x >> 5) {
            const float val = in[(int64_t)l * Kp + c];
            const int r = kap_idx[l * nc1 + c];
            const float f = kap_frac[l * nc1 + c];
            if (r >= 0 && r < n_rows) atomicAdd(&s[r * 32 + cc], (1.0f - f) * val);
            if (r + 1 >= 0 && r + 1 < n_rows) atomicAdd(&s[(r + 1) * 32 + cc], f * val);
        }
    }
    __syncthreads();
    if (c < nc1) {
        float *out = g1a + (int64_t)v * n_rows * nc1;
        for (int r = threadIdx.x >> 5; r < n_rows; r += blockDim.x >> 5) out[r * nc1 + c] = lw[r] * s[r * 32 + cc];
    }
    }
}

// 1^T: each sample gathers the (up to) four half-grid cells that read it.
// 2^T then 1^T for sinogram views first_view + [k_begin, k_end) (relative view k takes the half-grid
// views k - 1 and k, each from the chunk's g1^T [c0, c1) or, for view c0 - 1, from the carried one).
__global__ void k_deriv_T(const float *__restrict__ g1a, const float *__restrict__ carry, float *__restrict__ sino,
                          int64_t first_view, int64_t nv, int64_t c0, int64_t c1, int64_t k_begin, int64_t k_end,
                          int n_rows, int n_cols, float a_lam, float a_alp)
{
    const int nc1 = n_cols - 1;
    const int64_t per = (int64_t)n_rows * n_cols, total = (k_end - k_begin) * per;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = k_begin + t / per;
        const int rc = (int)(t % per), r = rc / n_cols, c = rc % n_cols;
        float acc = 0.0f;
#pragma unroll
        for (int dk = 0; dk < 2; ++dk)
#pragma unroll
            for (int dc = 0; dc < 2; ++dc) {
                const int64_t kp = k - dk;
                const int cp = c - dc;
                if (kp < 0 || kp >= nv || cp < 0 || cp >= nc1) continue;
                const float *src = kp >= c0 ? g1a + (kp - c0) * n_rows * nc1 : carry;
                const float coef = (dk ? a_lam : -a_lam) + (dc ? a_alp : -a_alp);
                acc = fmaf(coef, src[r * nc1 + cp], acc);
            }
        sino[(first_view + k) * per + rc] = acc;
    }
}

// Steps 6^T .. 4^T of views [c0, c1) of gF into the chunk buffers, ending with g1^T in region 1.
static int filter_adjoint_pass(const Plan &p, const float *gF, float *g4a, float *g3a, int64_t nvc, cudaStream_t st)
{
    const int64_t nc = p.g.n_cols, nr = p.g.n_rows, np = p.n_psi;
    const int64_t Kp4 = p.tct_k, Kp = p.tct_n;  // row strides of g4^T and g3^T
    float *g1a = g4a;  // g4^T is dead once g3^T is formed
    size_t sm1 = sizeof(float) * 32 * (size_t)np, sm2 = sizeof(float) * 32 * (size_t)nr;
    if (sm1 > 48 * 1024) KATS_CUDA(cudaFuncSetAttribute(k_unrebin_cos_T, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
    if (sm2 > 48 * 1024) KATS_CUDA(cudaFuncSetAttribute(k_rebin_T, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
    k_unrebin_cos_T<<<dim3((unsigned)ceil_div(Kp4, 32), (unsigned)std::min<int64_t>(nvc, 65535)), 256, sm1, st>>>(
        gF, g4a, p.psi_idx, p.psi_frac, p.cosa, (int)nvc, (int)nr, (int)nc, (int)np, (int)Kp4, (int)p.gf_cols);
    count_launches(1);
    KATS_CUDA(cudaGetLastError());
    const int64_t M = nvc * np;
    // 4^T: the transposed Toeplitz contraction, on the tensor cores when they can run it
    bool tc = false;
    int rc = launch_hilbert_tc_op(p, g4a, M, p.tct_k, p.btT_hi, p.btT_lo, p.tct_n, g3a, (int)p.tct_n, st, &tc);
    if (rc) return rc;
    if (!tc) {
        if (ceil_div(M, GBM) > 65535) {
            set_error("too many filtered views for one launch (%lld)", (long long)nvc);
            return KATS_EINVAL;
        }
        k_toeplitz_gemm<<<dim3((unsigned)ceil_div(p.nc1, GBN), (unsigned)ceil_div(M, GBM)), 256, 0, st>>>(
            g4a, g3a, p.hk, M, (int)nc, (int)p.nc1, (int)Kp4, (int)Kp, (int)nc, 1);
        count_launches(1);
        KATS_CUDA(cudaGetLastError());
    }
    k_rebin_T<<<dim3((unsigned)ceil_div(p.nc1, 32), (unsigned)std::min<int64_t>(nvc, 65535)), 256, sm2, st>>>(
        g3a, g1a, p.kap_idx, p.kap_frac, p.lw, (int)nvc, (int)nr, (int)nc, (int)np, (int)Kp);
    count_launches(1);
    KATS_CUDA(cudaGetLastError());
    return KATS_OK;
}

int launch_filter_adjoint(const Plan &p, const float *gF, float *sino, void *ws, size_t ws_bytes, cudaStream_t st)
{
    const int64_t nv = p.n_fviews, nc = p.g.n_cols, nr = p.g.n_rows;
    if (ws_bytes < filter_adjoint_workspace_bytes(p)) {
        set_error("filter adjoint workspace too small");
        return KATS_ESPACE;
    }
    const int64_t chunk = filter_chunk_views(p, adj_bytes_per_view(p));
    float *g4a = (float *)ws;
    float *g3a = g4a + chunk * adj_region1(p);
    float *carry = g3a + chunk * p.n_psi * p.tct_n;  // g1^T of the previous chunk's last view
    const size_t per = (size_t)(nr * nc), cell = (size_t)(nr * p.nc1);
    // sinogram views outside the window [first_view, first_view + nv] receive nothing
    if (p.first_view > 0) KATS_CUDA(cudaMemsetAsync(sino, 0, sizeof(float) * per * (size_t)p.first_view, st));
    const int64_t tail = p.g.n_views - (p.first_view + nv + 1);
    if (tail > 0)
        KATS_CUDA(cudaMemsetAsync(sino + (size_t)(p.first_view + nv + 1) * per, 0, sizeof(float) * per * (size_t)tail,
                                  st));
    const float a_lam = (float)(1.0 / (2.0 * p.dlam)), a_alp = (float)(1.0 / (2.0 * p.g.d_alpha));
    for (int64_t c0 = 0; c0 < nv; c0 += chunk) {
        const int64_t c1 = std::min(c0 + chunk, nv);
        int rc = filter_adjoint_pass(p, gF + (size_t)c0 * (size_t)(nr * p.gf_cols), g4a, g3a, c1 - c0, st);
        if (rc) return rc;
        // sinogram views c0 .. c1 - 1 (and c1 = nv after the last chunk) have every half-grid view they take
        const int64_t k_end = c1 == nv ? nv + 1 : c1;
        const int64_t total = (k_end - c0) * (int64_t)per;
        k_deriv_T<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), (int64_t)p.sm_count * 64), 256, 0, st>>>(
            g4a, carry, sino, p.first_view, nv, c0, c1, c0, k_end, (int)nr, (int)nc, a_lam, a_alp);
        count_launches(1);
        KATS_CUDA(cudaGetLastError());
        if (c1 < nv)
            KATS_CUDA(cudaMemcpyAsync(carry, g4a + (size_t)(c1 - 1 - c0) * cell, sizeof(float) * cell,
                                      cudaMemcpyDeviceToDevice, st));
    }
    return KATS_OK;
}

}  // namespace kats
