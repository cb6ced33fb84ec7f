// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <utility>
#include <vector>

#include "../../include/katsevich.h"

#include <nvtx3/nvToolsExt.h>

namespace kats {

constexpr double kPi = 3.141592653589793238462643383279502884;

// Voxel-column tile of the staged backprojection and its transpose (one thread per column).
constexpr int kTileX = 16, kTileY = 16;

// Device-resident plan: the pre-calculated tables of one pitch (Sec. II).
struct Plan {
    kats_geometry g;
    int device;
    int sm_count = 148;  // multiprocessors of the plan's device
    // derived scalars (FP64, host)
    int64_t N;        // slices per pitch
    int64_t n_psi;    // kappa lines
    int64_t nc1;      // half-grid columns (n_cols - 1)
    double alpha_m, psi_max, dpsi, h, dlam;
    double r_fov;  // farthest volume corner from the axis
    int64_t first_view, n_fviews;  // filtered half-views the volume needs
    int64_t gf_cols;               // row pitch of g^F in floats: n_cols rounded up to 4 (16-byte rows)
    int64_t update_count;
    double ext[6];
    // device tables
    int32_t *kap_idx = nullptr;  // [n_psi][nc1] floor of the fractional row
    float *kap_frac = nullptr;   // [n_psi][nc1]
    int32_t *psi_idx = nullptr;  // [n_rows][n_cols] floor of the fractional psi index, -2 = no root
    float *psi_frac = nullptr;   // [n_rows][n_cols]
    int32_t *pi_k0 = nullptr, *pi_k1 = nullptr;  // [N][ny][nx]
    float *pi_w0 = nullptr, *pi_w1 = nullptr;    // [N][ny][nx]
    int32_t *slice_kmin = nullptr, *slice_kmax = nullptr;  // [N] per table slice
    std::vector<int32_t> h_slice_kmin, h_slice_kmax;       // host copies (view ranges of volume slabs)
    bool pi_monotone = false;  // window starts / ends nondecreasing in the slice for every voxel column
    float *hk = nullptr;    // Hilbert kernel, [2 n_cols - 2], entry n + n_cols - 2 for n = c - c'
    // Toeplitz operand of the tensor-core Hilbert step: Bt[c][c'] = hk(c - c') for c < n_cols,
    // c' < n_cols - 1 (zero elsewhere), split as hi = value with the low 13 mantissa bits cleared
    // (exact in TF32) and lo = value - hi; [tc_n][tc_k] row-major.
    float *bt_hi = nullptr, *bt_lo = nullptr;
    int64_t tc_k = 0, tc_n = 0;  // K padded to 32, N padded to 256
    // the transpose's operand (adjoint of the Hilbert step): Bt'[c'][c] = hk(c - c') for c' < n_cols - 1,
    // c < n_cols, split the same way; [tct_n][tct_k], tct_n = n_cols - 1 padded to 256, tct_k = n_cols to 32
    float *btT_hi = nullptr, *btT_lo = nullptr;
    int64_t tct_k = 0, tct_n = 0;
    // the same operand for the 16-bit Hilbert step: value = hi + lo with hi, lo
    // in bf16 (resp. fp16), [tc_n][tc_k16], K padded to 64
    uint16_t *bt16_hi[2] = {nullptr, nullptr}, *bt16_lo[2] = {nullptr, nullptr};  // [0] bf16, [1] fp16
    int64_t tc_k16 = 0;
    float *lw = nullptr;    // [n_rows] length-correction weight
    float *cosa = nullptr;  // [n_cols] cos(alpha_c)
    float2 *trig = nullptr; // [views_per_turn] (cos, sin) of l_{k+1/2} + lambda0, k mod views_per_turn
    float2 *trig_lo = nullptr;  // their rounding residuals: (cos - float(cos), sin - float(sin))
    int *dev_status = nullptr;  // device error word (bounded waits that gave up), 0 = ok
    // Tile-relative projection (staged backprojection and its transpose): for each kTileX x kTileY
    // column tile t and view k of a turn, [t][k][2] float4 {u_r, v_r, e_u, e_v}, {r2, c_hi, c_lo, clo}:
    // the tile centre's u*, v* (FP64) as floats u_r, v_r plus residuals e_u, e_v; r2 = u_r^2 + v_r^2;
    // the window's first column clo (int bits) and the column coordinate of the ray through (u_r, v_r)
    // relative to it, c_hi + c_lo.  A voxel's column is then c_hi + c_lo + atan(cross / dot) / d_alpha
    // with cross, dot formed from its small offset from the centre, with no cancellation.
    float4 *geo = nullptr;
    int geo_ntx = 0, geo_nty = 0;
    float geo_tmax = 0.0f;  // largest |tan| of a voxel's angle from its tile centre's ray
    size_t plan_bytes = 0;
};

// device status codes written to Plan::dev_status
constexpr int kDevStatusTimeout = 1;

// thread-local error message
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);
// NVTX range for the host-side span of one stage (plan, filter, backprojection, ...): what a
// profiler shows on the CPU timeline and what `ncu --nvtx --nvtx-include` filters on.  NVTX is
// header-only and costs a few tens of nanoseconds when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Count of the library's kernel launches in this process (katsevich_launch_count).
void count_launches(int n);
int64_t launches_so_far();

#define KATS_CUDA(call)                                                 \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return ::kats::cuda_fail(_e, #call);     \
    } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Kernel launchers (defined in filter.cu, backproject.cu, adjoint.cu).
// Reduced-precision storage (KATS_PREC_BF16 / KATS_PREC_FP16): derivative data
// and filtered data are stored as 16-bit values scaled by d_alpha; the
// filtered data use a row-pair layout, one 32-bit word (g[r-1][c], g[r][c])
// per pair-row r = 0..n_rows ([n_fviews][n_rows + 1][gf_cols] words).
size_t filter16_workspace_bytes(const Plan &p);
int launch_filter16(const Plan &p, int prec, const float *sino, uint32_t *gFp, void *ws, size_t ws_bytes,
                    cudaStream_t st, int64_t nv = -1);
// A backprojection launch's share of the views: absolute view indices [k_lo, k_hi]; acc_in: vol
// holds the raw sums of the earlier views; acc_final: the launch scales and stores the result.
// Launches over consecutive view ranges, the first without acc_in and the last with acc_final,
// give bit for bit the result of one launch over all views.
struct BPRange {
    int k_lo = INT32_MIN, k_hi = INT32_MAX;
    int acc_in = 0, acc_final = 1;
    // lead_end: only the slices s of [s_begin, s_end) whose leading slice s_begin + (s - s_begin)
    // mod N lies below lead_end (slices one or more pitches apart go together; the host pipeline
    // copies such a group of leads back while the next one runs); takes every view
    int lead_end = INT32_MAX;
};
// Slices of [s_begin, s_end) whose leading slice s_begin + (s - s_begin) mod N is below lead_end,
// as ranges.
inline std::vector<std::pair<int, int>> lead_ranges(int s_begin, int s_end, int N, int lead_end)
{
    std::vector<std::pair<int, int>> r;
    const int le = std::min(lead_end, s_begin + N);
    for (int b = s_begin; b < s_end; b += N)
        if (b < std::min(s_end, b + (le - s_begin))) r.push_back({b, std::min(s_end, b + (le - s_begin))});
    return r;
}
// slabs: slices [s_begin, s_begin + s_count), s_begin a multiple of 16 (s_count < 0: every slice)
int launch_backproject16(const Plan &p, int prec, const uint32_t *gFp, float *vol, cudaStream_t st, int s_begin = 0,
                         int s_count = -1, const BPRange &range = BPRange());
int launch_hilbert_tc16(const Plan &p, int prec, const uint16_t *g3, float *g4, int64_t M, int ldc, cudaStream_t st,
                        bool *done);

// sino points at sinogram view p.first_view; gF receives p.n_fviews filtered views
// nv < 0: every filtered view; otherwise views [0, nv) of the given pointers (a chunk)
int launch_filter(const Plan &p, const float *sino, float *gF, void *ws, size_t ws_bytes, cudaStream_t st,
                  int64_t nv = -1);
// gF: [p.n_fviews][n_rows][p.gf_cols], view 0 = half-view p.first_view, pad columns zero
int launch_backproject(const Plan &p, const float *gF, float *vol, cudaStream_t st, int s_begin = 0,
                       int s_count = -1, const BPRange &range = BPRange());
int launch_backproject_adjoint(const Plan &p, const float *vol, float *gF, cudaStream_t st);
int launch_filter_adjoint(const Plan &p, const float *gF, float *sino, void *ws, size_t ws_bytes,
                          cudaStream_t st);
size_t filter_workspace_bytes(const Plan &p);
// views per chunk of the filter (steps 1-6 run chunk by chunk through one reused scratch buffer)
// for a chunk scratch of bytes_per_view per view
int64_t filter_chunk_views(const Plan &p, size_t bytes_per_view);
// tensor-core Hilbert step (hilbert_tc.cu); *done = false when it cannot run
int launch_hilbert_tc(const Plan &p, const float *g3, float *g4, int64_t M, int ldc, cudaStream_t st, bool *done);
// C[M][ldc] = A[M][K] . B on the tensor cores (3xTF32), B given as hi / lo [N][K] row-major, K a multiple
// of 32, N and ldc multiples of 256; *done = false when the tensor-core path cannot run.
int launch_hilbert_tc_op(const Plan &p, const float *A, int64_t M, int64_t K, const float *b_hi, const float *b_lo,
                         int64_t N, float *C, int ldc, cudaStream_t st, bool *done);
size_t filter_adjoint_workspace_bytes(const Plan &p);

// one item from host buffers (api.cu): device bytes it needs, and the
// stream-ordered H2D window copy + steps 1-7 + D2H volume copy
size_t host_item_bytes(const Plan &p, int precision);
int recon_one_host(const Plan &p, int precision, const float *host_sino, float *host_vol, void *ws, cudaStream_t st);

// device allocations that honour the test hook katsevich_debug_fail_allocs (plan.cu)
cudaError_t dev_malloc(void **ptr, size_t bytes);
cudaError_t dev_malloc_async(void **ptr, size_t bytes, cudaStream_t st);

}  // namespace kats
