/*
 * katsevich.h -- C ABI of the B300 (sm_103a) Katsevich helical cone-beam
 * reconstruction library (curved detector, computed pitch by pitch).
 *
 * Operator (W. Wang et al., "A three-dimensional dual-domain deep network for
 * high-pitch and sparse helical CT reconstruction", Sec. II):
 *   steps 1-6  sinogram g -> filtered data g^F   (derivative, length weight,
 *              forward rebinning onto kappa-lines, Hilbert transform in alpha,
 *              backward rebinning, post-cosine weight)
 *   step 7     g^F -> volume f by backprojection over each voxel's PI interval
 * with the kappa tables and the PI tables of ONE pitch computed once per
 * geometry (the "pre-calculating step") and reused for every pitch through the
 * periodicity of the PI endpoints and of v*, alpha*, w*.
 *
 * Conventions shared by every entry point
 *   helix     a(l) = (R cos(l+lambda0), R sin(l+lambda0), z0 + P l / (2 pi))
 *   views     sinogram view k at l_k = lambda_first + k * 2 pi / views_per_turn
 *   filtered  g^F view k at the half angle l_{k+1/2} (k = 0 .. n_views-2)
 *   detector  column c at alpha_c = (c - (n_cols-1)/2) d_alpha + alpha_offset
 *             row r at    w_r     = (r - (n_rows-1)/2) d_w     + w_offset
 *             (curved detector at distance D; ray ~ D sin(a) e_u + D cos(a) e_v + w e_z)
 *   volume    voxel (i, j, s) at (x0 + i dx, y0 + j dy, z_first + s dz)
 *   layouts   sinogram [batch][n_views][n_rows][n_cols]   (float32, c fastest)
 *             volume   [batch][nz][ny][nx]                (float32, x fastest)
 *   pitch     P / dz must be an integer N (slices per pitch); slice s uses
 *             PI-table slice s mod N shifted by (s div N) * views_per_turn views
 *
 * Memory: every data pointer is a DEVICE pointer on the current CUDA device
 * unless the name says host.  The caller owns all buffers; the library only
 * reads inputs and writes outputs.  A plan owns its device tables and is
 * immutable after katsevich_plan returns, so one plan may be used from several
 * streams at once (each call needs its own workspace).
 *
 * Errors: every entry point returns a KATS_* status; nothing throws across the
 * ABI.  On a non-zero status, katsevich_last_error() returns a message for the
 * calling thread, output buffers are not written by host-side checks, and a
 * status of KATS_ECUDA means a CUDA call failed (its error string is in the
 * message).
 */
#ifndef KATSEVICH_H
#define KATSEVICH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define KATS_API __attribute__((visibility("default")))
#else
#define KATS_API
#endif

#define KATS_OK 0
#define KATS_EINVAL 1   /* bad argument: null pointer, size, dtype, batch      */
#define KATS_EGEOM 2    /* invalid geometry (see katsevich_plan)               */
#define KATS_ENOMEM 3   /* device allocation failed                            */
#define KATS_ECUDA 4    /* a CUDA runtime/driver call failed                   */
#define KATS_ETIMEOUT 5 /* a bounded wait gave up                               */
#define KATS_ESPACE 6   /* caller workspace smaller than required              */

/* Storage precision of the intermediate data (precision form of the operator):
 * FP32 everywhere, or the rebinned derivative data and the filtered data g^F
 * stored in BF16 / FP16 (scaled by d_alpha), the Hilbert contraction on 16-bit
 * tensor cores with the Toeplitz operand split hi + lo, and FP32 accumulation
 * (FP16 interpolates the detector column pair in packed half arithmetic, BF16
 * unpacks exactly to FP32 first).  The reduced
 * forms are available for katsevich_recon and katsevich_recon_host; every other
 * entry point takes KATS_PREC_FP32. */
#define KATS_PREC_FP32 0
#define KATS_PREC_BF16 1
#define KATS_PREC_FP16 2

#define KATS_ENDPOINT_FRACTIONAL 0 /* midpoint rule: end views weighted by covered fraction */
#define KATS_ENDPOINT_HARD 1       /* views with l_{k+1/2} in [lam_i, lam_o], weight 1     */

typedef struct kats_geometry {
    double R;            /* helix radius (mm), Sec. II helix equation                    */
    double D;            /* source-to-detector distance (mm), curved detector            */
    double P;            /* pitch (mm per turn)                                           */
    double lambda0;      /* helix start angle (rad)                                       */
    double z0;           /* helix start height (mm)                                       */
    double lambda_first; /* angle of sinogram view 0 (rad)                                */
    int64_t views_per_turn, n_views;
    int64_t n_rows, n_cols;
    double d_alpha, alpha_offset; /* column pitch and offset (rad)                        */
    double d_w, w_offset;         /* row pitch and offset (mm at distance D)              */
    int64_t nx, ny, nz;
    double dx, dy, dz;            /* voxel size (mm)                                      */
    double x0, y0, z_first;       /* centre of voxel (0, 0, 0) (mm)                       */
    int64_t n_psi;                /* kappa lines; 0 selects 2 * n_rows                    */
    int64_t endpoint_mode;        /* KATS_ENDPOINT_*                                      */
    int64_t flags;                /* reserved, must be 0                                  */
} kats_geometry;

typedef struct kats_plan kats_plan; /* opaque; device-resident tables */

typedef struct kats_plan_info {
    /* Sec. II Eq. (maxvalue): lam_min/max over the PI endpoints of one pitch;
     * alpha/w extremes of (alpha*, w*) over the views each voxel of that pitch
     * backprojects (evaluated in FP32 on the device). */
    double lambda_min, lambda_max, alpha_min, alpha_max, w_min, w_max;
    double alpha_m;           /* arcsin(r_fov / R), r_fov = farthest volume corner   */
    double psi_max;           /* pi/2 + alpha_m                                        */
    int64_t slices_per_pitch; /* N = P / dz                                            */
    int64_t n_psi;
    int64_t first_view;       /* first filtered half-view the volume needs             */
    int64_t n_filtered_views; /* filtered half-views needed (sinogram views: +1)       */
    int64_t update_count;     /* sum over voxels of their PI-window view counts        */
    int64_t gf_cols;          /* row pitch of filtered data: n_cols rounded up to 4    */
    int64_t workspace_bytes;  /* per concurrent call, FP32 storage                     */
    int64_t plan_bytes;       /* device bytes held by the plan                         */
    int64_t pi_monotone;      /* 1: every voxel column's PI-window start and end (with
                               * end weights) are nondecreasing in z, the property the
                               * backprojection's ramp handling uses; 0: it takes the
                               * general per-slice weights                             */
} kats_plan_info;

/*
 * Largest pitch whose Tam-Danielsson window fits the detector rows, times
 * `factor`, rounded down to a whole number of slices of thickness g->dz.
 * (Sec. I: the row count needed for exact reconstruction grows with the pitch;
 * on the curved detector the widest TD extent over |alpha| <= alpha_m is
 * (D P / (2 pi R)) (pi/2 + alpha_m) / cos(alpha_m), which must not exceed the
 * outermost row centre (n_rows - 1)/2 * d_w.)  Uses R, D, n_rows, d_w, dz and
 * the volume extent of *g; g->P is ignored.  Host only.
 */
KATS_API int katsevich_fit_pitch(const kats_geometry *g, double factor, double *pitch_out);

/*
 * Pre-calculating step (Sec. II): validate *g and build, on the current
 * device, in FP64 arithmetic,
 *   - the forward-rebinning table w_kappa(alpha_{c+1/2}, psi_l) (Eq. (w_k)) as
 *     (row index, weight), psi_l uniform on [-psi_max, psi_max];
 *   - the backward-rebinning table psi_hat(alpha_c, w_r), the root of smallest
 *     |psi| (Sec. II step 5), as (psi index, weight);
 *   - the PI table of one pitch: PI-line endpoints lam_i < lam_o of every voxel
 *     column point (x, y, z_first + j dz), j < N (Eq. (e1)), turned into the
 *     first/last filtered view and their end weights.
 * Errors: KATS_EGEOM when R, D, P, sizes or spacings are not positive, r_fov >=
 * R, P/dz is not an integer, flags != 0, or some voxel's PI window needs a
 * filtered view outside [0, n_views - 2]; KATS_ENOMEM / KATS_ECUDA otherwise.
 * On success *out owns device memory until katsevich_plan_destroy.
 * Synchronous (returns after the tables are built).
 */
KATS_API int katsevich_plan(const kats_geometry *g, kats_plan **out);

/* Extents, sizes and the update count of a plan (host only). */
KATS_API int katsevich_plan_info(const kats_plan *plan, kats_plan_info *info);

/* Device workspace bytes one recon/adjoint call needs for `precision`. */
KATS_API int64_t katsevich_workspace_bytes(const kats_plan *plan, int precision);

/*
 * Full operator, steps 1-7 (Sec. II reconstruction step), for `batch`
 * sinograms: sino [batch][n_views][n_rows][n_cols] -> vol [batch][nz][ny][nx].
 * `precision` is one of KATS_PREC_*; the 16-bit forms need the staged
 * backprojection (KATS_EINVAL for detectors narrower than its column window).
 * Only sinogram views [first_view, first_view + n_filtered_views] are read.
 * `workspace` (device, >= katsevich_workspace_bytes) is scratch owned by the
 * caller; `stream` is a cudaStream_t (NULL = legacy default stream).
 * Stream-ordered and asynchronous: returns after enqueueing the kernels.
 */
KATS_API int katsevich_recon(const kats_plan *plan, const float *sino, float *vol, int batch,
                    int precision, void *workspace, size_t workspace_bytes, void *stream);

/*
 * Exact transpose of katsevich_recon (same discretisation, same precision
 * rule): vol_grad [batch][nz][ny][nx] -> sino_grad [batch][n_views][n_rows][n_cols].
 * Every element of sino_grad is written (views outside the window get 0).
 */
KATS_API int katsevich_adjoint(const kats_plan *plan, const float *vol_grad, float *sino_grad, int batch,
                      int precision, void *workspace, size_t workspace_bytes, void *stream);

/*
 * Steps 1-6 only (Sec. II Eqs. (Deriv), (LW), (FR), (HF), (BR), (PW)):
 * sino [batch][n_views][n_rows][n_cols] -> gF [batch][n_filtered_views][n_rows][gf_cols]
 * (rows padded to gf_cols = n_cols rounded up to 4 floats, pad columns written
 * as 0); filtered view v of the output is half-view first_view + v.
 */
KATS_API int katsevich_filter(const kats_plan *plan, const float *sino, float *gF, int batch,
                     int precision, void *workspace, size_t workspace_bytes, void *stream);

/*
 * Step 7 only (Sec. II backprojection step): gF [batch][n_filtered_views][n_rows][gf_cols]
 * (layout of katsevich_filter's output, FP32, 16-byte aligned, pad columns 0)
 * -> vol [batch][nz][ny][nx].
 */
KATS_API int katsevich_backproject(const kats_plan *plan, const float *gF, float *vol, int batch, void *stream);

/*
 * Transpose of step 7 alone: vol [batch][nz][ny][nx] -> gF [batch][n_filtered_views][n_rows][gf_cols]
 * (every element written; pad columns 0).  FP32 atomics: the summation order,
 * and so the last bits, may vary between calls.
 */
KATS_API int katsevich_backproject_adjoint(const kats_plan *plan, const float *vol, float *gF, int batch, void *stream);

/*
 * Transpose of steps 1-6 alone: gF [batch][n_filtered_views][n_rows][gf_cols]
 * -> sino [batch][n_views][n_rows][n_cols] (every element written).
 * `workspace` as for katsevich_adjoint.
 */
KATS_API int katsevich_filter_adjoint(const kats_plan *plan, const float *gF, float *sino, int batch, int precision,
                                      void *workspace, size_t workspace_bytes, void *stream);

/*
 * End-to-end call with HOST buffers: copies the needed sinogram views from
 * host_sino (pinned memory recommended) to the device, runs katsevich_recon and
 * copies the volume back to host_vol, then waits for `stream`.  `workspace`
 * (device) must hold katsevich_host_workspace_bytes.  Items whose view window
 * is 128 MiB or more overlap the copies with the kernels on internal streams
 * (ordered after the work already on `stream`): the window arrives in chunks
 * that are filtered as they land, slabs of slices are backprojected as soon as
 * their views are filtered, and finished slabs are copied back while later
 * ones run.  The volume is bit for bit that of katsevich_recon.
 */
KATS_API int64_t katsevich_host_workspace_bytes(const kats_plan *plan, int batch, int precision);
KATS_API int katsevich_recon_host(const kats_plan *plan, const float *host_sino, float *host_vol, int batch,
                         int precision, void *workspace, size_t workspace_bytes, void *stream);

/*
 * z-slab partition of one reconstruction (Sec. II backprojection step: a voxel
 * takes only the views of its PI interval, so a range of slices needs only the
 * views whose half-view lies in the union of its voxels' PI windows; the paper
 * backprojects slice by slice for the same reason).  Host only.
 * katsevich_slab_views: the sinogram views [*view_begin, *view_begin +
 * *view_count) that slices [s_begin, s_end) of the plan's volume read
 * (0 <= s_begin < s_end <= nz; *view_count is 0 when no voxel of the range has
 * a PI window).  Neighbouring slabs overlap in views (the PI windows are longer
 * than one turn's share), not in slices.
 */
KATS_API int katsevich_slab_views(const kats_plan *plan, int64_t s_begin, int64_t s_end, int64_t *view_begin,
                                  int64_t *view_count);

/*
 * Steps 1-7 for slices [s_begin, s_end) of one volume, from just the views the
 * slab reads: sino_views [view_count][n_rows][n_cols] (device) holds sinogram
 * views [view_begin, view_begin + view_count), which must cover the range
 * katsevich_slab_views returns; vol_slab [s_end - s_begin][ny][nx] (device)
 * receives the slab.  s_begin must be a multiple of 16 (the backprojection's
 * slice tile): the slab then equals slices [s_begin, s_end) of katsevich_recon
 * bit for bit, in every precision.  `workspace` as for katsevich_recon.  One
 * slab per GPU, with no exchange between them, is the multi-GPU partition of a
 * single volume.  Stream-ordered and asynchronous.
 */
KATS_API int katsevich_recon_slab(const kats_plan *plan, const float *sino_views, int64_t view_begin,
                                  int64_t view_count, int64_t s_begin, int64_t s_end, float *vol_slab, int precision,
                                  void *workspace, size_t workspace_bytes, void *stream);

/*
 * Copy a plan table to host memory (for checks against an independent
 * implementation).  which: 0 kappa row index (int32 [n_psi][n_cols-1]),
 * 1 kappa weight (float), 2 psi index (int32 [n_rows][n_cols]), 3 psi weight
 * (float), 4 first view k0 (int32 [N][ny][nx]), 5 last view k1, 6 first-view
 * weight (float), 7 last-view weight (float).  `bytes` must equal the size.
 */
KATS_API int katsevich_plan_table(const kats_plan *plan, int which, void *host_dst, size_t bytes);

/*
 * The device FP64 PI-line solver on n host points xyz[n][3] (Eq. (e1)):
 * writes lam_i[n], lam_o[n] (host).  Synchronous; for checks.
 */
KATS_API int katsevich_pi_endpoints(const kats_geometry *g, int64_t n, const double *host_xyz,
                           double *host_lam_i, double *host_lam_o);

/*
 * katsevich_recon without a caller workspace, for callers that cannot
 * allocate device memory when they reconstruct: services whose device memory
 * is reserved up front by another allocator, or loops where a cudaMalloc /
 * cudaFree (which may synchronise the device) would stall other streams.
 * The paper has no counterpart; this is an interface convenience.
 *
 * Same operator, layouts and FP32 precision as katsevich_recon.  The scratch
 * is a fixed array of KATS_NOALLOC_SCRATCH_BYTES in the library's device
 * memory (every GPU that loads the library holds one copy until the process
 * exits).  Nothing is allocated: no cudaMalloc, cudaFree or allocating library
 * call.  Geometries whose scratch (filtered views plus filter intermediates)
 * exceeds the array are rejected with KATS_ESPACE and a message giving both
 * sizes; use katsevich_recon for them.  The first call on a device looks up
 * the array's device address (once per device, with that device current);
 * make that first call before any stream capture.  All calls share the one
 * array, so calls whose work overlaps on the GPU (different streams, or
 * different threads) race and corrupt each other's results: serialise them.
 * Every scratch element read is written earlier by the same call, so no
 * state carries over from the previous call.
 */
#define KATS_NOALLOC_SCRATCH_BYTES (64u << 20)
KATS_API int katsevich_recon_noalloc(const kats_plan *plan, const float *sino, float *vol, int batch, void *stream);

/*
 * Device status of a plan's kernels: waits inside the kernels are bounded;
 * one that gives up records KATS_ETIMEOUT-class status here instead of
 * hanging.  Synchronises the device, returns the word in *status (0 = ok) and
 * clears it.
 */
KATS_API int katsevich_device_status(const kats_plan *plan, int *status);

/*
 * Serving loop (the operator's deployment form; the paper has no counterpart).
 *
 * A server owns CUDA streams ("slots"), one device arena and a device plan
 * cache.  katsevich_server_submit queues a request (any geometry, volume size
 * and precision; host sinogram in, host volume out) and returns at once.  A
 * worker thread admits queued requests in arrival order as soon as a slot is
 * free and the request's device block (view window + volume + workspace,
 * katsevich_host_workspace_bytes of its plan) fits in the arena; requests that
 * arrive while others run are admitted as slots and memory free up, and
 * their copies and kernels overlap on the device (continuous batching).  A
 * request whose block does not fit waits; later requests may be admitted
 * ahead of the first one in line at most max_bypass times, then admission
 * waits for it.  A request larger than the whole arena completes with
 * KATS_ENOMEM ("refused").  Plans are built on first use (on the worker
 * thread, on a private stream) and cached by geometry; when the cache's plans
 * exceed plan_cache_bytes, idle plans are destroyed least recently used first
 * (destroying one may wait for the device).
 *
 * Ownership: host_sino (the full sinogram [n_views][n_rows][n_cols]) and
 * host_vol ([nz][ny][nx]) are the caller's and must stay valid until
 * katsevich_server_wait has returned for the ticket; page-locked buffers let
 * the copies overlap other requests' kernels (pageable ones still work, with
 * the copies serialised).  Results are bit-identical to katsevich_recon_host
 * on the same plan and precision: each request runs the same kernels on its
 * own block.
 *
 * Errors: create/submit/wait return KATS_* codes.  wait returns the request's
 * own status (a failed plan build: its code; a device wait that gave up inside
 * the request's kernels: KATS_ETIMEOUT) and releases the ticket; if the request
 * has not finished after timeout_ms (negative = do not wait) it returns
 * KATS_ETIMEOUT and the ticket stays valid.  Destroying the server finishes the
 * running requests, fails the queued ones and invalidates every ticket.
 */
typedef struct kats_server kats_server;
typedef struct kats_server_config {
    int64_t arena_bytes;      /* device bytes for the running requests' blocks (one allocation)  */
    int64_t plan_cache_bytes; /* device bytes of cached plans before idle ones are evicted        */
    int32_t slots;            /* concurrent requests, one CUDA stream each (1 .. 64)              */
    int32_t max_bypass;       /* later requests admitted ahead of a waiting first-in-line one     */
} kats_server_config;
typedef struct kats_request_stats {
    int32_t status;       /* the request's KATS_* status                                   */
    int32_t slot;         /* slot it ran on (-1 if never admitted)                          */
    int32_t plan_hit;     /* 1 if its plan was already cached when it was first considered  */
    int32_t bypassed;     /* requests admitted ahead of it while it was first in line       */
    double t_submit_ms;   /* host clock (ms since the server started): submitted            */
    double t_admit_ms;    /*   admitted (slot and block assigned, work issued)              */
    double t_done_ms;     /*   completion seen by the worker                                */
    double gpu_ms;        /* device time of its stream work (copies + kernels), CUDA events */
    int64_t device_bytes; /* arena bytes it held                                            */
} kats_request_stats;
typedef struct kats_server_stats {
    int64_t submitted, completed, failed, refused;
    int64_t plan_hits, plan_misses, plan_evictions, plans_cached;
    int64_t arena_bytes, arena_in_use_bytes, arena_peak_bytes, plan_cache_used_bytes;
    int32_t slots, max_running, pending, running;
} kats_server_stats;
KATS_API int katsevich_server_create(const kats_server_config *cfg, kats_server **out);
KATS_API int katsevich_server_submit(kats_server *srv, const kats_geometry *g, const float *host_sino,
                                     float *host_vol, int precision, uint64_t *ticket);
KATS_API int katsevich_server_wait(kats_server *srv, uint64_t ticket, int64_t timeout_ms, kats_request_stats *stats);
KATS_API int katsevich_server_stats(kats_server *srv, kats_server_stats *out);
KATS_API void katsevich_server_destroy(kats_server *srv);

/*
 * The server's admission arena as a host-only object (no device memory is
 * touched): first-fit offsets in [0, bytes), blocks rounded up to 256 bytes,
 * freed neighbours merged.  alloc returns an offset or -1 when no free block
 * fits; free returns KATS_EINVAL for an offset that is not an allocated block.
 */
typedef struct kats_arena kats_arena;
KATS_API int katsevich_arena_create(int64_t bytes, kats_arena **out);
KATS_API int64_t katsevich_arena_alloc(kats_arena *a, int64_t bytes);
KATS_API int katsevich_arena_free(kats_arena *a, int64_t offset);
KATS_API int64_t katsevich_arena_largest_free(const kats_arena *a);
KATS_API int64_t katsevich_arena_in_use(const kats_arena *a);
KATS_API void katsevich_arena_destroy(kats_arena *a);

/*
 * Data simulation (the paper's Sec. III-C data generation), producing the
 * network's input sinograms from label volumes.  Conventions and layouts as
 * above; all pointers are device pointers unless named host_.
 *
 * katsevich_project: sino[v - v0][row][col] for views v0 .. v0+nv-1 = the line
 *   integral, along the ray from the source a(l_v) through the detector sample
 *   (alpha_col, w_row), of the piecewise-constant voxel function (voxel
 *   (i, j, s) is the cube of side dx, dy, dz centred at (x0 + i dx, y0 + j dy,
 *   z_first + s dz) with value vol[s][j][i]; zero outside the volume).  Only
 *   the geometry's scan and volume fields are used (P, not a plan); the volume
 *   must hold fewer than 2^31 voxels.
 * katsevich_sparse_upsample: the sparse detector (columns 0, keep, 2 keep, ...
 *   of each row of nv views) interpolated linearly back to every column;
 *   columns past the last kept one take its value.  sino and out must not
 *   overlap.
 * katsevich_add_noise: M = max(g_up) (of the non-negative entries, 0 if none),
 *   counts_i = Poisson(I0 exp(-g_up_i / M)) (a draw of the generator
 *   Philox4x32-10 keyed by seed with counter (i, draw, 0): PTRS transformed
 *   rejection for means >= 10, multiplication of uniforms below), plus
 *   mean + sqrt(var) z_i with z_i normal (Box-Muller on counter (i, 0, 1)),
 *   floored at 1; g_in_i = M log(I0 / that).  The paper's "g + poisson(g)" is
 *   read as the Poisson draw of g.  counts (nullable, int64) receives the
 *   Poisson draws.  workspace holds katsevich_noise_workspace_bytes() bytes;
 *   host_M (nullable) receives M and makes the call synchronous.  The result
 *   depends only on (g_up, I0, mean, var, seed), not on launch shape.
 */
KATS_API int katsevich_project(const kats_geometry *g, const float *vol, float *sino, int64_t v0, int64_t nv,
                               void *stream);
KATS_API int katsevich_sparse_upsample(const kats_geometry *g, const float *sino, float *out, int64_t nv, int keep,
                                       void *stream);
KATS_API int64_t katsevich_noise_workspace_bytes(void);
KATS_API int katsevich_add_noise(const float *g_up, float *g_in, int64_t n, double I0, double mean, double var,
                                 uint64_t seed, int64_t *counts, void *workspace, size_t workspace_bytes,
                                 double *host_M, void *stream);

/*
 * Measured read bandwidth of the current GPU's shared-memory data path, the
 * path the backprojection's bilinear taps are read through (its roofline):
 * 4 CTAs per SM of 1024 threads stream conflict-free 16-byte shared loads; the
 * best of 4 timed rounds of 3 launches, in bytes per second, goes to
 * *bytes_per_second.  Synchronous (its own stream); about 40 ms.  Errors:
 * KATS_EINVAL for a NULL pointer, KATS_ECUDA.
 */
KATS_API int katsevich_smem_read_bandwidth(double *bytes_per_second);

/*
 * Measured rate of bilinear (hardware-filtered) 2-D texture fetches on the
 * current GPU, FP32 texels (half_texels = 0) or FP16 texels (1): the gather
 * path a texture-based backprojection would take, one filtered sample per
 * voxel-view update (with 8-bit interpolation weights).  8 CTAs per SM of 256
 * threads fetch from a 256 x 256 texture; the best of 4 timed rounds of 3
 * launches, in samples per second, goes to *samples_per_second.  Synchronous;
 * about 50 ms.  Errors: KATS_EINVAL for a NULL pointer, KATS_ECUDA.
 */
KATS_API int katsevich_tex_bilinear_rate(int half_texels, double *samples_per_second);

/*
 * Bounds-checked build (compiled with KATS_DEBUG_CHECKS, libkatsevich_debug.so;
 * it stands in for a memory checker).  The staged-window kernels verify that
 * every voxel's detector column lies inside its CTA's staged view window and
 * that every tap row they read unclamped lies inside the staged rows (the
 * plan's extents claim both).  A violation sets a bit in a device word
 * instead of reading outside shared memory: 1 backprojection column, 2
 * backprojection row, 4 adjoint column, 8 adjoint row.
 * katsevich_debug_checks_enabled: 1 in the checked build, 0 otherwise.
 * katsevich_debug_check_flags: synchronises the device, returns the word in
 * *flags (always 0 in the plain build) and clears it; KATS_EINVAL for NULL.
 */
KATS_API int katsevich_debug_checks_enabled(void);
KATS_API int katsevich_debug_check_flags(int *flags);
/* Checked build only (a no-op otherwise): stage every view window `cols`
 * columns narrower than its tile needs, so that the column check fires; taps
 * stay clamped inside the window, results are wrong, nothing faults.  0 ends it. */
KATS_API void katsevich_debug_narrow_window(int cols);
/* Checked build only (a no-op otherwise): launch the backprojection as if the plan's PI windows
 * were not monotone in z (on != 0), so every view takes the general end-weight path instead of
 * the ramp walk; the result must not change.  0 ends it. */
KATS_API void katsevich_debug_nonmonotone(int on);
/* Checked build only (no-ops returning KATS_OK otherwise), for the test of the device-timeout
 * path, set on the current device:
 * katsevich_debug_wait_limit: the staged backprojection's bounded mbarrier waits give up after
 *   `polls` polls instead of 2^22 (<= 0 restores the default);
 * katsevich_debug_stall_producer: its producer warp stops issuing view pairs after `pairs` of
 *   them (arming no further copy), so the consumers' waits run out, the CTA records
 *   KATS_ETIMEOUT in the plan's device status (katsevich_device_status) and retires with no
 *   copy in flight; the volume is then incomplete.  A negative value ends it.
 * Errors: KATS_ECUDA. */
KATS_API int katsevich_debug_wait_limit(int polls);
KATS_API int katsevich_debug_stall_producer(int pairs);

/*
 * Host only (no device needed): how the backprojection groups slices [s_begin, s_end) of a volume
 * with slices_per_pitch slices per pitch.  By the periodicity of Sec. II a slice m pitches up sees
 * view k + m views_per_turn as the slice m pitches down sees view k, so one thread reconstructs
 * a column of groups of slices one pitch apart and computes each view's geometry once for all of
 * them.  Item i has groups[i] groups (2 to max_groups, at most 4) of cnt[i] slices each, group m
 * covering slices [s0[i] + m N, s0[i] + m N + cnt[i]), N = slices_per_pitch, in a form with t[i]
 * >= cnt[i] slices per group per thread; slices in no item go to the one-group kernel as ranges
 * [rest[2j], rest[2j + 1]).  lead_end restricts the leading slices to [s_begin, lead_end), and so
 * the slices to those whose leading slice s_begin + (s - s_begin) mod N lies below it (the host
 * pipeline launches its last slab in such groups of leads; INT64_MAX: no restriction).  Every
 * slice of the (restricted) set lies in exactly one item group or range.  The library's
 * own launches use this grouping with max_groups from the plan's row-band bound (4 for the
 * clinical scanners).  Capacities: max_items items, max_rest ranges; the counts go to *n_items and
 * *n_rest in any case.  Errors: KATS_EINVAL for a NULL pointer or bad size, KATS_ESPACE when a
 * capacity is too small.
 */
KATS_API int katsevich_slice_groups(int64_t s_begin, int64_t s_end, int64_t slices_per_pitch, int max_groups,
                                    int64_t lead_end, int32_t *groups, int32_t *t, int32_t *s0, int32_t *cnt,
                                    int max_items, int *n_items, int32_t *rest, int max_rest, int *n_rest);

/*
 * Number of kernels the library has launched in this process so far (every
 * device, every entry point), for launch accounting: the difference across a
 * region is the library's launches inside it.
 */
KATS_API int64_t katsevich_launch_count(void);

/*
 * Host-side fault injection for tests: the next n device allocations the
 * library makes (plan tables and scratch, a server's arena) fail as if the
 * device were out of memory, without calling CUDA; the call then returns
 * KATS_ENOMEM.  n <= 0 switches injection off.
 */
KATS_API void katsevich_debug_fail_allocs(int n);

/* Release a plan's device memory.  NULL is allowed. */
KATS_API void katsevich_plan_destroy(kats_plan *plan);

/* Message of the last failed call on this thread ("" if none). */
KATS_API const char *katsevich_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KATSEVICH_H */
