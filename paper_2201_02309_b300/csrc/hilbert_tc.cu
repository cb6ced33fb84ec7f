// Step 4 of the reconstruction step (Sec. II, Eq. (HF)): the Hilbert
// transform in alpha at constant psi, as a Toeplitz contraction on the 5th
// generation tensor cores:
//     g4[m][c] = sum_{c'} g3[m][c'] T[c'][c],   T[c'][c] = hk(c - c'),
// m = (filtered view, psi line), c' = half-grid column, c = column.
//
// FP32 accuracy from TF32 operands (3xTF32): A = A_hi + A_lo and
// T = T_hi + T_lo with hi exact in TF32 (low 13 mantissa bits cleared), and
//     C = A_hi T_hi + A_hi T_lo + A_lo T_hi
// (the dropped A_lo T_lo term is ~2^-22 of the product).  T_hi / T_lo are
// plan constants; A is split in place in shared memory.
//
// A 128 x 256 tile of C accumulates in TMEM.  A persistent CTA per SM walks its
// tiles with two accumulators, so one tile's epilogue overlaps the next tile's MMAs:
//   warp 0      TMA producer (A tile 128 x 16, T_hi / T_lo tiles 256 x 16,
//               fp32, 64-byte swizzle), 4-stage ring running across tiles
//   warp 1      TMEM allocation and the single-thread tcgen05.mma issuer
//   warps 2..5  split A into hi / lo in shared memory
//   warps 6..9  the epilogue (tcgen05.ld -> registers -> global g4)
// Every mbarrier wait is bounded; on a timeout the CTA records a device
// status, lets its MMAs finish and its copies land, and frees TMEM before
// returning.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace kats {

namespace {

constexpr int TC_M = 128, TC_N = 256;  // tile
constexpr int TC_STAGES = 2;            // ring depth of the 16-bit form
constexpr int TC_THREADS = 192;
constexpr int kTcWaitLimit = 1 << 22;

// Instruction descriptor fields, kind::tf32: D fp32 (bits 4-5 = 1), A and B tf32
// (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28 (TpShape::IDESC).

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t *b, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t *b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool bar_wait(uint64_t *b, uint32_t parity)
{
    for (int i = 0; i < kTcWaitLimit; ++i)
        if (bar_try(b, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap *map, uint64_t *b, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(saddr(b))
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of 128
// bytes, 8-row groups 1024 bytes apart (stride byte offset), descriptor
// version 1 (bits 46-47), layout type 2 = 128-byte swizzle (bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// The same for K blocks of KB fp32 elements: rows of 4 KB bytes with a (4 KB)-byte swizzle
// (layout type 2 = 128-byte, 4 = 64-byte), 8-row groups 8 x 4 KB bytes apart.
template <int KB>
__device__ __forceinline__ uint64_t swz_desc(uint32_t addr)
{
    static_assert(KB == 32 || KB == 16, "K block of 128 or 64 bytes");
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)((8 * 4 * KB) >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)(KB == 32 ? 2 : 4) << 61);
}

template <uint32_t IDESC>
__device__ __forceinline__ void mma_tf32_n(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *b)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(b))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive fp32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcArgs {
    float *C;  // [M][ldc], ldc a multiple of TC_N (whole tiles are stored)
    int64_t M;
    int ldc, kblocks;
    int *status;
};

// Steps of Eq. (HF) as above: one CTA per SM walks the tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... (n-tile fastest), with two TMEM accumulators (2 x 256
// columns), so that the epilogue of one tile overlaps the MMAs of the next and the
// TMA / split / MMA ring runs on across tiles without refilling.
//   warp 0      TMA producer        warp 1      TMEM allocation, MMA issuer
//   warps 2..5  A split hi / lo     warps 6..9  epilogue (TMEM -> registers -> g4)
// Every wait is bounded; on a timeout the CTA records a device status, lets its
// issued MMAs finish and its copies land, and frees TMEM before returning.
constexpr int TP_THREADS = 320;
// tile width, ring depth and K block of the launched form: 4 stages of K blocks of 16 (64-byte
// rows) keep each stage's copies three stages ahead of the MMAs that read it
constexpr int TP_N = 256, TP_STAGES = 4, TP_KB = 16;

// Tile TC_M x N, STAGES-deep ring; one stage holds A, A_lo (TC_M x KB) and T_hi, T_lo (N x KB).
template <int N, int STAGES, int KB>
struct TpShape {
    static constexpr uint32_t A_BYTES = TC_M * KB * 4;
    static constexpr uint32_t B_BYTES = N * KB * 4;
    static constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr uint32_t SMEM = STAGES * STAGE_BYTES + 1024;  // + alignment slack
    // kind::tf32 instruction descriptor for TC_M x N
    static constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
                                      ((uint32_t)(TC_M >> 4) << 24);
};

template <int N, int STAGES, int KB>
__global__ void __launch_bounds__(TP_THREADS, 1)
    k_hilbert_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapBh,
                   const __grid_constant__ CUtensorMap mapBl, TcArgs a, int n_ntiles, int64_t n_tiles)
{
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    using SH = TpShape<N, STAGES, KB>;
    __shared__ __align__(8) uint64_t s_full[STAGES], s_conv[STAGES], s_empty[STAGES];
    __shared__ __align__(8) uint64_t s_accf[2], s_acce[2], s_done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ long long s_issued;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t base = (saddr(tc_raw) + 1023u) & ~1023u;  // 1024-byte aligned (128-byte swizzle atoms)
    unsigned char *const gbase = tc_raw + (base - saddr(tc_raw));
    auto stA = [&](int s) { return base + (uint32_t)s * SH::STAGE_BYTES; };
    auto stAlo = [&](int s) { return stA(s) + SH::A_BYTES; };
    auto stBh = [&](int s) { return stA(s) + 2 * SH::A_BYTES; };
    auto stBl = [&](int s) { return stA(s) + 2 * SH::A_BYTES + SH::B_BYTES; };
    const int nkb = a.kblocks;
    const int64_t my_tiles = n_tiles > (int64_t)blockIdx.x ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto tile_m0 = [&](int64_t i) { return ((int64_t)blockIdx.x + i * gridDim.x) / n_ntiles * TC_M; };
    auto tile_n0 = [&](int64_t i) { return (int)(((int64_t)blockIdx.x + i * gridDim.x) % n_ntiles) * N; };
    auto aborted = [&]() { return *(volatile int *)&s_abort != 0; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            bar_init(&s_full[s], 1);
            bar_init(&s_conv[s], 4);
            bar_init(&s_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init(&s_accf[b], 1);
            bar_init(&s_acce[b], 4);
        }
        bar_init(&s_done, 1);
        s_abort = 0;
        s_issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&s_tmem)),
                     "r"((uint32_t)(2 * N))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        // ---------------- TMA producer: k-block g of the CTA's sequence goes to stage g % 2
        if (lane == 0) {
            long long g = 0;
            for (int64_t i = 0; i < my_tiles && !aborted(); ++i) {
                const int64_t m0 = tile_m0(i);
                const int n0 = tile_n0(i);
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = (int)(g % STAGES);
                    if (g >= STAGES && !bar_wait(&s_empty[s], (uint32_t)(((g / STAGES) - 1) & 1))) {
                        atomicExch(&s_abort, 1);
                        break;
                    }
                    if (aborted()) break;
                    bar_expect(&s_full[s], SH::A_BYTES + 2 * SH::B_BYTES);
                    tma_2d(stA(s), &mapA, &s_full[s], kb * KB, (int)m0);
                    tma_2d(stBh(s), &mapBh, &s_full[s], kb * KB, n0);
                    tma_2d(stBl(s), &mapBl, &s_full[s], kb * KB, n0);
                    s_issued = g + 1;
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer: tile i accumulates in TMEM columns (i % 2) * 256
        if (lane == 0) {
            long long g = 0;
            for (int64_t i = 0; i < my_tiles; ++i) {
                const int b = (int)(i & 1);
                if (i >= 2 && !bar_wait(&s_acce[b], (uint32_t)(((i >> 1) - 1) & 1))) {
                    atomicExch(&s_abort, 1);
                    break;
                }
                if (aborted()) break;
                fence_after();
                const uint32_t acc = tmem + (uint32_t)(b * N);
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = (int)(g % STAGES);
                    if (!bar_wait(&s_conv[s], (uint32_t)((g / STAGES) & 1))) {
                        atomicExch(&s_abort, 1);
                        ok = false;
                        break;
                    }
                    if (aborted()) {
                        ok = false;
                        break;
                    }
                    fence_after();
#pragma unroll
                    for (int kk = 0; kk < KB / 8; ++kk) {  // 8 tf32 = 32 bytes per MMA
                        const uint32_t off = (uint32_t)kk * 32u;
                        const uint64_t dA = swz_desc<KB>(stA(s) + off), dAl = swz_desc<KB>(stAlo(s) + off);
                        const uint64_t dBh = swz_desc<KB>(stBh(s) + off), dBl = swz_desc<KB>(stBl(s) + off);
                        mma_tf32_n<SH::IDESC>(acc, dA, dBh, (kb | kk) != 0);
                        mma_tf32_n<SH::IDESC>(acc, dA, dBl, 1u);
                        mma_tf32_n<SH::IDESC>(acc, dAl, dBh, 1u);
                    }
                    mma_commit(&s_empty[s]);  // stage s free once these MMAs have read it
                }
                if (!ok) break;
                mma_commit(&s_accf[b]);  // tile i complete in buffer b
            }
            mma_commit(&s_done);  // every MMA this thread issued has completed
        }
    } else if (warp < 6) {
        // ---------------- converters: split A into hi / lo in shared memory
        const int ct = threadIdx.x - 64;  // 0..127
        long long g = 0;
        for (int64_t i = 0; i < my_tiles && !aborted(); ++i) {
            for (int kb = 0; kb < nkb; ++kb, ++g) {
                const int s = (int)(g % STAGES);
                if (!bar_wait(&s_full[s], (uint32_t)((g / STAGES) & 1))) {
                    atomicExch(&s_abort, 1);
                    break;
                }
                if (aborted()) break;
                float4 *A = reinterpret_cast<float4 *>(gbase + (stA(s) - base));
                float4 *L = reinterpret_cast<float4 *>(gbase + (stAlo(s) - base));
#pragma unroll
                for (int q = 0; q < (int)(SH::A_BYTES / 16) / 128; ++q) {
                    const int e = ct + 128 * q;
                    float4 v = A[e], h, l;
                    h.x = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
                    h.y = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
                    h.z = __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u);
                    h.w = __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u);
                    l.x = v.x - h.x;
                    l.y = v.y - h.y;
                    l.z = v.z - h.z;
                    l.w = v.w - h.w;
                    A[e] = h;
                    L[e] = l;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor core reads
                __syncwarp();
                if (lane == 0) bar_arrive(&s_conv[s]);
            }
        }
    } else {
        // ---------------- epilogue: TMEM lane = tile row; warp w reads lanes 32 (w % 4) .. + 31
        const int quarter = warp & 3;
        for (int64_t i = 0; i < my_tiles; ++i) {
            const int b = (int)(i & 1);
            if (!bar_wait(&s_accf[b], (uint32_t)((i >> 1) & 1))) {
                atomicExch(&s_abort, 1);
                break;
            }
            if (aborted()) break;
            fence_after();
            const int64_t row = tile_m0(i) + quarter * 32 + lane;
            const int n0 = tile_n0(i);
            const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * N);
            for (int cb = 0; cb < N / 32; ++cb) {
                float v[32];
                tmem_ld32(taddr + (uint32_t)(cb * 32), v);
                if (row < a.M) {
                    float4 *out = reinterpret_cast<float4 *>(a.C + row * a.ldc + n0 + cb * 32);
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        out[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) bar_arrive(&s_acce[b]);  // buffer b free for tile i + 2
        }
    }

    // ---------------- teardown
    fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool done = bar_wait(&s_done, 0u);  // no MMA may still use TMEM when it is freed
        if (s_abort || !done) {
            // let the producer's copies (the last STAGES issued) land before shared memory is released
            for (long long g = s_issued > STAGES ? s_issued - STAGES : 0; g < s_issued; ++g)
                bar_wait(&s_full[g % STAGES], (uint32_t)((g / STAGES) & 1));
            atomicExch(a.status, kDevStatusTimeout);
        }
    }
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * N))
                     : "memory");
    }
}

typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                             const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder()
{
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeFn)ptr;
    });
    return fn;
}

bool encode_2d(EncodeFn enc, CUtensorMap *map, const float *ptr, int64_t inner, int64_t outer, int box_inner,
               int box_outer, CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B)
{
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)inner * 4};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)ptr, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ---------------------------------------------------------------- 16-bit A
// kind::f16 variant for reduced-precision storage: A (g3 * d_alpha) is exact
// in bf16 / fp16, the Toeplitz operand is split hi + lo in the same type, and
//     C = A T_hi + A T_lo
// accumulates in FP32 in TMEM.  Warps: 0 TMA producer, 1 MMA issuer, 2..5
// epilogue; K blocks of 64 elements (one 128-byte swizzle span) in two stages;
// persistent with two accumulators like the FP32 form.  (Four stages of 32-wide
// K blocks measured slower here: 39.31 against 39.10 ms per FP16 step.)
constexpr int T16_K = 64;
constexpr uint32_t T16_A_BYTES = TC_M * T16_K * 2;  // 16 KB
constexpr uint32_t T16_B_BYTES = TC_N * T16_K * 2;  // 32 KB
constexpr uint32_t T16_STAGE_BYTES = T16_A_BYTES + 2 * T16_B_BYTES;
constexpr uint32_t T16_SMEM = TC_STAGES * T16_STAGE_BYTES + 1024;

// kind::f16 descriptor: D fp32, A and B bf16 (format 1) or fp16 (format 0), K-major.
template <bool FP16>
__device__ __forceinline__ uint32_t idesc_f16()
{
    const uint32_t f = FP16 ? 0u : 1u;
    return (1u << 4) | (f << 7) | (f << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Persistent like k_hilbert_tc: one CTA per SM walks the tiles (n-tile fastest) with two
// TMEM accumulators; warps 2..5 drain tile i while the MMAs of tile i + 1 run.
template <bool FP16>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_hilbert_tc16(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapBh,
                   const __grid_constant__ CUtensorMap mapBl, TcArgs a, int n_ntiles, int64_t n_tiles)
{
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    __shared__ __align__(8) uint64_t s_full[TC_STAGES], s_empty[TC_STAGES];
    __shared__ __align__(8) uint64_t s_accf[2], s_acce[2], s_done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ long long s_issued;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t base = (saddr(tc_raw) + 1023u) & ~1023u;
    auto stA = [&](int s) { return base + (uint32_t)s * T16_STAGE_BYTES; };
    auto stBh = [&](int s) { return stA(s) + T16_A_BYTES; };
    auto stBl = [&](int s) { return stA(s) + T16_A_BYTES + T16_B_BYTES; };
    const int nkb = a.kblocks;
    const int64_t my_tiles = n_tiles > (int64_t)blockIdx.x ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto tile_m0 = [&](int64_t i) { return ((int64_t)blockIdx.x + i * gridDim.x) / n_ntiles * TC_M; };
    auto tile_n0 = [&](int64_t i) { return (int)(((int64_t)blockIdx.x + i * gridDim.x) % n_ntiles) * TC_N; };
    auto aborted = [&]() { return *(volatile int *)&s_abort != 0; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            bar_init(&s_full[s], 1);
            bar_init(&s_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init(&s_accf[b], 1);
            bar_init(&s_acce[b], 4);
        }
        bar_init(&s_done, 1);
        s_abort = 0;
        s_issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&s_tmem)),
                     "r"((uint32_t)(2 * TC_N))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        // ---------------- TMA producer: k-block g of the CTA's sequence goes to stage g % 2
        if (lane == 0) {
            long long g = 0;
            for (int64_t i = 0; i < my_tiles && !aborted(); ++i) {
                const int64_t m0 = tile_m0(i);
                const int n0 = tile_n0(i);
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = (int)(g & 1);
                    if (g >= TC_STAGES && !bar_wait(&s_empty[s], (uint32_t)(((g >> 1) - 1) & 1))) {
                        atomicExch(&s_abort, 1);
                        break;
                    }
                    if (aborted()) break;
                    bar_expect(&s_full[s], T16_A_BYTES + 2 * T16_B_BYTES);
                    tma_2d(stA(s), &mapA, &s_full[s], kb * T16_K, (int)m0);
                    tma_2d(stBh(s), &mapBh, &s_full[s], kb * T16_K, n0);
                    tma_2d(stBl(s), &mapBl, &s_full[s], kb * T16_K, n0);
                    s_issued = g + 1;
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer: tile i accumulates in TMEM columns (i % 2) * 256
        if (lane == 0) {
            const uint32_t idesc = idesc_f16<FP16>();
            long long g = 0;
            for (int64_t i = 0; i < my_tiles; ++i) {
                const int b = (int)(i & 1);
                if (i >= 2 && !bar_wait(&s_acce[b], (uint32_t)(((i >> 1) - 1) & 1))) {
                    atomicExch(&s_abort, 1);
                    break;
                }
                if (aborted()) break;
                fence_after();
                const uint32_t acc = tmem + (uint32_t)(b * TC_N);
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = (int)(g & 1);
                    if (!bar_wait(&s_full[s], (uint32_t)((g >> 1) & 1))) {
                        atomicExch(&s_abort, 1);
                        ok = false;
                        break;
                    }
                    if (aborted()) {
                        ok = false;
                        break;
                    }
                    fence_after();
#pragma unroll
                    for (int kk = 0; kk < T16_K / 16; ++kk) {  // 16 elements = 32 bytes per MMA
                        const uint32_t off = (uint32_t)kk * 32u;
                        const uint64_t dA = sw128_desc(stA(s) + off);
                        mma_f16(acc, dA, sw128_desc(stBh(s) + off), idesc, (kb | kk) != 0);
                        mma_f16(acc, dA, sw128_desc(stBl(s) + off), idesc, 1u);
                    }
                    mma_commit(&s_empty[s]);  // stage s free once these MMAs have read it
                }
                if (!ok) break;
                mma_commit(&s_accf[b]);  // tile i complete in buffer b
            }
            mma_commit(&s_done);  // every MMA this thread issued has completed
        }
    } else {
        // ---------------- epilogue: TMEM lane = tile row; warp w reads lanes 32 (w % 4) .. + 31
        const int quarter = warp & 3;
        for (int64_t i = 0; i < my_tiles; ++i) {
            const int b = (int)(i & 1);
            if (!bar_wait(&s_accf[b], (uint32_t)((i >> 1) & 1))) {
                atomicExch(&s_abort, 1);
                break;
            }
            if (aborted()) break;
            fence_after();
            const int64_t row = tile_m0(i) + quarter * 32 + lane;
            const int n0 = tile_n0(i);
            const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * TC_N);
            for (int cb = 0; cb < TC_N / 32; ++cb) {
                float v[32];
                tmem_ld32(taddr + (uint32_t)(cb * 32), v);
                if (row < a.M) {
                    float4 *out = reinterpret_cast<float4 *>(a.C + row * a.ldc + n0 + cb * 32);
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        out[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) bar_arrive(&s_acce[b]);  // buffer b free for tile i + 2
        }
    }

    // ---------------- teardown
    fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool done = bar_wait(&s_done, 0u);  // no MMA may still use TMEM when it is freed
        if (s_abort || !done) {
            for (long long g = s_issued > TC_STAGES ? s_issued - TC_STAGES : 0; g < s_issued; ++g)
                bar_wait(&s_full[g & 1], (uint32_t)((g >> 1) & 1));
            atomicExch(a.status, kDevStatusTimeout);
        }
    }
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * TC_N))
                     : "memory");
    }
}

bool encode_2d_u16(EncodeFn enc, CUtensorMap *map, const uint16_t *ptr, int64_t inner, int64_t outer, int box_inner,
                   int box_outer)
{
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)inner * 2};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, (void *)ptr, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// g4[M][ldc] = (g3 * d_alpha)[M][tc_k16] . T, 16-bit operands, fp32 accumulation.
int launch_hilbert_tc16(const Plan &p, int prec, const uint16_t *g3, float *g4, int64_t M, int ldc, cudaStream_t st,
                        bool *done)
{
    *done = false;
    EncodeFn enc = encoder();
    const int kind = prec == KATS_PREC_FP16 ? 1 : 0;
    if (!enc || M < 1 || ldc % TC_N != 0 || p.tc_n % TC_N != 0 || (reinterpret_cast<uintptr_t>(g3) % 16) != 0 ||
        (reinterpret_cast<uintptr_t>(g4) % 16) != 0)
        return KATS_OK;
    CUtensorMap mA, mBh, mBl;
    if (!encode_2d_u16(enc, &mA, g3, p.tc_k16, M, T16_K, TC_M) ||
        !encode_2d_u16(enc, &mBh, p.bt16_hi[kind], p.tc_k16, p.tc_n, T16_K, TC_N) ||
        !encode_2d_u16(enc, &mBl, p.bt16_lo[kind], p.tc_k16, p.tc_n, T16_K, TC_N))
        return KATS_OK;
    TcArgs a{g4, M, ldc, (int)(p.tc_k16 / T16_K), p.dev_status};
    auto kern = kind ? k_hilbert_tc16<true> : k_hilbert_tc16<false>;
    KATS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T16_SMEM));
    int dev = 0, sms = 0;
    KATS_CUDA(cudaGetDevice(&dev));
    KATS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int n_ntiles = (int)(p.tc_n / TC_N);
    const int64_t n_tiles = (int64_t)n_ntiles * ceil_div(M, TC_M);
    kern<<<(unsigned)std::min<int64_t>(sms, n_tiles), TC_THREADS, T16_SMEM, st>>>(mA, mBh, mBl, a, n_ntiles, n_tiles);
    count_launches(1);
    KATS_CUDA(cudaGetLastError());
    *done = true;
    return KATS_OK;
}

// C[M][ldc] = A[M][K] . B on the tensor cores, B as hi / lo [N][K] (3xTF32).  Returns KATS_OK
// with *done = false when the tensor-core path cannot run (no tensor-map encoder, misaligned
// buffers or sizes), leaving the caller to fall back.
int launch_hilbert_tc_op(const Plan &p, const float *A, int64_t M, int64_t K, const float *b_hi, const float *b_lo,
                         int64_t N, float *C, int ldc, cudaStream_t st, bool *done)
{
    *done = false;
    EncodeFn enc = encoder();
    if (!enc || M < 1 || K % TP_KB != 0 || N % TP_N != 0 || ldc % TP_N != 0 || ldc < N ||
        (reinterpret_cast<uintptr_t>(A) % 16) != 0 || (reinterpret_cast<uintptr_t>(C) % 16) != 0)
        return KATS_OK;
    CUtensorMap mA, mBh, mBl;
    const CUtensorMapSwizzle swz = TP_KB == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    if (!encode_2d(enc, &mA, A, K, M, TP_KB, TC_M, swz) || !encode_2d(enc, &mBh, b_hi, K, N, TP_KB, TP_N, swz) ||
        !encode_2d(enc, &mBl, b_lo, K, N, TP_KB, TP_N, swz))
        return KATS_OK;
    TcArgs a{C, M, ldc, (int)(K / TP_KB), p.dev_status};
    using SH = TpShape<TP_N, TP_STAGES, TP_KB>;
    auto kern = k_hilbert_tc<TP_N, TP_STAGES, TP_KB>;
    KATS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SH::SMEM));
    int dev = 0, sms = 0;
    KATS_CUDA(cudaGetDevice(&dev));
    KATS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int n_ntiles = (int)(N / TP_N);
    const int64_t n_tiles = (int64_t)n_ntiles * ceil_div(M, TC_M);
    kern<<<(unsigned)std::min<int64_t>(sms, n_tiles), TP_THREADS, SH::SMEM, st>>>(mA, mBh, mBl, a, n_ntiles, n_tiles);
    count_launches(1);
    KATS_CUDA(cudaGetLastError());
    *done = true;
    return KATS_OK;
}

// g4[M][ldc] = g3[M][tc_k] . T on the tensor cores (ldc a multiple of 256).
int launch_hilbert_tc(const Plan &p, const float *g3, float *g4, int64_t M, int ldc, cudaStream_t st, bool *done)
{
    return launch_hilbert_tc_op(p, g3, M, p.tc_k, p.bt_hi, p.bt_lo, p.tc_n, g4, ldc, st, done);
}

}  // namespace kats
