// katsevich_smem_read_bandwidth: measured peak of the SM shared-memory read
// path, the path the backprojection's bilinear taps go through.
// katsevich_tex_bilinear_rate: measured rate of hardware-filtered (bilinear)
// texture fetches, the path a texture-based backprojection would take instead.
//
// Every thread of a 1024-thread CTA streams 16-byte loads from a 32 KB shared
// buffer: consecutive lanes read consecutive 16-byte words (no bank conflicts), so
// one warp instruction moves 512 B.  Four FP32 adds per load keep the values
// live and leave the issue slots mostly free, so the shared data path is the only
// limit.  The figure is the roofline denominator's measured counterpart (the
// derived one is 148 SMs x 128 B/clk x the SM clock).
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

using namespace kats;

namespace {

constexpr int kBufVec = 2048;  // float4 words: 32 KB
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(1024) k_smem_read(float *out, int iters)
{
    __shared__ float4 buf[kBufVec];
    for (int i = threadIdx.x; i < kBufVec; i += blockDim.x)
        buf[i] = make_float4((float)i, (float)(i + 1), (float)(i + 2), (float)(i + 3));
    __syncthreads();
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const int lane_word = threadIdx.x & (kBufVec - 1);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const float4 v = buf[(lane_word + u * 64 + it * 7) & (kBufVec - 1)];
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
    }
    // data-dependent store keeps the loads; out has one float per CTA
    if (threadIdx.x == 0) out[blockIdx.x] = acc.x + acc.y + acc.z + acc.w;
}

// Bilinear texture fetches, the hardware path a texture-based backprojection would use for
// its taps (one filtered sample per voxel-view update).  Coordinates advance by a fraction of
// a texel per fetch and stay inside the 256 x 256 texture (clamp addressing besides).
constexpr int kTexUnroll = 8;

__global__ void __launch_bounds__(256) k_tex_bilinear(cudaTextureObject_t tex, float *out, int iters)
{
    const float x0 = 8.0f + (float)(threadIdx.x & 31) * 3.3f, y0 = 8.0f + (float)(threadIdx.x >> 5) * 5.1f +
                                                                      (float)(blockIdx.x & 15) * 0.37f;
    float acc = 0.0f;
    for (int it = 0; it < iters; ++it) {
        const float x = x0 + (float)it * 0.0137f;
#pragma unroll
        for (int u = 0; u < kTexUnroll; ++u) acc += tex2D<float>(tex, x + 0.25f * u, y0 + 0.5f * u);
    }
    if (threadIdx.x == 0) out[blockIdx.x] = acc;  // data-dependent store keeps the fetches
}

}  // namespace

extern "C" int katsevich_tex_bilinear_rate(int half_texels, double *samples_per_second)
{
    if (!samples_per_second) {
        set_error("bad argument");
        return KATS_EINVAL;
    }
    int dev = 0, sms = 0;
    KATS_CUDA(cudaGetDevice(&dev));
    KATS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    constexpr int side = 256;
    const int blocks = 8 * sms, threads = 256, iters = 256;
    cudaArray_t arr = nullptr;
    cudaTextureObject_t tex = 0;
    float *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const cudaChannelFormatDesc fmt = half_texels ? cudaCreateChannelDescHalf() : cudaCreateChannelDesc<float>();
    cudaError_t e = cudaMallocArray(&arr, &fmt, side, side);
    if (e == cudaSuccess) {
        // texel values: a smooth ramp (any finite values do)
        std::vector<float> hf((size_t)side * side);
        std::vector<__half> hh((size_t)side * side);
        for (int i = 0; i < side * side; ++i) {
            hf[(size_t)i] = (float)(i % 97) * 0.01f;
            hh[(size_t)i] = __float2half(hf[(size_t)i]);
        }
        const size_t pitch = (size_t)side * (half_texels ? 2 : 4);
        e = cudaMemcpy2DToArray(arr, 0, 0, half_texels ? (const void *)hh.data() : (const void *)hf.data(), pitch,
                                pitch, side, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {
        cudaResourceDesc rd = {};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = arr;
        cudaTextureDesc td = {};
        td.addressMode[0] = td.addressMode[1] = cudaAddressModeClamp;
        td.filterMode = cudaFilterModeLinear;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        e = cudaCreateTextureObject(&tex, &rd, &td, nullptr);
    }
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * (size_t)blocks);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = 0.0;
    for (int rep = 0; e == cudaSuccess && rep < 4; ++rep) {  // the first round warms up
        k_tex_bilinear<<<blocks, threads, 0, st>>>(tex, out, iters);
        count_launches(1);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int k = 0; e == cudaSuccess && k < 3; ++k) {
            k_tex_bilinear<<<blocks, threads, 0, st>>>(tex, out, iters);
            count_launches(1);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms > 0.0f)
            best = std::max(best, 3.0 * blocks * threads * (double)iters * kTexUnroll / (ms * 1e-3));
    }
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    if (tex) cudaDestroyTextureObject(tex);
    if (arr) cudaFreeArray(arr);
    if (e != cudaSuccess) return cuda_fail(e, "texture bilinear probe");
    *samples_per_second = best;
    return KATS_OK;
}

extern "C" int katsevich_smem_read_bandwidth(double *bytes_per_second)
{
    if (!bytes_per_second) {
        set_error("bad argument");
        return KATS_EINVAL;
    }
    int dev = 0, sms = 0;
    KATS_CUDA(cudaGetDevice(&dev));
    KATS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = 4 * sms, threads = 1024, iters = 512;
    float *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(float) * (size_t)blocks);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.0f;
    for (int rep = 0; e == cudaSuccess && rep < 4; ++rep) {  // the first launch warms up
        k_smem_read<<<blocks, threads, 0, st>>>(out, iters);
        count_launches(1);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int k = 0; e == cudaSuccess && k < 3; ++k) {
            k_smem_read<<<blocks, threads, 0, st>>>(out, iters);
            count_launches(1);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms > 0.0f) {
            const double bytes = 3.0 * blocks * threads * (double)iters * kUnroll * 16.0;
            best = std::max(best, (float)(bytes / (ms * 1e-3)));
        }
    }
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    if (e != cudaSuccess) return cuda_fail(e, "shared-memory bandwidth probe");
    *bytes_per_second = best;
    return KATS_OK;
}
