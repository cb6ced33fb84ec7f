// katsevich_smem_read_bandwidth: measured peak of the SM shared-memory read
// path, the path the backprojection's bilinear taps go through.
//
// Every thread of a 1024-thread CTA streams 16-byte loads from a 32 KB shared
// buffer: consecutive lanes read consecutive 16-byte words (no bank conflicts), so
// one warp instruction moves 512 B.  Four FP32 adds per load keep the values
// live and leave the issue slots mostly free, so the shared data path is the only
// limit.  The figure is the roofline denominator's measured counterpart (the
// derived one is 148 SMs x 128 B/clk x the SM clock).
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

}  // namespace

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
