// katsevich_recon_noalloc: the full operator with its scratch in a fixed,
// library-owned device array instead of a caller workspace.
//
// For callers that cannot allocate device memory at call time, e.g. a
// reconstruction service whose device memory is all reserved up front by
// another allocator (a framework's caching pool) or a latency-critical loop
// where cudaMalloc / cudaFree would synchronise the device and stall other
// streams.  The paper has no counterpart; it is an interface convenience.
#include <mutex>

#include "common.cuh"

using namespace kats;

namespace {

constexpr size_t kScratchBytes = (size_t)KATS_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// One copy per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Device address of g_scratch on the current device (looked up once per device).
int scratch_address(int dev, void **out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return KATS_OK;
}

}  // namespace

extern "C" int katsevich_recon_noalloc(const kats_plan *plan, const float *sino, float *vol, int batch, void *stream)
{
    if (!plan || !sino || !vol) {
        set_error("null plan or buffer");
        return KATS_EINVAL;
    }
    if (batch < 1) {
        set_error("batch must be >= 1 (got %d)", batch);
        return KATS_EINVAL;
    }
    const Plan &p = *reinterpret_cast<const Plan *>(plan);
    int dev = -1;
    KATS_CUDA(cudaGetDevice(&dev));
    if (dev != p.device) {
        set_error("plan was built on device %d, current device is %d", p.device, dev);
        return KATS_EINVAL;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device index %d is above the supported %d", dev, kMaxDevices);
        return KATS_EINVAL;
    }
    const size_t gf = round256(sizeof(float) * (size_t)(p.n_fviews * p.g.n_rows * p.gf_cols));
    const size_t need = gf + filter_workspace_bytes(p);
    if (need > kScratchBytes) {
        set_error("katsevich_recon_noalloc: this geometry needs %zu bytes of scratch, the static array holds %zu; "
                  "use katsevich_recon with a caller workspace",
                  need, kScratchBytes);
        return KATS_ESPACE;
    }
    void *base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    float *gF = (float *)base;
    char *fws = (char *)base + gf;
    const size_t view = (size_t)(p.g.n_rows * p.g.n_cols);
    for (int b = 0; b < batch; ++b) {
        // every scratch element the kernels read is written earlier in the same call
        rc = launch_filter(p, sino + b * (size_t)p.g.n_views * view + p.first_view * view, gF, fws, need - gf, st);
        if (rc) return rc;
        rc = launch_backproject(p, gF, vol + b * (size_t)(p.g.nx * p.g.ny * p.g.nz), st);
        if (rc) return rc;
    }
    return KATS_OK;
}
