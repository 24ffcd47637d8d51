// edt_static.cu -- ebof_edt_static: the exact EDT entry point for callers that
// cannot allocate device memory.  Its scratch (the column distances of the
// separable EDT) lives in a file-scope __device__ array instead of a buffer
// the caller passes in.
#include "ebof.h"
#include "ebof_internal.cuh"

#include <atomic>
#include <cmath>

namespace {

// Largest image, in pixels, the static scratch serves: 2^21 px (1920x1080
// fits).  The array costs 8 MiB on every device that loads the library, for
// the lifetime of the process.
constexpr size_t kStaticEdtMaxPixels = size_t(1) << 21;

__device__ __align__(256) int32_t g_edt_scratch[kStaticEdtMaxPixels];

constexpr int kMaxDev = 64;
// Device address of g_edt_scratch per device, looked up on first use.  In
// host code the name g_edt_scratch is only a host-side stand-in, so the
// address handed to kernels must come from cudaGetSymbolAddress with the
// device current.
std::atomic<int32_t *> g_scratch_addr[kMaxDev];

int32_t *scratch_for_current_device(int dev)
{
    int32_t *p = g_scratch_addr[dev].load();
    if (p) return p;
    void *addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_edt_scratch) != cudaSuccess || !addr) {
        cudaGetLastError();
        return nullptr;
    }
    ebof::init_front_attributes();  // opt-in shared memory of the row pass
    g_scratch_addr[dev].store((int32_t *)addr);
    return (int32_t *)addr;
}

}  // namespace

extern "C" ebof_status ebof_edt_static(const uint8_t *d_edge, int32_t width, int32_t height,
                                       int32_t *d_edt, float *d_surface, float alpha,
                                       void *cuda_stream)
{
    if (!d_edge || !d_edt || width < 1 || height < 1 || width > ebof::kMaxDim ||
        height > ebof::kMaxDim || !(std::isfinite(alpha) && alpha > 0.0f))
        return EBOF_ERR_INVALID_ARG;
    if ((size_t)width * (size_t)height > kStaticEdtMaxPixels) return EBOF_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return EBOF_ERR_CUDA;
    int32_t *scratch = scratch_for_current_device(dev);
    if (!scratch) return EBOF_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaGetLastError();
    const size_t plane = (size_t)width * height;
    ebof::launch_edt_columns(d_edge, width, plane, width, height, scratch, width, plane, 1, st);
    ebof::launch_edt_rows_surface(scratch, width, plane, width, height, alpha, d_edt, d_surface,
                                  nullptr, width, plane, 1, false, st);
    return cudaGetLastError() == cudaSuccess ? EBOF_OK : EBOF_ERR_CUDA;
}
