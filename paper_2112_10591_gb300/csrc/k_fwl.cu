// k_fwl.cu -- the Flow Warping Loss of §IV-C (ebof_fwl in include/ebof.h).
//
// Three launches on the caller's stream:
//   1. fwl_splat_kernel: one thread per event (grid-stride).  An event of
//      the window votes its polarity at its pixel into I_uncomp and, moved
//      back along the flow to t_begin, with bilinear weights into I_comp
//      (float atomics; votes outside the image are dropped).
//   2. fwl_partial_kernel: per-block sums of I and I^2 of both images, in
//      double, in a fixed order.
//   3. fwl_final_kernel: one block adds the partials in a fixed order and
//      writes FWL = var(I_comp) / var(I_uncomp) with the two variances.
// Traffic: 16 B per event read (x, y, t, p) plus 8 B of flow at its pixel,
// the two images written by atomics and read once (8 B per pixel each way).
#include "ebof.h"
#include "profiler.cuh"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

namespace {

constexpr int kFwlThreads = 256;
constexpr int kFwlPartialBlocks = 2 * 152;

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

__global__ void fwl_splat_kernel(const uint16_t *__restrict__ x, const uint16_t *__restrict__ y,
                                 const int64_t *__restrict__ t, const int8_t *__restrict__ p,
                                 int64_t n, int64_t t_begin, int64_t t_end,
                                 const float *__restrict__ flow, int W, int H,
                                 float *__restrict__ comp, float *__restrict__ uncomp)
{
    const size_t P = (size_t)W * H;
    const float inv_span = t_end > t_begin ? 1.0f / (float)(t_end - t_begin) : 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ti = t[i];
        if (ti < t_begin || ti >= t_end) continue;
        const int xi = x[i], yi = y[i];
        if (xi >= W || yi >= H) continue;
        const float s = p ? (float)p[i] : 1.0f;
        const size_t o = (size_t)yi * W + xi;
        atomicAdd(&uncomp[o], s);
        const float tau = (float)(ti - t_begin) * inv_span;
        const float xw = (float)xi - flow[o] * tau;
        const float yw = (float)yi - flow[P + o] * tau;
        const float fx = floorf(xw), fy = floorf(yw);
        const float ax = xw - fx, ay = yw - fy;
        const int X0 = (int)fx, Y0 = (int)fy;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const int X = X0 + dx, Y = Y0 + dy;
                if (X < 0 || Y < 0 || X >= W || Y >= H) continue;
                const float w = (dx ? ax : 1.0f - ax) * (dy ? ay : 1.0f - ay);
                atomicAdd(&comp[(size_t)Y * W + X], s * w);
            }
    }
}

// Block sum of four doubles in a fixed order; thread 0 gets the result.
__device__ void block_sum4(double v[4], double *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    if (lane == 0)
        for (int k = 0; k < 4; ++k) sh[warp * 4 + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < 4; ++k) {
            double a = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sh[w * 4 + k];
            v[k] = a;
        }
    }
}

__global__ void fwl_partial_kernel(const float *__restrict__ comp,
                                   const float *__restrict__ uncomp, size_t P,
                                   double *__restrict__ partial)
{
    __shared__ double sh[(kFwlThreads / 32) * 4];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
         i += (size_t)gridDim.x * blockDim.x) {
        const double c = comp[i], u = uncomp[i];
        v[0] += c;
        v[1] += c * c;
        v[2] += u;
        v[3] += u * u;
    }
    block_sum4(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) partial[blockIdx.x * 4 + k] = v[k];
}

__global__ void fwl_final_kernel(const double *__restrict__ partial, int nblocks, size_t P,
                                 double *__restrict__ out)
{
    __shared__ double sh[(kFwlThreads / 32) * 4];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < 4; ++k) v[k] += partial[b * 4 + k];
    block_sum4(v, sh);
    if (threadIdx.x == 0) {
        const double n = (double)P;
        const double mc = v[0] / n, mu = v[2] / n;
        const double var_c = v[1] / n - mc * mc;
        const double var_u = v[3] / n - mu * mu;
        out[0] = var_u > 0.0 ? var_c / var_u : 1.0;
        out[1] = var_c;
        out[2] = var_u;
    }
}

}  // namespace

extern "C" {

size_t ebof_fwl_scratch_bytes(int32_t width, int32_t height)
{
    if (width < 1 || height < 1) return 0;
    const size_t P = (size_t)width * height;
    return 2 * align256(sizeof(float) * P) + align256(sizeof(double) * 4 * kFwlPartialBlocks);
}

ebof_status ebof_fwl(const uint16_t *d_x, const uint16_t *d_y, const int64_t *d_t,
                     const int8_t *d_p, int64_t n_events, int64_t t_begin, int64_t t_end,
                     const float *d_flow, int32_t width, int32_t height, void *d_scratch,
                     double *d_out, void *cuda_stream)
{
    if (!d_flow || !d_scratch || !d_out || width < 1 || height < 1 || width > 16384 ||
        height > 16384 || n_events < 0 || t_end < t_begin ||
        (n_events > 0 && (!d_x || !d_y || !d_t)))
        return EBOF_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaGetLastError();
    const size_t P = (size_t)width * height;
    char *base = (char *)d_scratch;
    float *comp = (float *)base;
    float *uncomp = (float *)(base + align256(sizeof(float) * P));
    double *partial = (double *)(base + 2 * align256(sizeof(float) * P));
    cudaMemsetAsync(base, 0, 2 * align256(sizeof(float) * P), st);
    if (n_events > 0) {
        const int64_t want = (n_events + kFwlThreads - 1) / kFwlThreads;
        const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
        fwl_splat_kernel<<<blocks, kFwlThreads, 0, st>>>(d_x, d_y, d_t, d_p, n_events, t_begin,
                                                         t_end, d_flow, width, height, comp,
                                                         uncomp);
        ebof::g_launches.fetch_add(1);
    }
    fwl_partial_kernel<<<kFwlPartialBlocks, kFwlThreads, 0, st>>>(comp, uncomp, P, partial);
    fwl_final_kernel<<<1, kFwlThreads, 0, st>>>(partial, kFwlPartialBlocks, P, d_out);
    ebof::g_launches.fetch_add(2);
    return cudaGetLastError() == cudaSuccess ? EBOF_OK : EBOF_ERR_CUDA;
}

}  // extern "C"
