// dev_common.cuh -- small device helpers shared by the flow kernels.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace ebof {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// Arithmetic with a fixed rounding sequence.  The compiler fuses a product
// and a sum into one multiply-add wherever it sees fit, differently in
// different kernels; these intrinsics are never fused or split, so an
// expression written with them rounds the same way in every kernel that
// evaluates it.  The variational refinement's per-pixel arithmetic and the
// bilinear sample are written with them, so that every kernel form (tile,
// column walk, SOR region layouts) gives the same values bit for bit.
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// (1 - fy) ((1 - fx) a + fx b) + fy ((1 - fx) c + fx d), rounded in a fixed order.
__device__ __forceinline__ float lerp2(float a, float b, float c, float d, float fx, float fy)
{
    const float gx = fsub(1.0f, fx);
    const float top = ffma(fx, b, fmul(gx, a));
    const float bot = ffma(fx, d, fmul(gx, c));
    return ffma(fy, bot, fmul(fsub(1.0f, fy), top));
}

// Pyramid storage: FP32, or FP16 with every load widened to FP32 and every
// store rounded to nearest.
__device__ __forceinline__ float ldp(const float *p) { return *p; }
__device__ __forceinline__ float ldp(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ void stp(float *p, float v) { *p = v; }
__device__ __forceinline__ void stp(__half *p, float v) { *p = __float2half_rn(v); }

// Bilinear sample with the position clamped to [0, w-1] x [0, h-1].
template <typename T>
__device__ __forceinline__ float bilinear(const T *__restrict__ I, int w, int h, int pitch,
                                          float x, float y)
{
    x = fminf(fmaxf(x, 0.0f), (float)(w - 1));
    y = fminf(fmaxf(y, 0.0f), (float)(h - 1));
    const float xf = floorf(x), yf = floorf(y);
    const int x0 = (int)xf, y0 = (int)yf;
    const int x1 = min(x0 + 1, w - 1), y1 = min(y0 + 1, h - 1);
    const float fx = x - xf, fy = y - yf;
    const float a = ldp(&I[(size_t)y0 * pitch + x0]), b = ldp(&I[(size_t)y0 * pitch + x1]);
    const float c = ldp(&I[(size_t)y1 * pitch + x0]), d = ldp(&I[(size_t)y1 * pitch + x1]);
    return lerp2(a, b, c, d, fx, fy);
}

// The four samples around a clamped position and its fractional offsets.
struct BilTaps {
    float a, b, c, d, fx, fy;
};

// Taps of the sample below with 32-bit offsets (images of at most 2^31
// elements); split from the interpolation so that callers can issue the
// loads ahead of their use.
template <typename T>
__device__ __forceinline__ BilTaps bil_taps_i(const T *__restrict__ I, int w, int h, int pitch,
                                              float x, float y)
{
    x = fminf(fmaxf(x, 0.0f), (float)(w - 1));
    y = fminf(fmaxf(y, 0.0f), (float)(h - 1));
    const float xf = floorf(x), yf = floorf(y);
    const int x0 = (int)xf, y0 = (int)yf;
    const int x1 = min(x0 + 1, w - 1), y1 = min(y0 + 1, h - 1);
    const T *r0 = I + y0 * pitch, *r1 = I + y1 * pitch;
    BilTaps t;
    t.fx = x - xf;
    t.fy = y - yf;
    t.a = ldp(&r0[x0]);
    t.b = ldp(&r0[x1]);
    t.c = ldp(&r1[x0]);
    t.d = ldp(&r1[x1]);
    return t;
}

__device__ __forceinline__ float bil_lerp(const BilTaps &t)
{
    return lerp2(t.a, t.b, t.c, t.d, t.fx, t.fy);
}

// The bilinear sample with 32-bit offsets (the same arithmetic as
// bil_lerp(bil_taps_i(...)), written out whole for the search and
// densification kernels).
template <typename T>
__device__ __forceinline__ float bilinear_i(const T *__restrict__ I, int w, int h, int pitch,
                                            float x, float y)
{
    x = fminf(fmaxf(x, 0.0f), (float)(w - 1));
    y = fminf(fmaxf(y, 0.0f), (float)(h - 1));
    const float xf = floorf(x), yf = floorf(y);
    const int x0 = (int)xf, y0 = (int)yf;
    const int x1 = min(x0 + 1, w - 1), y1 = min(y0 + 1, h - 1);
    const float fx = x - xf, fy = y - yf;
    const T *r0 = I + y0 * pitch, *r1 = I + y1 * pitch;
    const float a = ldp(&r0[x0]), b = ldp(&r0[x1]);
    const float c = ldp(&r1[x0]), d = ldp(&r1[x1]);
    return lerp2(a, b, c, d, fx, fy);
}

// Robust penaliser derivative Psi'(s^2) = 1 / (2 sqrt(s^2 + eps^2)), eps = 1e-3.
__device__ __forceinline__ float psi_prime(float s2)
{
    return fmul(0.5f, rsqrtf(fadd(s2, 1e-6f)));
}

constexpr float kZeta2 = 0.01f;  // zeta^2 of the constraint normalisation

}  // namespace ebof
