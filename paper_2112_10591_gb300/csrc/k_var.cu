// k_var.cu -- variational refinement (reading F6), one fused kernel per
// fixed-point iteration.
//
// One block owns a 64x64 region of the level image and refines the flow of
// its (64 - 2R)^2 interior, R = 2 * sweeps - 1.  The block
//   1. stages U and the warped image I1(x + U) for the region + 2 px,
//   2. builds derivatives of the warped image and smoothness weights for the
//      region + 1 px in shared memory,
//   3. builds every region pixel's 2x2 linear system in registers (data and
//      gradient-constancy terms normalised, weights lagged at dU = 0),
//   4. runs the red-black SOR sweeps on (du, dv) entirely in registers: a
//      thread owns a 2-column x 4-row strip, so one of the two horizontal
//      neighbours is its own and the other is a lane shuffle away, and the
//      rows at strip ends are exchanged through shared memory once per half
//      sweep,
//   5. writes U + dU for its interior pixels.
// The region border keeps du = 0.  After h half sweeps only pixels within
// h - 1 px of that border differ from the whole-image red-black iteration,
// and those lie in the discarded halo, so the interior is exactly the
// whole-image iteration (up to floating-point rounding).
#include "dev_common.cuh"
#include "ebof_internal.cuh"
#include "profiler.cuh"

namespace ebof {

namespace {

constexpr int kVR = 64;                  // region side
constexpr int kVS = 4;                   // rows per thread strip
constexpr int kVWarps = kVR / kVS;       // warps per block (stacked strips)
constexpr int kVThreads = 32 * kVWarps;  // 512
constexpr int kVE = kVR + 4;             // staging window: region + 2 px each side
constexpr int kVD = kVR + 2;             // derivative window: region + 1 px each side
constexpr size_t kVSmemFloats =
    2 * kVE * kVE + kVE * kVE + 3 * kVD * kVD + 2 * 2 * kVWarps * 2 * 64;
constexpr unsigned kFull = 0xffffffffu;

// One red-black half sweep of colour C on a thread's 2-column x kVS-row
// strip; P is the parity of (x + y) at the strip's first pixel.  Pixel
// (row r, column q) has colour (P + r + q) & 1.  The strip's first and last
// rows are read by the warps above and below from xch (double-buffered by
// half sweep, so one barrier per half sweep suffices).
template <int P, int C>
__device__ __forceinline__ void sor_half(float (&du)[kVS][2], float (&dv)[kVS][2],
                                         const float (&i11)[kVS][2], const float (&i22)[kVS][2],
                                         const float (&a12)[kVS][2], const float (&b1)[kVS][2],
                                         const float (&b2)[kVS][2], const float (&wl)[kVS][2],
                                         const float (&wr)[kVS][2], const float (&wu)[kVS][2],
                                         const float (&wd)[kVS][2], const float *xtop,
                                         const float *xbot, int lane, int wp, float omega)
{
    const float om1 = 1.0f - omega;
#pragma unroll
    for (int r = 0; r < kVS; ++r) {
        const int q = (C + P + r) & 1;  // compile-time after unrolling
        float lu, lv, ru, rv;
        if (q == 0) {
            const float nu = __shfl_up_sync(kFull, du[r][1], 1);
            const float nv = __shfl_up_sync(kFull, dv[r][1], 1);
            lu = lane > 0 ? nu : 0.0f;
            lv = lane > 0 ? nv : 0.0f;
            ru = du[r][1];
            rv = dv[r][1];
        } else {
            const float nu = __shfl_down_sync(kFull, du[r][0], 1);
            const float nv = __shfl_down_sync(kFull, dv[r][0], 1);
            ru = lane < 31 ? nu : 0.0f;
            rv = lane < 31 ? nv : 0.0f;
            lu = du[r][0];
            lv = dv[r][0];
        }
        const int col = 2 * lane + q;
        float uu, uv, dnu, dnv;
        if (r > 0) {
            uu = du[r - 1][q];
            uv = dv[r - 1][q];
        } else {
            uu = wp > 0 ? xbot[((wp - 1) * 2 + 0) * 64 + col] : 0.0f;
            uv = wp > 0 ? xbot[((wp - 1) * 2 + 1) * 64 + col] : 0.0f;
        }
        if (r < kVS - 1) {
            dnu = du[r + 1][q];
            dnv = dv[r + 1][q];
        } else {
            dnu = wp < kVWarps - 1 ? xtop[((wp + 1) * 2 + 0) * 64 + col] : 0.0f;
            dnv = wp < kVWarps - 1 ? xtop[((wp + 1) * 2 + 1) * 64 + col] : 0.0f;
        }
        const float nu = om1 * du[r][q] +
                         omega * (b1[r][q] + wl[r][q] * lu + wr[r][q] * ru + wu[r][q] * uu +
                                  wd[r][q] * dnu - a12[r][q] * dv[r][q]) * i11[r][q];
        const float nv = om1 * dv[r][q] +
                         omega * (b2[r][q] + wl[r][q] * lv + wr[r][q] * rv + wu[r][q] * uv +
                                  wd[r][q] * dnv - a12[r][q] * nu) * i22[r][q];
        du[r][q] = nu;
        dv[r][q] = nv;
    }
}

template <int P>
__device__ __forceinline__ void sor_sweeps(float (&du)[kVS][2], float (&dv)[kVS][2],
                                           const float (&i11)[kVS][2], const float (&i22)[kVS][2],
                                           const float (&a12)[kVS][2], const float (&b1)[kVS][2],
                                           const float (&b2)[kVS][2], const float (&wl)[kVS][2],
                                           const float (&wr)[kVS][2], const float (&wu)[kVS][2],
                                           const float (&wd)[kVS][2], float *xch, int lane, int wp,
                                           int n_half, float omega)
{
    for (int hs = 0; hs < n_half; ++hs) {
        // exchange buffer of this half sweep: [top|bottom][warp][du|dv][64]
        float *xb = xch + (hs & 1) * (2 * kVWarps * 2 * 64);
        float *xtop = xb, *xbot = xb + kVWarps * 2 * 64;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            xtop[(wp * 2 + 0) * 64 + 2 * lane + q] = du[0][q];
            xtop[(wp * 2 + 1) * 64 + 2 * lane + q] = dv[0][q];
            xbot[(wp * 2 + 0) * 64 + 2 * lane + q] = du[kVS - 1][q];
            xbot[(wp * 2 + 1) * 64 + 2 * lane + q] = dv[kVS - 1][q];
        }
        __syncthreads();
        if ((hs & 1) == 0)
            sor_half<P, 0>(du, dv, i11, i22, a12, b1, b2, wl, wr, wu, wd, xtop, xbot, lane, wp, omega);
        else
            sor_half<P, 1>(du, dv, i11, i22, a12, b1, b2, wl, wr, wu, wd, xtop, xbot, lane, wp, omega);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kVThreads, 1)
var_fused_kernel(const float *__restrict__ I0b, const float *__restrict__ I0xb,
                 const float *__restrict__ I0yb, const float *__restrict__ I1b, int w, int h,
                 int pitch, size_t pfs, const float *__restrict__ Uinb, float *__restrict__ Uoutb,
                 size_t ufs, size_t plane, int R, int tile, int n_half, float delta, float gamma,
                 float alpha_s, float omega)
{
    extern __shared__ float sm[];
    float *sU = sm;
    float *sV = sU + kVE * kVE;
    float *sW = sV + kVE * kVE;
    float *sIx = sW + kVE * kVE;
    float *sIy = sIx + kVD * kVD;
    float *sAs = sIy + kVD * kVD;
    float *xch = sAs + kVD * kVD;  // strip-end exchange, two buffers

    const int f = blockIdx.z;
    const int rx0 = blockIdx.x * tile - R, ry0 = blockIdx.y * tile - R;
    const int ex0 = rx0 - 2, ey0 = ry0 - 2;
    const int dx0 = rx0 - 1, dy0 = ry0 - 1;
    const size_t po = (size_t)f * pfs;
    const float *I0 = I0b + po, *I0x = I0xb + po, *I0y = I0yb + po, *I1 = I1b + po;
    const float *Uin = Uinb + (size_t)f * ufs;
    float *Uout = Uoutb + (size_t)f * ufs;

    // 1. flow on the staging window, then the warped image I1(x + U); the
    // loops are unrolled so that each thread keeps all its loads in flight
    const int t = threadIdx.x;
    constexpr int kIt = (kVE * kVE + kVThreads - 1) / kVThreads;
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
        const int i = t + it * kVThreads;
        if (i >= kVE * kVE) break;
        const int gx = ex0 + i % kVE, gy = ey0 + i / kVE;
        float u = 0.0f, v = 0.0f;
        if (gx >= 0 && gx < w && gy >= 0 && gy < h) {
            const size_t p = (size_t)gy * pitch + gx;
            u = Uin[p];
            v = Uin[plane + p];
        }
        sU[i] = u;
        sV[i] = v;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
        const int i = t + it * kVThreads;
        if (i >= kVE * kVE) break;
        const int gx = ex0 + i % kVE, gy = ey0 + i / kVE;
        float wv = 0.0f;
        if (gx >= 0 && gx < w && gy >= 0 && gy < h)
            wv = bilinear(I1, w, h, pitch, (float)gx + sU[i], (float)gy + sV[i]);
        sW[i] = wv;
    }
    __syncthreads();

    // 2. derivatives of the warped image and smoothness weights, region + 1
    constexpr int kDIt = (kVD * kVD + kVThreads - 1) / kVThreads;
#pragma unroll
    for (int it = 0; it < kDIt; ++it) {
        const int i = t + it * kVThreads;
        if (i >= kVD * kVD) break;
        const int gx = dx0 + i % kVD, gy = dy0 + i / kVD;
        float ix = 0.0f, iy = 0.0f, as = 0.0f;
        if (gx >= 0 && gx < w && gy >= 0 && gy < h) {
            const int xp = min(gx + 1, w - 1), xm = max(gx - 1, 0);
            const int yp = min(gy + 1, h - 1), ym = max(gy - 1, 0);
            const int row = (gy - ey0) * kVE;
            ix = 0.5f * (sW[row + xp - ex0] - sW[row + xm - ex0]);
            iy = 0.5f * (sW[(yp - ey0) * kVE + gx - ex0] - sW[(ym - ey0) * kVE + gx - ex0]);
            const int e = row + gx - ex0;
            const float u = sU[e], v = sV[e];
            const float ux = gx + 1 < w ? sU[e + 1] - u : 0.0f;
            const float uy = gy + 1 < h ? sU[e + kVE] - u : 0.0f;
            const float vx = gx + 1 < w ? sV[e + 1] - v : 0.0f;
            const float vy = gy + 1 < h ? sV[e + kVE] - v : 0.0f;
            as = alpha_s * psi_prime(ux * ux + uy * uy + vx * vx + vy * vy);
        }
        sIx[i] = ix;
        sIy[i] = iy;
        sAs[i] = as;
    }
    __syncthreads();

    // 3. linear systems of this thread's 8 pixels
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    float i11[kVS][2], i22[kVS][2], a12[kVS][2], b1[kVS][2], b2[kVS][2];
    float wl[kVS][2], wr[kVS][2], wu[kVS][2], wd[kVS][2];
    float du[kVS][2], dv[kVS][2];
#pragma unroll
    for (int r = 0; r < kVS; ++r)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            du[r][q] = 0.0f; dv[r][q] = 0.0f;
            i11[r][q] = 0.0f; i22[r][q] = 0.0f; a12[r][q] = 0.0f;
            b1[r][q] = 0.0f; b2[r][q] = 0.0f;
            wl[r][q] = 0.0f; wr[r][q] = 0.0f; wu[r][q] = 0.0f; wd[r][q] = 0.0f;
            const int gx = rx0 + 2 * lane + q, gy = ry0 + wp * kVS + r;
            if (gx < 0 || gx >= w || gy < 0 || gy >= h) continue;
            const int xp = min(gx + 1, w - 1), xm = max(gx - 1, 0);
            const int yp = min(gy + 1, h - 1), ym = max(gy - 1, 0);
            const int d = (gy - dy0) * kVD + (gx - dx0);
            const int drow = (gy - dy0) * kVD;
            const float Ix = sIx[d], Iy = sIy[d];
            const float Ixx = 0.5f * (sIx[drow + xp - dx0] - sIx[drow + xm - dx0]);
            const float Ixy = 0.5f * (sIx[(yp - dy0) * kVD + gx - dx0] - sIx[(ym - dy0) * kVD + gx - dx0]);
            const float Iyy = 0.5f * (sIy[(yp - dy0) * kVD + gx - dx0] - sIy[(ym - dy0) * kVD + gx - dx0]);
            const size_t p = (size_t)gy * pitch + gx;
            const int e = (gy - ey0) * kVE + (gx - ex0);
            const float Iz = sW[e] - I0[p];
            const float Ixz = Ix - I0x[p], Iyz = Iy - I0y[p];
            const float nd = __fdividef(1.0f, Ix * Ix + Iy * Iy + kZeta2);
            const float ng = __fdividef(1.0f, Ixx * Ixx + 2.0f * Ixy * Ixy + Iyy * Iyy + kZeta2);
            float ad = delta * nd * psi_prime(nd * Iz * Iz);
            float ag = gamma * ng * psi_prime(ng * (Ixz * Ixz + Iyz * Iyz));
            const float u = sU[e], v = sV[e];
            const float wx = (float)gx + u, wy = (float)gy + v;
            if (wx < 0.0f || wx > (float)(w - 1) || wy < 0.0f || wy > (float)(h - 1)) {
                ad = 0.0f;
                ag = 0.0f;
            }
            const float asp = sAs[d];
            const float cl = gx > 0 ? 0.5f * (asp + sAs[d - 1]) : 0.0f;
            const float cr = gx + 1 < w ? 0.5f * (asp + sAs[d + 1]) : 0.0f;
            const float cu = gy > 0 ? 0.5f * (asp + sAs[d - kVD]) : 0.0f;
            const float cd = gy + 1 < h ? 0.5f * (asp + sAs[d + kVD]) : 0.0f;
            const float sw = cl + cr + cu + cd;
            const float su0 = cl * (sU[e - 1] - u) + cr * (sU[e + 1] - u) +
                              cu * (sU[e - kVE] - u) + cd * (sU[e + kVE] - u);
            const float sv0 = cl * (sV[e - 1] - v) + cr * (sV[e + 1] - v) +
                              cu * (sV[e - kVE] - v) + cd * (sV[e + kVE] - v);
            i11[r][q] = __fdividef(1.0f, ad * Ix * Ix + ag * (Ixx * Ixx + Ixy * Ixy) + sw);
            i22[r][q] = __fdividef(1.0f, ad * Iy * Iy + ag * (Ixy * Ixy + Iyy * Iyy) + sw);
            a12[r][q] = ad * Ix * Iy + ag * (Ixx * Ixy + Ixy * Iyy);
            b1[r][q] = su0 - ad * Ix * Iz - ag * (Ixx * Ixz + Ixy * Iyz);
            b2[r][q] = sv0 - ad * Iy * Iz - ag * (Ixy * Ixz + Iyy * Iyz);
            wl[r][q] = cl; wr[r][q] = cr; wu[r][q] = cu; wd[r][q] = cd;
        }

    // 4. red-black SOR; red = (x + y) even, first.  kVS is even, so the
    // parity of (x + y) at a strip's first pixel is the same for every warp
    // of the block, and the column of a given colour in a given row is a
    // compile-time constant once that parity is fixed.
    const int par = (rx0 + ry0) & 1;
    if (par == 0)
        sor_sweeps<0>(du, dv, i11, i22, a12, b1, b2, wl, wr, wu, wd, xch, lane, wp, n_half, omega);
    else
        sor_sweeps<1>(du, dv, i11, i22, a12, b1, b2, wl, wr, wu, wd, xch, lane, wp, n_half, omega);

    // 5. U + dU on the interior
#pragma unroll
    for (int r = 0; r < kVS; ++r)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int lx = 2 * lane + q, ly = wp * kVS + r;
            const int gx = rx0 + lx, gy = ry0 + ly;
            if (lx < R || lx >= R + tile || ly < R || ly >= R + tile || gx >= w || gy >= h)
                continue;
            const int e = (gy - ey0) * kVE + (gx - ex0);
            const size_t p = (size_t)gy * pitch + gx;
            Uout[p] = sU[e] + du[r][q];
            Uout[plane + p] = sV[e] + dv[r][q];
        }
}

}  // namespace

bool var_fused_supported(int var_sor)
{
    const int R = var_sor > 0 ? 2 * var_sor - 1 : 0;
    return kVR - 2 * R >= 16;
}

void init_var_attributes()
{
    cudaFuncSetAttribute(var_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(kVSmemFloats * sizeof(float)));
}

float *launch_variational_fused(const float *I0, const float *I0x, const float *I0y,
                                const float *I1, const Level &lv, size_t pyr_frame_stride,
                                float *U, float *Utmp, size_t u_frame_stride, int frames,
                                const FlowParams &fp, cudaStream_t st)
{
    const int n_half = 2 * fp.var_sor;
    const int R = n_half > 0 ? n_half - 1 : 0;
    const int tile = kVR - 2 * R;
    dim3 grd((lv.w + tile - 1) / tile, (lv.h + tile - 1) / tile, frames);
    float *a = U, *b = Utmp;
    for (int k = 0; k < fp.var_outer; ++k) {
        StageScope sc(kStVarSor, 1, st);
        var_fused_kernel<<<grd, kVThreads, kVSmemFloats * sizeof(float), st>>>(
            I0, I0x, I0y, I1, lv.w, lv.h, lv.pitch, pyr_frame_stride, a, b, u_frame_stride,
            lv.plane, R, tile, n_half, fp.delta, fp.gamma, fp.alpha_s, fp.omega);
        float *t = a;
        a = b;
        b = t;
    }
    return a;
}

}  // namespace ebof
