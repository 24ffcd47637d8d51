// k_var.cu -- variational refinement (reading F6): two kernels per
// fixed-point iteration.
//
// var_coeff_kernel, one thread per pixel: stages U and the warped image
// I1(x + U) for a 32x12 tile plus 2 px in shared memory, builds derivatives
// of the warped image and the smoothness weights, and writes every pixel's
// 2x2 linear system (data and gradient-constancy terms normalised, weights
// lagged at dU = 0): omega/a11, omega/a22 (the SOR relaxation factor folded
// into the inverted diagonal), a12, b1, b2 and the left and upper edge
// weights, as seven planes (the right and lower weights are the neighbours'
// left and upper ones).  Only the staging halo is shared between tiles.  On
// levels from 1024 px wide the same systems come from var_coeff_cw_kernel,
// a column walk with the rows in registers.
//
// var_sor_kernel: one block owns a 64x64 region and refines the flow of its
// (64 - 2R)^2 interior, R = 2 * sweeps - 1.  It loads the region's linear
// systems into registers and runs the red-black SOR sweeps there: a thread
// owns a 2-column x 4-row strip, so one horizontal neighbour is its own and
// the other is a lane shuffle away, and the rows at strip ends are exchanged
// through shared memory once per half sweep.  (A 2 x 2 strip with 1024
// threads, twice the resident warps, measured no faster.)  The region border keeps
// du = 0; after h half sweeps only pixels within h - 1 px of that border
// differ from the whole-image red-black iteration, and those lie in the
// discarded halo, so the interior is exactly the whole-image iteration (up to
// floating-point rounding).  It writes U + dU for its interior.
//
// var_sor_tma_kernel: the same sweeps in a persistent grid (one block per
// SM) that walks over the regions, for grids of at least four regions per
// SM.  One thread loads each region's coefficient planes into shared memory
// with a single TMA tensor copy (cp.async.bulk.tensor, completion on an
// mbarrier); once every thread has
// moved its values into registers, the copy of the block's next region is
// issued and runs during the sweeps.  The box starts at the region's first
// column rounded down to a multiple of 4 (the 16-byte rule of tensor
// copies) and is 4 columns wider; elements outside the level are filled
// with zero, as the direct loads do, so both kernels give the same result.
#include "dev_common.cuh"
#include "ebof_internal.cuh"
#include "profiler.cuh"
#include "seg.cuh"

#include <cooperative_groups.h>
#include <mutex>

namespace ebof {

namespace {

constexpr int kVR = 64;                  // region side
constexpr int kVS = 4;                   // rows per thread strip
constexpr int kVWarps = kVR / kVS;       // warps per block (stacked strips)
constexpr int kVThreads = 32 * kVWarps;  // 512
constexpr size_t kVSmemFloats = 2 * 2 * kVWarps * 2 * 64;  // strip-end exchange
constexpr size_t kVSmemFloats2 = 2 * 2 * 32 * 2 * 64;       // the same for 32 warps
// Coefficient planes of a pixel's system: omega/a11, omega/a22, a12, b1, b2
// and the left and upper edge weights.  The right and lower weights of a pixel are
// the left and upper ones of its neighbours (each the mean of the same two
// smoothness weights, so equal bit for bit) and are not stored.
enum { kCI11 = 0, kCI22, kCA12, kCB1, kCB2, kCWL, kCWU, kCPlanes };

constexpr int kTmaBoxW = kVR + 4;  // region columns + the rounding of the box start
constexpr size_t kTmaCoefFloats = (size_t)kCPlanes * kVR * kTmaBoxW;
constexpr size_t kTmaSmemBytes = (kTmaCoefFloats + kVSmemFloats) * sizeof(float);
constexpr int kMaxDevs = 64;
int g_num_sms[kMaxDevs];
// coefficient tile: 384 threads at 40 registers, four blocks per SM, so a
// 640 x 360 level (600 tiles) takes one wave where 32 x 16 tiles took two
constexpr int kAX = 32, kAY = 12;
constexpr int kAEX = kAX + 4, kAEY = kAY + 4;  // staging window: tile + 2 px
constexpr int kADX = kAX + 2, kADY = kAY + 2;  // derivative window: tile + 1 px
constexpr unsigned kFull = 0xffffffffu;

// Loads of data that the same launch may have written on another SM earlier
// (COH: through L2 with ld.global.cg, never from a possibly stale L1 or the
// read-only path); plain loads otherwise.  The values are the same.
template <bool COH>
__device__ __forceinline__ float ldf(const float *p)
{
    if constexpr (COH)
        return __ldcg(p);
    else
        return *p;
}
template <bool COH>
__device__ __forceinline__ float2 ldf2(const float *p)
{
    if constexpr (COH)
        return __ldcg(reinterpret_cast<const float2 *>(p));
    else
        return *reinterpret_cast<const float2 *>(p);
}


// One red-black half sweep of colour C on a thread's 2-column x VS-row
// strip; P is the parity of (x + y) at the strip's first pixel.  Pixel
// (row r, column q) has colour (P + r + q) & 1.  The strip's first and last
// rows are read by the warps above and below from xch (double-buffered by
// half sweep, so one barrier per half sweep suffices).  WARPS strips are
// stacked in a block.
template <int VS, int WARPS, int P, int C>
__device__ __forceinline__ void sor_half(float (&du)[VS][2], float (&dv)[VS][2],
                                         const float (&i11)[VS][2], const float (&i22)[VS][2],
                                         const float (&a12)[VS][2], const float (&b1)[VS][2],
                                         const float (&b2)[VS][2], const float (&wl)[VS][2],
                                         const float (&wr)[VS][2], const float (&wu)[VS][2],
                                         const float (&wd)[VS][2], const float *xtop,
                                         const float *xbot, int lane, int wp, float omega)
{
    const float om1 = 1.0f - omega;
#pragma unroll
    for (int r = 0; r < VS; ++r) {
        const int q = (C + P + r) & 1;  // compile-time after unrolling
        // lane 0's left and lane 31's right neighbours lie outside the
        // region: the shuffles return the lane's own (finite) values there,
        // and the edge weights wl / wr of those pixels are 0
        float lu, lv, ru, rv;
        if (q == 0) {
            lu = __shfl_up_sync(kFull, du[r][1], 1);
            lv = __shfl_up_sync(kFull, dv[r][1], 1);
            ru = du[r][1];
            rv = dv[r][1];
        } else {
            ru = __shfl_down_sync(kFull, du[r][0], 1);
            rv = __shfl_down_sync(kFull, dv[r][0], 1);
            lu = du[r][0];
            lv = dv[r][0];
        }
        const int col = q * 32 + lane;  // the exchange rows hold the q = 0 column first
        float uu, uv, dnu, dnv;
        if (r > 0) {
            uu = du[r - 1][q];
            uv = dv[r - 1][q];
        } else {
            uu = wp > 0 ? xbot[((wp - 1) * 2 + 0) * 64 + col] : 0.0f;
            uv = wp > 0 ? xbot[((wp - 1) * 2 + 1) * 64 + col] : 0.0f;
        }
        if (r < VS - 1) {
            dnu = du[r + 1][q];
            dnv = dv[r + 1][q];
        } else {
            dnu = wp < WARPS - 1 ? xtop[((wp + 1) * 2 + 0) * 64 + col] : 0.0f;
            dnv = wp < WARPS - 1 ? xtop[((wp + 1) * 2 + 1) * 64 + col] : 0.0f;
        }
        // i11 = omega / a11, i22 = omega / a22; fixed rounding order (every
        // SOR layout gives the same values)
        float tu = ffma(wl[r][q], lu, b1[r][q]);
        tu = ffma(wr[r][q], ru, tu);
        tu = ffma(wu[r][q], uu, tu);
        tu = ffma(wd[r][q], dnu, tu);
        tu = ffma(-a12[r][q], dv[r][q], tu);
        const float nu = ffma(tu, i11[r][q], fmul(om1, du[r][q]));
        float tv = ffma(wl[r][q], lv, b2[r][q]);
        tv = ffma(wr[r][q], rv, tv);
        tv = ffma(wu[r][q], uv, tv);
        tv = ffma(wd[r][q], dnv, tv);
        tv = ffma(-a12[r][q], nu, tv);
        const float nv = ffma(tv, i22[r][q], fmul(om1, dv[r][q]));
        du[r][q] = nu;
        dv[r][q] = nv;
    }
}

// n_half half sweeps, red first.  pw = parity of (x + y) at this warp's
// strip start (block-uniform when VS is even, alternating per warp when VS
// is odd); the branch on it is warp-uniform and every barrier is outside it.
template <int VS, int WARPS>
__device__ __forceinline__ void sor_sweeps(float (&du)[VS][2], float (&dv)[VS][2],
                                           const float (&i11)[VS][2], const float (&i22)[VS][2],
                                           const float (&a12)[VS][2], const float (&b1)[VS][2],
                                           const float (&b2)[VS][2], const float (&wl)[VS][2],
                                           const float (&wr)[VS][2], const float (&wu)[VS][2],
                                           const float (&wd)[VS][2], float *xch, int lane, int wp,
                                           int pw, int n_half, float omega)
{
    for (int hs = 0; hs < n_half; ++hs) {
        // exchange buffer of this half sweep: [top|bottom][warp][du|dv][q][lane]
        // (a lane's two columns 32 floats apart: conflict-free accesses)
        float *xb = xch + (hs & 1) * (2 * WARPS * 2 * 64);
        float *xtop = xb, *xbot = xb + WARPS * 2 * 64;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            xtop[(wp * 2 + 0) * 64 + q * 32 + lane] = du[0][q];
            xtop[(wp * 2 + 1) * 64 + q * 32 + lane] = dv[0][q];
            xbot[(wp * 2 + 0) * 64 + q * 32 + lane] = du[VS - 1][q];
            xbot[(wp * 2 + 1) * 64 + q * 32 + lane] = dv[VS - 1][q];
        }
        __syncthreads();
        if (pw == 0) {
            if ((hs & 1) == 0)
                sor_half<VS, WARPS, 0, 0>(du, dv, i11, i22, a12, b1, b2, wl, wr, wu, wd, xtop,
                                          xbot, lane, wp, omega);
            else
                sor_half<VS, WARPS, 0, 1>(du, dv, i11, i22, a12, b1, b2, wl, wr, wu, wd, xtop,
                                          xbot, lane, wp, omega);
        } else {
            if ((hs & 1) == 0)
                sor_half<VS, WARPS, 1, 0>(du, dv, i11, i22, a12, b1, b2, wl, wr, wu, wd, xtop,
                                          xbot, lane, wp, omega);
            else
                sor_half<VS, WARPS, 1, 1>(du, dv, i11, i22, a12, b1, b2, wl, wr, wu, wd, xtop,
                                          xbot, lane, wp, omega);
        }
    }
    __syncthreads();
}

// Smoothness weight alpha_s Psi'(|grad u|^2 + |grad v|^2) with forward
// differences (ur, ud: U to the right and below; hx, hy: those neighbours are
// in the level, else the difference is 0).
__device__ __forceinline__ float smooth_weight(float u, float ur, float ud, float v, float vr,
                                               float vd, bool hx, bool hy, float alpha_s)
{
    const float ux = hx ? fsub(ur, u) : 0.0f;
    const float uy = hy ? fsub(ud, u) : 0.0f;
    const float vx = hx ? fsub(vr, v) : 0.0f;
    const float vy = hy ? fsub(vd, v) : 0.0f;
    return fmul(alpha_s, psi_prime(ffma(vy, vy, ffma(vx, vx, ffma(uy, uy, fmul(ux, ux))))));
}

__device__ __forceinline__ float cdiff(float hi, float lo) { return fmul(0.5f, fsub(hi, lo)); }

// Derivatives of the warped image and the smoothness weight at a pixel of a
// staging window (row stride ES; (e) the pixel, at image position gx, gy).
// IN: the pixel and its neighbours lie inside the level, so the clamps and
// border tests are known to pass and are left out (same values).
template <bool IN>
__device__ __forceinline__ void stage_derivs(const float *sW, const float *sU, const float *sV,
                                             int ES, int e, int ex0, int ey0, int gx, int gy,
                                             int w, int h, float alpha_s, float &ix, float &iy,
                                             float &as)
{
    const int xp = (IN ? gx + 1 : min(gx + 1, w - 1)) - ex0;
    const int xm = (IN ? gx - 1 : max(gx - 1, 0)) - ex0;
    const int yp = (IN ? gy + 1 : min(gy + 1, h - 1)) - ey0;
    const int ym = (IN ? gy - 1 : max(gy - 1, 0)) - ey0;
    const int ex = gx - ex0, ey = gy - ey0;
    ix = cdiff(sW[ey * ES + xp], sW[ey * ES + xm]);
    iy = cdiff(sW[yp * ES + ex], sW[ym * ES + ex]);
    as = smooth_weight(sU[e], sU[e + 1], sU[e + ES], sV[e], sV[e + 1], sV[e + ES],
                       IN || gx + 1 < w, IN || gy + 1 < h, alpha_s);
}

struct PixelSystem {
    float i11, i22, a12, b1, b2, cl, cr, cu, cd;
};

// The 2x2 system of pixel (gx, gy) from its neighbourhood.  ix, iy: the
// warped image's derivatives at the pixel; ixl, ixr: Ix at the clamped left
// and right neighbours, ixu, ixd and iyu, iyd: Ix and Iy at the clamped upper
// and lower ones; iw: the warped sample; as*: smoothness weights at the pixel
// and its four neighbours, used only where that neighbour is in the level
// (bl, br, bu, bd); u*, v*: the flow at the pixel and its four neighbours (0
// outside the level); i0, i0x, i0y: the template image and its gradient.
// The diagonal is stored inverted and scaled by the SOR relaxation factor:
// i11 = omega / a11, i22 = omega / a22.
__device__ __forceinline__ PixelSystem pixel_system_vals(
    float ix, float iy, float ixl, float ixr, float ixu, float ixd, float iyu, float iyd,
    float iw, float asp, float asl, float asr, float asu, float asd, float u, float ul, float ur,
    float uu, float ud, float v, float vl, float vr, float vu, float vd, bool bl, bool br,
    bool bu, bool bd, int gx, int gy, int w, int h, float i0, float i0x, float i0y, float delta,
    float gamma, float omega)
{
    // every operation with a fixed rounding (fmul, fadd, fsub, ffma), so that
    // the two kernel forms that call this function give the same systems
    const float Ix = ix, Iy = iy;
    const float Ixx = cdiff(ixr, ixl);
    const float Ixy = cdiff(ixd, ixu);
    const float Iyy = cdiff(iyd, iyu);
    const float Iz = fsub(iw, i0);
    const float Ixz = fsub(Ix, i0x), Iyz = fsub(Iy, i0y);
    const float nd = __fdividef(1.0f, fadd(ffma(Iy, Iy, fmul(Ix, Ix)), kZeta2));
    const float ng = __fdividef(
        1.0f, fadd(ffma(Iyy, Iyy, ffma(fmul(2.0f, Ixy), Ixy, fmul(Ixx, Ixx))), kZeta2));
    float ad = fmul(fmul(delta, nd), psi_prime(fmul(fmul(nd, Iz), Iz)));
    float ag = fmul(fmul(gamma, ng), psi_prime(fmul(ng, ffma(Iyz, Iyz, fmul(Ixz, Ixz)))));
    const float wx = fadd((float)gx, u), wy = fadd((float)gy, v);
    if (wx < 0.0f || wx > (float)(w - 1) || wy < 0.0f || wy > (float)(h - 1)) {
        ad = 0.0f;
        ag = 0.0f;
    }
    PixelSystem ps;
    ps.cl = bl ? fmul(0.5f, fadd(asp, asl)) : 0.0f;
    ps.cr = br ? fmul(0.5f, fadd(asp, asr)) : 0.0f;
    ps.cu = bu ? fmul(0.5f, fadd(asp, asu)) : 0.0f;
    ps.cd = bd ? fmul(0.5f, fadd(asp, asd)) : 0.0f;
    const float sw = fadd(fadd(fadd(ps.cl, ps.cr), ps.cu), ps.cd);
    const float su0 = ffma(ps.cd, fsub(ud, u),
                           ffma(ps.cu, fsub(uu, u), ffma(ps.cr, fsub(ur, u),
                                                         fmul(ps.cl, fsub(ul, u)))));
    const float sv0 = ffma(ps.cd, fsub(vd, v),
                           ffma(ps.cu, fsub(vu, v), ffma(ps.cr, fsub(vr, v),
                                                         fmul(ps.cl, fsub(vl, v)))));
    const float adx = fmul(ad, Ix), ady = fmul(ad, Iy);
    ps.i11 = __fdividef(omega, fadd(ffma(ag, ffma(Ixy, Ixy, fmul(Ixx, Ixx)), fmul(adx, Ix)), sw));
    ps.i22 = __fdividef(omega, fadd(ffma(ag, ffma(Iyy, Iyy, fmul(Ixy, Ixy)), fmul(ady, Iy)), sw));
    ps.a12 = ffma(ag, ffma(Ixy, Iyy, fmul(Ixx, Ixy)), fmul(adx, Iy));
    ps.b1 = ffma(-ag, ffma(Ixy, Iyz, fmul(Ixx, Ixz)), ffma(-adx, Iz, su0));
    ps.b2 = ffma(-ag, ffma(Iyy, Iyz, fmul(Ixy, Ixz)), ffma(-ady, Iz, sv0));
    return ps;
}

// The same system read from the staging and derivative windows: d indexes
// the derivative window (row stride DS, origin dx0, dy0), e the staging
// window (row stride ES).  Every index read lies in the windows (their rings
// hold 0 outside the level).  IN as in stage_derivs.
template <bool IN>
__device__ __forceinline__ PixelSystem pixel_system(const float *sIx, const float *sIy,
                                                    const float *sAs, int DS, int dx0, int dy0,
                                                    const float *sW, const float *sU,
                                                    const float *sV, int ES, int e, int gx,
                                                    int gy, int w, int h, float i0, float i0x,
                                                    float i0y, float delta, float gamma,
                                                    float omega)
{
    const int xp = (IN ? gx + 1 : min(gx + 1, w - 1)) - dx0;
    const int xm = (IN ? gx - 1 : max(gx - 1, 0)) - dx0;
    const int yp = (IN ? gy + 1 : min(gy + 1, h - 1)) - dy0;
    const int ym = (IN ? gy - 1 : max(gy - 1, 0)) - dy0;
    const int dx = gx - dx0, dy = gy - dy0;
    const int d = dy * DS + dx;
    return pixel_system_vals(
        sIx[d], sIy[d], sIx[dy * DS + xm], sIx[dy * DS + xp], sIx[ym * DS + dx],
        sIx[yp * DS + dx], sIy[ym * DS + dx], sIy[yp * DS + dx], sW[e], sAs[d], sAs[d - 1],
        sAs[d + 1], sAs[d - DS], sAs[d + DS], sU[e], sU[e - 1], sU[e + 1], sU[e - ES],
        sU[e + ES], sV[e], sV[e - 1], sV[e + 1], sV[e - ES], sV[e + ES], IN || gx > 0,
        IN || gx + 1 < w, IN || gy > 0, IN || gy + 1 < h, gx, gy, w, h, i0, i0x, i0y, delta,
        gamma, omega);
}

// One coefficient tile.  IN: the tile's staging window (tile + 2 px) lies
// inside the level, so no load or neighbour needs a bounds test.
template <bool IN, typename T>
__device__ __forceinline__ void coeff_tile(
    float (&sU)[kAEY][kAEX], float (&sV)[kAEY][kAEX], float (&sW)[kAEY][kAEX],
    float (&sIx)[kADY][kADX], float (&sIy)[kADY][kADX], float (&sAs)[kADY][kADX],
    const T *__restrict__ I0b, const T *__restrict__ I0xb, const T *__restrict__ I0yb,
    const T *__restrict__ I1b, int w, int h, int pitch, size_t pfs, const float *__restrict__ Ub,
    size_t ufs, size_t plane, float *__restrict__ coefb, size_t cfs, float delta, float gamma,
    float alpha_s, float omega, unsigned bx, unsigned by, unsigned f)
{
    const int tx0 = bx * kAX, ty0 = by * kAY;
    const int ex0 = tx0 - 2, ey0 = ty0 - 2, dx0 = tx0 - 1, dy0 = ty0 - 1;
    // frame base pointers once; offsets within a frame fit in 32 bits
    const size_t po = (size_t)f * pfs;
    const T *I1 = I1b + po;
    const float *U = Ub + (size_t)f * ufs;
    const float *V = U + plane;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 12 threads, one per tile pixel

    const int t = ty * kAX + tx;
    constexpr int kN = kAX * kAY;
    for (int i = t; i < kAEX * kAEY; i += kN) {
        const int lx = i % kAEX, ly = i / kAEX;
        const int gx = ex0 + lx, gy = ey0 + ly;
        float u = 0.0f, v = 0.0f, wv = 0.0f;
        if (IN || (gx >= 0 && gx < w && gy >= 0 && gy < h)) {
            const int p = gy * pitch + gx;
            u = U[p];
            v = V[p];
            wv = bilinear_i(I1, w, h, pitch, (float)gx + u, (float)gy + v);
        }
        sU[ly][lx] = u;
        sV[ly][lx] = v;
        sW[ly][lx] = wv;
    }
    __syncthreads();
    for (int i = t; i < kADX * kADY; i += kN) {
        const int lx = i % kADX, ly = i / kADX;
        const int gx = dx0 + lx, gy = dy0 + ly;
        float ix = 0.0f, iy = 0.0f, as = 0.0f;
        if (IN || (gx >= 0 && gx < w && gy >= 0 && gy < h))
            stage_derivs<IN>(&sW[0][0], &sU[0][0], &sV[0][0], kAEX,
                             (gy - ey0) * kAEX + (gx - ex0), ex0, ey0, gx, gy, w, h, alpha_s,
                             ix, iy, as);
        sIx[ly][lx] = ix;
        sIy[ly][lx] = iy;
        sAs[ly][lx] = as;
    }
    __syncthreads();

    const int gx = tx0 + threadIdx.x, gy = ty0 + threadIdx.y;
    if (!IN && (gx >= w || gy >= h)) return;
    const int p = gy * pitch + gx;
    const PixelSystem ps = pixel_system<IN>(
        &sIx[0][0], &sIy[0][0], &sAs[0][0], kADX, dx0, dy0, &sW[0][0], &sU[0][0], &sV[0][0], kAEX,
        (gy - ey0) * kAEX + (gx - ex0), gx, gy, w, h, ldp(&(I0b + po)[p]), ldp(&(I0xb + po)[p]),
        ldp(&(I0yb + po)[p]), delta, gamma, omega);
    const int pl = (int)plane;
    float *cf = coefb + (size_t)f * cfs + p;
    cf[kCI11 * pl] = ps.i11;
    cf[kCI22 * pl] = ps.i22;
    cf[kCA12 * pl] = ps.a12;
    cf[kCB1 * pl] = ps.b1;
    cf[kCB2 * pl] = ps.b2;
    cf[kCWL * pl] = ps.cl;
    cf[kCWU * pl] = ps.cu;
}

// (bx, by): the tile, f: the frame.
template <typename T>
__device__ __forceinline__ void var_coeff_body(
    const T *__restrict__ I0b, const T *__restrict__ I0xb, const T *__restrict__ I0yb,
    const T *__restrict__ I1b, int w, int h, int pitch, size_t pfs, const float *__restrict__ Ub,
    size_t ufs, size_t plane, float *__restrict__ coefb, size_t cfs, float delta, float gamma,
    float alpha_s, float omega, unsigned bx, unsigned by, unsigned f)
{
    __shared__ float sU[kAEY][kAEX], sV[kAEY][kAEX], sW[kAEY][kAEX];
    __shared__ float sIx[kADY][kADX], sIy[kADY][kADX], sAs[kADY][kADX];
    const int tx0 = bx * kAX, ty0 = by * kAY;
    if (tx0 >= 2 && ty0 >= 2 && tx0 + kAX + 2 <= w && ty0 + kAY + 2 <= h)
        coeff_tile<true>(sU, sV, sW, sIx, sIy, sAs, I0b, I0xb, I0yb, I1b, w, h, pitch, pfs, Ub,
                         ufs, plane, coefb, cfs, delta, gamma, alpha_s, omega, bx, by, f);
    else
        coeff_tile<false>(sU, sV, sW, sIx, sIy, sAs, I0b, I0xb, I0yb, I1b, w, h, pitch, pfs, Ub,
                          ufs, plane, coefb, cfs, delta, gamma, alpha_s, omega, bx, by, f);
}

template <typename T>
__global__ void __launch_bounds__(kAX * kAY)
var_coeff_kernel(const T *__restrict__ I0b, const T *__restrict__ I0xb,
                 const T *__restrict__ I0yb, const T *__restrict__ I1b, int w, int h,
                 int pitch, size_t pfs, const float *__restrict__ Ub, size_t ufs, size_t plane,
                 float *__restrict__ coefb, size_t cfs, float delta, float gamma, float alpha_s,
                 float omega)
{
    var_coeff_body(I0b, I0xb, I0yb, I1b, w, h, pitch, pfs, Ub, ufs, plane, coefb, cfs, delta,
                   gamma, alpha_s, omega, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <typename T>
__global__ void __launch_bounds__(kAX * kAY)
seg_var_coeff_kernel(const __grid_constant__ SegTable<SegCoeff> tab)
{
    int b;
    const SegCoeff &a = seg_of(tab, b);
    const int r = b / a.gx;
    var_coeff_body((const T *)a.I0, (const T *)a.I0x, (const T *)a.I0y, (const T *)a.I1, a.w, a.h,
                   a.pitch, a.pfs, a.U, a.ufs, a.plane, a.coef, a.cfs, a.delta, a.gamma,
                   a.alpha_s, a.omega, b % a.gx, r % a.gy, r / a.gy);
}

// Column-walk form of the same kernel.  A warp owns 28 output columns: lane
// l holds column x = x0 - 2 + l, lanes 2..29 are outputs and lanes 0, 1, 30,
// 31 the halo that the central differences and the forward differences of
// the smoothness term need.  The warp walks R output rows down and keeps
// the rows it needs in registers: W (the warped sample I1(x + U)) of rows
// y .. y + 2, Ix, Iy and the smoothness weight of rows y - 1 .. y + 1, U and
// V of rows y - 1 .. y + 2; horizontal neighbours come from lane shuffles.
// Each row's U, V loads are issued two iterations and its bilinear taps one
// iteration before their use.  Values of positions outside the level are 0,
// as in the staging windows of coeff_tile, and every clamp and border test
// is the tile form's; the arithmetic has a fixed rounding sequence (fmul,
// fadd, ffma), so both forms write the same coefficients bit for bit.  Seven
// blocks of 72 registers per SM: a 1280 x 720 level's 1058 blocks take one
// wave (at eight blocks, 64 registers, the kernel spilled).
constexpr int kCWOut = 28;   // output columns per warp
constexpr int kCWWarps = 4;  // warps per block, row strips stacked
constexpr int kCWRows = 8;   // output rows per warp (default; ebof_params.coeff_cw_rows)

template <int R, bool IN, typename T, bool COH = false>
__device__ __forceinline__ void coeff_strip(const T *__restrict__ I0, const T *__restrict__ I0x,
                                            const T *__restrict__ I0y, const T *__restrict__ I1,
                                            int w, int h, int pitch, const float *__restrict__ U,
                                            const float *__restrict__ V, float *__restrict__ cf,
                                            int pl, int x, int y0, bool out_lane, float delta,
                                            float gamma, float alpha_s, float omega)
{
    const bool xin = IN || (x >= 0 && x < w);
    const bool hx = IN || x + 1 < w;
    const bool bl = IN || x > 0;
    const int ylast = y0 + R + 1;  // last row whose W, U and V are read
    auto row_in = [&](int r) { return IN || (r >= 0 && r < h); };
    auto load_uv = [&](int r, float &u, float &v) {
        u = 0.0f;
        v = 0.0f;
        if (row_in(r) && xin) {
            const int p = r * pitch + x;
            u = ldf<COH>(U + p);
            v = ldf<COH>(V + p);
        }
    };
    auto taps = [&](int r, float u, float v) {
        BilTaps t = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (row_in(r) && xin) t = bil_taps_i(I1, w, h, pitch, (float)x + u, (float)r + v);
        return t;
    };
    // neighbour in x with the clamp of the central differences
    auto right = [&](float c) {
        const float n = __shfl_down_sync(kFull, c, 1);
        return (IN || x + 1 < w) ? n : c;
    };
    auto left = [&](float c) {
        const float n = __shfl_up_sync(kFull, c, 1);
        return (IN || x > 0) ? n : c;
    };
    // Ix, Iy and the smoothness weight of row r from W of rows r - 1 .. r + 1
    // and U, V of rows r, r + 1
    auto derive = [&](int r, float wm, float w0, float wp, float u0, float u1, float v0,
                      float v1, float &ix, float &iy, float &as) {
        ix = cdiff(right(w0), left(w0));
        iy = cdiff((IN || r + 1 < h) ? wp : w0, (IN || r > 0) ? wm : w0);
        as = smooth_weight(u0, __shfl_down_sync(kFull, u0, 1), u1, v0,
                           __shfl_down_sync(kFull, v0, 1), v1, hx, IN || r + 1 < h, alpha_s);
    };

    // prologue: U, V of rows y0 - 2 .. y0 + 3, W of rows y0 - 2 .. y0 + 1,
    // the derivatives of rows y0 - 1 and y0, the taps of row y0 + 2
    float ua, va, ub, vb, uc, vc, ud, vd, u2, v2, u3, v3;
    load_uv(y0 - 2, ua, va);
    load_uv(y0 - 1, ub, vb);
    load_uv(y0, uc, vc);
    load_uv(y0 + 1, ud, vd);
    load_uv(y0 + 2, u2, v2);
    load_uv(y0 + 3, u3, v3);
    const float wa = bil_lerp(taps(y0 - 2, ua, va));
    const float wb = bil_lerp(taps(y0 - 1, ub, vb));
    float wc = bil_lerp(taps(y0, uc, vc));
    float wd = bil_lerp(taps(y0 + 1, ud, vd));
    BilTaps t2 = taps(y0 + 2, u2, v2);
    float ixm, iym, asm_, ix0, iy0, as0;
    derive(y0 - 1, wa, wb, wc, ub, uc, vb, vc, ixm, iym, asm_);
    derive(y0, wb, wc, wd, uc, ud, vc, vd, ix0, iy0, as0);
    auto ld_t = [&](const T *a, int p) { return ldp(&a[p]); };
    int p = y0 * pitch + x;
    const bool pin = row_in(y0) && xin;
    float i0 = pin ? ld_t(I0, p) : 0.0f, i0x = pin ? ld_t(I0x, p) : 0.0f;
    float i0y = pin ? ld_t(I0y, p) : 0.0f;

#pragma unroll 1
    for (int y = y0; y < y0 + R; ++y) {
        if (!IN && y >= h) break;
        // W, derivatives of row y + 1
        const float we = bil_lerp(t2);
        float ixp, iyp, asp_;
        derive(y + 1, wc, wd, we, ud, u2, vd, v2, ixp, iyp, asp_);
        // loads for the next iterations
        BilTaps t3 = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (y + 3 <= ylast) t3 = taps(y + 3, u3, v3);
        float u4 = 0.0f, v4 = 0.0f;
        if (y + 4 <= ylast) load_uv(y + 4, u4, v4);
        const int pn = p + pitch;
        const bool nin = y + 1 < y0 + R && row_in(y + 1) && xin;
        const float n_i0 = nin ? ld_t(I0, pn) : 0.0f, n_i0x = nin ? ld_t(I0x, pn) : 0.0f;
        const float n_i0y = nin ? ld_t(I0y, pn) : 0.0f;
        // the system of row y
        const PixelSystem ps = pixel_system_vals(
            ix0, iy0, left(ix0), right(ix0), (IN || y > 0) ? ixm : ix0,
            (IN || y + 1 < h) ? ixp : ix0, (IN || y > 0) ? iym : iy0,
            (IN || y + 1 < h) ? iyp : iy0, wc, as0, __shfl_up_sync(kFull, as0, 1),
            __shfl_down_sync(kFull, as0, 1), asm_, asp_, uc, __shfl_up_sync(kFull, uc, 1),
            __shfl_down_sync(kFull, uc, 1), ub, ud, vc, __shfl_up_sync(kFull, vc, 1),
            __shfl_down_sync(kFull, vc, 1), vb, vd, bl, hx, IN || y > 0, IN || y + 1 < h, x, y,
            w, h, i0, i0x, i0y, delta, gamma, omega);
        if (out_lane && xin) {
            float *c = cf + p;
            c[kCI11 * pl] = ps.i11;
            c[kCI22 * pl] = ps.i22;
            c[kCA12 * pl] = ps.a12;
            c[kCB1 * pl] = ps.b1;
            c[kCB2 * pl] = ps.b2;
            c[kCWL * pl] = ps.cl;
            c[kCWU * pl] = ps.cu;
        }
        // move the windows down one row
        ixm = ix0; iym = iy0; asm_ = as0;
        ix0 = ixp; iy0 = iyp; as0 = asp_;
        wc = wd; wd = we;
        ub = uc; vb = vc; uc = ud; vc = vd; ud = u2; vd = v2; u2 = u3; v2 = v3; u3 = u4; v3 = v4;
        t2 = t3;
        p = pn;
        i0 = n_i0; i0x = n_i0x; i0y = n_i0y;
    }
}

template <int R, typename T>
__global__ void __launch_bounds__(32 * kCWWarps, 7)
var_coeff_cw_kernel(const T *__restrict__ I0b, const T *__restrict__ I0xb,
                    const T *__restrict__ I0yb, const T *__restrict__ I1b, int w, int h,
                    int pitch, size_t pfs, const float *__restrict__ Ub, size_t ufs,
                    size_t plane, float *__restrict__ coefb, size_t cfs, float delta,
                    float gamma, float alpha_s, float omega)
{
    const int lane = threadIdx.x;
    const int y0 = (blockIdx.y * kCWWarps + threadIdx.y) * R;
    if (y0 >= h) return;  // the whole warp
    const int f = blockIdx.z;
    const int cx0 = blockIdx.x * kCWOut - 2;  // column of lane 0
    const size_t po = (size_t)f * pfs;
    const float *U = Ub + (size_t)f * ufs;
    const bool out_lane = lane >= 2 && lane < 2 + kCWOut;
    if (cx0 >= 0 && cx0 + 31 < w && y0 >= 2 && y0 + R + 1 < h)
        coeff_strip<R, true>(I0b + po, I0xb + po, I0yb + po, I1b + po, w, h, pitch, U, U + plane,
                             coefb + (size_t)f * cfs, (int)plane, cx0 + lane, y0, out_lane,
                             delta, gamma, alpha_s, omega);
    else
        coeff_strip<R, false>(I0b + po, I0xb + po, I0yb + po, I1b + po, w, h, pitch, U,
                              U + plane, coefb + (size_t)f * cfs, (int)plane, cx0 + lane, y0,
                              out_lane, delta, gamma, alpha_s, omega);
}

// Left and right halo of a region in columns: R rounded up to even, so that
// every region starts on an even column and a lane's two columns are one
// aligned 8-byte pair in every plane (pitches and plane sizes are even).
__host__ __device__ __forceinline__ int sor_halo_x(int R) { return R + (R & 1); }

// Interior output of a lane's pair (columns gx0, gx0 + 1 of row gy; the
// pair is interior or not as a whole): U + dU, as pairs where both columns
// are in the level.
template <bool COH = false>
__device__ __forceinline__ void store_pair(const float *Uin, float *Uout, size_t plane, int p,
                                           int gx0, int w, float du0, float du1, float dv0,
                                           float dv1)
{
    if (gx0 + 1 < w) {
        const float2 u = ldf2<COH>(Uin + p);
        const float2 v = ldf2<COH>(Uin + plane + p);
        *reinterpret_cast<float2 *>(Uout + p) = make_float2(u.x + du0, u.y + du1);
        *reinterpret_cast<float2 *>(Uout + plane + p) = make_float2(v.x + dv0, v.y + dv1);
    } else if (gx0 < w) {
        Uout[p] = ldf<COH>(Uin + p) + du0;
        (Uout + plane)[p] = ldf<COH>(Uin + plane + p) + dv0;
    }
}

// The right and lower edge weights of a thread's strip from the stored left
// and upper ones: w_r(x) = w_l(x + 1) (the next lane's first column for the
// strip's second column; 0 past the region's last column, whose right
// neighbour holds dU = 0) and w_d(y) = w_u(y + 1) (wub: w_u of the row below
// the strip).
template <int VS>
__device__ __forceinline__ void lower_right_weights(const float (&wl)[VS][2],
                                                    const float (&wu)[VS][2],
                                                    const float (&wub)[2], int lane,
                                                    float (&wr)[VS][2], float (&wd)[VS][2])
{
#pragma unroll
    for (int r = 0; r < VS; ++r) {
        const float n = __shfl_down_sync(kFull, wl[r][0], 1);
        wr[r][0] = wl[r][1];
        wr[r][1] = lane < 31 ? n : 0.0f;
#pragma unroll
        for (int q = 0; q < 2; ++q) wd[r][q] = r + 1 < VS ? wu[r + 1][q] : wub[q];
    }
}

// The region's first column (lane 0's first) has its left neighbour outside
// the region, where dU stays 0; a zero edge weight there lets the SOR update
// take the shuffled value without a select (0 times a finite value adds
// exactly 0).  Its right neighbour's weight is unaffected: a pixel's right
// weight is read from the next lane.
template <int VS>
__device__ __forceinline__ void zero_region_left_weights(float (&wl)[VS][2], int lane)
{
    if (lane == 0) {
#pragma unroll
        for (int r = 0; r < VS; ++r) wl[r][0] = 0.0f;
    }
}

// A lane's two adjacent values of one plane (c: the first); EVEN: one
// aligned 8-byte load.
template <bool EVEN, bool COH = false>
__device__ __forceinline__ void set_pair(float (&a)[2], const float *c)
{
    if (EVEN) {
        const float2 v = ldf2<COH>(c);
        a[0] = v.x;
        a[1] = v.y;
    } else {
        a[0] = ldf<COH>(c);
        a[1] = ldf<COH>(c + 1);
    }
}

// Region of 64 columns x RH rows, strips of VS rows: RH / VS warps.  EVEN:
// column halo rounded up to even (pairs loaded and stored as 8 bytes); else
// a halo of R columns (narrower halo, scalar accesses).
template <int VS, int RH, bool EVEN, bool COH>
__device__ __forceinline__ void sor_region(int bx, int by, int f, int w, int h, int pitch,
                                           const float *__restrict__ Uinb,
                                           float *__restrict__ Uoutb, size_t ufs, size_t plane,
                                           const float *__restrict__ coefb, size_t cfs, int R,
                                           int n_half, float omega, float *xch)
{
    constexpr int WARPS = RH / VS;
    const int hx = EVEN ? sor_halo_x(R) : R;
    const int tile_x = kVR - 2 * hx, tile_y = RH - 2 * R;
    const int rx0 = bx * tile_x - hx, ry0 = by * tile_y - R;
    const float *Uin = Uinb + (size_t)f * ufs;
    float *Uout = Uoutb + (size_t)f * ufs;
    const float *cf = coefb + (size_t)f * cfs;
    const int pl = (int)plane;  // offsets within a frame fit in 32 bits
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    float i11[VS][2], i22[VS][2], a12[VS][2], b1[VS][2], b2[VS][2];
    float wl[VS][2], wr[VS][2], wu[VS][2], wd[VS][2];
    float du[VS][2], dv[VS][2];
    const int gx0 = rx0 + 2 * lane;  // the lane's pair of columns (even when EVEN)
    const bool inside = rx0 >= 0 && ry0 >= 0 && rx0 + kVR <= w && ry0 + RH <= h;  // block-uniform
#pragma unroll
    for (int r = 0; r < VS; ++r) {
        const int gy = ry0 + wp * VS + r;
        if (inside) {
            // the whole region lies in the level: loads without bounds tests
            du[r][0] = du[r][1] = 0.0f;
            dv[r][0] = dv[r][1] = 0.0f;
            const float *c = cf + gy * pitch + gx0;
            set_pair<EVEN, COH>(i11[r], c + kCI11 * pl);
            set_pair<EVEN, COH>(i22[r], c + kCI22 * pl);
            set_pair<EVEN, COH>(a12[r], c + kCA12 * pl);
            set_pair<EVEN, COH>(b1[r], c + kCB1 * pl);
            set_pair<EVEN, COH>(b2[r], c + kCB2 * pl);
            set_pair<EVEN, COH>(wl[r], c + kCWL * pl);
            set_pair<EVEN, COH>(wu[r], c + kCWU * pl);
            continue;
        }
        if (!EVEN) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                du[r][q] = 0.0f;
                dv[r][q] = 0.0f;
                const int gx = gx0 + q;
                const bool in = gx >= 0 && gx < w && gy >= 0 && gy < h;
                const float *c = cf + (in ? gy * pitch + gx : 0);
                i11[r][q] = in ? ldf<COH>(c + kCI11 * pl) : 0.0f;
                i22[r][q] = in ? ldf<COH>(c + kCI22 * pl) : 0.0f;
                a12[r][q] = in ? ldf<COH>(c + kCA12 * pl) : 0.0f;
                b1[r][q] = in ? ldf<COH>(c + kCB1 * pl) : 0.0f;
                b2[r][q] = in ? ldf<COH>(c + kCB2 * pl) : 0.0f;
                wl[r][q] = in ? ldf<COH>(c + kCWL * pl) : 0.0f;
                wu[r][q] = in ? ldf<COH>(c + kCWU * pl) : 0.0f;
            }
            continue;
        }
        // gx0 >= 0 implies both columns >= 0; the second may be w (odd w),
        // still inside the row's pitch: loaded and masked
        const bool in0 = gx0 >= 0 && gx0 < w && gy >= 0 && gy < h;
        const bool in1 = in0 && gx0 + 1 < w;
        const float *c = cf + (in0 ? gy * pitch + gx0 : 0);
        float2 v[kCPlanes];
#pragma unroll
        for (int k = 0; k < kCPlanes; ++k)
            v[k] = in0 ? ldf2<COH>(c + k * pl) : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const bool in = q ? in1 : in0;
            du[r][q] = 0.0f;
            dv[r][q] = 0.0f;
            i11[r][q] = in ? (q ? v[kCI11].y : v[kCI11].x) : 0.0f;
            i22[r][q] = in ? (q ? v[kCI22].y : v[kCI22].x) : 0.0f;
            a12[r][q] = in ? (q ? v[kCA12].y : v[kCA12].x) : 0.0f;
            b1[r][q] = in ? (q ? v[kCB1].y : v[kCB1].x) : 0.0f;
            b2[r][q] = in ? (q ? v[kCB2].y : v[kCB2].x) : 0.0f;
            wl[r][q] = in ? (q ? v[kCWL].y : v[kCWL].x) : 0.0f;
            wu[r][q] = in ? (q ? v[kCWU].y : v[kCWU].x) : 0.0f;
        }
    }

    // upper weights of the row below the strip (the next strip's first row;
    // none below the region's last strip, whose lower neighbours hold dU = 0)
    float wub[2] = {0.0f, 0.0f};
    if (wp < WARPS - 1) {
        const int gy = ry0 + (wp + 1) * VS;
        if (inside) {
            set_pair<EVEN, COH>(wub, cf + gy * pitch + gx0 + kCWU * pl);
        } else {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int gx = gx0 + q;
                if (gx >= 0 && gx < w && gy >= 0 && gy < h)
                    wub[q] = ldf<COH>(cf + gy * pitch + gx + kCWU * pl);
            }
        }
    }
    lower_right_weights<VS>(wl, wu, wub, lane, wr, wd);
    zero_region_left_weights<VS>(wl, lane);

    // red-black SOR; red = (x + y) even, first.  Given the parity of (x + y)
    // at a strip's first pixel, the column of a given colour in a given row
    // is a compile-time constant.
    sor_sweeps<VS, WARPS>(du, dv, i11, i22, a12, b1, b2, wl, wr, wu, wd, xch, lane, wp,
                          (rx0 + ry0 + wp * VS) & 1, n_half, omega);

    if (!EVEN) {
#pragma unroll
        for (int r = 0; r < VS; ++r)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int lx = 2 * lane + q, ly = wp * VS + r;
                const int gx = rx0 + lx, gy = ry0 + ly;
                if (lx < hx || lx >= hx + tile_x || ly < R || ly >= R + tile_y || gx >= w ||
                    gy >= h)
                    continue;
                const int p = gy * pitch + gx;
                Uout[p] = ldf<COH>(Uin + p) + du[r][q];
                (Uout + plane)[p] = ldf<COH>(Uin + plane + p) + dv[r][q];
            }
        return;
    }
    const int lx0 = 2 * lane;
    if (lx0 >= hx && lx0 < hx + tile_x) {
#pragma unroll
        for (int r = 0; r < VS; ++r) {
            const int ly = wp * VS + r, gy = ry0 + ly;
            if (ly < R || ly >= R + tile_y || gy >= h) continue;
            store_pair<COH>(Uin, Uout, plane, gy * pitch + gx0, gx0, w, du[r][0], du[r][1],
                            dv[r][0], dv[r][1]);
        }
    }
}

template <int VS, int RH, bool EVEN>
__global__ void __launch_bounds__(32 * (RH / VS), 1)
var_sor_kernel(int w, int h, int pitch, const float *__restrict__ Uinb,
               float *__restrict__ Uoutb, size_t ufs, size_t plane,
               const float *__restrict__ coefb, size_t cfs, int R, int n_half, float omega)
{
    extern __shared__ float xch[];  // strip-end exchange, two buffers
    sor_region<VS, RH, EVEN, false>(blockIdx.x, blockIdx.y, blockIdx.z, w, h, pitch, Uinb, Uoutb,
                                    ufs, plane, coefb, cfs, R, n_half, omega, xch);
}

// The even-halo 64 x 64 regions of several groups' levels in one launch.
__global__ void __launch_bounds__(kVThreads, 1)
seg_var_sor_kernel(const __grid_constant__ SegTable<SegSor> tab)
{
    extern __shared__ float xch[];
    int b;
    const SegSor &a = seg_of(tab, b);
    const int r = b / a.gx;
    sor_region<kVS, kVR, true, false>(b % a.gx, r % a.gy, r / a.gy, a.w, a.h, a.pitch, a.Uin,
                                      a.Uout, a.ufs, a.plane, a.coef, a.cfs, a.R, a.n_half,
                                      a.omega, xch);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Bounded wait for the mbarrier phase with the given parity: at most
// `limit` try-wait rounds.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit)
{
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__global__ void __launch_bounds__(kVThreads, 1)
var_sor_tma_kernel(const __grid_constant__ CUtensorMap cmap, int w, int h, int pitch,
                   const float *__restrict__ Uinb, float *__restrict__ Uoutb, size_t ufs,
                   size_t plane, int R, int tile, int nrx, int nry, int total, int n_half,
                   float omega, long long wait_limit, int *err)
{
    extern __shared__ __align__(1024) float tsm[];
    float *cbuf = tsm;                  // [kCPlanes][kVR][kTmaBoxW]
    float *xch = tsm + kTmaCoefFloats;  // strip-end exchange, two buffers
    __shared__ __align__(8) unsigned long long mbar_s;
    const uint32_t mbar = smem_u32(&mbar_s);
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    const int per_frame = nrx * nry;
    const unsigned long long map_addr = (unsigned long long)&cmap;
    const uint32_t dst = smem_u32(cbuf);

    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int hx = sor_halo_x(R), tile_x = kVR - 2 * hx;
    auto issue = [&](int r) {  // thread 0: the tensor copy of region r
        const int f = r / per_frame, rem = r - f * per_frame;
        const int ry = rem / nrx, rx = rem - ry * nrx;
        const int bx0 = (rx * tile_x - hx) & ~3;
        const int by0 = ry * tile - R;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar),
                     "r"((unsigned)(kTmaCoefFloats * sizeof(float)))
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes "
            "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
            "l"(map_addr), "r"(bx0), "r"(by0), "r"(0), "r"(f), "r"(mbar)
            : "memory");
    };
    int r = blockIdx.x;
    if (t == 0 && r < total) issue(r);
    uint32_t parity = 0;
    for (; r < total; r += gridDim.x) {
        const bool ok = mbar_wait(mbar, parity, wait_limit);
        if (__syncthreads_or(!ok)) {
            if (t == 0) {
                atomicOr(err, kErrTimeout);
                // let the copy in flight land before the block exits (bounded
                // by the default limit, whatever the first wait's was)
                mbar_wait(mbar, parity, kWaitLimitDefault);
            }
            return;
        }
        parity ^= 1u;
        const int f = r / per_frame, rem = r - f * per_frame;
        const int ry = rem / nrx, rx = rem - ry * nrx;
        const int rx0 = rx * tile_x - hx, ry0 = ry * tile - R;
        const int ox = rx0 - (rx0 & ~3);  // region column 0 within the box: 0 or 2
        float i11[kVS][2], i22[kVS][2], a12[kVS][2], b1[kVS][2], b2[kVS][2];
        float wl[kVS][2], wr[kVS][2], wu[kVS][2], wd[kVS][2];
        float du[kVS][2], dv[kVS][2];
#pragma unroll
        for (int rr = 0; rr < kVS; ++rr) {
            const float *c = cbuf + (wp * kVS + rr) * kTmaBoxW + ox + 2 * lane;
            constexpr int P = kVR * kTmaBoxW;
            float2 v[kCPlanes];
#pragma unroll
            for (int k = 0; k < kCPlanes; ++k) v[k] = *reinterpret_cast<const float2 *>(c + k * P);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                du[rr][q] = 0.0f;
                dv[rr][q] = 0.0f;
                i11[rr][q] = q ? v[kCI11].y : v[kCI11].x;
                i22[rr][q] = q ? v[kCI22].y : v[kCI22].x;
                a12[rr][q] = q ? v[kCA12].y : v[kCA12].x;
                b1[rr][q] = q ? v[kCB1].y : v[kCB1].x;
                b2[rr][q] = q ? v[kCB2].y : v[kCB2].x;
                wl[rr][q] = q ? v[kCWL].y : v[kCWL].x;
                wu[rr][q] = q ? v[kCWU].y : v[kCWU].x;
            }
        }
        {
            float wub[2] = {0.0f, 0.0f};
            if (wp < kVWarps - 1) {
                const float2 v = *reinterpret_cast<const float2 *>(
                    cbuf + kCWU * kVR * kTmaBoxW + (wp + 1) * kVS * kTmaBoxW + ox + 2 * lane);
                wub[0] = v.x;
                wub[1] = v.y;
            }
            lower_right_weights<kVS>(wl, wu, wub, lane, wr, wd);
            zero_region_left_weights<kVS>(wl, lane);
        }
        __syncthreads();  // every thread holds its coefficients: the buffer is free
        if (t == 0 && r + (int)gridDim.x < total) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(r + gridDim.x);
        }
        const float *Uin = Uinb + (size_t)f * ufs;
        float *Uout = Uoutb + (size_t)f * ufs;
        sor_sweeps<kVS, kVWarps>(du, dv, i11, i22, a12, b1, b2, wl, wr, wu, wd, xch, lane, wp,
                                 (rx0 + ry0) & 1, n_half, omega);
        const int lx0 = 2 * lane, gx0 = rx0 + lx0;
        if (lx0 >= hx && lx0 < hx + tile_x) {
#pragma unroll
            for (int rr = 0; rr < kVS; ++rr) {
                const int ly = wp * kVS + rr, gy = ry0 + ly;
                if (ly < R || ly >= R + tile || gy >= h) continue;
                store_pair(Uin, Uout, plane, gy * pitch + gx0, gx0, w, du[rr][0], du[rr][1],
                           dv[rr][0], dv[rr][1]);
            }
        }
    }
}

// The whole variational refinement of one small level (every outer
// iteration) in one launch: one thread-block cluster per frame, C blocks of
// 512 threads.  Per outer iteration the cluster first builds the level's
// linear systems, a warp per column-walk strip (28 columns x SR rows, the
// strips dealt round the cluster's warps; short strips, as the walk down a
// strip is a chain of dependent loads), into the coefficient planes; a
// cluster barrier; then runs the SOR sweeps, a block per 64x32 region of
// 2-row strips (the regions dealt round the blocks), writing U + dU; a
// cluster barrier.  The
// device functions are those of var_coeff_cw_kernel and var_sor_kernel and
// the arithmetic has a fixed rounding sequence, so the flow is the same bit
// for bit as with the two kernels launched per iteration; it only saves their
// launches and the blocks' start-up, which dominate on levels this small.
// Data written earlier in the launch by other blocks (the planes, U) is read
// through L2 (ld.global.cg) after the barrier, whose release / acquire order
// makes it visible across the cluster.  Every block of a cluster passes every
// barrier (the work loops sit between them), so none can wait forever.
template <int SR, typename T>
__global__ void __launch_bounds__(kVThreads, 1)
var_level_cluster_kernel(const T *__restrict__ I0b, const T *__restrict__ I0xb,
                         const T *__restrict__ I0yb, const T *__restrict__ I1b, int w, int h,
                         int pitch, size_t pfs, float *Ua, float *Ub, size_t ufs, size_t plane,
                         float *coefb, size_t cfs, int outer, int n_half, int R, int nrx,
                         int nry, int ncx, int ncy, float delta, float gamma, float alpha_s,
                         float omega)
{
    extern __shared__ float xch[];  // strip-end exchange of the SOR regions
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank(), C = (int)cluster.num_blocks();
    const int f = blockIdx.z;  // one cluster per frame
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const size_t po = (size_t)f * pfs;
    const int nstrips = ncx * ncy, nreg = nrx * nry;
    const bool out_lane = lane >= 2 && lane < 2 + kCWOut;
    float *a = Ua, *b = Ub;
    for (int k = 0; k < outer; ++k) {
        const float *U = a + (size_t)f * ufs;
        float *cf = coefb + (size_t)f * cfs;
        for (int si = rank * kVWarps + wp; si < nstrips; si += C * kVWarps) {
            const int cx0 = (si % ncx) * kCWOut - 2, y0 = (si / ncx) * SR;
            if (cx0 >= 0 && cx0 + 31 < w && y0 >= 2 && y0 + SR + 1 < h)
                coeff_strip<SR, true, T, true>(I0b + po, I0xb + po, I0yb + po, I1b + po, w, h,
                                               pitch, U, U + plane, cf, (int)plane, cx0 + lane,
                                               y0, out_lane, delta, gamma, alpha_s, omega);
            else
                coeff_strip<SR, false, T, true>(I0b + po, I0xb + po, I0yb + po, I1b + po, w, h,
                                                pitch, U, U + plane, cf, (int)plane, cx0 + lane,
                                                y0, out_lane, delta, gamma, alpha_s, omega);
        }
        cluster.sync();
        for (int r = rank; r < nreg; r += C)
            sor_region<2, 32, true, true>(r % nrx, r / nrx, f, w, h, pitch, a, b, ufs, plane,
                                          coefb, cfs, R, n_half, omega, xch);
        cluster.sync();
        float *t = a;
        a = b;
        b = t;
    }
}

// Largest cluster of var_level_cluster_kernel that can be resident, per
// device (0: none); set by init_var_attributes.
int g_cluster_max[kMaxDevs];

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        cudaGetLastError();
    });
    return fn;
}

}  // namespace

void make_coef_maps(float *work, const Geometry &geo, int frames, CoefMaps *m)
{
    for (int l = 0; l < kMaxLevels; ++l) m->ok[l] = false;
    EncodeTiledFn enc = encode_tiled();
    if (!enc || !work) return;
    for (int l = 0; l < geo.levels; ++l) {
        const Level &lv = geo.lv[l];
        const cuuint64_t dims[4] = {(cuuint64_t)lv.w, (cuuint64_t)lv.h, (cuuint64_t)kCPlanes,
                                    (cuuint64_t)frames};
        const cuuint64_t strides[3] = {(cuuint64_t)lv.pitch * sizeof(float),
                                       (cuuint64_t)lv.plane * sizeof(float),
                                       (cuuint64_t)kCPlanes * lv.plane * sizeof(float)};
        const cuuint32_t box[4] = {(cuuint32_t)kTmaBoxW, (cuuint32_t)kVR, (cuuint32_t)kCPlanes,
                                   1};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        m->ok[l] = enc(&m->map[l], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, work, dims, strides, box,
                       estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
}

bool var_fused_supported(int var_sor)
{
    const int R = var_sor > 0 ? 2 * var_sor - 1 : 0;
    return kVR - 2 * sor_halo_x(R) >= 16;
}

void init_var_attributes()
{
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kMaxDevs) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        g_num_sms[dev] = n;
    }
    cudaFuncSetAttribute(var_sor_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kTmaSmemBytes);
    cudaFuncSetAttribute(var_sor_kernel<1, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(kVSmemFloats2 * sizeof(float)));
    // clusters of up to 16 blocks for the level-resident refinement: the
    // largest size whose cluster can be resident with one block per SM
    cudaFuncSetAttribute(var_level_cluster_kernel<2, float>,
                         cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(var_level_cluster_kernel<2, __half>,
                         cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(var_level_cluster_kernel<4, float>,
                         cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(var_level_cluster_kernel<4, __half>,
                         cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    int cm = 0;
    for (int c = 16; c >= 1 && cm == 0; --c) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c, 1, 1);
        cfg.blockDim = dim3(kVThreads, 1, 1);
        cfg.dynamicSmemBytes = kVSmemFloats * sizeof(float);
        cudaLaunchAttribute at;
        at.id = cudaLaunchAttributeClusterDimension;
        at.val.clusterDim.x = c;
        at.val.clusterDim.y = 1;
        at.val.clusterDim.z = 1;
        cfg.attrs = &at;
        cfg.numAttrs = 1;
        int n32 = 0, n16 = 0;
        int n32b = 0, n16b = 0;
        if (cudaOccupancyMaxActiveClusters(&n32, var_level_cluster_kernel<2, float>, &cfg) ==
                cudaSuccess &&
            cudaOccupancyMaxActiveClusters(&n16, var_level_cluster_kernel<2, __half>, &cfg) ==
                cudaSuccess &&
            cudaOccupancyMaxActiveClusters(&n32b, var_level_cluster_kernel<4, float>, &cfg) ==
                cudaSuccess &&
            cudaOccupancyMaxActiveClusters(&n16b, var_level_cluster_kernel<4, __half>, &cfg) ==
                cudaSuccess &&
            n32 > 0 && n16 > 0 && n32b > 0 && n16b > 0)
            cm = c;
    }
    cudaGetLastError();
    if (dev >= 0 && dev < kMaxDevs) g_cluster_max[dev] = cm;

}

int sor_tile_x(int R) { return kVR - 2 * sor_halo_x(R); }
int sor_tile_y(int R) { return kVR - 2 * R; }
void coeff_tile_shape(int &x, int &y)
{
    x = kAX;
    y = kAY;
}
int coeff_planes() { return kCPlanes; }

void launch_seg_coeff(const SegTable<SegCoeff> &t, int blocks, bool half, cudaStream_t st)
{
    StageScope sc(kStVarCoeff, 1, st);
    if (half) seg_var_coeff_kernel<__half><<<blocks, dim3(kAX, kAY), 0, st>>>(t);
    else seg_var_coeff_kernel<float><<<blocks, dim3(kAX, kAY), 0, st>>>(t);
}

void launch_seg_sor(const SegTable<SegSor> &t, int blocks, cudaStream_t st)
{
    StageScope sc(kStVarSor, 1, st);
    seg_var_sor_kernel<<<blocks, kVThreads, kVSmemFloats * sizeof(float), st>>>(t);
}

float *launch_variational_fused(const void *I0, const void *I0x, const void *I0y,
                                const void *I1, const Level &lv, size_t pyr_frame_stride,
                                float *U, float *Utmp, size_t u_frame_stride, float *coef,
                                int frames, const FlowParams &fp, const CUtensorMap *coef_map,
                                int *err, cudaStream_t st)
{
    // the level's planes are packed: frame stride kCPlanes planes of this level
    const size_t coef_frame_stride = (size_t)kCPlanes * lv.plane;
    int dev = 0;
    cudaGetDevice(&dev);
    const int nsm = (dev >= 0 && dev < kMaxDevs && g_num_sms[dev] > 0) ? g_num_sms[dev] : 0;
    const int n_half = 2 * fp.var_sor;
    const int R = n_half > 0 ? n_half - 1 : 0;
    const int tile = kVR - 2 * R;                    // interior rows of a 64-row region
    const int tile_x = kVR - 2 * sor_halo_x(R);      // interior columns
    const dim3 cgrd((lv.w + kAX - 1) / kAX, (lv.h + kAY - 1) / kAY, frames);
    // the coefficient kernel's form depends on the level's width and the
    // stream's parameters only, so single, batched and grouped windows of a
    // level always run the same one (and give the same coefficients): by
    // default the column walk from 1024 px wide (the finest level of 1280 x
    // 720 frames), where it is the faster; smaller levels keep the tile form
    const bool column_walk = lv.w >= fp.coeff_cw_min_width;
    const int cw_rows = fp.coeff_cw_rows == 4 || fp.coeff_cw_rows == 16 ? fp.coeff_cw_rows
                                                                       : kCWRows;
    const dim3 wgrd((lv.w + kCWOut - 1) / kCWOut,
                    ((lv.h + cw_rows - 1) / cw_rows + kCWWarps - 1) / kCWWarps, frames);
    const dim3 sgrd((lv.w + tile_x - 1) / tile_x, (lv.h + tile - 1) / tile, frames);
    // small levels: every outer iteration in one cluster launch per frame
    // (same flow bit for bit), where one cluster holds the level's work and
    // all the frames' clusters fit one wave
    {
        // strips of 2 rows if the cluster can hold them, else of 4
        const int cmax = std::min((dev >= 0 && dev < kMaxDevs) ? g_cluster_max[dev] : 0,
                                  fp.var_cluster_max);
        // SOR regions of 64 x 32 (2-row strips, 16 warps): the interior is
        // 32 - 2R rows high
        const int ty32 = 32 - 2 * R;
        const int nrx = (lv.w + tile_x - 1) / tile_x;
        const int nry = ty32 > 0 ? (lv.h + ty32 - 1) / ty32 : 1 << 20;
        const int ncx = (lv.w + kCWOut - 1) / kCWOut, nreg = nrx * nry;
        auto need = [&](int sr) {
            const int ncy_ = (lv.h + sr - 1) / sr;
            return std::max(nreg, (ncx * ncy_ + kVWarps - 1) / kVWarps);
        };
        const int sr = need(2) <= cmax ? 2 : 4;
        const int ncy = (lv.h + sr - 1) / sr, C = need(sr);
        if (fp.var_outer > 0 && C <= cmax && nsm > 0 && frames * C <= nsm) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(C, 1, frames);
            cfg.blockDim = dim3(kVThreads, 1, 1);
            cfg.dynamicSmemBytes = kVSmemFloats * sizeof(float);
            cfg.stream = st;
            cudaLaunchAttribute at;
            at.id = cudaLaunchAttributeClusterDimension;
            at.val.clusterDim.x = C;
            at.val.clusterDim.y = 1;
            at.val.clusterDim.z = 1;
            cfg.attrs = &at;
            cfg.numAttrs = 1;
            cudaError_t e;
            {
                StageScope sc(kStVarSor, 1, st);
                if (fp.half)
                    e = cudaLaunchKernelEx(&cfg, sr == 2 ? var_level_cluster_kernel<2, __half>
                                                         : var_level_cluster_kernel<4, __half>,
                                           (const __half *)I0, (const __half *)I0x,
                                           (const __half *)I0y, (const __half *)I1, lv.w, lv.h,
                                           lv.pitch, pyr_frame_stride, U, Utmp, u_frame_stride,
                                           lv.plane, coef, coef_frame_stride, fp.var_outer,
                                           n_half, R, nrx, nry, ncx, ncy, fp.delta, fp.gamma,
                                           fp.alpha_s, fp.omega);
                else
                    e = cudaLaunchKernelEx(&cfg, sr == 2 ? var_level_cluster_kernel<2, float>
                                                         : var_level_cluster_kernel<4, float>,
                                           (const float *)I0, (const float *)I0x,
                                           (const float *)I0y, (const float *)I1, lv.w, lv.h,
                                           lv.pitch, pyr_frame_stride, U, Utmp, u_frame_stride,
                                           lv.plane, coef, coef_frame_stride, fp.var_outer,
                                           n_half, R, nrx, nry, ncx, ncy, fp.delta, fp.gamma,
                                           fp.alpha_s, fp.omega);
            }
            if (e == cudaSuccess) return (fp.var_outer & 1) ? Utmp : U;
            cudaGetLastError();  // not launched: the per-iteration kernels below
        }
    }
    float *a = U, *b = Utmp;
    for (int k = 0; k < fp.var_outer; ++k) {
        if (column_walk) {
            StageScope sc(kStVarCoeff, 1, st);
#define EBOF_CW(R, T)                                                                          \
    var_coeff_cw_kernel<R, T><<<wgrd, dim3(32, kCWWarps), 0, st>>>(                             \
        (const T *)I0, (const T *)I0x, (const T *)I0y, (const T *)I1, lv.w, lv.h, lv.pitch,     \
        pyr_frame_stride, a, u_frame_stride, lv.plane, coef, coef_frame_stride, fp.delta,       \
        fp.gamma, fp.alpha_s, fp.omega)
            if (fp.half) {
                if (cw_rows == 4) EBOF_CW(4, __half);
                else if (cw_rows == 16) EBOF_CW(16, __half);
                else EBOF_CW(kCWRows, __half);
            } else {
                if (cw_rows == 4) EBOF_CW(4, float);
                else if (cw_rows == 16) EBOF_CW(16, float);
                else EBOF_CW(kCWRows, float);
            }
#undef EBOF_CW
        } else {
            StageScope sc(kStVarCoeff, 1, st);
            if (fp.half)
                var_coeff_kernel<__half><<<cgrd, dim3(kAX, kAY), 0, st>>>(
                    (const __half *)I0, (const __half *)I0x, (const __half *)I0y,
                    (const __half *)I1, lv.w, lv.h, lv.pitch, pyr_frame_stride, a,
                    u_frame_stride, lv.plane, coef, coef_frame_stride, fp.delta, fp.gamma,
                    fp.alpha_s, fp.omega);
            else
                var_coeff_kernel<float><<<cgrd, dim3(kAX, kAY), 0, st>>>(
                    (const float *)I0, (const float *)I0x, (const float *)I0y,
                    (const float *)I1, lv.w, lv.h, lv.pitch, pyr_frame_stride, a,
                    u_frame_stride, lv.plane, coef, coef_frame_stride, fp.delta, fp.gamma,
                    fp.alpha_s, fp.omega);
        }
        {
            StageScope sc(kStVarSor, 1, st);
            const int total = (int)(sgrd.x * sgrd.y * sgrd.z);
            // the persistent copy-ahead kernel pays off once every SM has
            // several regions to walk (batched and grouped windows); both
            // kernels see the same coefficients, so the choice never changes
            // the result
            // grids of under one wave are latency bound: where 64 x 32
            // regions of 1-row strips (1024 threads, one pixel update each
            // per half sweep) still fit in one wave, they replace the 4-row
            // strips.  Every layout computes the interior's whole-image
            // iteration, so the choice never changes the result.
            const dim3 g1((lv.w + tile_x - 1) / tile_x,
                          (lv.h + (32 - 2 * R) - 1) / (32 - 2 * R), frames);
            const int row_waves = fp.sor_row_waves;
            const bool small = nsm > 0 && row_waves > 0 && total < row_waves * nsm;
            // even-halo regions (8-byte pairs) unless they take more waves
            // than regions with an R-column halo
            const int todd = kVR - 2 * R;
            const dim3 godd((lv.w + todd - 1) / todd, sgrd.y, frames);
            const int wave = nsm > 0 ? nsm : 1;
            const bool even = (total + wave - 1) / wave <=
                              ((int)(godd.x * godd.y * godd.z) + wave - 1) / wave;
            if (coef_map && nsm > 0 && (long long)total >= (long long)fp.sor_tma_min_per_sm * nsm)
                var_sor_tma_kernel<<<nsm, kVThreads, kTmaSmemBytes, st>>>(
                    *coef_map, lv.w, lv.h, lv.pitch, a, b, u_frame_stride, lv.plane, R, tile,
                    (int)sgrd.x, (int)sgrd.y, total, n_half, fp.omega,
                    fp.wait_limit >= 0 ? fp.wait_limit : kWaitLimitDefault, err);
            else if (small && 32 - 2 * R >= 8 && (int)(g1.x * g1.y * g1.z) <= row_waves * nsm)
                var_sor_kernel<1, 32, true><<<g1, 32 * 32, kVSmemFloats2 * sizeof(float), st>>>(
                    lv.w, lv.h, lv.pitch, a, b, u_frame_stride, lv.plane, coef,
                    coef_frame_stride, R, n_half, fp.omega);
            else if (even)
                var_sor_kernel<kVS, kVR, true>
                    <<<sgrd, kVThreads, kVSmemFloats * sizeof(float), st>>>(
                        lv.w, lv.h, lv.pitch, a, b, u_frame_stride, lv.plane, coef,
                        coef_frame_stride, R, n_half, fp.omega);
            else
                var_sor_kernel<kVS, kVR, false>
                    <<<godd, kVThreads, kVSmemFloats * sizeof(float), st>>>(
                        lv.w, lv.h, lv.pitch, a, b, u_frame_stride, lv.plane, coef,
                        coef_frame_stride, R, n_half, fp.omega);
        }
        float *t = a;
        a = b;
        b = t;
    }
    return a;
}

}  // namespace ebof
