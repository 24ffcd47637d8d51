// k_flow.cu -- the frame-based flow block (§III-D) as Dense Inverse Search.
//
// §III-D leaves the frame-based method open; this block is Dense Inverse
// Search (Kroeger et al., ECCV 2016) on the 8-bit intensity I = 255 * d_exp
// of Eq. 1:
//   pyramid     2x2 box means, central-difference gradients (replicated border)
//   search      per-patch inverse-compositional Gauss-Newton on mean-
//               normalised patches, determinant guard, reset rule
//   densify     weights 1 / max(1, |I1(x + u_i) - I0(x)|)
//   variational normalised data + gradient-constancy + smoothness terms,
//               lagged robust weights, red-black SOR
// All arithmetic is FP32; the readings of the open points are those of the
// FP64 oracle this library is tested against.
#include "ebof_internal.cuh"
#include "profiler.cuh"
#include "dev_common.cuh"
#include "seg.cuh"

#include <type_traits>

namespace ebof {

namespace {

// ---------------------------------------------------------------- A5
template <typename T>
__global__ void downsample_kernel(const T *__restrict__ I, int pitch, T *__restrict__ out,
                                  int wc, int hc, int pitch_c, size_t fs)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= wc || y >= hc) return;
    const T *im = I + (size_t)blockIdx.z * fs;
    const size_t r0 = (size_t)(2 * y) * pitch + 2 * x, r1 = r0 + pitch;
    stp(&out[(size_t)blockIdx.z * fs + (size_t)y * pitch_c + x],
        0.25f * (ldp(&im[r0]) + ldp(&im[r0 + 1]) + ldp(&im[r1]) + ldp(&im[r1 + 1])));
}

// Value as stored in T (the next level is built from the stored values).
__device__ __forceinline__ float as_stored(float v, const float *) { return v; }
__device__ __forceinline__ float as_stored(float v, const __half *)
{
    return __half2float(__float2half_rn(v));
}

// Box-mean levels 1 .. min(levels, kPyrFused) - 1 of a slot in one launch,
// and the central differences of level 0: a block stages a 64 x 64 region of
// level 0 with a one-pixel ring (replicated at the image border, as the
// clamps of the gradient stencil read it) in shared memory, writes the
// region's level-0 gradients, then halves its 32 x 32 tile of level 1 in
// shared memory down to 2 x 2 at level 5.  Same sums in the same order as
// downsample_kernel and pyramid_gradients_body, so the levels and gradients
// are identical; the gradient launch then covers levels 1 and up only.
constexpr int kPyrTile = 32;
constexpr int kPyrFused = 6;
constexpr int kPyrStage = 2 * kPyrTile + 2;  // staged level-0 rows and columns

// Four consecutive elements of a row as one 16-byte (FP32) or 8-byte (FP16)
// load.
template <typename T> struct Quad;
template <> struct Quad<float> {
    using V = float4;
    static __device__ __forceinline__ void unpack(const V &v, float (&o)[4])
    {
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
};
template <> struct Quad<__half> {
    using V = uint2;
    static __device__ __forceinline__ void unpack(const V &v, float (&o)[4])
    {
        const __half2 a = *reinterpret_cast<const __half2 *>(&v.x);
        const __half2 b = *reinterpret_cast<const __half2 *>(&v.y);
        o[0] = __low2float(a); o[1] = __high2float(a);
        o[2] = __low2float(b); o[3] = __high2float(b);
    }
};

// Level 0 at the clamped positions (x0b - 1 + c, y0b - 1 + r), r, c < 66,
// into s0; every load of a thread is issued before the first shared-memory
// store.  Regions whose 64 columns lie inside the level read them as quads
// (x0b is a multiple of 64 and rows start on 128-byte boundaries, so the
// quads are aligned) and the two ring columns as single elements.
template <typename T>
__device__ __forceinline__ void stage_level0(float (&s0)[kPyrStage][kPyrStage + 1],
                                             const T *__restrict__ I0, int w0, int h0, int p0,
                                             int x0b, int y0b, int t)
{
    constexpr int E = kPyrStage;
    if (x0b + 2 * kPyrTile <= w0) {
        using V = typename Quad<T>::V;
        constexpr int NQ = E * (2 * kPyrTile / 4);  // quads of the 64 columns
        constexpr int KQ = (NQ + 255) / 256;
        V v[KQ];
#pragma unroll
        for (int k = 0; k < KQ; ++k) {
            const int i = t + 256 * k;
            if (i < NQ) {
                const int r = i / (2 * kPyrTile / 4), c = i % (2 * kPyrTile / 4);
                const int gy = min(max(y0b - 1 + r, 0), h0 - 1);
                v[k] = *reinterpret_cast<const V *>(I0 + gy * p0 + x0b + 4 * c);
            }
        }
        float hv = 0.0f;  // ring columns x0b - 1 and x0b + 64
        const int hr = t >> 1, hc = (t & 1) ? E - 1 : 0;
        if (t < 2 * E) {
            const int gy = min(max(y0b - 1 + hr, 0), h0 - 1);
            const int gx = min(max(x0b - 1 + hc, 0), w0 - 1);
            hv = ldp(&I0[gy * p0 + gx]);
        }
#pragma unroll
        for (int k = 0; k < KQ; ++k) {
            const int i = t + 256 * k;
            if (i < NQ) {
                const int r = i / (2 * kPyrTile / 4), c = i % (2 * kPyrTile / 4);
                float o[4];
                Quad<T>::unpack(v[k], o);
#pragma unroll
                for (int q = 0; q < 4; ++q) s0[r][1 + 4 * c + q] = o[q];
            }
        }
        if (t < 2 * E) s0[hr][hc] = hv;
    } else {
        constexpr int KS = (E * E + 255) / 256;
        float v[KS];
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const int i = t + 256 * k;
            v[k] = 0.0f;
            if (i < E * E) {
                const int r = i / E, c = i % E;
                const int gy = min(max(y0b - 1 + r, 0), h0 - 1);
                const int gx = min(max(x0b - 1 + c, 0), w0 - 1);
                v[k] = ldp(&I0[gy * p0 + gx]);
            }
        }
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const int i = t + 256 * k;
            if (i < E * E) s0[i / E][i % E] = v[k];
        }
    }
}

// (bx, by): the level-1 tile, f: the frame.
template <typename T>
__device__ __forceinline__ void pyramid_means_body(T *__restrict__ slots, size_t fs,
                                                   const PyrDesc &d, unsigned bx, unsigned by,
                                                   unsigned f)
{
    __shared__ float s0[kPyrStage][kPyrStage + 1];
    __shared__ float ta[kPyrTile][kPyrTile + 1];
    __shared__ float tb[kPyrTile / 2][kPyrTile / 2 + 1];
    T *slot = slots + (size_t)f * fs;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int t = ty * 32 + tx;
    const int x1b = bx * kPyrTile, y1b = by * kPyrTile;
    const int x0b = 2 * x1b, y0b = 2 * y1b;
    const int w0 = d.w[0], h0 = d.h[0], p0 = d.pitch[0];
    stage_level0<T>(s0, slot + d.off[0], w0, h0, p0, x0b, y0b, t);
    __syncthreads();
    {
        // level-0 gradients of the region: s0[r][c] holds level 0 at the
        // clamped position (x0b - 1 + c, y0b - 1 + r)
        T *Ix = slot + d.off[0] + d.plane[0], *Iy = slot + d.off[0] + 2 * d.plane[0];
#pragma unroll
        for (int i = 0; i < 2 * kPyrTile / 8; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int lx = tx + 32 * j, ly = ty + 8 * i;
                const int x = x0b + lx, y = y0b + ly;
                if (x < w0 && y < h0) {
                    const int p = y * p0 + x;
                    stp(&Ix[p], 0.5f * (s0[ly + 1][lx + 2] - s0[ly + 1][lx]));
                    stp(&Iy[p], 0.5f * (s0[ly + 2][lx + 1] - s0[ly][lx + 1]));
                }
            }
    }
    {
        T *I1 = slot + d.off[1];
#pragma unroll
        for (int i = 0; i < kPyrTile / 8; ++i) {
            const int ly = ty + 8 * i, x = x1b + tx, y = y1b + ly;
            float v = 0.0f;
            if (x < d.w[1] && y < d.h[1]) {
                const int sx = 2 * tx + 1, sy = 2 * ly + 1;
                v = 0.25f * (s0[sy][sx] + s0[sy][sx + 1] + s0[sy + 1][sx] + s0[sy + 1][sx + 1]);
                stp(&I1[(size_t)y * d.pitch[1] + x], v);
                v = as_stored(v, I1);
            }
            ta[ly][tx] = v;
        }
    }
    __syncthreads();
    int side = kPyrTile / 2;
    for (int l = 2; l < d.levels && l < kPyrFused; ++l, side >>= 1) {
        // level l - 1 is in ta for even l, in tb for odd l
        const bool from_a = (l & 1) == 0;
        const int lx = t % side, ly = t / side;
        const int x = (x1b >> (l - 1)) + lx, y = (y1b >> (l - 1)) + ly;
        if (t < side * side) {
            float v = 0.0f;
            if (x < d.w[l] && y < d.h[l]) {
                const int sx = 2 * lx, sy = 2 * ly;
                v = from_a ? 0.25f * (ta[sy][sx] + ta[sy][sx + 1] + ta[sy + 1][sx] + ta[sy + 1][sx + 1])
                           : 0.25f * (tb[sy][sx] + tb[sy][sx + 1] + tb[sy + 1][sx] + tb[sy + 1][sx + 1]);
                T *Il = slot + d.off[l];
                stp(&Il[(size_t)y * d.pitch[l] + x], v);
                v = as_stored(v, Il);
            }
            if (from_a) tb[ly][lx] = v;
            else ta[ly][lx] = v;
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
pyramid_means_kernel(T *__restrict__ slots, size_t fs, PyrDesc d)
{
    pyramid_means_body(slots, fs, d, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Central differences of the levels of a slot in one launch: the blocks of
// level l are blk0[l] .. blk0[l + 1] - 1 (32 x 8 pixels each), launched from
// block gb0 on (level 1 when the box-mean kernel wrote level 0's).  bb: the
// block of the launch, f: the frame.
template <typename T>
__device__ __forceinline__ void pyramid_gradients_body(T *__restrict__ slots, size_t fs,
                                                       const PyrDesc &d, unsigned bb, unsigned f)
{
    bb += d.gb0;
    int l = 0;
    while (l + 1 < d.levels && (int)bb >= d.blk0[l + 1]) ++l;
    const int b = bb - d.blk0[l];
    const int w = d.w[l], h = d.h[l], pitch = d.pitch[l];
    const int nbx = (w + 31) / 32;
    const int x = (b % nbx) * 32 + threadIdx.x, y = (b / nbx) * 8 + threadIdx.y;
    if (x >= w || y >= h) return;
    T *im = slots + (size_t)f * fs + d.off[l];
    T *Ix = im + d.plane[l], *Iy = im + 2 * d.plane[l];
    const int xp = min(x + 1, w - 1), xm = max(x - 1, 0);
    const int yp = min(y + 1, h - 1), ym = max(y - 1, 0);
    const size_t p = (size_t)y * pitch + x;
    stp(&Ix[p], 0.5f * (ldp(&im[(size_t)y * pitch + xp]) - ldp(&im[(size_t)y * pitch + xm])));
    stp(&Iy[p], 0.5f * (ldp(&im[(size_t)yp * pitch + x]) - ldp(&im[(size_t)ym * pitch + x])));
}

// One plane of a pyramid level (row pitch `pitch`) into a dense w x h FP32
// array (FP16 storage widened exactly).
template <typename T>
__global__ void __launch_bounds__(256)
pyramid_export_kernel(const T *__restrict__ src, int w, int h, int pitch, float *__restrict__ dst)
{
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x < w && y < h) dst[(size_t)y * w + x] = ldp(&src[(size_t)y * pitch + x]);
}

template <typename T>
__global__ void __launch_bounds__(256)
pyramid_gradients_kernel(T *__restrict__ slots, size_t fs, PyrDesc d)
{
    pyramid_gradients_body(slots, fs, d, blockIdx.x, blockIdx.z);
}

template <typename T>
__global__ void __launch_bounds__(256)
seg_pyramid_means_kernel(const __grid_constant__ SegTable<SegPyr> tab)
{
    int b;
    const SegPyr &a = seg_of(tab, b);
    const int r = b / a.gx;
    pyramid_means_body((T *)a.slots, a.fs, a.d, b % a.gx, r % a.gy, r / a.gy);
}

template <typename T>
__global__ void __launch_bounds__(256)
seg_pyramid_gradients_kernel(const __grid_constant__ SegTable<SegPyr> tab)
{
    int b;
    const SegPyr &a = seg_of(tab, b);
    pyramid_gradients_body((T *)a.slots, a.fs, a.d, b % a.gx, b / a.gx);
}

// ---------------------------------------------------------------- A6
// Group of G = CG x RG lanes per patch: lane c owns the CPL adjacent patch
// columns of column group c % CG (those below ps) over the RPL rows of row
// group c / CG, and keeps their template, gradients and running samples in
// registers.  Patch sums are reduced over the group with xor shuffles, so a
// warp serves 32 / G patches.  Every lane of a warp runs the same number of
// iterations (guarded patches iterate on a dummy determinant and are
// discarded), so the shuffles never diverge.
template <int G>
__device__ __forceinline__ float group_sum(float v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Lane layouts per patch size.  Wide: fewest idle lanes and fewest
// instructions per patch (ps 9..12: 4 lanes x 3 columns), for levels with
// enough patches to fill the GPU.  Narrow: one column per lane, split into
// two row halves (32 lanes for ps 9..16), the shortest serial work per lane,
// for levels with few patches where latency matters.  The choice depends on
// the level's patch count only, never on the number of frames in a launch,
// so batched and single-window results agree bit for bit.
template <int PS>
struct SearchShape {
    static constexpr int kWideCG = PS <= 8 ? 8 : (PS <= 12 ? 4 : 8);
    static constexpr int kWideRG = 1;
    static constexpr int kNarrowCG = PS <= 8 ? 8 : 16;
    static constexpr int kNarrowRG = PS <= 8 ? 1 : 2;
};
constexpr int kWideSearchPatches = 8192;

// bx: the block of patches, f: the frame.
template <int PS, int CG, int RG, typename T>
__device__ __forceinline__ void patch_search_body(
    const T *__restrict__ I0b, const T *__restrict__ I0xb, const T *__restrict__ I0yb,
    const T *__restrict__ I1b, int w, int h, int pitch, size_t pfs, int npx, int npy,
    const float *__restrict__ Ucb, int wc, int hc, int pitch_c, size_t plane_c, size_t ucfs,
    float *__restrict__ upb, size_t upfs, int stride, int iters, float kappa, int *err,
    unsigned bx, unsigned f)
{
    constexpr int G = CG * RG;
    constexpr int CPL = (PS + CG - 1) / CG;
    constexpr int RPL = (PS + RG - 1) / RG;
    const int c = threadIdx.x % G;
    const int np = npx * npy;
    const int pid_raw = bx * (128 / G) + threadIdx.x / G;
    const bool real = pid_raw < np;
    const int pid = real ? pid_raw : np - 1;
    const int i = pid % npx, j = pid / npx;
    const int x0 = min(i * stride, w - PS), y0 = min(j * stride, h - PS);
    const int c0 = (c % CG) * CPL;  // first column of this lane
    const int r0 = (c / CG) * RPL;  // first row of this lane
    const T *I0 = I0b + (size_t)f * pfs, *I0x = I0xb + (size_t)f * pfs;
    const T *I0y = I0yb + (size_t)f * pfs, *I1 = I1b + (size_t)f * pfs;
    if (x0 < 0 || y0 < 0) {  // cannot happen when the level holds a patch
        if (real && c == 0) atomicOr(err, kErrBounds);
    }

    // F3: start value from the next coarser level
    float u0 = 0.0f, v0 = 0.0f;
    if (Ucb) {
        const int cx = clampi((2 * x0 + PS) / 4, 0, wc - 1);
        const int cy = clampi((2 * y0 + PS) / 4, 0, hc - 1);
        const float *Uc = Ucb + (size_t)f * ucfs;
        u0 = 2.0f * Uc[(size_t)cy * pitch_c + cx];
        v0 = 2.0f * Uc[plane_c + (size_t)cy * pitch_c + cx];
    }

    // F4: template, mean-normalised gradients, Hessian
    float Tm[RPL][CPL], GX[RPL][CPL], GY[RPL][CPL];
    float sgx = 0.0f, sgy = 0.0f;
#pragma unroll
    for (int r = 0; r < RPL; ++r)
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            const bool act = c0 + k < PS && r0 + r < PS;
            const int p = (y0 + (act ? r0 + r : 0)) * pitch + x0 + (act ? c0 + k : 0);
            Tm[r][k] = act ? ldp(&I0[p]) : 0.0f;
            GX[r][k] = act ? ldp(&I0x[p]) : 0.0f;
            GY[r][k] = act ? ldp(&I0y[p]) : 0.0f;
            sgx += GX[r][k];
            sgy += GY[r][k];
        }
    constexpr float inv_n = 1.0f / (PS * PS);
    sgx = group_sum<G>(sgx); sgy = group_sum<G>(sgy);
    const float mgx = sgx * inv_n, mgy = sgy * inv_n;
    float h11 = 0.0f, h12 = 0.0f, h22 = 0.0f;
#pragma unroll
    for (int r = 0; r < RPL; ++r)
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            if (c0 + k < PS && r0 + r < PS) { GX[r][k] -= mgx; GY[r][k] -= mgy; }
            h11 += GX[r][k] * GX[r][k]; h12 += GX[r][k] * GY[r][k]; h22 += GY[r][k] * GY[r][k];
        }
    h11 = group_sum<G>(h11); h12 = group_sum<G>(h12); h22 = group_sum<G>(h22);
    // this lane's share of sum g T, accumulated in the order the iterations
    // accumulate sum g w, so that b = sum g w - sum g T is exactly zero
    // wherever the warped patch equals the template
    float tb1 = 0.0f, tb2 = 0.0f;
#pragma unroll
    for (int r = 0; r < RPL; ++r)
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            tb1 += GX[r][k] * Tm[r][k];
            tb2 += GY[r][k] * Tm[r][k];
        }
    const float det = h11 * h22 - h12 * h12;
    const bool guard = !(det > 1e-6f * (float)(PS * PS) * (float)(PS * PS));
    // damped step (H + mu Id)^-1 b, mu = kappa * trace(H)
    const float mu = kappa * (h11 + h22);
    const float a11 = h11 + mu, a22 = h22 + mu;
    const float inv_det = guard ? 0.0f : __fdividef(1.0f, a11 * a22 - h12 * h12);

    float u = u0, v = v0;
    const float lim = (float)(w + h);
    for (int it = 0; it < iters; ++it) {
        // b = sum g ((w - mean w) - (T - mean T)); the mean-normalised
        // gradients sum to zero, so both means drop out: b = sum g w - sum g T
        // (exactly zero when the warped patch equals the template)
        float b1 = 0.0f, b2 = 0.0f;
        // The displacement is the same for the whole patch, so the bilinear
        // sample has fixed weights (ax, ay) on a fixed (PS+1) x (PS+1) window
        // of texels from (sx0, sy0), and each row's horizontal lerps serve
        // two output rows.  Clamping the sample position to the level, the
        // reading of the oracle, gives the same value as clamping the
        // window's row and column indices (outside the level both taps of a
        // lerp are the same edge texel, and a + t (a - a) = a exactly).  The
        // window's rows and columns are clamped only where some lane's
        // window leaves the level; inside it the clamps do nothing, so the
        // form a warp takes never changes a value.
        const float uc = fminf(fmaxf(u, -lim), lim), vc = fminf(fmaxf(v, -lim), lim);
        const float fu = floorf(uc), fv = floorf(vc);
        const int sx0 = x0 + (int)fu, sy0 = y0 + (int)fv;
        const float ax = uc - fu, ay = vc - fv;
        const bool inside = sx0 >= 0 && sy0 >= 0 && sx0 + PS <= w - 1 && sy0 + PS <= h - 1;
        // columns c0 .. c0 + CPL and rows r0 .. r0 + RPL of the window (the
        // last of each only as the right / lower neighbour); no column or row
        // beyond PS is read
        auto window = [&](auto clamped) {
            constexpr bool C = decltype(clamped)::value;
            int cx[CPL + 1];
#pragma unroll
            for (int k = 0; k <= CPL; ++k)
                cx[k] = C ? clampi(sx0 + c0 + k, 0, w - 1) : sx0 + c0 + k;
            auto row = [&](int rr) {
                return I1 + (C ? clampi(sy0 + rr, 0, h - 1) : sy0 + rr) * pitch;
            };
            float hp[CPL];
            {
                const T *q = row(r0);
                float s[CPL + 1];
#pragma unroll
                for (int k = 0; k <= CPL; ++k)
                    s[k] = c0 + k <= PS && r0 <= PS ? ldp(&q[cx[k]]) : 0.0f;
#pragma unroll
                for (int k = 0; k < CPL; ++k) hp[k] = s[k] + ax * (s[k + 1] - s[k]);
            }
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                const T *q = row(r0 + r + 1);
                const bool rin = r0 + r + 1 <= PS;
                float s[CPL + 1];
#pragma unroll
                for (int k = 0; k <= CPL; ++k) s[k] = c0 + k <= PS && rin ? ldp(&q[cx[k]]) : 0.0f;
#pragma unroll
                for (int k = 0; k < CPL; ++k) {
                    const float hn = s[k] + ax * (s[k + 1] - s[k]);
                    const float wv = hp[k] + ay * (hn - hp[k]);
                    hp[k] = hn;
                    b1 += GX[r][k] * wv;
                    b2 += GY[r][k] * wv;
                }
            }
        };
        if (__all_sync(0xffffffffu, inside))
            window(std::integral_constant<bool, false>());
        else
            window(std::integral_constant<bool, true>());
        b1 = group_sum<G>(b1 - tb1); b2 = group_sum<G>(b2 - tb2);
        u -= (a22 * b1 - h12 * b2) * inv_det;
        v -= (a11 * b2 - h12 * b1) * inv_det;
    }
    if (guard || !(hypotf(u - u0, v - v0) <= (float)PS)) { u = u0; v = v0; }
    if (real && c == 0) {
        float *up = upb + (size_t)f * upfs;
        up[pid] = u;
        up[(size_t)np + pid] = v;
    }
}

template <int PS, int CG, int RG, typename T>
__global__ void __launch_bounds__(128)
patch_search_kernel(const T *__restrict__ I0b, const T *__restrict__ I0xb,
                    const T *__restrict__ I0yb, const T *__restrict__ I1b, int w, int h,
                    int pitch, size_t pfs, int npx, int npy, const float *__restrict__ Ucb, int wc,
                    int hc, int pitch_c, size_t plane_c, size_t ucfs, float *__restrict__ upb,
                    size_t upfs, int stride, int iters, float kappa, int *err)
{
    patch_search_body<PS, CG, RG, T>(I0b, I0xb, I0yb, I1b, w, h, pitch, pfs, npx, npy, Ucb, wc, hc,
                                     pitch_c, plane_c, ucfs, upb, upfs, stride, iters, kappa, err,
                                     blockIdx.x, blockIdx.y);
}

template <int PS, int CG, int RG, typename T>
__global__ void __launch_bounds__(128)
seg_patch_search_kernel(const __grid_constant__ SegTable<SegSearch> tab)
{
    int b;
    const SegSearch &a = seg_of(tab, b);
    patch_search_body<PS, CG, RG, T>(
        (const T *)a.I0, (const T *)a.I0x, (const T *)a.I0y, (const T *)a.I1, a.w, a.h, a.pitch,
        a.pfs, a.npx, a.npy, a.Uc, a.wc, a.hc, a.pitch_c, a.plane_c, a.ucfs, a.up, a.upfs,
        a.stride, a.iters, a.kappa, a.err, b % a.gx, b / a.gx);
}

// ---------------------------------------------------------------- A7
__device__ __forceinline__ void cover_range(int x, int n, int ps, int stride, int cnt, int &lo,
                                            int &hi, bool &last)
{
    // regular patches k < cnt - 1 have origin k * stride; the last one is
    // flush with the border at n - ps
    const int t = x - ps + 1;
    lo = t <= 0 ? 0 : (t + stride - 1) / stride;
    hi = min(cnt - 2, x / stride);
    last = x >= n - ps;
}

// Thread per pixel.  NC = ceil(ps / stride) bounds the regular patches that
// cover a pixel per axis: their loops are unrolled and predicated so that the
// loads of all of them are in flight together, and the patch flush with the
// right or lower border (which covers only pixels within ps of it) is a
// separate branch.  NC = 0: runtime loops.  Every pixel sums its covering
// patches in ascending (row, column) order, the flush patch last on each
// axis.  Where the four taps lie inside the level the sample takes its
// weights from frac(u), frac(v) directly (the clamp cannot act); elsewhere
// it is the clamped bilinear sample.
template <typename T>
__device__ __forceinline__ float dense_sample(const T *__restrict__ I1, int w, int h, int pitch,
                                              int x, int y, float u, float v)
{
    const float fu = floorf(u), fv = floorf(v);
    const float sxf = (float)x + fu, syf = (float)y + fv;
    if (sxf >= 0.0f && sxf + 1.0f <= (float)(w - 1) && syf >= 0.0f &&
        syf + 1.0f <= (float)(h - 1)) {
        const float ax = u - fu, ay = v - fv;
        const T *r0 = I1 + (int)syf * pitch + (int)sxf, *r1 = r0 + pitch;
        const float a = ldp(&r0[0]), b = ldp(&r0[1]), c = ldp(&r1[0]), d = ldp(&r1[1]);
        return (1.0f - ay) * ((1.0f - ax) * a + ax * b) + ay * ((1.0f - ax) * c + ax * d);
    }
    return bilinear_i(I1, w, h, pitch, (float)x + u, (float)y + v);
}

// (bx, by): the 32 x 8 tile, f: the frame.
template <typename T, int NC>
__device__ __forceinline__ void densify_body(const T *__restrict__ I0b, const T *__restrict__ I1b,
                                             int w, int h, int pitch, size_t pfs,
                                             const float *__restrict__ upb, size_t upfs, int npx,
                                             int npy, float *__restrict__ Ub, size_t ufs,
                                             size_t plane, int ps, int stride, unsigned bx,
                                             unsigned by, unsigned f)
{
    const int x = bx * 32 + threadIdx.x;
    const int y = by * 8 + threadIdx.y;
    if (x >= w || y >= h) return;
    const T *I0 = I0b + (size_t)f * pfs, *I1 = I1b + (size_t)f * pfs;
    const float *up = upb + (size_t)f * upfs;
    const float *vp = up + npx * npy;
    int ilo, ihi, jlo, jhi;
    bool ilast, jlast;
    cover_range(x, w, ps, stride, npx, ilo, ihi, ilast);
    cover_range(y, h, ps, stride, npy, jlo, jhi, jlast);
    const float i0 = ldp(&I0[y * pitch + x]);
    float nu = 0.0f, nv = 0.0f, den = 0.0f;
    auto add = [&](int id) {
        const float u = up[id], v = vp[id];
        const float r = dense_sample(I1, w, h, pitch, x, y, u, v) - i0;
        const float lam = 1.0f / fmaxf(1.0f, fabsf(r));
        nu += lam * u; nv += lam * v; den += lam;
    };
    // the patches of row j: regular columns, then the flush one
    auto row = [&](int j) {
        const int base = j * npx;
        if (NC > 0) {
#pragma unroll
            for (int di = 0; di < (NC > 0 ? NC : 1); ++di)
                if (ilo + di <= ihi) add(base + ilo + di);
        } else {
            for (int i = ilo; i <= ihi; ++i) add(base + i);
        }
        if (ilast) add(base + npx - 1);
    };
    if (NC > 0) {
#pragma unroll
        for (int dj = 0; dj < (NC > 0 ? NC : 1); ++dj)
            if (jlo + dj <= jhi) row(jlo + dj);
    } else {
        for (int j = jlo; j <= jhi; ++j) row(j);
    }
    if (jlast) row(npy - 1);
    float *U = Ub + (size_t)f * ufs;
    const int p = y * pitch + x;
    U[p] = den > 0.0f ? nu / den : 0.0f;
    (U + plane)[p] = den > 0.0f ? nv / den : 0.0f;
}

template <typename T, int NC>
__global__ void __launch_bounds__(256)
densify_kernel(const T *__restrict__ I0b, const T *__restrict__ I1b, int w, int h, int pitch,
               size_t pfs, const float *__restrict__ upb, size_t upfs, int npx, int npy,
               float *__restrict__ Ub, size_t ufs, size_t plane, int ps, int stride)
{
    densify_body<T, NC>(I0b, I1b, w, h, pitch, pfs, upb, upfs, npx, npy, Ub, ufs, plane, ps,
                        stride, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <typename T, int NC>
__global__ void __launch_bounds__(256)
seg_densify_kernel(const __grid_constant__ SegTable<SegDensify> tab)
{
    int b;
    const SegDensify &a = seg_of(tab, b);
    const int r = b / a.gx;
    densify_body<T, NC>((const T *)a.I0, (const T *)a.I1, a.w, a.h, a.pitch, a.pfs, a.up, a.upfs,
                        a.npx, a.npy, a.U, a.ufs, a.plane, a.ps, a.stride, b % a.gx, r % a.gy,
                        r / a.gy);
}

// ---------------------------------------------------------------- A8
// Work planes (each lv.plane floats) of one frame.
enum { kW1 = 0, kA11, kA12, kA22, kB1, kB2, kAS, kDU, kDV, kWorkPlanes };

template <typename T>
__global__ void warp_kernel(const T *__restrict__ I1b, int w, int h, int pitch, size_t pfs,
                            const float *__restrict__ Ub, size_t ufs, size_t plane,
                            float *__restrict__ workb, size_t wfs)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= w || y >= h) return;
    const int f = blockIdx.z;
    const float *U = Ub + (size_t)f * ufs;
    const size_t p = (size_t)y * pitch + x;
    workb[(size_t)f * wfs + kW1 * plane + p] =
        bilinear(I1b + (size_t)f * pfs, w, h, pitch, (float)x + U[p], (float)y + U[plane + p]);
}

template <typename T>
__global__ void coeff_kernel(const T *__restrict__ I0b, const T *__restrict__ I0xb,
                             const T *__restrict__ I0yb, int w, int h, int pitch, size_t pfs,
                             const float *__restrict__ Ub, size_t ufs, size_t plane,
                             float *__restrict__ workb, size_t wfs, float delta, float gamma,
                             float alpha_s)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= w || y >= h) return;
    const int f = blockIdx.z;
    float *wk = workb + (size_t)f * wfs;
    const float *W1 = wk + kW1 * plane;
    const float *U = Ub + (size_t)f * ufs;
    auto at = [&](int xx, int yy) { return W1[(size_t)yy * pitch + xx]; };
    auto dx = [&](int xx, int yy) {
        return 0.5f * (at(min(xx + 1, w - 1), yy) - at(max(xx - 1, 0), yy));
    };
    auto dy = [&](int xx, int yy) {
        return 0.5f * (at(xx, min(yy + 1, h - 1)) - at(xx, max(yy - 1, 0)));
    };
    const int xp = min(x + 1, w - 1), xm = max(x - 1, 0);
    const int yp = min(y + 1, h - 1), ym = max(y - 1, 0);
    const size_t p = (size_t)y * pitch + x;
    const float Ix = dx(x, y), Iy = dy(x, y);
    const float Ixx = 0.5f * (dx(xp, y) - dx(xm, y));
    const float Ixy = 0.5f * (dx(x, yp) - dx(x, ym));
    const float Iyy = 0.5f * (dy(x, yp) - dy(x, ym));
    const size_t fo = (size_t)f * pfs;
    const float Iz = at(x, y) - ldp(&I0b[fo + p]);
    const float Ixz = Ix - ldp(&I0xb[fo + p]);
    const float Iyz = Iy - ldp(&I0yb[fo + p]);
    const float nd = 1.0f / (Ix * Ix + Iy * Iy + kZeta2);
    const float ng = 1.0f / (Ixx * Ixx + 2.0f * Ixy * Ixy + Iyy * Iyy + kZeta2);
    float ad = delta * nd * psi_prime(nd * Iz * Iz);
    float ag = gamma * ng * psi_prime(ng * (Ixz * Ixz + Iyz * Iyz));
    const float u = U[p], v = U[plane + p];
    const float wx = (float)x + u, wy = (float)y + v;
    if (wx < 0.0f || wx > (float)(w - 1) || wy < 0.0f || wy > (float)(h - 1)) { ad = 0.0f; ag = 0.0f; }
    const float ux = x + 1 < w ? U[p + 1] - u : 0.0f;
    const float uy = y + 1 < h ? U[p + pitch] - u : 0.0f;
    const float vx = x + 1 < w ? U[plane + p + 1] - v : 0.0f;
    const float vy = y + 1 < h ? U[plane + p + pitch] - v : 0.0f;
    wk[kA11 * plane + p] = ad * Ix * Ix + ag * (Ixx * Ixx + Ixy * Ixy);
    wk[kA12 * plane + p] = ad * Ix * Iy + ag * (Ixx * Ixy + Ixy * Iyy);
    wk[kA22 * plane + p] = ad * Iy * Iy + ag * (Ixy * Ixy + Iyy * Iyy);
    wk[kB1 * plane + p] = -ad * Ix * Iz - ag * (Ixx * Ixz + Ixy * Iyz);
    wk[kB2 * plane + p] = -ad * Iy * Iz - ag * (Ixy * Ixz + Iyy * Iyz);
    wk[kAS * plane + p] = alpha_s * psi_prime(ux * ux + uy * uy + vx * vx + vy * vy);
    wk[kDU * plane + p] = 0.0f;
    wk[kDV * plane + p] = 0.0f;
}

// One red-black half sweep: pixels with (x + y) & 1 == colour.
__global__ void sor_kernel(int w, int h, int pitch, const float *__restrict__ Ub, size_t ufs,
                           size_t plane, float *__restrict__ workb, size_t wfs, int colour,
                           float omega)
{
    const int xh = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int x = 2 * xh + ((y + colour) & 1);
    if (x >= w || y >= h) return;
    const int f = blockIdx.z;
    float *wk = workb + (size_t)f * wfs;
    const float *U = Ub + (size_t)f * ufs;
    const float *as = wk + kAS * plane;
    float *du = wk + kDU * plane, *dv = wk + kDV * plane;
    const size_t p = (size_t)y * pitch + x;
    const float asp = as[p], up = U[p], vp = U[plane + p];
    float sw = 0.0f, su = 0.0f, sv = 0.0f;
    auto nb = [&](size_t q) {
        const float wn = 0.5f * (asp + as[q]);
        sw += wn;
        su += wn * (U[q] + du[q] - up);
        sv += wn * (U[plane + q] + dv[q] - vp);
    };
    if (x > 0) nb(p - 1);
    if (x + 1 < w) nb(p + 1);
    if (y > 0) nb(p - pitch);
    if (y + 1 < h) nb(p + pitch);
    const float a11 = wk[kA11 * plane + p] + sw, a12 = wk[kA12 * plane + p];
    const float a22 = wk[kA22 * plane + p] + sw;
    const float r1 = su + wk[kB1 * plane + p], r2 = sv + wk[kB2 * plane + p];
    float d1 = du[p], d2 = dv[p];
    if (a11 > 0.0f) d1 = (1.0f - omega) * d1 + omega * (r1 - a12 * d2) / a11;
    if (a22 > 0.0f) d2 = (1.0f - omega) * d2 + omega * (r2 - a12 * d1) / a22;
    du[p] = d1;
    dv[p] = d2;
}

__global__ void add_kernel(int w, int h, int pitch, float *__restrict__ Ub, size_t ufs,
                           size_t plane, const float *__restrict__ workb, size_t wfs)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= w || y >= h) return;
    const int f = blockIdx.z;
    float *U = Ub + (size_t)f * ufs;
    const float *wk = workb + (size_t)f * wfs;
    const size_t p = (size_t)y * pitch + x;
    U[p] += wk[kDU * plane + p];
    U[plane + p] += wk[kDV * plane + p];
}

// bx: the block of 256 pixels of row y, f: the frame.
__device__ __forceinline__ void flow_out_body(const float *__restrict__ Ub, int W, int H,
                                              int pitch, size_t ufs, size_t plane,
                                              float *__restrict__ flow, unsigned bx, unsigned y,
                                              unsigned f)
{
    const int x = bx * 256 + threadIdx.x;
    if (x >= W) return;
    const float *U = Ub + (size_t)f * ufs;
    const size_t o = (size_t)f * 2 * W * H + (size_t)y * W + x;
    flow[o] = U[(size_t)y * pitch + x];
    flow[o + (size_t)W * H] = U[plane + (size_t)y * pitch + x];
}

__global__ void flow_out_kernel(const float *__restrict__ Ub, int W, int H, int pitch,
                                size_t ufs, size_t plane, float *__restrict__ flow)
{
    flow_out_body(Ub, W, H, pitch, ufs, plane, flow, blockIdx.x, blockIdx.y, blockIdx.z);
}

__global__ void __launch_bounds__(256)
seg_flow_out_kernel(const __grid_constant__ SegTable<SegFlowOut> tab)
{
    int b;
    const SegFlowOut &a = seg_of(tab, b);
    const int r = b / a.gx;
    flow_out_body(a.U, a.W, a.H, a.pitch, a.ufs, a.plane, a.flow, b % a.gx, r % a.H, r / a.H);
}

// Same as flow_out_kernel, with frame f's destination read from dst[f] in
// device memory (so a captured graph writes each call's flow to the caller's
// buffers).
__global__ void flow_out_ptr_kernel(const float *__restrict__ U, int W, int H, int pitch,
                                    size_t plane, size_t u_frame_stride, float *const *dst)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    float *flow = dst[blockIdx.z];
    const float *Ub = U + (size_t)blockIdx.z * u_frame_stride;
    const size_t o = (size_t)y * W + x;
    flow[o] = Ub[(size_t)y * pitch + x];
    flow[o + (size_t)W * H] = Ub[plane + (size_t)y * pitch + x];
}

template <int PS, typename T>
void search_ps(const T *I0, const T *I0x, const T *I0y, const T *I1,
               const Level &lv, size_t pfs, const float *Uc, const Level *lvc, size_t ucfs,
               float *up, size_t upfs, int frames, const FlowParams &fp, int *err, cudaStream_t st)
{
    using SS = SearchShape<PS>;
    const int np = lv.npx * lv.npy;
    const bool wide = search_wide(np);
    const int G = wide ? SS::kWideCG * SS::kWideRG : SS::kNarrowCG * SS::kNarrowRG;
    const int per_block = 128 / G;
    dim3 grd((np + per_block - 1) / per_block, frames);
    auto kern = wide ? patch_search_kernel<PS, SS::kWideCG, SS::kWideRG, T>
                     : patch_search_kernel<PS, SS::kNarrowCG, SS::kNarrowRG, T>;
    kern<<<grd, 128, 0, st>>>(
        I0, I0x, I0y, I1, lv.w, lv.h, lv.pitch, pfs, lv.npx, lv.npy, Uc, lvc ? lvc->w : 0,
        lvc ? lvc->h : 0, lvc ? lvc->pitch : 0, lvc ? lvc->plane : 0, ucfs, up, upfs, fp.stride,
        fp.gn_iters, fp.gn_damping, err);
}

dim3 grid2d(int w, int h, int frames, dim3 blk)
{
    return dim3((w + blk.x - 1) / blk.x, (h + blk.y - 1) / blk.y, frames);
}

}  // namespace

void init_flow_attributes() { init_var_attributes(); }

PyrDesc make_pyr_desc(const Geometry &geo)
{
    PyrDesc d = {};
    d.levels = std::max(geo.levels, 1);
    int nb = 0;
    for (int l = 0; l < d.levels; ++l) {
        const Level &lv = geo.lv[l];
        d.w[l] = lv.w;
        d.h[l] = lv.h;
        d.pitch[l] = lv.pitch;
        d.off[l] = geo.pyr_off[l];
        d.plane[l] = lv.plane;
        d.blk0[l] = nb;
        nb += ((lv.w + 31) / 32) * ((lv.h + 7) / 8);
    }
    d.blk0[d.levels] = nb;
    d.gb0 = d.levels > 1 ? d.blk0[1] : 0;  // level 0's gradients come with the box means
    return d;
}

void launch_pyramid(void *slots, const Geometry &geo, size_t frame_stride, int frames, bool half,
                    cudaStream_t st)
{
    const PyrDesc d = make_pyr_desc(geo);
    const int nb = d.blk0[d.levels] - d.gb0;
    const int extra = std::max(0, d.levels - kPyrFused);
    StageScope sc(kStPyramid, 1 + (d.levels > 1 ? 1 : 0) + extra, st);
    const dim3 blk(32, 8);
    const size_t es = half ? 2 : 4;
    if (d.levels > 1) {
        // tiles over the whole of level 0 (an odd last column or row of level 0
        // lies past level 1's tiles when the width or height is 64k + 1)
        const dim3 grd((d.w[0] + 2 * kPyrTile - 1) / (2 * kPyrTile),
                       (d.h[0] + 2 * kPyrTile - 1) / (2 * kPyrTile), frames);
        if (half)
            pyramid_means_kernel<__half><<<grd, blk, 0, st>>>((__half *)slots, frame_stride, d);
        else
            pyramid_means_kernel<float><<<grd, blk, 0, st>>>((float *)slots, frame_stride, d);
    }
    for (int l = kPyrFused; l < d.levels; ++l) {  // levels beyond the fused tile
        char *base = (char *)slots;
        const dim3 grd = grid2d(d.w[l], d.h[l], frames, blk);
        if (half)
            downsample_kernel<__half><<<grd, blk, 0, st>>>(
                (const __half *)(base + d.off[l - 1] * es), d.pitch[l - 1],
                (__half *)(base + d.off[l] * es), d.w[l], d.h[l], d.pitch[l], frame_stride);
        else
            downsample_kernel<float><<<grd, blk, 0, st>>>(
                (const float *)(base + d.off[l - 1] * es), d.pitch[l - 1],
                (float *)(base + d.off[l] * es), d.w[l], d.h[l], d.pitch[l], frame_stride);
    }
    const dim3 ggrd(nb, 1, frames);
    if (half)
        pyramid_gradients_kernel<__half><<<ggrd, blk, 0, st>>>((__half *)slots, frame_stride, d);
    else
        pyramid_gradients_kernel<float><<<ggrd, blk, 0, st>>>((float *)slots, frame_stride, d);
}

void launch_pyramid_export(const void *plane, bool half, int w, int h, int pitch, float *dst,
                           cudaStream_t st)
{
    const dim3 blk(32, 8), grd((w + 31) / 32, (h + 7) / 8);
    if (half)
        pyramid_export_kernel<__half><<<grd, blk, 0, st>>>((const __half *)plane, w, h, pitch, dst);
    else
        pyramid_export_kernel<float><<<grd, blk, 0, st>>>((const float *)plane, w, h, pitch, dst);
}

template <typename T>
void launch_patch_search_t(const T *I0, const T *I0x, const T *I0y, const T *I1,
                           const Level &lv, size_t pyr_frame_stride, const float *Uc,
                           const Level *lvc, size_t uc_frame_stride, float *up,
                           size_t up_frame_stride, int frames, const FlowParams &fp, int *err,
                           cudaStream_t st)
{
#define EBOF_PS(N)                                                                              \
    case N:                                                                                     \
        search_ps<N, T>(I0, I0x, I0y, I1, lv, pyr_frame_stride, Uc, lvc, uc_frame_stride, up,   \
                        up_frame_stride, frames, fp, err, st);                                  \
        break;
    switch (fp.ps) {
        EBOF_PS(4) EBOF_PS(5) EBOF_PS(6) EBOF_PS(7) EBOF_PS(8) EBOF_PS(9) EBOF_PS(10)
        EBOF_PS(11) EBOF_PS(12) EBOF_PS(13) EBOF_PS(14) EBOF_PS(15) EBOF_PS(16)
        default: break;
    }
#undef EBOF_PS
}

void launch_patch_search(const void *I0, const void *I0x, const void *I0y, const void *I1,
                         const Level &lv, size_t pyr_frame_stride, const float *Uc,
                         const Level *lvc, size_t uc_frame_stride, float *up,
                         size_t up_frame_stride, int frames, const FlowParams &fp, int *err,
                         cudaStream_t st)
{
    if (lv.npx * lv.npy <= 0) return;
    StageScope sc(kStSearch, 1, st);
    if (fp.half)
        launch_patch_search_t((const __half *)I0, (const __half *)I0x, (const __half *)I0y,
                              (const __half *)I1, lv, pyr_frame_stride, Uc, lvc, uc_frame_stride,
                              up, up_frame_stride, frames, fp, err, st);
    else
        launch_patch_search_t((const float *)I0, (const float *)I0x, (const float *)I0y,
                              (const float *)I1, lv, pyr_frame_stride, Uc, lvc, uc_frame_stride,
                              up, up_frame_stride, frames, fp, err, st);
}

void launch_densify(const void *I0, const void *I1, const Level &lv, size_t pyr_frame_stride,
                    const float *up, size_t up_frame_stride, float *U, size_t u_frame_stride,
                    int frames, const FlowParams &fp, cudaStream_t st)
{
    StageScope sc(kStDensify, 1, st);
    dim3 blk(32, 8);
    const dim3 grd = grid2d(lv.w, lv.h, frames, blk);
    // regular patches covering a pixel per axis: at most ceil(ps / stride)
    const int nc = (fp.ps + fp.stride - 1) / fp.stride;
#define EBOF_DENSE(T, N)                                                                         \
    densify_kernel<T, N><<<grd, blk, 0, st>>>((const T *)I0, (const T *)I1, lv.w, lv.h,         \
                                              lv.pitch, pyr_frame_stride, up, up_frame_stride,   \
                                              lv.npx, lv.npy, U, u_frame_stride, lv.plane, fp.ps,\
                                              fp.stride)
    if (fp.half) {
        if (nc == 2) EBOF_DENSE(__half, 2);
        else if (nc == 3) EBOF_DENSE(__half, 3);
        else if (nc == 4) EBOF_DENSE(__half, 4);
        else EBOF_DENSE(__half, 0);
    } else {
        if (nc == 2) EBOF_DENSE(float, 2);
        else if (nc == 3) EBOF_DENSE(float, 3);
        else if (nc == 4) EBOF_DENSE(float, 4);
        else EBOF_DENSE(float, 0);
    }
#undef EBOF_DENSE
}

template <typename T>
void variational_steps(const T *I0, const T *I0x, const T *I0y, const T *I1, const Level &lv,
                       size_t pyr_frame_stride, float *U, size_t u_frame_stride, float *work,
                       size_t work_frame_stride, int frames, const FlowParams &fp,
                       cudaStream_t st)
{
    dim3 blk(32, 8);
    const dim3 grd = grid2d(lv.w, lv.h, frames, blk);
    const dim3 grd_half = grid2d((lv.w + 1) / 2, lv.h, frames, blk);
    for (int k = 0; k < fp.var_outer; ++k) {
        {
            StageScope sc(kStVarWarp, 1, st);
            warp_kernel<T><<<grd, blk, 0, st>>>(I1, lv.w, lv.h, lv.pitch, pyr_frame_stride, U,
                                                u_frame_stride, lv.plane, work, work_frame_stride);
        }
        {
            StageScope sc(kStVarCoeff, 1, st);
            coeff_kernel<T><<<grd, blk, 0, st>>>(I0, I0x, I0y, lv.w, lv.h, lv.pitch,
                                                 pyr_frame_stride, U, u_frame_stride, lv.plane,
                                                 work, work_frame_stride, fp.delta, fp.gamma,
                                                 fp.alpha_s);
        }
        if (fp.var_sor > 0) {
            StageScope sc(kStVarSor, 2 * fp.var_sor, st);
            for (int s = 0; s < fp.var_sor; ++s)
                for (int colour = 0; colour < 2; ++colour)
                    sor_kernel<<<grd_half, blk, 0, st>>>(lv.w, lv.h, lv.pitch, U, u_frame_stride,
                                                         lv.plane, work, work_frame_stride,
                                                         colour, fp.omega);
        }
        {
            StageScope sc(kStVarAdd, 1, st);
            add_kernel<<<grd, blk, 0, st>>>(lv.w, lv.h, lv.pitch, U, u_frame_stride, lv.plane,
                                            work, work_frame_stride);
        }
    }
}

float *launch_variational(const void *I0, const void *I0x, const void *I0y, const void *I1,
                          const Level &lv, size_t pyr_frame_stride, float *U, float *Utmp,
                          size_t u_frame_stride, float *work, size_t work_frame_stride,
                          int frames, const FlowParams &fp, const CUtensorMap *coef_map,
                          int *err, cudaStream_t st)
{
    if (fp.var_outer <= 0) return U;
    if (var_fused_supported(fp.var_sor))
        return launch_variational_fused(I0, I0x, I0y, I1, lv, pyr_frame_stride, U, Utmp,
                                        u_frame_stride, work, frames, fp, coef_map, err, st);
    // many sweeps: one launch per step, state in global memory
    if (fp.half)
        variational_steps((const __half *)I0, (const __half *)I0x, (const __half *)I0y,
                          (const __half *)I1, lv, pyr_frame_stride, U, u_frame_stride, work,
                          work_frame_stride, frames, fp, st);
    else
        variational_steps((const float *)I0, (const float *)I0x, (const float *)I0y,
                          (const float *)I1, lv, pyr_frame_stride, U, u_frame_stride, work,
                          work_frame_stride, frames, fp, st);
    return U;
}

bool search_wide(int n_patches) { return n_patches >= kWideSearchPatches; }

int search_patches_per_block(int ps, bool wide)
{
    int G = 0;
#define EBOF_G(N)                                                                                \
    case N:                                                                                      \
        G = wide ? SearchShape<N>::kWideCG * SearchShape<N>::kWideRG                             \
                 : SearchShape<N>::kNarrowCG * SearchShape<N>::kNarrowRG;                          \
        break;
    switch (ps) {
        EBOF_G(4) EBOF_G(5) EBOF_G(6) EBOF_G(7) EBOF_G(8) EBOF_G(9) EBOF_G(10) EBOF_G(11)
        EBOF_G(12) EBOF_G(13) EBOF_G(14) EBOF_G(15) EBOF_G(16)
        default: break;
    }
#undef EBOF_G
    return G > 0 ? 128 / G : 0;
}

void launch_seg_pyr_means(const SegTable<SegPyr> &t, int blocks, bool half, cudaStream_t st)
{
    StageScope sc(kStPyramid, 1, st);
    if (half) seg_pyramid_means_kernel<__half><<<blocks, dim3(32, 8), 0, st>>>(t);
    else seg_pyramid_means_kernel<float><<<blocks, dim3(32, 8), 0, st>>>(t);
}

void launch_seg_pyr_grads(const SegTable<SegPyr> &t, int blocks, bool half, cudaStream_t st)
{
    StageScope sc(kStPyramid, 1, st);
    if (half) seg_pyramid_gradients_kernel<__half><<<blocks, dim3(32, 8), 0, st>>>(t);
    else seg_pyramid_gradients_kernel<float><<<blocks, dim3(32, 8), 0, st>>>(t);
}

int seg_max_levels() { return kPyrFused; }

void launch_seg_search(const SegTable<SegSearch> &t, int blocks, int ps, bool wide, bool half,
                       cudaStream_t st)
{
    StageScope sc(kStSearch, 1, st);
#define EBOF_SPS(N)                                                                              \
    case N: {                                                                                    \
        using SS = SearchShape<N>;                                                               \
        if (half)                                                                                \
            (wide ? seg_patch_search_kernel<N, SS::kWideCG, SS::kWideRG, __half>                 \
                  : seg_patch_search_kernel<N, SS::kNarrowCG, SS::kNarrowRG, __half>)            \
                <<<blocks, 128, 0, st>>>(t);                                                     \
        else                                                                                     \
            (wide ? seg_patch_search_kernel<N, SS::kWideCG, SS::kWideRG, float>                  \
                  : seg_patch_search_kernel<N, SS::kNarrowCG, SS::kNarrowRG, float>)             \
                <<<blocks, 128, 0, st>>>(t);                                                     \
        break;                                                                                   \
    }
    switch (ps) {
        EBOF_SPS(4) EBOF_SPS(5) EBOF_SPS(6) EBOF_SPS(7) EBOF_SPS(8) EBOF_SPS(9) EBOF_SPS(10)
        EBOF_SPS(11) EBOF_SPS(12) EBOF_SPS(13) EBOF_SPS(14) EBOF_SPS(15) EBOF_SPS(16)
        default: break;
    }
#undef EBOF_SPS
}

void launch_seg_densify(const SegTable<SegDensify> &t, int blocks, int nc, bool half,
                        cudaStream_t st)
{
    StageScope sc(kStDensify, 1, st);
    const dim3 blk(32, 8);
#define EBOF_SDENSE(T, N) seg_densify_kernel<T, N><<<blocks, blk, 0, st>>>(t)
    if (half) {
        if (nc == 2) EBOF_SDENSE(__half, 2);
        else if (nc == 3) EBOF_SDENSE(__half, 3);
        else if (nc == 4) EBOF_SDENSE(__half, 4);
        else EBOF_SDENSE(__half, 0);
    } else {
        if (nc == 2) EBOF_SDENSE(float, 2);
        else if (nc == 3) EBOF_SDENSE(float, 3);
        else if (nc == 4) EBOF_SDENSE(float, 4);
        else EBOF_SDENSE(float, 0);
    }
#undef EBOF_SDENSE
}

void launch_seg_flow_out(const SegTable<SegFlowOut> &t, int blocks, cudaStream_t st)
{
    StageScope sc(kStFlowOut, 1, st);
    seg_flow_out_kernel<<<blocks, 256, 0, st>>>(t);
}

void launch_flow_out_ptr(const float *U, int W, int H, int pitch, size_t u_frame_stride,
                         float *const *dst, int frames, cudaStream_t st)
{
    StageScope sc(kStFlowOut, 1, st);
    dim3 grd((W + 255) / 256, H, frames);
    flow_out_ptr_kernel<<<grd, 256, 0, st>>>(U, W, H, pitch, (size_t)pitch * H, u_frame_stride,
                                             dst);
}

void launch_flow_out(const float *U, int W, int H, int pitch, size_t u_frame_stride,
                     float *flow, int frames, cudaStream_t st)
{
    StageScope sc(kStFlowOut, 1, st);
    dim3 grd((W + 255) / 256, H, frames);
    flow_out_kernel<<<grd, 256, 0, st>>>(U, W, H, pitch, u_frame_stride,
                                         (size_t)pitch * H, flow);
}

}  // namespace ebof
