// k_front.cu -- event accumulation, denoising/filling, exact EDT, surface.
//
// §III-A: edge image of a window.  §III-B: Alg. 1 (denoise) then Alg. 2
// (fill).  §III-C: exact Euclidean distance transform as int32 squared
// distances (separable: a per-column pass, then a per-row lower envelope of
// parabolas), fused with Eq. 1, d_exp = 1 - exp(-sqrt(D) / alpha), and the
// 8-bit intensity scale 255 * d_exp the flow block runs on.
#include "ebof.h"
#include "ebof_internal.cuh"
#include "profiler.cuh"

#include <cuda_fp16.h>

#include <algorithm>

namespace ebof {

namespace {

// ---------------------------------------------------------------- A1 scatter
// One thread per event.  The window index of an event is
// floor((t - t_begin) / dt) when it lies in [0, n_windows); duplicates collapse
// (a byte store of 1 is idempotent).  Counters are aggregated per warp over
// lanes that share a window, so sorted event streams cost one atomic per warp.
__global__ void scatter_kernel(const uint16_t *__restrict__ x, const uint16_t *__restrict__ y,
                               const int64_t *__restrict__ t, int64_t n, int64_t t_begin,
                               int64_t dt, int n_windows, int W, int H, int pitch,
                               uint8_t *__restrict__ E, size_t fstride, DevStats *stats,
                               unsigned long long *dropped_time)
{
    const int64_t span = dt * (int64_t)n_windows;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        int k = -2;  // -2: no event (tail), -1: outside every window
        bool oob = false;
        if (i < n) {
            const int64_t rel = t[i] - t_begin;
            k = -1;
            if (rel >= 0 && rel < span) {
                k = (int)(rel / dt);
                const int xi = x[i], yi = y[i];
                if (xi < W && yi < H)
                    E[(size_t)k * fstride + (size_t)yi * pitch + xi] = 1;
                else
                    oob = true;
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, k);
        const unsigned oob_mask = __ballot_sync(0xffffffffu, oob);
        if (lane == __ffs(peers) - 1) {
            if (k >= 0) {
                atomicAdd(&stats[k].in_window, (unsigned long long)__popc(peers));
                const int no = __popc(peers & oob_mask);
                if (no) atomicAdd(&stats[k].dropped_oob, (unsigned long long)no);
            } else if (k == -1) {
                atomicAdd(dropped_time, (unsigned long long)__popc(peers));
            }
        }
    }
}

// Scatter for a group of streams: frame f takes the events of descriptor f.
__global__ void scatter_desc_kernel(const ebof_window_desc *__restrict__ desc, int W, int H,
                                    int pitch, uint8_t *__restrict__ E, size_t fstride,
                                    DevStats *stats, unsigned long long *dropped_time)
{
    const int f = blockIdx.y;
    const ebof_window_desc d = desc[f];
    const int lane = threadIdx.x & 31;
    uint8_t *e = E + (size_t)f * fstride;
    unsigned long long in_w = 0, oob = 0, out_t = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < d.n_events;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        if (i < d.n_events) {
            const int64_t tt = d.t[i];
            if (tt >= d.t_begin && tt < d.t_end) {
                ++in_w;
                const int xi = d.x[i], yi = d.y[i];
                if (xi < W && yi < H) e[(size_t)yi * pitch + xi] = 1;
                else ++oob;
            } else {
                ++out_t;
            }
        }
    }
    // warp sums, one atomic per warp and counter
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        in_w += __shfl_xor_sync(0xffffffffu, in_w, o);
        oob += __shfl_xor_sync(0xffffffffu, oob, o);
        out_t += __shfl_xor_sync(0xffffffffu, out_t, o);
    }
    if (lane == 0) {
        if (in_w) atomicAdd(&stats[f].in_window, in_w);
        if (oob) atomicAdd(&stats[f].dropped_oob, oob);
        if (out_t) atomicAdd(dropped_time, out_t);
    }
}

// ---------------------------------------------------------------- A2
// Alg. 1 then Alg. 2 in one pass: a block stages E for its 32 x 8 tile plus
// a 2-pixel halo in shared memory, denoises the tile plus 1 pixel there
// (counts in E), then fills the tile (counts in the denoised image).
// Neighbours outside the image count as non-edge in both, as in
// count_neighbours, so the result equals denoise_kernel then fill_kernel.
constexpr int kDfX = 32, kDfY = 8;

__device__ __forceinline__ int count_tile(const uint8_t (*t)[kDfX + 4], int lx, int ly, int conn)
{
    int c = t[ly - 1][lx] + t[ly + 1][lx] + t[ly][lx - 1] + t[ly][lx + 1];
    if (conn == 8) c += t[ly - 1][lx - 1] + t[ly - 1][lx + 1] + t[ly + 1][lx - 1] + t[ly + 1][lx + 1];
    return c;
}

__global__ void __launch_bounds__(kDfX * kDfY)
denoise_fill_kernel(const uint8_t *__restrict__ E, uint8_t *__restrict__ Edf, int W, int H,
                    int pitch, size_t fstride, int conn, int n_d, int n_f,
                    uint8_t *__restrict__ export_dense, DevStats *stats)
{
    __shared__ uint8_t sE[kDfY + 4][kDfX + 4];
    __shared__ uint8_t sD[kDfY + 4][kDfX + 4];  // denoised, 1-pixel ring inside a 2-pixel frame
    const int f = blockIdx.z;
    const uint8_t *e = E + (size_t)f * fstride;
    const int x0 = blockIdx.x * kDfX - 2, y0 = blockIdx.y * kDfY - 2;
    const int t = threadIdx.y * kDfX + threadIdx.x;
    for (int i = t; i < (kDfX + 4) * (kDfY + 4); i += kDfX * kDfY) {
        const int lx = i % (kDfX + 4), ly = i / (kDfX + 4);
        const int gx = x0 + lx, gy = y0 + ly;
        uint8_t v = 0;
        if (gx >= 0 && gy >= 0 && gx < W && gy < H) v = e[(size_t)gy * pitch + gx] ? 1 : 0;
        sE[ly][lx] = v;
        sD[ly][lx] = 0;
    }
    __syncthreads();
    for (int i = t; i < (kDfX + 2) * (kDfY + 2); i += kDfX * kDfY) {
        const int lx = 1 + i % (kDfX + 2), ly = 1 + i / (kDfX + 2);
        uint8_t v = sE[ly][lx];
        if (v && count_tile(sE, lx, ly, conn) < n_d) v = 0;
        sD[ly][lx] = v;
    }
    __syncthreads();
    const int x = blockIdx.x * kDfX + threadIdx.x, y = blockIdx.y * kDfY + threadIdx.y;
    uint8_t v = 0;
    if (x < W && y < H) {
        const int lx = threadIdx.x + 2, ly = threadIdx.y + 2;
        v = sD[ly][lx];
        if (!v && count_tile(sD, lx, ly, conn) >= n_f) v = 1;
        Edf[(size_t)f * fstride + (size_t)y * pitch + x] = v;
        if (export_dense) export_dense[(size_t)f * W * H + (size_t)y * W + x] = v;
    }
    const unsigned m = __ballot_sync(0xffffffffu, v != 0);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&stats[f].edge_px, (unsigned long long)__popc(m));
}

// ---------------------------------------------------------------- A3
// Column pass: g(x, y) = distance to the nearest edge pixel in column x, or
// G_INF = W + H for a column without any (larger than any in-image
// distance).  A block covers 32 columns; thread (c, k) owns column c's
// chunk k of CH rows (CH a multiple of 32, at most 512).  It packs its
// chunk into bit masks, publishes the first and last edge row of the chunk,
// and after one barrier finds, for each row, the nearest edge pixel above
// (highest set bit at or above the row, else the previous chunks) and below
// (lowest set bit at or below, else the next chunks) with bit scans.  Row
// writes of a warp are 32 consecutive int32.
constexpr int kColMaxWords = 16;   // CH <= 512 rows
constexpr int kColMaxChunks = 32;  // chunks per column

__global__ void __launch_bounds__(1024)
edt_cols_kernel(const uint8_t *__restrict__ E, int epitch, size_t efs, int W, int H,
                int32_t *__restrict__ g, int gpitch, size_t gfs, int CH)
{
    __shared__ int s_first[kColMaxChunks][32], s_last[kColMaxChunks][32];
    const int c = threadIdx.x, k = threadIdx.y, nch = blockDim.y;
    const int x = blockIdx.x * 32 + c;
    const bool colok = x < W;
    const uint8_t *e = E + (size_t)blockIdx.y * efs;
    const int y0 = k * CH, y1 = min(H, y0 + CH);
    const int nw = (CH + 31) / 32;
    unsigned mask[kColMaxWords];
    int first = -1, last = -1;
#pragma unroll
    for (int wi = 0; wi < kColMaxWords; ++wi) {
        unsigned m = 0;
        if (wi < nw && colok) {
            for (int b = 0; b < 32; ++b) {
                const int y = y0 + wi * 32 + b;
                if (y < y1 && e[(size_t)y * epitch + x]) m |= 1u << b;
            }
        }
        mask[wi] = m;
        if (m) {
            if (first < 0) first = y0 + wi * 32 + __ffs(m) - 1;
            last = y0 + wi * 32 + 31 - __clz(m);
        }
    }
    s_first[k][c] = first;
    s_last[k][c] = last;
    __syncthreads();
    if (!colok || y0 >= H) return;
    int above = -1, below = -1;
    for (int j = k - 1; j >= 0; --j)
        if (s_last[j][c] >= 0) { above = s_last[j][c]; break; }
    for (int j = k + 1; j < nch; ++j)
        if (s_first[j][c] >= 0) { below = s_first[j][c]; break; }
    const int ginf = W + H;
    int32_t *gc = g + (size_t)blockIdx.y * gfs + x;
    int run_above = above;  // nearest edge row before word wi
#pragma unroll
    for (int wi = 0; wi < kColMaxWords; ++wi) {
        if (wi >= nw) break;
        int next_first = below;  // nearest edge row after word wi
#pragma unroll
        for (int wj = kColMaxWords - 1; wj > wi; --wj)
            if (wj < nw && mask[wj]) next_first = y0 + wj * 32 + __ffs(mask[wj]) - 1;
        const unsigned m = mask[wi];
        for (int b = 0; b < 32; ++b) {
            const int y = y0 + wi * 32 + b;
            if (y >= y1) break;
            const unsigned up = m & (0xffffffffu >> (31 - b));  // bits 0..b
            const unsigned dn = m & (0xffffffffu << b);         // bits b..31
            const int a = up ? y0 + wi * 32 + 31 - __clz(up) : run_above;
            const int bl = dn ? y0 + wi * 32 + __ffs(dn) - 1 : next_first;
            int d = ginf;
            if (a >= 0) d = y - a;
            if (bl >= 0 && bl - y < d) d = bl - y;
            gc[(size_t)y * gpitch] = d;
        }
        if (m) run_above = y0 + wi * 32 + 31 - __clz(m);
    }
}

// ---------------------------------------------------------------- A4
// Row pass: D(x) = min over columns x' of (x - x')^2 + h(x'), h(x') =
// g(x', y)^2 -- the lower envelope of the row's parabolas, evaluated at every
// pixel.  WPR warps serve one row; the row is cut into NB = 32 * WPR bands of
// B = ceil(W / NB) columns, one band per lane.
//  1. The row's h is staged in shared memory (-1: column without edge pixels).
//  2. Each lane builds the lower envelope of its band's parabolas (the stack
//     construction of the separable exact EDT; breakpoints compared exactly
//     in 64-bit integers).
//  3. Each lane walks its band's pixels left to right.  For every band within
//     NEAR bands it keeps a pointer into that band's envelope and moves it
//     forward while the next parabola is not higher at x; since the owner of x
//     within one envelope never moves left as x grows, the walk costs O(1) per
//     pixel on average.  Farther bands are visited (nearest first, binary
//     search for the owner) only while their distance^2 is below the best
//     value so far.
//  4. Eq. 1 and the 8-bit scale, with coalesced stores.
// Every step is an exact integer minimum, so D is bit-identical to any exact
// EDT, whatever WPR and NEAR: single windows use twice the warps per row
// (half the pixels per lane) to cut latency, batches the narrower layout.

// With sites a < b < c on an envelope, is b hidden once c arrives?
// Breakpoint s(p, q) = ((h_q + q^2) - (h_p + p^2)) / (2 (q - p)) for p < q;
// b is hidden iff s(b, c) <= s(a, b).
__device__ __forceinline__ bool hidden(int a, int b, int c, const int32_t *h)
{
    const long long fa = (long long)h[a] + (long long)a * a;
    const long long fb = (long long)h[b] + (long long)b * b;
    const long long fc = (long long)h[c] + (long long)c * c;
    return (fc - fb) * (long long)(b - a) <= (fb - fa) * (long long)(c - b);
}

// (x - site)^2 + h(site) < 2^29 for images up to 16384 px a side.
__device__ __forceinline__ int para(int x, int site, const int32_t *h)
{
    const int d = x - site;
    return d * d + h[site];
}

__host__ __device__ __forceinline__ size_t rows_smem_words(int W, int wpr)
{
    return 3 * (size_t)W + 2 * 32 * (size_t)wpr + 1;
}

// Level-0 intensity of the flow block.  FP32 storage keeps I = 255 d_exp.
// FP16 storage keeps the complement C = 255 - I = 255 exp(-d / alpha): the
// flow is the same for I and 255 - I (mean-normalised patches, squared
// residuals and products of derivatives), and far from the edges, where I
// saturates towards 255 and its variations are far below FP16's 0.125 step
// there, C is small and keeps them at FP16's relative precision.
__device__ __forceinline__ void st_int(float *p, float s, float c) { (void)c; *p = 255.0f * s; }
__device__ __forceinline__ void st_int(__half *p, float s, float c)
{
    (void)s;
    *p = __float2half_rn(255.0f * c);
}

// The ablation surfaces are stored as gain * y itself (no complement); FP16
// clamps at its largest finite value, so distances beyond 65504 / gain
// (about 1540 px for DS_L) read as one plateau.
__device__ __forceinline__ void st_lin(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_lin(__half *p, float v)
{
    *p = __float2half_rn(fminf(v, 65504.0f));
}

// y(d) of the ablation surfaces of §IV-D (mode 1 DS_L, 2 DS_LB, 3 DS_Log).
__device__ __forceinline__ float ablation_surface(const SurfaceMap &sm, float d)
{
    return sm.mode == 1 ? d : (sm.mode == 2 ? fminf(d, sm.d_sat) : log1pf(d));
}

template <int WPR, int NEAR, typename T>
__global__ void edt_rows_surface_kernel(const int32_t *__restrict__ g, int gpitch, size_t gfs,
                                        int W, int H, int rows_per_block, SurfaceMap sm,
                                        int32_t *__restrict__ D_dense,
                                        float *__restrict__ S_dense, T *__restrict__ I0,
                                        int ipitch, size_t ifs)
{
    constexpr int NB = 32 * WPR;
    extern __shared__ int32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rib = warp / WPR, sub = warp % WPR;
    const int y = blockIdx.x * rows_per_block + rib;
    const int f = blockIdx.y;
    const bool valid = y < H;
    int32_t *h = smem + (size_t)rib * rows_smem_words(W, WPR);
    int32_t *stk = h + W;       // envelope sites, per band
    int32_t *res = stk + W;     // D per pixel of the row
    int32_t *cnts = res + W;    // envelope size per band
    int32_t *minh = cnts + NB;  // smallest h of the band's sites (a lower bound of its parabolas)
    int32_t *anyf = minh + NB;  // row has an edge pixel
    const int tr = sub * 32 + lane;  // thread index within the row
    const int ginf = W + H;
    if (tr == 0) *anyf = 0;
    __syncthreads();
    if (valid) {
        const int32_t *grow = g + (size_t)f * gfs + (size_t)y * gpitch;
        int any = 0;
        for (int x = tr; x < W; x += NB) {
            const int gv = grow[x];
            h[x] = gv >= ginf ? -1 : gv * gv;
            any |= gv < ginf ? 1 : 0;
        }
        if (any) *anyf = 1;  // benign race: every writer stores 1
    }
    __syncthreads();
    const bool any = valid && *anyf;

    const int B = (W + NB - 1) / NB;
    const int bi = tr;  // this lane's band
    const int a = min(W, bi * B), b = min(W, a + B);
    int cnt = 0, mh = 0x7fffffff;
    if (any) {
        for (int q = a; q < b; ++q) {
            if (h[q] < 0) continue;
            mh = min(mh, h[q]);
            while (cnt >= 2 && hidden(stk[a + cnt - 2], stk[a + cnt - 1], q, h)) --cnt;
            stk[a + cnt++] = q;
        }
    }
    if (valid) {
        cnts[bi] = cnt;
        minh[bi] = mh;
    }
    __syncthreads();

    if (any) {
        int ptr[2 * NEAR + 1];
#pragma unroll
        for (int k = 0; k <= 2 * NEAR; ++k) ptr[k] = 0;
        for (int x = a; x < b; ++x) {
            int best = 0x7fffffff;
#pragma unroll
            for (int k = 0; k <= 2 * NEAR; ++k) {
                const int M = bi + k - NEAR;
                if (M < 0 || M >= NB) continue;
                const int ma = min(W, M * B), mb = min(W, ma + B);
                const int cM = cnts[M];
                if (cM == 0) continue;
                const int gap = M < bi ? x - (mb - 1) : (M > bi ? ma - x : 0);
                // no parabola of band M is below gap^2 + its smallest h
                if (M != bi && gap * gap + minh[M] >= best) continue;
                const int32_t *sl = stk + ma;
                int pk = ptr[k];
                int cur = para(x, sl[pk], h);
                while (pk + 1 < cM) {
                    const int nxt = para(x, sl[pk + 1], h);
                    if (nxt > cur) break;
                    cur = nxt;
                    ++pk;
                }
                ptr[k] = pk;
                best = min(best, cur);
            }
            for (int dist = NEAR + 1; dist < NB; ++dist) {
                bool progress = false;
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    const int M = side ? bi + dist : bi - dist;
                    if (M < 0 || M >= NB) continue;
                    const int ma = min(W, M * B), mb = min(W, ma + B);
                    if (ma >= mb) continue;
                    const int gap = side ? ma - x : x - (mb - 1);  // < 2^14: gap^2 fits
                    if (gap * gap >= best) continue;
                    progress = true;
                    const int cM = cnts[M];
                    if (cM == 0 || gap * gap + minh[M] >= best) continue;
                    const int32_t *sl = stk + ma;
                    int lo = 0, hi = cM - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (para(x, sl[mid + 1], h) <= para(x, sl[mid], h)) lo = mid + 1;
                        else hi = mid;
                    }
                    best = min(best, para(x, sl[lo], h));
                }
                if (!progress) break;
            }
            res[x] = best;
        }
    }
    __syncthreads();

    if (!valid) return;
    T *irow = I0 ? I0 + (size_t)f * ifs + (size_t)y * ipitch : nullptr;
    const size_t dbase = (size_t)f * W * H + (size_t)y * W;
    for (int x = tr; x < W; x += NB) {
        const int32_t D = any ? res[x] : kInfD;
        float S = 1.0f, C = 0.0f;  // d_exp of Eq. 1 and its complement 1 - d_exp
        if (sm.mode == 0) {
            if (D != kInfD) {
                C = expf(-sqrtf((float)D) / sm.alpha);
                S = 1.0f - C;
            }
            if (irow) st_int(&irow[x], S, C);
        } else {
            // no edge pixel (kInfD): y at the finite d = sqrt(INT32_MAX)
            S = ablation_surface(sm, sqrtf((float)D));
            if (irow) st_lin(&irow[x], sm.gain * S);
        }
        if (D_dense) D_dense[dbase + x] = D;
        if (S_dense) S_dense[dbase + x] = S;
    }
}

// Caller-given surface (dense, d_exp in [0, 1]) to the level-0 intensity.
template <typename T>
__global__ void surface_to_intensity_kernel(const float *__restrict__ S, int W, int H,
                                            T *__restrict__ I0, int pitch, SurfaceMap sm)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const float sv = S[(size_t)y * W + x];
    if (sm.mode == 0)
        st_int(&I0[(size_t)y * pitch + x], sv, 1.0f - sv);
    else
        st_lin(&I0[(size_t)y * pitch + x], sm.gain * sv);
}

inline unsigned grid1d(int64_t n, int block, int cap)
{
    int64_t b = (n + block - 1) / block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

}  // namespace

void launch_scatter(const uint16_t *x, const uint16_t *y, const int64_t *t, int64_t n,
                    int64_t t_begin, int64_t dt, int n_windows, int W, int H, int pitch,
                    uint8_t *E, size_t frame_stride, DevStats *stats,
                    unsigned long long *dropped_time, cudaStream_t st)
{
    if (n <= 0) return;
    StageScope sc(kStScatter, 1, st);
    scatter_kernel<<<grid1d(n, 256, 152 * 16), 256, 0, st>>>(x, y, t, n, t_begin, dt, n_windows,
                                                             W, H, pitch, E, frame_stride, stats,
                                                             dropped_time);
}

void launch_scatter_desc(const ebof_window_desc *desc, int frames, int W, int H, int pitch,
                         uint8_t *E, size_t frame_stride, DevStats *stats,
                         unsigned long long *dropped_time, cudaStream_t st)
{
    StageScope sc(kStScatter, 1, st);
    // the event counts are read on the device: size the grid for the largest
    // windows (about 4 blocks per SM in all), blocks past a window's end exit
    dim3 grd(std::max(64, 608 / std::max(frames, 1)), frames);
    scatter_desc_kernel<<<grd, 256, 0, st>>>(desc, W, H, pitch, E, frame_stride, stats,
                                             dropped_time);
}

void launch_denoise_fill(const uint8_t *E, uint8_t *Ed, uint8_t *Edf, int W, int H, int pitch,
                         size_t frame_stride, int frames, int conn, int n_d, int n_f,
                         uint8_t *export_dense, DevStats *stats, cudaStream_t st)
{
    (void)Ed;  // the denoised image stays in shared memory
    StageScope sc(kStDenoiseFill, 1, st);
    dim3 blk(kDfX, kDfY), grd((W + kDfX - 1) / kDfX, (H + kDfY - 1) / kDfY, frames);
    denoise_fill_kernel<<<grd, blk, 0, st>>>(E, Edf, W, H, pitch, frame_stride, conn, n_d, n_f,
                                             export_dense, stats);
}

void launch_edt_columns(const uint8_t *E, int edge_pitch, size_t edge_frame_stride, int W,
                        int H, int32_t *g, int g_pitch, size_t g_frame_stride, int frames,
                        cudaStream_t st)
{
    StageScope sc(kStEdtCols, 1, st);
    // chunks of CH rows, CH a multiple of 32: at most 32 chunks of at most 512 rows
    int nch = (H + 31) / 32;
    if (nch > kColMaxChunks) nch = kColMaxChunks;
    int CH = ((H + nch - 1) / nch + 31) / 32 * 32;
    nch = (H + CH - 1) / CH;
    dim3 blk(32, nch), grd((W + 31) / 32, frames);
    edt_cols_kernel<<<grd, blk, 0, st>>>(E, edge_pitch, edge_frame_stride, W, H, g, g_pitch,
                                         g_frame_stride, CH);
}

// Warps per row: one below 640 px, two above; single windows (one or two
// frames per launch) of rows from 1024 px use four, with a window of four
// near bands each side (two otherwise).
int edt_rows_wpr(int W, int frames)
{
    const int wpr = W >= 640 ? 2 : 1;
    return (wpr == 2 && W >= 1024 && frames <= 2) ? 4 : wpr;
}

template <typename T>
void edt_rows_t(const int32_t *g, int g_pitch, size_t g_frame_stride, int W, int H,
                const SurfaceMap &sm, int32_t *D_dense, float *S_dense, T *I0, int i_pitch,
                size_t i_frame_stride, int frames, cudaStream_t st)
{
    const int wpr = edt_rows_wpr(W, frames);
    int rows = wpr == 1 ? 4 : 2;
    while (rows > 1 && (size_t)rows * rows_smem_words(W, wpr) * 4 > 200 * 1024) --rows;
    const size_t smem = (size_t)rows * rows_smem_words(W, wpr) * 4;
    dim3 grd((H + rows - 1) / rows, frames);
    if (wpr == 4)
        edt_rows_surface_kernel<4, 4, T><<<grd, 32 * 4 * rows, smem, st>>>(
            g, g_pitch, g_frame_stride, W, H, rows, sm, D_dense, S_dense, I0, i_pitch,
            i_frame_stride);
    else if (wpr == 2)
        edt_rows_surface_kernel<2, 2, T><<<grd, 32 * 2 * rows, smem, st>>>(
            g, g_pitch, g_frame_stride, W, H, rows, sm, D_dense, S_dense, I0, i_pitch,
            i_frame_stride);
    else
        edt_rows_surface_kernel<1, 2, T><<<grd, 32 * rows, smem, st>>>(
            g, g_pitch, g_frame_stride, W, H, rows, sm, D_dense, S_dense, I0, i_pitch,
            i_frame_stride);
}

void launch_edt_rows_surface(const int32_t *g, int g_pitch, size_t g_frame_stride, int W, int H,
                             const SurfaceMap &sm, int32_t *D_dense, float *S_dense, void *I0,
                             int i_pitch, size_t i_frame_stride, int frames, bool half,
                             cudaStream_t st)
{
    StageScope sc(kStEdtRows, 1, st);
    if (half)
        edt_rows_t(g, g_pitch, g_frame_stride, W, H, sm, D_dense, S_dense, (__half *)I0,
                   i_pitch, i_frame_stride, frames, st);
    else
        edt_rows_t(g, g_pitch, g_frame_stride, W, H, sm, D_dense, S_dense, (float *)I0,
                   i_pitch, i_frame_stride, frames, st);
}

void launch_edt_rows_surface(const int32_t *g, int g_pitch, size_t g_frame_stride, int W, int H,
                             float alpha, int32_t *D_dense, float *S_dense, void *I0,
                             int i_pitch, size_t i_frame_stride, int frames, bool half,
                             cudaStream_t st)
{
    launch_edt_rows_surface(g, g_pitch, g_frame_stride, W, H, exp_surface(alpha), D_dense,
                            S_dense, I0, i_pitch, i_frame_stride, frames, half, st);
}

void init_front_attributes()
{
    cudaFuncSetAttribute(edt_rows_surface_kernel<1, 2, float>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    cudaFuncSetAttribute(edt_rows_surface_kernel<2, 2, float>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    cudaFuncSetAttribute(edt_rows_surface_kernel<4, 4, float>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    cudaFuncSetAttribute(edt_rows_surface_kernel<1, 2, __half>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    cudaFuncSetAttribute(edt_rows_surface_kernel<2, 2, __half>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    cudaFuncSetAttribute(edt_rows_surface_kernel<4, 4, __half>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
}

void launch_surface_to_intensity(const float *S, int W, int H, void *I0, int pitch, bool half,
                                 const SurfaceMap &sm, cudaStream_t st)
{
    StageScope sc(kStEdtRows, 1, st);
    dim3 grd((W + 255) / 256, H);
    if (half)
        surface_to_intensity_kernel<__half>
            <<<grd, 256, 0, st>>>(S, W, H, (__half *)I0, pitch, sm);
    else
        surface_to_intensity_kernel<float><<<grd, 256, 0, st>>>(S, W, H, (float *)I0, pitch, sm);
}

}  // namespace ebof
