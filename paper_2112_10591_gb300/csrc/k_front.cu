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
#include "seg.cuh"

#include <cuda_fp16.h>

#include <algorithm>

namespace ebof {

namespace {

// ---------------------------------------------------------------- A1 scatter
// One thread per event.  The window index of an event is
// floor((t - t_begin) / dt) when it lies in [0, n_windows); duplicates collapse
// (a byte store of 1 is idempotent).  A block walks one contiguous chunk of
// the events, 32 per warp and step.  Timestamps are sorted, so a warp's 32
// events nearly always share a window and its counts run in registers until
// the window changes (then one atomic per counter); a step whose events
// straddle a window boundary counts per group of lanes that share a window.
__device__ __forceinline__ void flush_counts(int cur, unsigned long long &c_in,
                                             unsigned long long &c_oob, unsigned long long &c_time,
                                             int lane, DevStats *stats,
                                             unsigned long long *dropped_time)
{
    if (lane == 0) {
        if (cur >= 0) {
            if (c_in) atomicAdd(&stats[cur].in_window, c_in);
            if (c_oob) atomicAdd(&stats[cur].dropped_oob, c_oob);
        } else if (cur == -1 && c_time) {
            atomicAdd(dropped_time, c_time);
        }
    }
    c_in = c_oob = c_time = 0;
}

__global__ void scatter_kernel(const uint16_t *__restrict__ x, const uint16_t *__restrict__ y,
                               const int64_t *__restrict__ t, int64_t n, int64_t t_begin,
                               int64_t dt, int n_windows, int W, int H, int pitch,
                               uint8_t *__restrict__ E, size_t fstride, DevStats *stats,
                               unsigned long long *dropped_time)
{
    const int64_t span = dt * (int64_t)n_windows;
    const int lane = threadIdx.x & 31;
    const int64_t per_block =
        ((n + gridDim.x - 1) / gridDim.x + blockDim.x - 1) / blockDim.x * blockDim.x;
    const int64_t beg = (int64_t)blockIdx.x * per_block;
    const int64_t end = min(n, beg + per_block);
    int cur = -3;  // window of the running counts (-1: outside every window, -3: none)
    unsigned long long c_in = 0, c_oob = 0, c_time = 0;
    for (int64_t base = beg; base < end; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        int k = -2;  // -2: no event (tail), -1: outside every window
        bool oob = false;
        if (i < end) {
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
        const unsigned valid = __ballot_sync(0xffffffffu, k != -2);
        const unsigned oob_mask = __ballot_sync(0xffffffffu, oob);
        if (valid == 0) continue;  // warp-uniform
        const int kl = __shfl_sync(0xffffffffu, k, __ffs(valid) - 1);
        if (__all_sync(0xffffffffu, k == -2 || k == kl)) {
            if (kl != cur) {
                flush_counts(cur, c_in, c_oob, c_time, lane, stats, dropped_time);
                cur = kl;
            }
            if (kl >= 0) {
                c_in += __popc(valid);
                c_oob += __popc(oob_mask);
            } else {
                c_time += __popc(valid);
            }
            continue;
        }
        flush_counts(cur, c_in, c_oob, c_time, lane, stats, dropped_time);
        cur = -3;
        const unsigned peers = __match_any_sync(0xffffffffu, k);
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
    flush_counts(cur, c_in, c_oob, c_time, lane, stats, dropped_time);
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
    // block sums, one atomic per block and counter (same-address atomics
    // serialise in L2)
    __shared__ unsigned long long s_sum[3][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        in_w += __shfl_xor_sync(0xffffffffu, in_w, o);
        oob += __shfl_xor_sync(0xffffffffu, oob, o);
        out_t += __shfl_xor_sync(0xffffffffu, out_t, o);
    }
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (lane == 0) {
        s_sum[0][warp] = in_w;
        s_sum[1][warp] = oob;
        s_sum[2][warp] = out_t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < nwarps; ++k) {
            in_w += s_sum[0][k];
            oob += s_sum[1][k];
            out_t += s_sum[2][k];
        }
        if (in_w) atomicAdd(&stats[f].in_window, in_w);
        if (oob) atomicAdd(&stats[f].dropped_oob, oob);
        if (out_t) atomicAdd(dropped_time, out_t);
    }
}

// Scatter of a fused launch over several groups: a work list of event
// chunks (kScatterChunk events of one window) over all the windows.  Every
// block turns the windows' event counts, read from their device
// descriptors, into chunk offsets in shared memory, then walks the chunks
// blockIdx.x, blockIdx.x + gridDim.x, ...: windows of very different sizes
// spread evenly over the blocks.  The counts of a chunk go out as one atomic
// per counter and block, as in scatter_desc_kernel.
__global__ void __launch_bounds__(256)
scatter_list_kernel(const ScatterWin *__restrict__ wins, int n_wins)
{
    __shared__ int s_off[kScatterListMax + 1];
    __shared__ unsigned long long s_sum[3][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {
        int run = 0;
        for (int base = 0; base < n_wins; base += 32) {
            const int i = base + lane;
            int c = 0;
            if (i < n_wins) {
                const int64_t ne = wins[i].desc->n_events;
                c = (int)((ne + kScatterChunk - 1) / kScatterChunk);
            }
            int v = c;  // inclusive scan over the lanes
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            if (i < n_wins) s_off[i] = run + v - c;
            run += __shfl_sync(0xffffffffu, v, 31);
        }
        if (lane == 0) s_off[n_wins] = run;
    }
    __syncthreads();
    const int total = s_off[n_wins];
    for (int c = blockIdx.x; c < total; c += gridDim.x) {
        // the window of chunk c: the last one whose chunks start at or before c
        int lo = 0, hi = n_wins - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= c) lo = mid;
            else hi = mid - 1;
        }
        const ScatterWin &w = wins[lo];
        const ebof_window_desc d = *w.desc;
        const int64_t i0 = (int64_t)(c - s_off[lo]) * kScatterChunk;
        const int64_t i1 = min(d.n_events, i0 + (int64_t)kScatterChunk);
        unsigned long long in_w = 0, oob = 0, out_t = 0;
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const int64_t tt = d.t[i];
            if (tt >= d.t_begin && tt < d.t_end) {
                ++in_w;
                const int xi = d.x[i], yi = d.y[i];
                if (xi < w.W && yi < w.H) w.E[(size_t)yi * w.pitch + xi] = 1;
                else ++oob;
            } else {
                ++out_t;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            in_w += __shfl_xor_sync(0xffffffffu, in_w, o);
            oob += __shfl_xor_sync(0xffffffffu, oob, o);
            out_t += __shfl_xor_sync(0xffffffffu, out_t, o);
        }
        if (lane == 0) {
            s_sum[0][warp] = in_w;
            s_sum[1][warp] = oob;
            s_sum[2][warp] = out_t;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
                in_w += s_sum[0][k];
                oob += s_sum[1][k];
                out_t += s_sum[2][k];
            }
            if (in_w) atomicAdd(&w.stats->in_window, in_w);
            if (oob) atomicAdd(&w.stats->dropped_oob, oob);
            if (out_t) atomicAdd(w.dropped_time, out_t);
        }
        __syncthreads();  // s_sum is rewritten by the next chunk
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

// (bx, by): the tile, f: the frame.
__device__ __forceinline__ void denoise_fill_body(const uint8_t *__restrict__ E,
                                                  uint8_t *__restrict__ Edf, int W, int H,
                                                  int pitch, size_t fstride, int conn, int n_d,
                                                  int n_f, uint8_t *__restrict__ export_dense,
                                                  DevStats *stats, int bx, int by, int f)
{
    __shared__ uint8_t sE[kDfY + 4][kDfX + 4];
    __shared__ uint8_t sD[kDfY + 4][kDfX + 4];  // denoised, 1-pixel ring inside a 2-pixel frame
    const uint8_t *e = E + (size_t)f * fstride;
    const int x0 = bx * kDfX - 2, y0 = by * kDfY - 2;
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
    const int x = bx * kDfX + threadIdx.x, y = by * kDfY + threadIdx.y;
    uint8_t v = 0;
    if (x < W && y < H) {
        const int lx = threadIdx.x + 2, ly = threadIdx.y + 2;
        v = sD[ly][lx];
        if (!v && count_tile(sD, lx, ly, conn) >= n_f) v = 1;
        Edf[(size_t)f * fstride + (size_t)y * pitch + x] = v;
        if (export_dense) export_dense[(size_t)f * W * H + (size_t)y * W + x] = v;
    }
    // one atomic per block: same-address atomics serialise in L2
    const int nedge = __syncthreads_count(v != 0);
    if (t == 0 && nedge) atomicAdd(&stats[f].edge_px, (unsigned long long)nedge);
}

__global__ void __launch_bounds__(kDfX * kDfY)
denoise_fill_kernel(const uint8_t *__restrict__ E, uint8_t *__restrict__ Edf, int W, int H,
                    int pitch, size_t fstride, int conn, int n_d, int n_f,
                    uint8_t *__restrict__ export_dense, DevStats *stats)
{
    denoise_fill_body(E, Edf, W, H, pitch, fstride, conn, n_d, n_f, export_dense, stats,
                      blockIdx.x, blockIdx.y, blockIdx.z);
}

__global__ void __launch_bounds__(kDfX * kDfY)
seg_denoise_fill_kernel(const __grid_constant__ SegTable<SegDenoise> tab)
{
    int b;
    const SegDenoise &a = seg_of(tab, b);
    const int bx = b % a.gx, r = b / a.gx;
    denoise_fill_body(a.E, a.Edf, a.W, a.H, a.pitch, a.fs, a.conn, a.n_d, a.n_f, nullptr,
                      a.stats, bx, r % a.gy, r / a.gy);
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

// bx: the block of 32 columns, f: the frame; nch chunks (at most blockDim.y:
// threads of chunks past the last one only take part in the barrier).
__device__ __forceinline__ void edt_cols_body(const uint8_t *__restrict__ E, int epitch,
                                              size_t efs, int W, int H,
                                              int32_t *__restrict__ g, int gpitch, size_t gfs,
                                              int CH, int nch, unsigned bx, unsigned f)
{
    __shared__ int s_first[kColMaxChunks][32], s_last[kColMaxChunks][32];
    const int c = threadIdx.x, k = threadIdx.y;
    const int x = bx * 32 + c;
    const bool colok = x < W;  // chunks k >= nch start at or below row H: nothing to do
    const uint8_t *e = E + (size_t)f * efs;
    const int y0 = k * CH, y1 = min(H, y0 + CH);
    const int nw = (CH + 31) / 32;
    unsigned mask[kColMaxWords];
    int first = -1, last = -1;
#pragma unroll
    for (int wi = 0; wi < kColMaxWords; ++wi) {
        unsigned m = 0;
        if (wi < nw && colok) {
            // all 32 loads in flight before the first test (rows past the
            // chunk read its last row and are masked out)
            uint8_t ev[32];
#pragma unroll
            for (int b = 0; b < 32; ++b)
                ev[b] = e[(size_t)min(y0 + wi * 32 + b, y1 - 1) * epitch + x];
#pragma unroll
            for (int b = 0; b < 32; ++b)
                if (y0 + wi * 32 + b < y1 && ev[b]) m |= 1u << b;
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
    int32_t *gc = g + (size_t)f * gfs + x;
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

__global__ void __launch_bounds__(1024)
edt_cols_kernel(const uint8_t *__restrict__ E, int epitch, size_t efs, int W, int H,
                int32_t *__restrict__ g, int gpitch, size_t gfs, int CH)
{
    edt_cols_body(E, epitch, efs, W, H, g, gpitch, gfs, CH, blockDim.y, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(1024)
seg_edt_cols_kernel(const __grid_constant__ SegTable<SegEdtCols> tab)
{
    int b;
    const SegEdtCols &a = seg_of(tab, b);
    edt_cols_body(a.E, a.epitch, a.efs, a.W, a.H, a.g, a.gpitch, a.gfs, a.CH, a.nch, b % a.gx,
                  b / a.gx);
}

// ---------------------------------------------------------------- A4
// Row pass: D(x) = min over columns s of (x - s)^2 + h(s), h(s) = g(s, y)^2,
// the lower envelope of the row's parabolas evaluated at every pixel.  With
// F(s) = s^2 + h(s) it reads D(x) = x^2 + min_s (F(s) - 2 x s): a minimum of
// lines in x, so the sites that own part of the envelope are exactly the
// vertices of the lower convex hull of the points (s, F(s)).  One warp (two
// or four for single frames of wide rows) serves a row, and each lane owns a
// band of B consecutive columns (B odd, so that the lanes' accesses to F fall
// in distinct shared-memory banks).
//  1. The row's F is staged in shared memory (-1: column without edge pixels).
//  2. Each lane builds the lower hull of its band's points with a stack
//     (orientation tests exact in 64-bit integers; a point on the segment of
//     its neighbours is dropped, which never changes a minimum).
//  3. Rounds merge the hulls of neighbouring groups of 1, 2, 4, ... bands
//     (five for 32 bands, seven for 128).  The group's first lane finds the
//     lower bridge of the two hulls
//     by walking from their inner ends (the left hull's last vertex moves left
//     and the right hull's first vertex moves right while the vertex is not
//     strictly below the line through the other two); the right hull's
//     surviving vertices are then moved down behind the left hull's, so a
//     group's hull always starts at its first column.
//  4. Each lane walks its band's pixels left to right with a pointer into the
//     row's hull (binary search for the first pixel): along a strictly convex
//     hull the owner of x never moves left as x grows.
//  5. Eq. 1 (or an ablation surface) and the 8-bit scale, coalesced stores.
// Every step is an exact integer minimum, so D is bit-identical to any exact
// EDT.  The work per pixel is a few hull steps whatever the distance to the
// nearest edge, and the lanes of a warp stay in step.

// With hull points a < b < c (columns; F as above): is b on or above the
// segment from a to c, i.e. not a strict vertex of the lower hull?
__device__ __forceinline__ bool above_chord(int a, int b, int c, const int32_t *F)
{
    const long long fa = F[a], fb = F[b], fc = F[c];
    return (fc - fb) * (long long)(b - a) <= (fb - fa) * (long long)(c - b);
}

// (x - s)^2 + h(s) from F(s) = s^2 + h(s); every term is below 2^29 for
// images up to 16384 px a side.
__device__ __forceinline__ int para(int x, int s, const int32_t *F)
{
    const int d = x - s;
    return d * d + (F[s] - s * s);
}

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRowsPerBlock = 4;                  // rows (warps) per block
constexpr int kRowLoads = 8;                      // column distances in flight per lane
constexpr size_t kRowsSmemCap = 200 * 1024;       // bytes; 16384-px rows fit one per block

// Shared memory of one row, in bytes: F and D (int32) and the hull's columns
// (int16: every column is below 2^14), padded to a multiple of 4 bytes.
__host__ __device__ __forceinline__ size_t rows_smem_bytes(int W)
{
    return 8 * (size_t)W + 2 * (((size_t)W + 1) & ~(size_t)1);
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

// Lower bridge of two hulls of one row whose columns are x-separated: the
// left hull hs[aL, aL + nL), the right one hs[aR, aR + nR), both non-empty.
// On return the merged hull is hs[aL, aL + i] followed by hs[aR + j, aR + nR).
// The left end moves left and the right end moves right while the vertex is
// not strictly below the line through the other two; each move drops a
// vertex, so the walk ends after at most nL + nR steps.
__device__ __forceinline__ void bridge(const int16_t *hs, const int32_t *F, int aL, int nL,
                                       int aR, int nR, int &i, int &j)
{
    i = nL - 1;
    j = 0;
    int li = hs[aL + i], rj = hs[aR];
    for (;;) {
        bool moved = false;
        while (j + 1 < nR) {
            const int rn = hs[aR + j + 1];
            if (!above_chord(li, rj, rn, F)) break;
            rj = rn;
            ++j;
            moved = true;
        }
        while (i > 0) {
            const int lp = hs[aL + i - 1];
            if (!above_chord(lp, li, rj, F)) break;
            li = lp;
            --i;
            moved = true;
        }
        if (!moved) break;
    }
}

// WPR warps serve a row (32 WPR bands).  WPR = 1: rows_per_block rows of one
// warp each, warp-level barriers only.  WPR > 1: one row per block; the merge
// rounds of groups wider than a warp go through shared memory and block
// barriers.  D is exact whatever WPR, so the layout never changes a result.
// bx: the block of rows, f: the frame.  A warp past the block's
// rows_per_block rows (a fused launch sized for another segment's) exits
// (WPR = 1 has warp-level barriers only).
template <int WPR, typename T>
__device__ __forceinline__ void edt_rows_surface_body(
    const int32_t *__restrict__ g, int gpitch, size_t gfs, int W, int H, int rows_per_block,
    const SurfaceMap &sm, int32_t *__restrict__ D_dense, float *__restrict__ S_dense,
    T *__restrict__ I0, int ipitch, size_t ifs, int bx, int f)
{
    constexpr int NB = 32 * WPR;
    extern __shared__ int32_t smem[];
    __shared__ int s_cnt[NB];         // hull sizes of the group leaders (WPR > 1)
    __shared__ int s_move[NB / 64 + 1][3];  // src, dst, len of a cross-warp group's move
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rib = warp / WPR;                 // row within the block
    const int tr = (warp % WPR) * 32 + lane;    // this lane's band
    const int y = bx * rows_per_block + rib;
    // WPR = 1: the whole warp; WPR > 1: never (one row per block)
    if (rib >= rows_per_block || y >= H) return;
    int32_t *F = smem + (size_t)rib * (rows_smem_bytes(W) / 4);
    int32_t *res = F + W;  // D of the row's pixels
    // hull columns; a group's hull starts at its first column
    int16_t *hs = reinterpret_cast<int16_t *>(res + W);
    auto row_sync = [] {
        if (WPR == 1) __syncwarp();
        else __syncthreads();
    };
    const int ginf = W + H;
    const int32_t *grow = g + (size_t)f * gfs + (size_t)y * gpitch;
    // loads issued in batches of kRowLoads before their first use
    for (int x0 = tr; x0 < W; x0 += NB * kRowLoads) {
        int gv[kRowLoads];
#pragma unroll
        for (int u = 0; u < kRowLoads; ++u) {
            const int x = x0 + NB * u;
            gv[u] = x < W ? grow[x] : ginf;
        }
#pragma unroll
        for (int u = 0; u < kRowLoads; ++u) {
            const int x = x0 + NB * u;
            if (x < W) F[x] = gv[u] >= ginf ? -1 : gv[u] * gv[u] + x * x;
        }
    }
    row_sync();

    // 2. the lower hull of the lane's band
    const int B = ((W + NB - 1) / NB) | 1;
    const int a = min(W, tr * B), b = min(W, a + B);
    int cnt = 0;
    for (int q = a; q < b; ++q) {
        if (F[q] < 0) continue;
        while (cnt >= 2 && above_chord(hs[a + cnt - 2], hs[a + cnt - 1], q, F)) --cnt;
        hs[a + cnt++] = (int16_t)q;
    }
    __syncwarp();

    // 3. merge rounds within the warp; the first lane of a group holds the
    // group's hull size
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int gs = 2 << k, half = 1 << k;
        const int nR = __shfl_down_sync(kFull, cnt, half);  // read by group leaders only
        const int leader = lane & ~(gs - 1);
        int src = 0, dst = 0, len = 0;
        if (lane == leader) {
            const int AR = min(W, (tr + half) * B);  // the right half's first column
            int i = cnt - 1, j = 0;
            if (cnt > 0 && nR > 0) bridge(hs, F, a, cnt, AR, nR, i, j);
            src = AR + j;
            dst = a + i + 1;
            len = nR - j;
            cnt = i + 1 + len;
        }
        src = __shfl_sync(kFull, src, leader);
        dst = __shfl_sync(kFull, dst, leader);
        len = __shfl_sync(kFull, len, leader);
        // move the right hull's survivors down (dst <= src: every read of a
        // later step lies above every write of an earlier one)
        const int steps = __reduce_max_sync(kFull, (unsigned)((len + gs - 1) / gs));
        const int e0 = lane - leader;
        for (int t = 0; t < steps; ++t) {
            const int e = t * gs + e0;
            int v = 0;
            if (e < len) v = hs[src + e];
            __syncwarp();
            if (e < len) hs[dst + e] = (int16_t)v;
            __syncwarp();
        }
    }
    int n;  // the row's hull: hs[0, n)
    if (WPR == 1) {
        n = __shfl_sync(kFull, cnt, 0);
    } else {
        // merge rounds across the row's warps
        if (lane == 0) s_cnt[tr] = cnt;
        __syncthreads();
#pragma unroll
        for (int k = 5; (2 << k) <= NB; ++k) {
            const int gs = 2 << k, half = 1 << k;
            const int grp = tr / gs, leader = grp * gs;
            if (tr == leader) {
                const int nL = s_cnt[tr], nR = s_cnt[tr + half];
                const int AR = min(W, (tr + half) * B);
                int i = nL - 1, j = 0;
                if (nL > 0 && nR > 0) bridge(hs, F, a, nL, AR, nR, i, j);
                s_move[grp][0] = AR + j;
                s_move[grp][1] = a + i + 1;
                s_move[grp][2] = nR - j;
                s_cnt[tr] = i + 1 + nR - j;
            }
            __syncthreads();
            const int src = s_move[grp][0], dst = s_move[grp][1], len = s_move[grp][2];
            int steps = 0;
#pragma unroll
            for (int q = 0; q < NB / gs; ++q) steps = max(steps, (s_move[q][2] + gs - 1) / gs);
            const int e0 = tr - leader;
            for (int t = 0; t < steps; ++t) {
                const int e = t * gs + e0;
                int v = 0;
                if (e < len) v = hs[src + e];
                __syncthreads();
                if (e < len) hs[dst + e] = (int16_t)v;
                __syncthreads();
            }
            __syncthreads();  // s_move is rewritten by the next round
        }
        n = s_cnt[0];
    }

    // 4. D of the lane's pixels
    if (n > 0 && a < b) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (para(a, hs[mid + 1], F) <= para(a, hs[mid], F)) lo = mid + 1;
            else hi = mid;
        }
        int kk = lo, sk = hs[lo];
        for (int x = a; x < b; ++x) {
            int cur = para(x, sk, F);
            while (kk + 1 < n) {
                const int sn = hs[kk + 1];
                const int nx = para(x, sn, F);
                if (nx > cur) break;
                cur = nx;
                sk = sn;
                ++kk;
            }
            res[x] = cur;
        }
    }
    row_sync();

    // 5. surface and intensity (n == 0: the image has no edge pixel)
    T *irow = I0 ? I0 + (size_t)f * ifs + (size_t)y * ipitch : nullptr;
    const size_t dbase = (size_t)f * W * H + (size_t)y * W;
    const float inv_alpha = 1.0f / sm.alpha;
    for (int x = tr; x < W; x += NB) {
        const int32_t D = n > 0 ? res[x] : kInfD;
        float S = 1.0f, C = 0.0f;  // d_exp of Eq. 1 and its complement 1 - d_exp
        if (sm.mode == 0) {
            if (D != kInfD) {
                C = expf(-sqrtf((float)D) * inv_alpha);
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

template <int WPR, typename T>
__global__ void __launch_bounds__(32 * kRowsPerBlock)
edt_rows_surface_kernel(const int32_t *__restrict__ g, int gpitch, size_t gfs, int W, int H,
                        int rows_per_block, SurfaceMap sm, int32_t *__restrict__ D_dense,
                        float *__restrict__ S_dense, T *__restrict__ I0, int ipitch, size_t ifs)
{
    edt_rows_surface_body<WPR, T>(g, gpitch, gfs, W, H, rows_per_block, sm, D_dense, S_dense, I0,
                                  ipitch, ifs, blockIdx.x, blockIdx.y);
}

template <typename T>
__global__ void __launch_bounds__(32 * kRowsPerBlock)
seg_edt_rows_kernel(const __grid_constant__ SegTable<SegEdtRows> tab)
{
    int b;
    const SegEdtRows &a = seg_of(tab, b);
    edt_rows_surface_body<1, T>(a.g, a.gpitch, a.gfs, a.W, a.H, a.rows, a.sm, nullptr, nullptr,
                                (T *)a.I0, a.ipitch, a.ifs, b % a.gx, b / a.gx);
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

void edt_cols_chunks(int H, int &CH, int &nch)
{
    // chunks of CH rows, CH a multiple of 32: at most 32 chunks of at most 512 rows
    nch = (H + 31) / 32;
    if (nch > kColMaxChunks) nch = kColMaxChunks;
    CH = ((H + nch - 1) / nch + 31) / 32 * 32;
    nch = (H + CH - 1) / CH;
}

void launch_edt_columns(const uint8_t *E, int edge_pitch, size_t edge_frame_stride, int W,
                        int H, int32_t *g, int g_pitch, size_t g_frame_stride, int frames,
                        cudaStream_t st)
{
    StageScope sc(kStEdtCols, 1, st);
    int CH, nch;
    edt_cols_chunks(H, CH, nch);
    dim3 blk(32, nch), grd((W + 31) / 32, frames);
    edt_cols_kernel<<<grd, blk, 0, st>>>(E, edge_pitch, edge_frame_stride, W, H, g, g_pitch,
                                         g_frame_stride, CH);
}

int edt_rows_block_rows(int W)
{
    int rows = kRowsPerBlock;
    while (rows > 1 && (size_t)rows * rows_smem_bytes(W) > kRowsSmemCap) --rows;
    return rows;
}

size_t edt_rows_smem(int W, int rows) { return (size_t)rows * rows_smem_bytes(W); }

// Warps per row: one for batches (fewest instructions per frame) and rows
// under 512 px; single windows (one or two frames per launch) of wider rows
// use two, or four from 1024 px, one row per block, to shorten the serial
// work of a lane.
int edt_rows_wpr(int W, int frames)
{
    if (frames > 2 || W < 512) return 1;
    return W >= 1024 ? 4 : 2;
}

template <typename T>
void edt_rows_t(const int32_t *g, int g_pitch, size_t g_frame_stride, int W, int H,
                const SurfaceMap &sm, int32_t *D_dense, float *S_dense, T *I0, int i_pitch,
                size_t i_frame_stride, int frames, cudaStream_t st)
{
    const int wpr = edt_rows_wpr(W, frames);
    // one warp a row: four rows per block, fewer where a row's shared memory
    // is large; wider layouts: one row per block
    const int rows = wpr == 1 ? edt_rows_block_rows(W) : 1;
    const size_t smem = edt_rows_smem(W, rows);
    dim3 grd((H + rows - 1) / rows, frames);
    if (wpr == 4)
        edt_rows_surface_kernel<4, T><<<grd, 128, smem, st>>>(
            g, g_pitch, g_frame_stride, W, H, 1, sm, D_dense, S_dense, I0, i_pitch,
            i_frame_stride);
    else if (wpr == 2)
        edt_rows_surface_kernel<2, T><<<grd, 64, smem, st>>>(
            g, g_pitch, g_frame_stride, W, H, 1, sm, D_dense, S_dense, I0, i_pitch,
            i_frame_stride);
    else
        edt_rows_surface_kernel<1, T><<<grd, 32 * rows, smem, st>>>(
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
    auto opt_in = [](const void *fn) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowsSmemCap);
    };
    opt_in((const void *)edt_rows_surface_kernel<1, float>);
    opt_in((const void *)edt_rows_surface_kernel<2, float>);
    opt_in((const void *)edt_rows_surface_kernel<4, float>);
    opt_in((const void *)edt_rows_surface_kernel<1, __half>);
    opt_in((const void *)edt_rows_surface_kernel<2, __half>);
    opt_in((const void *)edt_rows_surface_kernel<4, __half>);
    opt_in((const void *)seg_edt_rows_kernel<float>);
    opt_in((const void *)seg_edt_rows_kernel<__half>);
}

void launch_seg_scatter(const ScatterWin *wins, int n_wins, int blocks, cudaStream_t st)
{
    StageScope sc(kStScatter, 1, st);
    scatter_list_kernel<<<blocks, 256, 0, st>>>(wins, n_wins);
}

void launch_seg_denoise_fill(const SegTable<SegDenoise> &t, int blocks, cudaStream_t st)
{
    StageScope sc(kStDenoiseFill, 1, st);
    seg_denoise_fill_kernel<<<blocks, dim3(kDfX, kDfY), 0, st>>>(t);
}

void launch_seg_edt_cols(const SegTable<SegEdtCols> &t, int blocks, int nch_max,
                         cudaStream_t st)
{
    StageScope sc(kStEdtCols, 1, st);
    seg_edt_cols_kernel<<<blocks, dim3(32, nch_max), 0, st>>>(t);
}

void launch_seg_edt_rows(const SegTable<SegEdtRows> &t, int blocks, int rows_max, size_t smem,
                         bool half, cudaStream_t st)
{
    StageScope sc(kStEdtRows, 1, st);
    if (half)
        seg_edt_rows_kernel<__half><<<blocks, 32 * rows_max, smem, st>>>(t);
    else
        seg_edt_rows_kernel<float><<<blocks, 32 * rows_max, smem, st>>>(t);
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
