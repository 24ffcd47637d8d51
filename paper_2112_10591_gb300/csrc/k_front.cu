// k_front.cu -- event accumulation, denoising/filling, exact EDT, surface.
//
// §III-A: edge image of a window.  §III-B: Alg. 1 (denoise) then Alg. 2
// (fill).  §III-C: exact Euclidean distance transform as int32 squared
// distances (separable: a per-column pass, then a per-row lower envelope of
// parabolas), fused with Eq. 1, d_exp = 1 - exp(-sqrt(D) / alpha), and the
// 8-bit intensity scale 255 * d_exp the flow block runs on.
#include "ebof_internal.cuh"
#include "profiler.cuh"

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

// ---------------------------------------------------------------- A2
__device__ __forceinline__ int count_neighbours(const uint8_t *img, int W, int H, int pitch,
                                                int x, int y, int conn)
{
    int c = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            if (dx == 0 && dy == 0) continue;
            if (conn == 4 && dx != 0 && dy != 0) continue;
            const int qx = x + dx, qy = y + dy;
            if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
            c += img[(size_t)qy * pitch + qx] ? 1 : 0;
        }
    return c;
}

// Alg. 1: an edge pixel with fewer than n_d edge neighbours (counted in E)
// stops being an edge pixel.
__global__ void denoise_kernel(const uint8_t *__restrict__ E, uint8_t *__restrict__ Ed, int W,
                               int H, int pitch, size_t fstride, int conn, int n_d)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    const uint8_t *e = E + (size_t)blockIdx.z * fstride;
    const size_t p = (size_t)y * pitch + x;
    uint8_t v = e[p] ? 1 : 0;
    if (v && count_neighbours(e, W, H, pitch, x, y, conn) < n_d) v = 0;
    Ed[(size_t)blockIdx.z * fstride + p] = v;
}

// Alg. 2 on the denoised image: a non-edge pixel with at least n_f edge
// neighbours (counted in E_d) becomes an edge pixel.  Also counts the edge
// pixels of E_df and writes the optional dense export.
__global__ void fill_kernel(const uint8_t *__restrict__ Ed, uint8_t *__restrict__ Edf, int W,
                            int H, int pitch, size_t fstride, int conn, int n_f,
                            uint8_t *__restrict__ export_dense, DevStats *stats)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int f = blockIdx.z;
    uint8_t v = 0;
    const bool in = x < W && y < H;
    if (in) {
        const uint8_t *e = Ed + (size_t)f * fstride;
        const size_t p = (size_t)y * pitch + x;
        v = e[p] ? 1 : 0;
        if (!v && count_neighbours(e, W, H, pitch, x, y, conn) >= n_f) v = 1;
        Edf[(size_t)f * fstride + p] = v;
        if (export_dense) export_dense[(size_t)f * W * H + (size_t)y * W + x] = v;
    }
    const unsigned m = __ballot_sync(0xffffffffu, v != 0);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&stats[f].edge_px, (unsigned long long)__popc(m));
}

// ---------------------------------------------------------------- A3
// One thread per (column, frame): distance to the nearest edge pixel above
// (forward sweep) and below (backward sweep).  Columns without any edge
// pixel get G_INF = W + H, larger than any distance in the image.
__global__ void edt_cols_kernel(const uint8_t *__restrict__ E, int epitch, size_t efs, int W,
                                int H, int32_t *__restrict__ g, int gpitch, size_t gfs)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    const uint8_t *e = E + (size_t)blockIdx.y * efs + x;
    int32_t *gc = g + (size_t)blockIdx.y * gfs + x;
    const int ginf = W + H;
    int last = -1;
    for (int y = 0; y < H; ++y) {
        if (e[(size_t)y * epitch]) last = y;
        gc[(size_t)y * gpitch] = last < 0 ? ginf : y - last;
    }
    last = -1;
    for (int y = H - 1; y >= 0; --y) {
        if (e[(size_t)y * epitch]) last = y;
        if (last >= 0) {
            const int d = last - y;
            int32_t *q = gc + (size_t)y * gpitch;
            if (d < *q) *q = d;
        }
    }
}

// ---------------------------------------------------------------- A4
// Row pass, one warp per row.  The row's column distances h(x') = g(x', y)^2
// are staged in shared memory.  Each lane owns a band of ceil(W / 32)
// consecutive columns and builds the lower envelope of the parabolas
// f_x'(x) = (x - x')^2 + h(x') of its band's columns (the stack construction
// of the separable exact EDT, with exact integer breakpoint comparisons).
// D(x) is the minimum over all bands' envelopes: the lane's own envelope is
// walked in step with x; the other bands are visited nearest first, skipped
// once (distance to the band)^2 reaches the best value so far, and each is
// evaluated at x by binary search over its breakpoints.  The result is the
// exact minimum, hence bit-identical to any other exact EDT.  The epilogue
// applies Eq. 1 and the 8-bit scale, and writes through shared memory so
// that global stores are coalesced.
constexpr int kRowWarpsMax = 4;  // rows per block

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

__device__ __forceinline__ long long para(int x, int site, const int32_t *h)
{
    const long long d = (long long)(x - site);
    return d * d + (long long)h[site];
}

__global__ void edt_rows_surface_kernel(const int32_t *__restrict__ g, int gpitch, size_t gfs,
                                        int W, int H, int rows_per_block, float alpha,
                                        int32_t *__restrict__ D_dense,
                                        float *__restrict__ S_dense, float *__restrict__ I0,
                                        int ipitch, size_t ifs)
{
    extern __shared__ int32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y = blockIdx.x * rows_per_block + warp;
    const int f = blockIdx.y;
    int32_t *h = smem + (size_t)warp * (3 * (size_t)W + 32);  // g^2, or -1: empty column
    int32_t *stk = h + W;                                       // envelope sites per band
    int32_t *res = stk + W;                                     // D per pixel of the row
    int32_t *cnts = res + W;                                    // envelope size per band
    if (y >= H) return;  // the whole warp leaves together
    const int32_t *grow = g + (size_t)f * gfs + (size_t)y * gpitch;
    const int ginf = W + H;
    int any = 0;
    for (int x = lane; x < W; x += 32) {
        const int gv = grow[x];
        h[x] = gv >= ginf ? -1 : gv * gv;
        any |= gv < ginf ? 1 : 0;
    }
    any = __any_sync(0xffffffffu, any);
    __syncwarp();

    const int B = (W + 31) / 32;
    const int a = min(W, lane * B), b = min(W, a + B);  // this lane's band [a, b)
    int cnt = 0;
    for (int q = a; q < b; ++q) {
        if (h[q] < 0) continue;
        while (cnt >= 2 && hidden(stk[a + cnt - 2], stk[a + cnt - 1], q, h)) --cnt;
        stk[a + cnt++] = q;
    }
    cnts[lane] = cnt;
    __syncwarp();

    int k = 0;
    for (int x = a; x < b; ++x) {
        long long best = 0x7fffffffffffffffLL;
        if (any) {
            if (cnt > 0) {
                while (k + 1 < cnt && para(x, stk[a + k + 1], h) <= para(x, stk[a + k], h)) ++k;
                best = para(x, stk[a + k], h);
            }
            for (int dist = 1; dist < 32; ++dist) {
                bool progress = false;
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    const int L = side ? lane + dist : lane - dist;
                    if (L < 0 || L >= 32) continue;
                    const int la = min(W, L * B), lb = min(W, la + B);
                    if (la >= lb) continue;
                    const long long gap = side ? (long long)(la - x) : (long long)(x - (lb - 1));
                    if (gap * gap >= best) continue;
                    progress = true;
                    const int cL = cnts[L];
                    if (cL == 0) continue;
                    const int32_t *s = stk + la;
                    int lo = 0, hi = cL - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (para(x, s[mid + 1], h) <= para(x, s[mid], h)) lo = mid + 1;
                        else hi = mid;
                    }
                    const long long v = para(x, s[lo], h);
                    if (v < best) best = v;
                }
                if (!progress) break;
            }
        }
        res[x] = any ? (int32_t)best : kInfD;
    }
    __syncwarp();

    float *irow = I0 ? I0 + (size_t)f * ifs + (size_t)y * ipitch : nullptr;
    const size_t dbase = (size_t)f * W * H + (size_t)y * W;
    for (int x = lane; x < W; x += 32) {
        const int32_t D = res[x];
        float S = 1.0f;
        if (D != kInfD) S = 1.0f - expf(-sqrtf((float)D) / alpha);
        if (irow) irow[x] = 255.0f * S;
        if (D_dense) D_dense[dbase + x] = D;
        if (S_dense) S_dense[dbase + x] = S;
    }
}

// Caller-given surface (dense, d_exp in [0, 1]) to the level-0 intensity.
__global__ void surface_to_intensity_kernel(const float *__restrict__ S, int W, int H,
                                            float *__restrict__ I0, int pitch)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    I0[(size_t)y * pitch + x] = 255.0f * S[(size_t)y * W + x];
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

void launch_denoise_fill(const uint8_t *E, uint8_t *Ed, uint8_t *Edf, int W, int H, int pitch,
                         size_t frame_stride, int frames, int conn, int n_d, int n_f,
                         uint8_t *export_dense, DevStats *stats, cudaStream_t st)
{
    StageScope sc(kStDenoiseFill, 2, st);
    dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8, frames);
    denoise_kernel<<<grd, blk, 0, st>>>(E, Ed, W, H, pitch, frame_stride, conn, n_d);
    fill_kernel<<<grd, blk, 0, st>>>(Ed, Edf, W, H, pitch, frame_stride, conn, n_f,
                                     export_dense, stats);
}

void launch_edt_columns(const uint8_t *E, int edge_pitch, size_t edge_frame_stride, int W,
                        int H, int32_t *g, int g_pitch, size_t g_frame_stride, int frames,
                        cudaStream_t st)
{
    StageScope sc(kStEdtCols, 1, st);
    dim3 grd((W + 127) / 128, frames);
    edt_cols_kernel<<<grd, 128, 0, st>>>(E, edge_pitch, edge_frame_stride, W, H, g, g_pitch,
                                         g_frame_stride);
}

size_t edt_rows_smem(int W, int rows) { return (size_t)rows * (3 * (size_t)W + 32) * 4; }

int edt_rows_per_block(int W)
{
    int rows = kRowWarpsMax;
    while (rows > 1 && edt_rows_smem(W, rows) > 200 * 1024) --rows;
    return rows;
}

void launch_edt_rows_surface(const int32_t *g, int g_pitch, size_t g_frame_stride, int W, int H,
                             float alpha, int32_t *D_dense, float *S_dense, float *I0,
                             int i_pitch, size_t i_frame_stride, int frames, cudaStream_t st)
{
    const int rows = edt_rows_per_block(W);
    const size_t smem = edt_rows_smem(W, rows);
    StageScope sc(kStEdtRows, 1, st);
    dim3 grd((H + rows - 1) / rows, frames);
    edt_rows_surface_kernel<<<grd, 32 * rows, smem, st>>>(g, g_pitch, g_frame_stride, W, H, rows,
                                                          alpha, D_dense, S_dense, I0, i_pitch,
                                                          i_frame_stride);
}

void init_front_attributes()
{
    cudaFuncSetAttribute(edt_rows_surface_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         210 * 1024);
}

void launch_surface_to_intensity(const float *S, int W, int H, float *I0, int pitch,
                                 cudaStream_t st)
{
    StageScope sc(kStEdtRows, 1, st);
    dim3 grd((W + 255) / 256, H);
    surface_to_intensity_kernel<<<grd, 256, 0, st>>>(S, W, H, I0, pitch);
}

}  // namespace ebof
