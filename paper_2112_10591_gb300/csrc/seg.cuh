// seg.cuh -- fused launches over several groups of streams of different
// resolutions (one launch per stage for all of them).
//
// A fused launch runs the blocks of up to kMaxSeg segments as one grid.  A
// segment is one group's share of the stage: its own level size, buffers,
// frame strides, parameters and block grid (gx x gy x frames).  Block b
// belongs to the segment s with first[s] <= b < first[s + 1] and runs block
// b - first[s] of that segment's grid, with the same code and the same
// arithmetic as the per-group kernel, so every result is bit-identical to
// the group's own launch.  A table is built on the host once per step
// pattern and passed as a __grid_constant__ kernel parameter: it sits in
// the launch's constant bank, where the block-uniform segment fields are
// read without occupying a thread's registers.  The scatter stage instead
// walks a device work list of event chunks over all windows (ScatterWin).
#pragma once

#include "ebof.h"
#include "ebof_internal.cuh"

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace ebof {

constexpr int kMaxSeg = 8;

template <class A>
struct SegTable {
    int n;                   // segments
    int first[kMaxSeg + 1];  // first block of each segment; first[n] = blocks
    A a[kMaxSeg];
};

#ifdef __CUDACC__
// The segment of this block and the block's index within it.
template <class A>
__device__ __forceinline__ const A &seg_of(const SegTable<A> &t, int &local)
{
    const int b = blockIdx.x, n = t.n;
    int s = 0;
    while (s + 1 < n && b >= t.first[s + 1]) ++s;
    local = b - t.first[s];
    return t.a[s];
}
#endif

// A1: one window of the scatter work list.
struct ScatterWin {
    const ebof_window_desc *desc;  // the window's events (device descriptor)
    uint8_t *E;                    // its edge image
    DevStats *stats;               // its counters
    unsigned long long *dropped_time;  // its group's out-of-window count
    int W, H, pitch;
};
constexpr int kScatterListMax = 1024;  // windows per fused scatter launch
constexpr int kScatterChunk = 4096;    // events per work item

// A2: gx x gy tiles of 32 x 8 per frame.
struct SegDenoise {
    const uint8_t *E;
    uint8_t *Edf;
    DevStats *stats;
    size_t fs;
    int W, H, pitch, conn, n_d, n_f, gx, gy;
};

// A3: gx blocks of 32 columns per frame, chunks of CH rows.
struct SegEdtCols {
    const uint8_t *E;
    int32_t *g;
    size_t efs, gfs;
    int epitch, gpitch, W, H, CH, nch, gx;
};

// A4: gx blocks of `rows` rows (one warp each) per frame.
struct SegEdtRows {
    const int32_t *g;
    void *I0;
    size_t gfs, ifs;
    SurfaceMap sm;
    int gpitch, ipitch, W, H, rows, gx;
};

// A5: the pyramid of one slot per frame; means: gx x gy level-1 tiles (and
// level 0's gradients), gradients: gx blocks over the other levels.
struct SegPyr {
    void *slots;
    size_t fs;
    PyrDesc d;
    int gx, gy;
};

// A6: gx blocks of patches per frame.
struct SegSearch {
    const void *I0, *I0x, *I0y, *I1;
    const float *Uc;  // coarser level's flow, or null
    float *up;
    int *err;
    size_t pfs, plane_c, ucfs, upfs;
    int w, h, pitch, npx, npy, wc, hc, pitch_c, stride, iters, gx;
    float kappa;
};

// A7: gx x gy tiles of 32 x 8 pixels per frame.
struct SegDensify {
    const void *I0, *I1;
    const float *up;
    float *U;
    size_t pfs, upfs, ufs, plane;
    int w, h, pitch, npx, npy, ps, stride, gx, gy;
};

// A8: the coefficient tiles (gx x gy per frame) of one outer iteration.
struct SegCoeff {
    const void *I0, *I0x, *I0y, *I1;
    const float *U;
    float *coef;
    size_t pfs, ufs, plane, cfs;
    int w, h, pitch, gx, gy;
    float delta, gamma, alpha_s, omega;
};

// A8: the SOR regions (gx x gy per frame) of one outer iteration.
struct SegSor {
    const float *Uin;
    float *Uout;
    const float *coef;
    size_t ufs, plane, cfs;
    int w, h, pitch, R, n_half, gx, gy;
    float omega;
};

// A9: rows of gx x 256 pixels per frame into [frames][2][H][W].
struct SegFlowOut {
    const float *U;
    float *flow;
    size_t ufs, plane;
    int W, H, pitch, gx;
};

// Launchers: `blocks` = first[n] of the table (the scatter list: its grid
// is sized on the host, every block walks the work list).
void launch_seg_scatter(const ScatterWin *wins, int n_wins, int blocks, cudaStream_t st);
void launch_seg_denoise_fill(const SegTable<SegDenoise> &t, int blocks, cudaStream_t st);
void launch_seg_edt_cols(const SegTable<SegEdtCols> &t, int blocks, int nch_max,
                         cudaStream_t st);
void launch_seg_edt_rows(const SegTable<SegEdtRows> &t, int blocks, int rows_max,
                         size_t smem, bool half, cudaStream_t st);
void launch_seg_pyr_means(const SegTable<SegPyr> &t, int blocks, bool half, cudaStream_t st);
void launch_seg_pyr_grads(const SegTable<SegPyr> &t, int blocks, bool half, cudaStream_t st);
// ps: patch size, wide: the wide lane layout
void launch_seg_search(const SegTable<SegSearch> &t, int blocks, int ps, bool wide, bool half,
                       cudaStream_t st);
// nc: covering patches per axis as launch_densify chooses it
void launch_seg_densify(const SegTable<SegDensify> &t, int blocks, int nc, bool half,
                        cudaStream_t st);
void launch_seg_coeff(const SegTable<SegCoeff> &t, int blocks, bool half, cudaStream_t st);
void launch_seg_sor(const SegTable<SegSor> &t, int blocks, cudaStream_t st);
void launch_seg_flow_out(const SegTable<SegFlowOut> &t, int blocks, cudaStream_t st);

// Block shapes the host needs to build the tables.
int edt_rows_block_rows(int W);        // rows per block of the one-warp row layout
size_t edt_rows_smem(int W, int rows);  // dynamic shared memory of such a block
void edt_cols_chunks(int H, int &CH, int &nch);
int search_patches_per_block(int ps, bool wide);
bool search_wide(int n_patches);
int sor_tile_x(int R);                 // interior columns of a SOR region
int sor_tile_y(int R);                 // interior rows of a SOR region
void coeff_tile_shape(int &x, int &y);  // pixels of a coefficient tile
int coeff_planes();                    // coefficient planes per level and frame
int seg_max_levels();                  // pyramid levels the fused pyramid kernels build
PyrDesc make_pyr_desc(const Geometry &geo);

}  // namespace ebof
