// ebof_internal.cuh -- internal declarations shared by the CUDA translation
// units of libebof.so.  Nothing here is part of the C ABI (include/ebof.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>  // CUtensorMap (type only; the driver is reached through the runtime)
#include <cuda_runtime.h>

#include "ebof.h"

namespace ebof {

constexpr int kMaxLevels = 8;
constexpr int kMaxDim = 16384;
constexpr int kMaxPatch = 16;
constexpr int32_t kInfD = 2147483647;  // squared distance with no edge pixel

// Device error bits, latched in StreamState::d_err.
constexpr int kErrBounds = 1;
constexpr int kErrTimeout = 2;  // a bounded wait on an asynchronous copy ran out

__host__ __device__ inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Geometry of one pyramid level.  Internal images are row-major with a row
// pitch rounded up to 32 elements (128-byte rows for 4-byte types).
struct Level {
    int w, h, pitch;
    size_t plane;      // pitch * h elements
    int npx, npy;      // patch grid (reading F2); 0 if no patch fits
};

// Geometry of a whole frame: the level chain plus the level-0 pitches.
struct Geometry {
    int width, height;
    int levels;        // levels used by the flow (capped, reading F1)
    Level lv[kMaxLevels];
    size_t pyr_floats; // floats of one pyramid slot (I, Ix, Iy at every level)
    size_t pyr_off[kMaxLevels];  // offset of level l in a slot (I; Ix, Iy follow)
    int max_patches;   // largest npx * npy over the levels
};

Geometry make_geometry(int width, int height, int levels, int ps, int stride);

// The pyramid of one slot as the fused pyramid kernels see it.
struct PyrDesc {
    int levels;
    int w[kMaxLevels], h[kMaxLevels], pitch[kMaxLevels];
    size_t off[kMaxLevels];    // element offset of level l's I in a slot
    size_t plane[kMaxLevels];  // Ix and Iy follow I at one and two planes
    int blk0[kMaxLevels + 1];  // first block of level l in the gradient launch
    int gb0;                   // first block launched (blk0[1] when the box means
                               // kernel writes level 0's gradients, else 0)
};

// Per-window event counters kept on the device (one per batch slot).
struct DevStats {
    unsigned long long in_window;
    unsigned long long dropped_oob;
    unsigned long long edge_px;
    unsigned long long pad;
};

// Kernel parameter bundles ---------------------------------------------------

// Distance to surface value y(d), d = sqrt(D), and surface to level-0
// intensity: Eq. 1 (mode EBOF_SURFACE_EXP, intensity 255 y) or an ablation
// surface of §IV-D (intensity gain * y, gain = 255 / y(d_sat)).
struct SurfaceMap {
    int mode;
    float alpha;  // Eq. 1
    float d_sat;  // bound of DS_LB
    float gain;   // intensity scale of the ablation surfaces
};

inline SurfaceMap exp_surface(float alpha) { return SurfaceMap{0, alpha, 6.0f, 255.0f}; }

// Default bound, in mbarrier try-wait rounds, of a kernel's wait for a
// tensor copy.
constexpr long long kWaitLimitDefault = 1LL << 22;

struct FlowParams {
    bool half;  // pyramid stored as FP16 (loads widened to FP32)
    int ps, stride, gn_iters;
    float gn_damping;
    int var_outer, var_sor;
    float delta, gamma, alpha_s, omega;
    long long wait_limit;  // first wait of the copy-ahead SOR kernel (rounds)
    // variational layouts (ebof_params): none changes a result
    int coeff_cw_min_width, sor_tma_min_per_sm, sor_row_waves, var_cluster_max, coeff_cw_rows;
};

// Launchers (each enqueues on `st`; frames = batch size). ---------------------

// A1: clear edge images, scatter events of n_windows consecutive windows.
void launch_scatter(const uint16_t *x, const uint16_t *y, const int64_t *t, int64_t n,
                    int64_t t_begin, int64_t dt, int n_windows, int W, int H, int pitch,
                    uint8_t *E, size_t frame_stride, DevStats *stats,
                    unsigned long long *dropped_time, cudaStream_t st);

// A1 for a group of streams: frame f scatters the events of desc[f] (device).
void launch_scatter_desc(const ebof_window_desc *desc, int frames, int W, int H,
                         int pitch, uint8_t *E, size_t frame_stride, DevStats *stats,
                         unsigned long long *dropped_time, cudaStream_t st);

// A2: Alg. 1 then Alg. 2; writes E_df (pitched) and optional dense export.
void launch_denoise_fill(const uint8_t *E, uint8_t *Ed, uint8_t *Edf, int W, int H, int pitch,
                         size_t frame_stride, int frames, int conn, int n_d, int n_f,
                         uint8_t *export_dense, DevStats *stats, cudaStream_t st);

// A3: per-column distance to the nearest edge pixel (G_INF = W + H if none).
void launch_edt_columns(const uint8_t *E, int edge_pitch, size_t edge_frame_stride, int W,
                        int H, int32_t *g, int g_pitch, size_t g_frame_stride, int frames,
                        cudaStream_t st);

// A4: per-row lower envelope -> D, fused surface (Eq. 1 or an ablation
// surface) and level-0 intensity.
void launch_edt_rows_surface(const int32_t *g, int g_pitch, size_t g_frame_stride, int W, int H,
                             const SurfaceMap &sm, int32_t *D_dense, float *S_dense, void *I0,
                             int i_pitch, size_t i_frame_stride, int frames, bool half,
                             cudaStream_t st);
// The same with the Eq. 1 surface.
void launch_edt_rows_surface(const int32_t *g, int g_pitch, size_t g_frame_stride, int W, int H,
                             float alpha, int32_t *D_dense, float *S_dense, void *I0,
                             int i_pitch, size_t i_frame_stride, int frames, bool half,
                             cudaStream_t st);

// Per-device kernel attributes (opt-in shared memory); call with the device current.
void init_front_attributes();
void init_flow_attributes();

// Surface given by the caller -> level-0 intensity (255 d_exp, or gain * y).
void launch_surface_to_intensity(const float *S, int W, int H, void *I0, int pitch, bool half,
                                 const SurfaceMap &sm, cudaStream_t st);

// A5: every box-mean level and every level's gradients of `frames` slots
// starting at `slots` (level 0 must be in place), in two launches.
void launch_pyramid(void *slots, const Geometry &geo, size_t frame_stride, int frames, bool half,
                    cudaStream_t st);
// One plane of a level (row pitch `pitch`) into a dense w x h FP32 array.
void launch_pyramid_export(const void *plane, bool half, int w, int h, int pitch, float *dst,
                           cudaStream_t st);

// A6: patch inverse search at one level.
void launch_patch_search(const void *I0, const void *I0x, const void *I0y, const void *I1,
                         const Level &lv, size_t pyr_frame_stride, const float *Uc,
                         const Level *lvc, size_t uc_frame_stride, float *up,
                         size_t up_frame_stride, int frames, const FlowParams &fp,
                         int *err, cudaStream_t st);

// A7: densification.
void launch_densify(const void *I0, const void *I1, const Level &lv, size_t pyr_frame_stride,
                    const float *up, size_t up_frame_stride, float *U, size_t u_frame_stride,
                    int frames, const FlowParams &fp, cudaStream_t st);

// Tensor maps (TMA descriptors) of the variational coefficient planes of
// each pyramid level in a stream's or group's work buffer: level l holds
// frames x 9 planes of pitch_l x h_l floats, frame stride 9 planes.
struct CoefMaps {
    bool ok[kMaxLevels];
    CUtensorMap map[kMaxLevels];
};
// Fills m for `frames` frames of `work`; levels whose map cannot be encoded
// are marked not ok (their SOR sweeps then load the planes directly).
void make_coef_maps(float *work, const Geometry &geo, int frames, CoefMaps *m);

// A8: variational refinement of U.  Returns the buffer holding the result:
// U itself, or Utmp (same shape as U) when the fused kernel ping-pongs.
// coef_map: the level's coefficient tensor map, or nullptr; err: device
// error word (kErrTimeout if a bounded wait runs out).
float *launch_variational(const void *I0, const void *I0x, const void *I0y, const void *I1,
                          const Level &lv, size_t pyr_frame_stride, float *U, float *Utmp,
                          size_t u_frame_stride, float *work, size_t work_frame_stride,
                          int frames, const FlowParams &fp, const CUtensorMap *coef_map,
                          int *err, cudaStream_t st);
bool var_fused_supported(int var_sor);
void init_var_attributes();
float *launch_variational_fused(const void *I0, const void *I0x, const void *I0y,
                                const void *I1, const Level &lv, size_t pyr_frame_stride,
                                float *U, float *Utmp, size_t u_frame_stride, float *coef,
                                int frames, const FlowParams &fp, const CUtensorMap *coef_map,
                                int *err, cudaStream_t st);

// A9 for one window, destination pointer read from device memory.
void launch_flow_out_ptr(const float *U, int W, int H, int pitch, size_t u_frame_stride,
                         float *const *dst, int frames, cudaStream_t st);

// A9: level-0 flow to the caller's dense planar layout.
void launch_flow_out(const float *U, int W, int H, int pitch, size_t u_frame_stride,
                     float *flow, int frames, cudaStream_t st);

}  // namespace ebof
