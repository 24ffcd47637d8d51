/*
 * ebof.h -- C ABI of the GB300 event-based optical flow library (libebof.so).
 *
 * The library computes the event-to-flow path of Brebion, Moreau and
 * Davoine, "Real-Time Optical Flow for Vehicular Perception with Low- and
 * High-Resolution Event Cameras": the events (x, y, t, p) of a time window
 * go in (§III-A), a dense optical-flow field from the previous window to
 * this one comes out (§III-D).  Between the two, on one GPU:
 *   - the binary edge image of the window (§III-A),
 *   - denoising and filling (Alg. 1, Alg. 2 of §III-B),
 *   - the exact Euclidean distance transform, as int32 squared distances,
 *     and the inverse exponential distance surface d_exp (Eq. 1, §III-C),
 *   - a Dense Inverse Search flow block on 255 * d_exp (§III-D leaves the
 *     frame-based method open): image pyramid, per-patch inverse-
 *     compositional Gauss-Newton, patch densification, variational
 *     refinement,
 *   - per-stream device state holding the previous window's pyramid.
 *
 * Conventions for every call:
 *   - Pointers named d_* are DEVICE pointers on the stream's device; h_* are
 *     host pointers.  The caller owns all of them; they must stay valid until
 *     the work enqueued on `cuda_stream` has completed.
 *   - Images are dense row-major [height][width]; flow is planar
 *     [2][height][width] (u = x component first, then v), in pixels per
 *     window, mapping the previous window to the current one.
 *   - `cuda_stream` is a cudaStream_t (NULL = the legacy default stream).
 *     Calls only enqueue work; none synchronises the host except
 *     ebof_stream_sync and the *_host variants.
 *   - Argument errors are reported synchronously and enqueue nothing.
 *     Errors found on the device (a failed bounds check) are latched in the
 *     stream and reported by ebof_stream_sync.
 *   - Events outside the window or outside the image are not errors: they
 *     are dropped and counted.
 *   - One ebof_stream must not be used from two host threads at once
 *     (detected: EBOF_ERR_BUSY).  Distinct streams are independent.
 */
#ifndef EBOF_H
#define EBOF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EBOF_OK = 0,
    EBOF_NO_PREVIOUS = 1,          /* first window: surface built, flow zero-filled */
    EBOF_QUEUED = 2,               /* server: stream waits for memory to be admitted */
    EBOF_ERR_INVALID_ARG = -1,
    EBOF_ERR_OOM = -2,
    EBOF_ERR_CUDA = -3,
    EBOF_ERR_TIMEOUT = -4,
    EBOF_ERR_DEVICE_BOUNDS = -5,   /* a kernel's own bounds check fired */
    EBOF_ERR_UNSUPPORTED = -6,     /* parameter outside what the kernels support */
    EBOF_ERR_BUSY = -7,            /* stream used from two host threads */
    EBOF_ERR_CANCELLED = -8        /* server: window dropped before it ran */
} ebof_status;

/* Method parameters.  Fill with ebof_default_params, then override. */
typedef struct {
    uint32_t struct_size;   /* = sizeof(ebof_params); checked for ABI evolution */
    int32_t width, height;  /* 1 .. 16384 each */
    int32_t connectivity;   /* 4: the 4 direct neighbours of Alg. 1/2; 8: 3x3 ring */
    int32_t n_d;            /* Alg. 1 threshold; 0 disables denoising */
    int32_t n_f;            /* Alg. 2 threshold; > connectivity disables filling */
    float alpha;            /* Eq. 1 spreading parameter (1.08 = d_sat 6 px, Eq. 3) */
    int32_t levels;         /* pyramid levels (capped so each level holds a patch) */
    int32_t patch;          /* patch side ps, 4 .. 16 */
    int32_t stride;         /* patch grid stride, >= 1 */
    int32_t gn_iters;       /* Gauss-Newton iterations per patch, >= 0 */
    float gn_damping;       /* kappa: step solves (H + kappa trace(H) Id) d = b, >= 0 */
    int32_t var_outer;      /* variational fixed-point iterations, >= 0 */
    int32_t var_sor;        /* red-black SOR sweeps per fixed-point iteration, >= 0 */
    float var_delta;        /* data term weight */
    float var_gamma;        /* gradient-constancy weight */
    float var_alpha;        /* smoothness weight */
    float sor_omega;        /* SOR relaxation, 0 < omega < 2 */
    int32_t max_batch;      /* most windows one ebof_process_windows call may take */
    int32_t storage;        /* EBOF_STORAGE_FP32, or EBOF_STORAGE_FP16: surfaces, pyramid
                               levels and gradients stored in FP16 (half the bytes) as the
                               complement 255 (1 - d_exp), to which the flow is invariant;
                               patch sums, densification and the variational refinement
                               stay FP32 (the ablation surfaces are stored as they are) */
    int32_t surface;        /* ebof_surface: Eq. 1, or an ablation surface of §IV-D */
    float d_sat;            /* px: the bound of DS_LB, and the distance whose value
                               maps to intensity 255 for every ablation surface */
    /* Kernel layouts of the variational refinement: how the work is tiled,
     * never what is computed.  Every setting gives the same flow bit for bit
     * (the per-pixel arithmetic has a fixed rounding sequence in every kernel
     * form), so the autotuner picks them by time alone. */
    int32_t coeff_cw_min_width; /* levels at least this wide build their linear systems
                                   with the column-walk kernel (a warp per 28 columns x 8
                                   rows), narrower ones with 32x12 tiles; >= 1 (1024) */
    int32_t sor_tma_min_per_sm; /* SOR grids with at least this many 64x64 regions per
                                   SM take the persistent copy-ahead kernel; >= 1 (4
                                   below 1024 px wide, 2^20, i.e. never, from 1024 px) */
    int32_t sor_row_waves;      /* SOR grids that fit this many waves of 64x32 regions
                                   of one-row strips take that form; 0 = never (1) */
    int32_t var_cluster_max;    /* small levels: the whole refinement of a frame in one
                                   thread-block cluster launch (every outer iteration,
                                   cluster barriers between the phases) when the level's
                                   work fits a cluster of at most this many blocks and
                                   the call's clusters fit one wave; 0 = never (0) */
    int32_t coeff_cw_rows;      /* rows a warp of the column-walk kernel walks down (the
                                   strip's height): 4, 8 or 16 (8) */
} ebof_params;

/* Distance surface built from the EDT (§III-C) and handed to the flow block.
 * The ablation surfaces of §IV-D replace Eq. 1 by y(d) of the distance d and
 * are scaled to the flow's intensity by gain = 255 / y(d_sat); where a
 * window has no edge pixel they take their value at d = sqrt(INT32_MAX). */
typedef enum {
    EBOF_SURFACE_EXP = 0,      /* Eq. 1: d_exp = 1 - exp(-d / alpha), intensity 255 d_exp */
    EBOF_SURFACE_LINEAR = 1,   /* DS_L: y = d */
    EBOF_SURFACE_BOUNDED = 2,  /* DS_LB: y = min(d, d_sat) */
    EBOF_SURFACE_LOG = 3       /* DS_Log: y = ln(d + 1) */
} ebof_surface;

enum { EBOF_STORAGE_FP32 = 0, EBOF_STORAGE_FP16 = 1 };

/* Counts of one processed window. */
typedef struct {
    int64_t events;         /* events passed for this window (batched: whole call) */
    int64_t in_window;      /* events with t_begin <= t < t_end */
    int64_t dropped_time;   /* events outside [t_begin, t_end) (batched: whole call) */
    int64_t dropped_oob;    /* in-window events with x >= width or y >= height */
    int64_t edge_px;        /* edge pixels after denoising and filling */
    int32_t levels_used;    /* pyramid levels the flow used; 0 = no flow */
    int32_t has_flow;       /* 1 if a previous window existed */
} ebof_window_stats;

typedef struct ebof_stream ebof_stream;

/* Defaults for a width x height sensor: connectivity 8, n_d 1, filling off,
 * alpha 1.08 (§IV-A), the Eq. 1 surface with d_sat 6 px, 3 levels of 8x8
 * patches below 640 px width and 5 levels
 * of 12x12 patches from 640 px, stride 4, 12 Gauss-Newton iterations with
 * damping 0.1, 5 x 5
 * variational iterations (delta 5, gamma 10, alpha 20, omega 1.6),
 * max_batch 1, FP32 storage; layouts: column walk from 1024 px, copy-ahead
 * SOR from 4 regions per SM below 1024 px wide (never from 1024 px), one-row
 * SOR strips for one-wave grids, no cluster-resident refinement. */
void ebof_default_params(ebof_params *p, int32_t width, int32_t height);

/* Eq. 2 with eps = 1/255 (Eq. 3): alpha = d_sat / ln(255). */
float ebof_alpha_from_dsat(float d_sat);

/* Allocates all device state of one camera stream on `device` (about
 * 200 bytes per pixel per batch slot).  Returns EBOF_ERR_OOM if the device
 * memory is not available, EBOF_ERR_UNSUPPORTED for parameters the kernels
 * do not support.  *out is NULL on failure. */
ebof_status ebof_stream_create(const ebof_params *p, int device, ebof_stream **out);

/* Device bytes ebof_stream_create would allocate for these parameters (for
 * admission control against a memory budget), or -1 if they are invalid.
 * Allocates nothing.  The pipelined and streaming host calls allocate their
 * own buffers on first use, on top of this. */
int64_t ebof_stream_device_bytes(const ebof_params *p);

/* Frees the stream after waiting for its work.  NULL is accepted. */
ebof_status ebof_stream_destroy(ebof_stream *s);

/* Forgets the previous window: the next call returns EBOF_NO_PREVIOUS.
 * Waits for work already enqueued on the stream. */
ebof_status ebof_stream_reset(ebof_stream *s);

/* One window of events, passed by descriptor (ebof_process_window_list,
 * groups, the server).  Events outside [t_begin, t_end) or outside the
 * image are counted and ignored, as in ebof_process_window. */
typedef struct {
    const uint16_t *x;   /* device pointers, n_events each */
    const uint16_t *y;
    const int64_t *t;
    int64_t n_events;
    int64_t t_begin, t_end;  /* the window [t_begin, t_end) */
} ebof_window_desc;

/* One window (§III-A..§III-D).  d_x, d_y, d_t: n_events events (SoA);
 * d_p (polarity) may be NULL and is never read (§III-A ignores polarity).
 * Window = [t_begin, t_end), microseconds.  d_flow [2][H][W] is required.
 * Optional outputs (NULL to skip): d_edge [H][W] the denoised and filled
 * edge image (the paper's mask for restricting the flow, §III-D), d_edt
 * [H][W] squared distances (INT32_MAX when the window has no edge pixel),
 * d_surface [H][W] the surface (d_exp of Eq. 1, or y of the ablation
 * surface p->surface).  Returns EBOF_NO_PREVIOUS (flow zero)
 * for the first window after create/reset, else EBOF_OK.
 * With max_batch 1, no optional output and stage timing off, steady-state
 * calls replay a CUDA graph of the whole window (one per ping-pong slot,
 * captured on first use) after copying the call's pointers and counts to
 * the device; the results are identical to the step-by-step launches. */
ebof_status ebof_process_window(ebof_stream *s, const uint16_t *d_x, const uint16_t *d_y,
                                const int64_t *d_t, const int8_t *d_p, int64_t n_events,
                                int64_t t_begin, int64_t t_end, float *d_flow,
                                uint8_t *d_edge, int32_t *d_edt, float *d_surface,
                                void *cuda_stream);

/* n_windows consecutive windows of one stream in one call (1 <= n_windows
 * <= max_batch): window k is [t_begin + k*dt, t_begin + (k+1)*dt); every
 * event goes to the window its timestamp falls in.  Outputs are stacked per
 * window: d_flow [n][2][H][W], optional d_edge/d_edt/d_surface [n][H][W].
 * Flow k maps window k-1 to window k (window -1 = the stream's previous
 * window).  Same result as n_windows ebof_process_window calls. */
ebof_status ebof_process_windows(ebof_stream *s, int32_t n_windows, const uint16_t *d_x,
                                 const uint16_t *d_y, const int64_t *d_t, const int8_t *d_p,
                                 int64_t n_events, int64_t t_begin, int64_t dt,
                                 float *d_flow, uint8_t *d_edge, int32_t *d_edt,
                                 float *d_surface, void *cuda_stream);

/* n_windows (1 <= n_windows <= max_batch) consecutive windows of one stream
 * with arbitrary extents, in one call: windows[k] (HOST array, copied during
 * the call) gives window k's device events and interval, d_flows[k] (HOST
 * array of device pointers) its flow destination [2][H][W].  Flow k maps
 * window k-1 to window k (window -1 = the stream's previous window); every
 * stage runs once for all n windows.  In steady state (a previous window
 * exists, stage timing off) the call replays a CUDA graph of the n-window
 * sequence, one graph per n captured on first use, after copying the
 * descriptors to the device and, if needed, moving the previous window's
 * pyramid to the first slot.  Same results as n ebof_process_window calls.
 * The event buffers must stay valid until the work completes. */
ebof_status ebof_process_window_list(ebof_stream *s, int32_t n_windows,
                                     const ebof_window_desc *windows, float *const *d_flows,
                                     void *cuda_stream);

/* Flow block only (§III-D) on a caller-given surface d_surface [H][W] of the
 * stream's surface kind: d_exp in [0, 1] for Eq. 1 (the flow runs on
 * 255 * d_surface), y for an ablation surface (the flow runs on gain * y).
 * It becomes the stream's previous window.  Same return values as
 * ebof_process_window. */
ebof_status ebof_process_surface(ebof_stream *s, const float *d_surface, float *d_flow,
                                 void *cuda_stream);

/* Level `level` (0 = finest) of the pyramid of the stream's newest window, as
 * the flow block (§III-D) uses it: the 2x2 box-mean intensity image I_l and
 * its central differences (replicated border) Ix_l, Iy_l, each copied into a
 * dense caller-owned device array of [H_l][W_l] floats, H_l = H >> level,
 * W_l = W >> level (FP16 storage is widened exactly).  Any of d_I, d_Ix, d_Iy
 * may be NULL.  The copies are enqueued on `cuda_stream` after the stream's
 * work so far (pipelined calls included); later calls on the stream write
 * that pyramid only after them.  Returns EBOF_NO_PREVIOUS (nothing copied)
 * before the first window, EBOF_ERR_INVALID_ARG for a level outside
 * 0 .. levels_used - 1. */
ebof_status ebof_stream_get_pyramid(ebof_stream *s, int32_t level, float *d_I, float *d_Ix,
                                    float *d_Iy, void *cuda_stream);

/* ebof_process_window with HOST buffers: the events go to the device, the
 * window runs and the flow comes back into h_flow [2][H][W], all on
 * `cuda_stream`, which is then synchronised.  Pageable buffers are staged
 * through device memory with copies.  When every buffer lies, whole, inside
 * one page-locked range registered with CUDA (addressable by the device at
 * the same address), a window that has a previous one reads its events and
 * writes its flow in place over the host link, with no staging copies; the
 * result is the same.
 * The buffers must not be modified or freed until the call returns. */
ebof_status ebof_process_window_host(ebof_stream *s, const uint16_t *h_x, const uint16_t *h_y,
                                     const int64_t *h_t, int64_t n_events, int64_t t_begin,
                                     int64_t t_end, float *h_flow, void *cuda_stream);

/* Pipelined windows (§III-A..§III-D per window, as ebof_process_window):
 * for callers that stream windows and collect the flows later.  The call
 * enqueues and returns; the window's front end (events to the pyramid) runs
 * on an internal stream after the caller's work on `cuda_stream` so far, and
 * its flow after its front end on one of four internal flow streams, in
 * turn, each with its own scratch buffers, over eight pyramid slots of the
 * stream's own: a window's front end and the flows of four consecutive
 * windows (each pair's flow depends only on their pyramids, §III-D) overlap
 * one another, the latency-bound coarse levels of one window filling the
 * SMs that another window's levels leave idle.  Nothing is enqueued on
 * `cuda_stream`: d_flow holds the flow, and the event buffers may be reused,
 * once ebof_stream_sync(s) returns.  Calls may share d_flow: its writes then
 * follow the call order (the later window waits for the earlier one), so
 * it ends with the newest flow.  Results are bit-identical to
 * ebof_process_window; the two kinds of call may be mixed on one stream
 * (the newest window's pyramid is handed over with one device copy).
 * Same return values; EBOF_ERR_OOM if the pipeline's buffers (eight pyramid
 * slots and three scratch sets: about 260 MB at 1280x720 FP32) cannot be
 * allocated. */
ebof_status ebof_process_window_async(ebof_stream *s, const uint16_t *d_x, const uint16_t *d_y,
                                      const int64_t *d_t, const int8_t *d_p, int64_t n_events,
                                      int64_t t_begin, int64_t t_end, float *d_flow,
                                      void *cuda_stream);

/* ebof_process_window_async with HOST buffers.  When every buffer lies,
 * whole, inside one page-locked range registered with CUDA, the call only
 * enqueues and returns: the events are copied in on an internal copy stream,
 * the window runs pipelined as in ebof_process_window_async, and the flow is
 * copied out into h_flow on a second internal copy stream, through five
 * device staging slots used in turn, so that a window's copies
 * overlap its neighbours' kernels.  `cuda_stream` is not used.  h_flow holds
 * the flow once ebof_stream_sync(s) returns; the buffers must stay valid and
 * unmodified until then.  Otherwise (pageable buffers) it is
 * ebof_process_window_host itself, synchronous.  Same return values;
 * EBOF_ERR_OOM if the staging slots cannot be made. */
ebof_status ebof_process_window_host_async(ebof_stream *s, const uint16_t *h_x,
                                           const uint16_t *h_y, const int64_t *h_t,
                                           int64_t n_events, int64_t t_begin, int64_t t_end,
                                           float *h_flow, void *cuda_stream);

/* Makes the work enqueued on `cuda_stream` after this call wait for
 * everything the stream `s` has enqueued so far, including the pipelined
 * windows and their copies out (without blocking the host). */
ebof_status ebof_stream_join(ebof_stream *s, void *cuda_stream);

/* Waits for the stream's work, then reports the first device-side error
 * (if any) and copies the counts of the last call's windows into out[0..
 * n_out-1] (n_out may be 0 and out NULL).  The latched error is cleared. */
ebof_status ebof_stream_sync(ebof_stream *s, ebof_window_stats *out, int32_t n_out);

/* Exact squared EDT and Eq. 1 surface of a caller-given binary edge image
 * d_edge [H][W] (non-zero = edge pixel): the separable passes of §III-C.
 * d_scratch: caller-owned device buffer of at least width*height int32
 * (column distances).  d_edt [H][W] required; d_surface [H][W] optional.
 * No per-stream state is used. */
ebof_status ebof_edt(const uint8_t *d_edge, int32_t width, int32_t height, int32_t *d_scratch,
                     int32_t *d_edt, float *d_surface, float alpha, void *cuda_stream);

/* ebof_edt without caller scratch, for callers that cannot allocate device
 * memory: code that must not call cudaMalloc once running (a real-time loop
 * where an allocation may synchronise the device and has no latency bound),
 * or code inside a host framework that owns all device memory through its
 * own allocator.  The paper has no counterpart; this is a deployment variant
 * of the separable EDT entry point above.
 * Same inputs, outputs and result as ebof_edt, but the column distances are
 * kept in a static device array of 2^21 int32 (8 MiB) that every device
 * which loads the library holds until the process exits, so width*height
 * must not exceed 2^21 (EBOF_ERR_INVALID_ARG otherwise).  The call
 * allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 * Its first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The looked-up address is kept for the life of
 * the process, so after cudaDeviceReset on a device this entry point must
 * not be called on that device again.  All calls share the one array, and each call
 * overwrites every entry it reads, so nothing carries over from the previous
 * call; calls that overlap on the GPU (on different streams, or from
 * different threads without ordering) race on the array and give wrong
 * results. */
ebof_status ebof_edt_static(const uint8_t *d_edge, int32_t width, int32_t height,
                            int32_t *d_edt, float *d_surface, float alpha, void *cuda_stream);

/* ---- Flow Warping Loss (§IV-C) -------------------------------------------
 * Quality of a flow without ground truth.  The window's events are moved
 * back along the flow to t_begin and accumulated with their polarity into
 * I_comp (bilinear votes; votes outside the image are dropped); I_uncomp
 * accumulates the same events unmoved (one vote at their pixel).  FWL =
 * var(I_comp) / var(I_uncomp), the variances over all width*height pixels;
 * FWL = 1 when var(I_uncomp) = 0.  Above 1 the flow beats the zero flow.
 * d_flow [2][H][W]: pixels per window as ebof_process_window returns it,
 * read at each event's pixel; an event at time t moves by
 * -flow * (t - t_begin) / (t_end - t_begin).  Only events with
 * t_begin <= t < t_end inside the image count.  d_p: polarity per event
 * (+1 / -1), or NULL to count every event as +1.  d_scratch: caller-owned
 * device memory of ebof_fwl_scratch_bytes(width, height) bytes.  d_out:
 * device double[3] = {FWL, var(I_comp), var(I_uncomp)}, written on
 * cuda_stream (read it after synchronising).  Allocates nothing; I_comp is
 * summed with float atomics, so its last bits depend on the vote order. */
size_t ebof_fwl_scratch_bytes(int32_t width, int32_t height);
ebof_status ebof_fwl(const uint16_t *d_x, const uint16_t *d_y, const int64_t *d_t,
                     const int8_t *d_p, int64_t n_events, int64_t t_begin, int64_t t_end,
                     const float *d_flow, int32_t width, int32_t height, void *d_scratch,
                     double *d_out, void *cuda_stream);

/* ---- multi-stream groups -------------------------------------------------
 * A group holds n camera streams of one resolution and steps them in
 * lockstep: one ebof_group_process call takes one window of every stream
 * and runs each stage once for all of them (every kernel gets the n windows
 * in its grid), so small frames still fill the GPU.  From the second call
 * on, the whole step is replayed as one CUDA graph per ping-pong parity
 * (captured on first use); only the window descriptors are copied in
 * before each replay.  Streams of other resolutions go in other groups,
 * which may run concurrently on other CUDA streams.  Results per stream are
 * bit-identical to an ebof_stream fed the same windows. */
typedef struct ebof_group ebof_group;

/* Allocates the state of n_streams streams (1 .. 4096) with parameters p
 * (p->max_batch is ignored) on `device`, including the group-owned flow
 * buffer [n][2][H][W]. */
ebof_status ebof_group_create(const ebof_params *p, int32_t n_streams, int device,
                              ebof_group **out);
ebof_status ebof_group_destroy(ebof_group *g);           /* NULL-safe; waits for work */
ebof_status ebof_group_reset(ebof_group *g);             /* every stream forgets its window */

/* One window per stream.  h_desc: HOST array of n_streams descriptors
 * (copied during the call).  d_flow: optional device [n][2][H][W]; the flow
 * also stays in the group's buffer (ebof_group_flow).  Returns
 * EBOF_NO_PREVIOUS on the first step (flows zero). */
ebof_status ebof_group_process(ebof_group *g, const ebof_window_desc *h_desc, float *d_flow,
                               void *cuda_stream);

/* Device pointer to stream k's flow of the last step ([2][H][W]); valid until
 * the next ebof_group_process. */
const float *ebof_group_flow(const ebof_group *g, int32_t k);

/* As ebof_stream_sync, for the group's streams (out[k] = stream k). */
ebof_status ebof_group_sync(ebof_group *g, ebof_window_stats *out, int32_t n_out);

/* Groups of different resolutions stepped together as ONE CUDA graph: each
 * group's step (every stage once for its streams) is one branch of the graph,
 * the branches forked from and joined into the caller's stream, so the
 * resolutions run concurrently and a step costs one graph launch.  Each
 * stage is still one launch per group (per resolution).  The groups stay
 * owned by the caller and must outlive the multigroup; they must not be
 * stepped on their own while it is in use.  The first step of a group, and
 * steps with stage timing on, run eagerly; later steps replay one graph per
 * pattern of the groups' ping-pong parities, captured on first use.
 * Results per stream are bit-identical to stepping each group alone. */
typedef struct ebof_multigroup ebof_multigroup;

/* n_groups (1 .. 64) distinct groups on one device. */
ebof_status ebof_multigroup_create(ebof_group *const *groups, int32_t n_groups,
                                   ebof_multigroup **out);
ebof_status ebof_multigroup_destroy(ebof_multigroup *m);  /* NULL-safe; waits for work */

/* One window per stream of every group: h_descs[i] is a HOST array of
 * groups[i]'s n_streams descriptors (copied during the call).  Flows stay in
 * each group's buffer (ebof_group_flow); errors and counts through
 * ebof_group_sync.  Returns EBOF_NO_PREVIOUS when some group had no previous
 * window, EBOF_ERR_BUSY if another thread uses one of the groups. */
ebof_status ebof_multigroup_process(ebof_multigroup *m, const ebof_window_desc *const *h_descs,
                                    void *cuda_stream);

/* Fused steps (§8(f) batched multi-stream; the method per stream is
 * unchanged, §III-A..§III-D).  fused = 1: from the next captured step on,
 * every stage of the step is ONE kernel launch for the streams of all
 * groups, whatever their resolutions and event counts: a block finds its
 * (group, frame, tile) in a table built on the host once per parity pattern
 * and passed in the launch's constant bank, and the scatter walks a device
 * work list of 4096-event chunks over all windows, so uneven windows spread
 * over every block.  Pyramid levels are aligned at the coarsest level: the
 * j-th flow level step runs level L - 1 - j of every group with L > j
 * levels (the small levels of a large resolution share launches with the
 * larger levels of a small one); a step with one group left runs that
 * group's own launches.  Groups that differ in storage type, patch size or
 * search lane layout at a step take one launch per kind there; more than 8
 * groups take one launch per 8.  fused = 2: the front-end stages (§III-A
 * to the pyramid) so, the flow levels of each group as a concurrent branch
 * of the step's graph.  Results are bit-identical to fused = 0 (default:
 * one launch per stage and group, the groups as concurrent graph branches).  The first step of a group and
 * steps with stage timing still run each group's own launches.  Returns
 * EBOF_ERR_UNSUPPORTED if a group has more than 6 pyramid levels or (mode
 * 1) more SOR sweeps than the register-resident SOR regions hold,
 * EBOF_ERR_INVALID_ARG for another mode, EBOF_ERR_BUSY if
 * another thread uses one of the groups.  Changing the mode waits for the
 * groups' work and drops the captured graphs. */
ebof_status ebof_multigroup_set_fused(ebof_multigroup *m, int32_t fused);

/* ---- serving loop ---------------------------------------------------------
 * A server runs many camera streams on one GPU as their windows arrive.
 * §IV (Real-Time Compliance) runs one sensor per pipeline and counts a flow
 * as real time when each window (4-13 ms of events) is processed before the
 * next one ends; the server carries that setting to many sensors sharing a
 * GPU.  It is a deployment layer with no counterpart in the paper's method.
 *  - Admission: a stream's device state (ebof_stream_device_bytes of its
 *    parameters, which include its batch limit max_batch) is allocated when
 *    it is admitted and stays resident until it is closed.  Streams are
 *    admitted in the order they were opened while the total fits the
 *    memory budget; one that does not fit waits (EBOF_QUEUED) until closed
 *    streams free enough memory.
 *  - Submission: each window goes to its stream's FIFO with the caller's
 *    tag and arrival time; its events and flow destination must stay valid
 *    until its completion is reported.
 *  - Continuous batching: a dispatcher thread keeps up to n_workers batches
 *    in flight, each on its own CUDA stream.  When a worker frees up it takes
 *    the stream whose oldest queued window arrived first and has no batch in
 *    flight, and launches that stream's queued windows (up to its max_batch)
 *    as one ebof_process_window_list call.  Batches grow with the backlog.
 *  - Completion: one ebof_completion per window, in completion order.
 * Every window's flow is bit-identical to feeding the same stream's windows
 * to ebof_process_window one by one. */
typedef struct ebof_server ebof_server;

typedef struct {
    int32_t struct_size;    /* sizeof(ebof_server_config) */
    int32_t device;
    int64_t memory_budget;  /* bytes of device state admitted streams may hold */
    int32_t n_workers;      /* batches in flight at once, 1..64 */
} ebof_server_config;

typedef struct {
    int32_t stream_id;
    int32_t status;       /* EBOF_OK; EBOF_NO_PREVIOUS for a stream's first
                             window (flow zero); EBOF_ERR_CANCELLED; or the
                             error of the launch */
    uint64_t tag;         /* as given to ebof_server_submit */
    int64_t arrival_ns;   /* ebof_now_ns clock */
    int64_t launch_ns;    /* the dispatcher launched its batch */
    int64_t done_ns;      /* the dispatcher saw the batch complete */
    int32_t batch;        /* windows in that batch */
    int32_t index;        /* this window's position in it */
} ebof_completion;

typedef struct {
    int32_t streams_admitted, streams_waiting;
    int64_t memory_budget, memory_in_use;
    int64_t windows_submitted, windows_completed, batches_launched;
    int32_t batches_in_flight, max_batch_seen;
} ebof_server_info;

/* Monotonic clock (nanoseconds) of the arrival and completion times. */
int64_t ebof_now_ns(void);

/* device 0, a 40 GB (40e9 bytes) budget, 8 workers. */
void ebof_server_default_config(ebof_server_config *c);

/* Creates the server and its dispatcher thread and worker CUDA streams. */
ebof_status ebof_server_create(const ebof_server_config *c, ebof_server **out);

/* Drops queued windows (no completions), waits for the batches in flight,
 * frees every stream.  NULL is accepted. */
ebof_status ebof_server_destroy(ebof_server *v);

/* Opens a stream with parameters p (validated as by ebof_stream_create) and
 * returns its id.  EBOF_OK: admitted, state allocated.  EBOF_QUEUED: waits
 * for memory; windows may be submitted meanwhile.  EBOF_ERR_OOM: its state
 * is larger than the whole budget, or the allocation failed. */
ebof_status ebof_server_open_stream(ebof_server *v, const ebof_params *p, int32_t *id);

/* No further windows for the stream.  Its queued windows still run; then its
 * state is freed and waiting streams are admitted.  A stream still waiting
 * for admission is dropped and its windows complete as EBOF_ERR_CANCELLED. */
ebof_status ebof_server_close_stream(ebof_server *v, int32_t id);

/* Queues one window (descriptor copied; device pointers kept) whose flow
 * [2][H][W] goes to d_flow.  arrival_ns: when the window became available
 * (ebof_now_ns clock; 0 = now), the start of its latency. */
ebof_status ebof_server_submit(ebof_server *v, int32_t id, const ebof_window_desc *w,
                               float *d_flow, uint64_t tag, int64_t arrival_ns);

/* Moves up to max_out completions into out, waiting up to wait_us
 * microseconds for the first; returns how many (>= 0) or an error (< 0). */
int32_t ebof_server_poll(ebof_server *v, ebof_completion *out, int32_t max_out,
                         int32_t wait_us);

/* Waits up to timeout_ms until every submitted window has completed
 * (EBOF_ERR_TIMEOUT otherwise).  Completions stay queued for poll. */
ebof_status ebof_server_drain(ebof_server *v, int32_t timeout_ms);

ebof_status ebof_server_get_info(ebof_server *v, ebof_server_info *out);

/* ---- tracing: per-stage CUDA-event timing (§IV Table VII reports per-block
 * times; these are the GPU equivalents).  Timing brackets each stage's
 * launches with cudaEvents on the caller's stream; it is off by default. */
typedef enum {
    EBOF_STAGE_SCATTER = 0,      /* edge image (§III-A) */
    EBOF_STAGE_DENOISE_FILL,     /* Alg. 1 + Alg. 2 */
    EBOF_STAGE_EDT_COLS,         /* EDT column pass */
    EBOF_STAGE_EDT_ROWS_SURFACE, /* EDT row pass + Eq. 1 */
    EBOF_STAGE_PYRAMID,          /* downsampling + gradients */
    EBOF_STAGE_PATCH_SEARCH,     /* inverse search */
    EBOF_STAGE_DENSIFY,          /* densification */
    EBOF_STAGE_VAR_WARP,         /* variational: warp */
    EBOF_STAGE_VAR_COEFF,        /* variational: linearised system */
    EBOF_STAGE_VAR_SOR,          /* variational: SOR sweeps */
    EBOF_STAGE_VAR_ADD,          /* variational: U += dU */
    EBOF_STAGE_FLOW_OUT,         /* flow to the caller's layout */
    EBOF_STAGE_COUNT
} ebof_stage;

/* Enables (1) or disables (0) stage timing and clears the accumulators. */
ebof_status ebof_stream_set_profiling(ebof_stream *s, int32_t enable);

/* Waits for the recorded stages, then writes the accumulated milliseconds
 * and kernel launch counts per stage into ms[0..n-1] and launches[0..n-1]
 * (either may be NULL; n <= EBOF_STAGE_COUNT). */
ebof_status ebof_stream_get_profile(ebof_stream *s, double *ms, int64_t *launches, int32_t n);

/* As ebof_stream_get_profile, for the launches of one pyramid level only
 * (level -1: the stages that are not per level, e.g. the EDT). */
ebof_status ebof_stream_get_profile_level(ebof_stream *s, int32_t level, double *ms,
                                          int64_t *launches, int32_t n);

/* Name of a stage ("scatter", "patch_search", ...). */
const char *ebof_stage_name(int32_t stage);

/* Kernels this library has launched in the process so far (all streams). */
uint64_t ebof_kernel_launches(void);

/* ---- diagnostics: failure injection for tests ------------------------------
 * Both act on the host side only and change nothing a kernel computes.  The
 * paper has no counterpart; they let tests drive the error paths above
 * without faulting a GPU. */

/* Bound, in mbarrier try-wait rounds, of the first wait of the batched SOR
 * kernel (the copy-ahead form, used when a call's variational grid has at
 * least four regions per SM) for a region's coefficient copy.  When it runs
 * out the kernel latches EBOF_ERR_TIMEOUT, reported by ebof_stream_sync, lets
 * the copy in flight land under a second wait at the default bound, and
 * leaves the flow of that call undefined.  Applies to launches enqueued
 * after the call (graphs captured earlier keep their bound); iterations < 0
 * restores the default, 2^22; 0 makes every such wait run out at once.
 * EBOF_ERR_BUSY while another thread uses the stream. */
ebof_status ebof_stream_set_wait_limit(ebof_stream *s, int64_t iterations);

/* The next n device allocations of this library (all threads, all streams)
 * succeed and the one after fails the way cudaMalloc fails when the device is
 * out of memory; the hook then disarms itself.  n < 0 disarms it.  The call
 * that meets the failure returns EBOF_ERR_OOM after freeing what it had
 * allocated; an existing stream stays usable. */
void ebof_debug_fail_allocation(int32_t n);

/* Static text for a status code. */
const char *ebof_status_string(ebof_status st);

#ifdef __cplusplus
}
#endif

#endif /* EBOF_H */
