// capi.cu -- the C ABI of include/ebof.h: per-stream device state, argument
// checks, stage sequencing and error reporting.  All compute is in the
// kernels of k_front.cu and k_flow.cu; this file only allocates, validates
// and enqueues.
#include "ebof.h"
#include "ebof_internal.cuh"
#include "profiler.cuh"
#include "seg.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <memory>
#include <new>
#include <vector>

using namespace ebof;

namespace ebof {

Geometry make_geometry(int width, int height, int levels, int ps, int stride)
{
    Geometry g;
    std::memset(&g, 0, sizeof(g));
    g.width = width;
    g.height = height;
    int L = 0;
    while (L < levels && L < kMaxLevels && (width >> L) >= ps && (height >> L) >= ps) ++L;
    g.levels = L;
    const int nalloc = std::max(L, 1);  // level 0 always exists (the surface)
    size_t off = 0;
    g.max_patches = 0;
    for (int l = 0; l < nalloc; ++l) {
        Level &lv = g.lv[l];
        lv.w = width >> l;
        lv.h = height >> l;
        lv.pitch = round_up(lv.w, 32);
        lv.plane = (size_t)lv.pitch * lv.h;
        lv.npx = lv.w >= ps ? (lv.w - ps + stride - 1) / stride + 1 : 0;
        lv.npy = lv.h >= ps ? (lv.h - ps + stride - 1) / stride + 1 : 0;
        g.max_patches = std::max(g.max_patches, lv.npx * lv.npy);
        g.pyr_off[l] = off;
        off += 3 * lv.plane;
    }
    g.pyr_floats = off;
    return g;
}

}  // namespace ebof

struct ebof_stream {
    ebof_params p;
    int device;
    Geometry geo;
    int pitch0;
    size_t e_fs, g_fs, pyr_fs, up_fs, u_fs, work_fs;
    uint8_t *E = nullptr, *Ed = nullptr, *Edf = nullptr;
    int32_t *g = nullptr;
    char *pyr = nullptr;  // pyramid slots, es bytes per element
    size_t es = 4;
    int nslots = 0, head = 0;
    bool has_prev = false;
    float *up = nullptr, *Ua = nullptr, *Ub = nullptr, *work = nullptr;
    DevStats *dstats = nullptr;
    unsigned long long *d_dropped_time = nullptr;
    int *d_err = nullptr;
    float *flow_stage = nullptr;  // device flow for the host-buffer call
    void *ev_stage = nullptr;     // device events for the host-buffer call
    size_t ev_stage_bytes = 0;
    // bookkeeping of the last call
    int last_n = 0;
    int64_t last_events = 0;
    bool last_had_prev = false;
    cudaEvent_t done = nullptr;
    cudaStream_t last_stream = nullptr;
    bool have_last = false;
    std::atomic<int> busy{0};
    long long wait_limit = kWaitLimitDefault;  // ebof_stream_set_wait_limit
    Profiler prof;
    // Per-call window descriptors and flow destinations, read on the device by
    // the descriptor-driven paths: [max_batch] ebof_window_desc followed by
    // [max_batch] float*, staged from h_call by one copy per call.
    char *d_call = nullptr;
    std::vector<char> h_call;
    ebof_window_desc *d_wins = nullptr;
    float **d_flows = nullptr;
    // single-window graph replays (one graph per ping-pong slot)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    long long graph_kernels[2] = {0, 0};
    // list calls: graph [n] replays n windows with the previous one in slot 0
    std::vector<cudaGraphExec_t> list_graph;
    std::vector<long long> list_graph_kernels;
    std::vector<int64_t> last_win_events;  // per window, after a list call
    bool last_list = false;
    cudaStream_t cap = nullptr;
    CoefMaps cmaps;  // tensor maps of the variational coefficient planes per level
    // asynchronous host-buffer calls (ebof_process_window_host_async): the
    // events go in on stream h2d, the flow comes back on stream d2h, both
    // through device staging slots used in turn, so that the copies of one
    // window overlap the kernels of its neighbours
    struct HostPipe {
        static constexpr int kSlots = 5;  // more than the flows in flight
        cudaStream_t h2d = nullptr, d2h = nullptr;
        cudaEvent_t in_done[kSlots] = {}, run_done[kSlots] = {}, out_done[kSlots] = {};
        bool used[kSlots] = {};
        void *ev[kSlots] = {};
        size_t ev_bytes[kSlots] = {};
        float *flow[kSlots] = {};
        int slot = 0;
        bool ready = false;
    } pipe;
    // pipelined calls (ebof_process_window_async, ebof_process_window_host_async):
    // a window's front end (A1-A5) runs on stream `front`, its flow (A6-A9)
    // on flow[k % kFlows] with scratch set k % kFlows, and the pipeline keeps
    // 2 kFlows pyramid slots of its own, so that a window's front end and the
    // flows of kFlows consecutive windows overlap one another
    struct Pipeline {
        static constexpr int kFlows = 4, kSlots = 2 * kFlows;
        bool ready = false;
        cudaStream_t front = nullptr, flow[kFlows] = {};
        char *pyr = nullptr;   // kSlots slots
        char *call = nullptr;  // per slot: the window's descriptor and flow destination
        std::vector<char> h_call;
        // scratch sets 1 .. kFlows - 1 (set 0: the stream's own buffers)
        float *up[kFlows] = {}, *Ua[kFlows] = {}, *Ub[kFlows] = {}, *work[kFlows] = {};
        int head = 0;            // slot of the newest window
        bool has_prev = false;   // the newest window is in these slots
        bool latest = false;     // these slots, not the ordinary ones, hold the newest window
        cudaEvent_t inputs = nullptr;
        cudaEvent_t front_done[kSlots] = {}, flow_done[kSlots] = {};
        bool flow_used[kSlots] = {};
        float *dflow[kSlots] = {};  // the flow destination of each slot's window
        cudaGraphExec_t front_graph[kSlots] = {}, flow_graph[kSlots] = {};
        long long front_k[kSlots] = {}, flow_k[kSlots] = {};
    } pl;
};

struct ebof_group {
    ebof_params p;
    int device = 0;
    int n = 0;
    Geometry geo;
    int pitch0 = 0;
    size_t e_fs = 0, g_fs = 0, pyr_fs = 0, up_fs = 0, u_fs = 0, work_fs = 0, es = 4;
    uint8_t *E = nullptr, *Ed = nullptr, *Edf = nullptr;
    int32_t *g = nullptr;
    char *pyr = nullptr;  // two banks of n pyramid slots
    float *up = nullptr, *Ua = nullptr, *Ub = nullptr, *work = nullptr;
    float *flow = nullptr;  // [n][2][H][W]
    DevStats *dstats = nullptr;
    unsigned long long *d_dropped_time = nullptr;
    int *d_err = nullptr;
    ebof_window_desc *d_desc = nullptr;
    int64_t *h_events = nullptr;  // events given per stream in the last step
    int parity = 0;
    bool has_prev = false, last_had_prev = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    long long graph_kernels[2] = {0, 0};
    cudaStream_t cap = nullptr;
    cudaEvent_t done = nullptr;
    cudaStream_t last_stream = nullptr;
    bool have_last = false;
    std::atomic<int> busy{0};
    Profiler prof;
    CoefMaps cmaps;
};

namespace ebof {

// The fused launches of one step pattern of a multigroup: the enqueue
// operations in order and the device copy of the scatter work lists they
// read (an operation reads the list base at run time, so the plan can be
// built before the lists have a device address).
struct FusedPlan {
    std::vector<char> host;  // work lists, each at a 16-byte aligned offset
    char *dev = nullptr;
    std::vector<std::function<void(cudaStream_t)>> ops;
    ~FusedPlan() { cudaFree(dev); }
    size_t add(const void *p, size_t bytes)
    {
        const size_t off = (host.size() + 15) & ~(size_t)15;
        host.resize(off + bytes);
        std::memcpy(host.data() + off, p, bytes);
        return off;
    }
};

}  // namespace ebof

struct ebof_multigroup {
    std::vector<ebof_group *> groups;  // not owned
    int device = 0;
    cudaStream_t cap = nullptr;
    std::vector<cudaEvent_t> fork;  // [0]: fork point, [1 + k]: group k's join
    // one graph per pattern of the groups' ping-pong parities
    std::vector<std::pair<unsigned long long, cudaGraphExec_t>> graphs;
    std::vector<long long> graph_kernels;
    // fused mode (ebof_multigroup_set_fused): 0 none, 1 every stage one launch
    // for all groups, 2 the front-end stages so and the flow levels as
    // per-group branches; plans[j] holds the work lists of graphs[j]
    int fused = 0;
    std::vector<std::unique_ptr<FusedPlan>> plans;
};

namespace {

constexpr int kMaxDevices = 64;
std::atomic<int> g_attr_done[kMaxDevices];

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
        if (ok && dev >= 0 && dev < kMaxDevices && !g_attr_done[dev].exchange(1)) {
            init_front_attributes();
            init_flow_attributes();
        }
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

struct ProfScope {
    explicit ProfScope(Profiler *p) { tl_prof = p; tl_level = -1; }
    ~ProfScope() { tl_prof = nullptr; tl_level = -1; }
};

struct BusyGuard {
    std::atomic<int> *flag;
    bool ok;
    explicit BusyGuard(std::atomic<int> &f) : flag(&f)
    {
        int expect = 0;
        ok = f.compare_exchange_strong(expect, 1);
    }
    ~BusyGuard()
    {
        if (ok) flag->store(0);
    }
};

bool finite_nonneg(float v) { return std::isfinite(v) && v >= 0.0f; }

ebof_status check_params(const ebof_params *p)
{
    if (!p || p->struct_size != sizeof(ebof_params)) return EBOF_ERR_INVALID_ARG;
    if (p->width < 1 || p->height < 1 || p->width > kMaxDim || p->height > kMaxDim)
        return EBOF_ERR_INVALID_ARG;
    if (p->connectivity != 4 && p->connectivity != 8) return EBOF_ERR_INVALID_ARG;
    if (p->n_d < 0 || p->n_f < 0) return EBOF_ERR_INVALID_ARG;
    if (!(std::isfinite(p->alpha) && p->alpha > 0.0f)) return EBOF_ERR_INVALID_ARG;
    if (p->levels < 1 || p->levels > kMaxLevels) return EBOF_ERR_INVALID_ARG;
    if (p->stride < 1 || p->gn_iters < 0 || p->gn_iters > 10000) return EBOF_ERR_INVALID_ARG;
    if (p->var_outer < 0 || p->var_outer > 1000 || p->var_sor < 0 || p->var_sor > 1000)
        return EBOF_ERR_INVALID_ARG;
    if (!finite_nonneg(p->gn_damping) || !finite_nonneg(p->var_delta) || !finite_nonneg(p->var_gamma) ||
        !finite_nonneg(p->var_alpha))
        return EBOF_ERR_INVALID_ARG;
    if (!(p->sor_omega > 0.0f && p->sor_omega < 2.0f)) return EBOF_ERR_INVALID_ARG;
    if (p->max_batch < 1 || p->max_batch > 4096) return EBOF_ERR_INVALID_ARG;
    if (p->storage != EBOF_STORAGE_FP32 && p->storage != EBOF_STORAGE_FP16)
        return EBOF_ERR_INVALID_ARG;
    if (p->surface < EBOF_SURFACE_EXP || p->surface > EBOF_SURFACE_LOG) return EBOF_ERR_INVALID_ARG;
    if (!(std::isfinite(p->d_sat) && p->d_sat > 0.0f)) return EBOF_ERR_INVALID_ARG;
    if (p->coeff_cw_min_width < 1 || p->sor_tma_min_per_sm < 1 || p->sor_row_waves < 0 ||
        p->var_cluster_max < 0 ||
        (p->coeff_cw_rows != 4 && p->coeff_cw_rows != 8 && p->coeff_cw_rows != 16))
        return EBOF_ERR_INVALID_ARG;
    if (p->patch < 4 || p->patch > kMaxPatch) return EBOF_ERR_UNSUPPORTED;
    return EBOF_OK;
}

// Failure injection (ebof_debug_fail_allocation): allocations left before
// the one that fails; negative = disarmed.
std::atomic<int> g_alloc_fail_after{-1};

// Every device allocation of the library goes through here.
template <class T>
cudaError_t dmalloc(T **ptr, size_t bytes)
{
    int c = g_alloc_fail_after.load();
    while (c >= 0 && !g_alloc_fail_after.compare_exchange_weak(c, c - 1)) {
    }
    if (c == 0) {  // the injected failure; the hook is disarmed now
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc((void **)ptr, std::max<size_t>(bytes, 256));
}

void free_all(ebof_stream *s)
{
    cudaFree(s->E); cudaFree(s->Ed); cudaFree(s->Edf); cudaFree(s->g); cudaFree(s->pyr);
    cudaFree(s->up); cudaFree(s->Ua); cudaFree(s->Ub); cudaFree(s->work);
    cudaFree(s->dstats); cudaFree(s->d_dropped_time); cudaFree(s->d_err);
    cudaFree(s->flow_stage); cudaFree(s->ev_stage); cudaFree(s->d_call);
    for (int b = 0; b < 2; ++b)
        if (s->graph[b]) cudaGraphExecDestroy(s->graph[b]);
    for (cudaGraphExec_t ge : s->list_graph)
        if (ge) cudaGraphExecDestroy(ge);
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->done) cudaEventDestroy(s->done);
    auto &q = s->pipe;
    for (int j = 0; j < ebof_stream::HostPipe::kSlots; ++j) {
        if (q.used[j]) cudaEventSynchronize(q.out_done[j]);
        cudaFree(q.ev[j]);
        cudaFree(q.flow[j]);
        if (q.in_done[j]) cudaEventDestroy(q.in_done[j]);
        if (q.run_done[j]) cudaEventDestroy(q.run_done[j]);
        if (q.out_done[j]) cudaEventDestroy(q.out_done[j]);
    }
    if (q.h2d) cudaStreamDestroy(q.h2d);
    if (q.d2h) cudaStreamDestroy(q.d2h);
    auto &L = s->pl;
    if (L.front) cudaStreamSynchronize(L.front);
    for (cudaStream_t f : L.flow)
        if (f) cudaStreamSynchronize(f);
    for (int j = 0; j < ebof_stream::Pipeline::kSlots; ++j) {
        if (L.front_graph[j]) cudaGraphExecDestroy(L.front_graph[j]);
        if (L.flow_graph[j]) cudaGraphExecDestroy(L.flow_graph[j]);
        if (L.front_done[j]) cudaEventDestroy(L.front_done[j]);
        if (L.flow_done[j]) cudaEventDestroy(L.flow_done[j]);
    }
    if (L.inputs) cudaEventDestroy(L.inputs);
    cudaFree(L.pyr);
    cudaFree(L.call);
    for (int f = 0; f < ebof_stream::Pipeline::kFlows; ++f) {
        cudaFree(L.up[f]);
        cudaFree(L.Ua[f]);
        cudaFree(L.Ub[f]);
        cudaFree(L.work[f]);
    }
    if (L.front) cudaStreamDestroy(L.front);
    for (cudaStream_t f : L.flow)
        if (f) cudaStreamDestroy(f);
}

SurfaceMap surface_map(const ebof_params &p)
{
    SurfaceMap m;
    m.mode = p.surface;
    m.alpha = p.alpha;
    m.d_sat = p.d_sat;
    if (p.surface == EBOF_SURFACE_EXP)
        m.gain = 255.0f;
    else if (p.surface == EBOF_SURFACE_LOG)
        m.gain = (float)(255.0 / std::log1p((double)p.d_sat));
    else
        m.gain = (float)(255.0 / (double)p.d_sat);
    return m;
}

FlowParams flow_params(const ebof_params &p)
{
    FlowParams fp;
    fp.half = p.storage == EBOF_STORAGE_FP16;
    fp.ps = p.patch;
    fp.stride = p.stride;
    fp.gn_iters = p.gn_iters;
    fp.gn_damping = p.gn_damping;
    fp.var_outer = p.var_outer;
    fp.var_sor = p.var_sor;
    fp.delta = p.var_delta;
    fp.gamma = p.var_gamma;
    fp.alpha_s = p.var_alpha;
    fp.omega = p.sor_omega;
    fp.wait_limit = kWaitLimitDefault;
    fp.coeff_cw_min_width = p.coeff_cw_min_width;
    fp.sor_tma_min_per_sm = p.sor_tma_min_per_sm;
    fp.sor_row_waves = p.sor_row_waves;
    fp.var_cluster_max = p.var_cluster_max;
    fp.coeff_cw_rows = p.coeff_cw_rows;
    return fp;
}

// Enqueues the whole path for n consecutive windows (or one caller-given
// surface) on `st`: the current windows go to slots cur_first.., the previous
// ones are at prev_first.., and nothing of the stream's bookkeeping changes
// (so the same sequence can be captured into a graph).  With `via_args`, the
// events and flow destination of window k are read from s->d_wins[k] and
// s->d_flows[k].
// Parts of the sequence (enqueue's `parts`): A1-A5 of the current windows,
// A6-A9 of the windows that have a previous one.
constexpr int kPartFront = 1, kPartFlow = 2, kPartAll = 3;

// The buffers the flow part works in (the stream's own unless given).
struct FlowScratch {
    float *up, *Ua, *Ub, *work;
    const CoefMaps *cmaps;  // tensor maps of `work`, or null (direct loads, same result)
};

void enqueue(ebof_stream *s, int n, const uint16_t *x, const uint16_t *y, const int64_t *t,
             int64_t nev, int64_t t_begin, int64_t dt, const float *surface_in, float *d_flow,
             uint8_t *d_edge, int32_t *d_edt, float *d_surface, bool via_args, int cur_first,
             int prev_first, bool had_prev, cudaStream_t st, int parts = kPartAll,
             char *pyr = nullptr, const ebof_window_desc *d_wins = nullptr,
             float *const *d_flows = nullptr, const FlowScratch *scratch = nullptr)
{
    const ebof_params &p = s->p;
    const Geometry &geo = s->geo;
    const int W = p.width, H = p.height;
    if (!pyr) pyr = s->pyr;
    if (!d_wins) d_wins = s->d_wins;
    if (!d_flows) d_flows = s->d_flows;
    tl_level = -1;
    const bool half = p.storage == EBOF_STORAGE_FP16;
    const size_t es = s->es;
    char *I0cur = pyr + (size_t)cur_first * s->pyr_fs * es;
    if (parts & kPartFront) {
        cudaMemsetAsync(s->dstats, 0, sizeof(DevStats) * n, st);
        cudaMemsetAsync(s->d_dropped_time, 0, sizeof(unsigned long long), st);

        if (surface_in) {
            launch_surface_to_intensity(surface_in, W, H, I0cur, s->pitch0, half,
                                        surface_map(p), st);
        } else {
            cudaMemsetAsync(s->E, 0, s->e_fs * n, st);
            if (via_args)
                launch_scatter_desc(d_wins, n, W, H, s->pitch0, s->E, s->e_fs, s->dstats,
                                    s->d_dropped_time, st);
            else
                launch_scatter(x, y, t, nev, t_begin, dt, n, W, H, s->pitch0, s->E, s->e_fs,
                               s->dstats, s->d_dropped_time, st);
            launch_denoise_fill(s->E, s->Ed, s->Edf, W, H, s->pitch0, s->e_fs, n, p.connectivity,
                                p.n_d, p.n_f, d_edge, s->dstats, st);
            launch_edt_columns(s->Edf, s->pitch0, s->e_fs, W, H, s->g, s->pitch0, s->g_fs, n, st);
            launch_edt_rows_surface(s->g, s->pitch0, s->g_fs, W, H, surface_map(p), d_edt,
                                    d_surface, I0cur, s->pitch0, s->pyr_fs, n, half, st);
        }

        // A5: pyramid and gradients of the current window(s)
        tl_level = 0;
        launch_pyramid(I0cur, geo, s->pyr_fs, n, half, st);
    }
    if (!(parts & kPartFlow)) return;

    // A6-A9: flow for every window that has a previous one
    const int ff = had_prev ? 0 : 1;
    const int nf = n - ff;
    const size_t flow_frame = (size_t)2 * W * H;
    if (geo.levels > 0 && nf > 0) {
        const int curf_first = cur_first + ff;
        FlowParams fp = flow_params(p);
        fp.wait_limit = s->wait_limit;
        const FlowScratch own = {s->up, s->Ua, s->Ub, s->work, &s->cmaps};
        const FlowScratch &sc = scratch ? *scratch : own;
        float *Ucur = nullptr, *Uc = nullptr;
        const Level *lvc = nullptr;
        for (int l = geo.levels - 1; l >= 0; --l) {
            tl_level = l;
            const Level &lv = geo.lv[l];
            const char *I0 = pyr + ((size_t)prev_first * s->pyr_fs + geo.pyr_off[l]) * es;
            const char *I1 = pyr + ((size_t)curf_first * s->pyr_fs + geo.pyr_off[l]) * es;
            const char *I0x = I0 + lv.plane * es, *I0y = I0 + 2 * lv.plane * es;
            Ucur = (Uc == sc.Ua) ? sc.Ub : sc.Ua;
            launch_patch_search(I0, I0x, I0y, I1, lv, s->pyr_fs, Uc, lvc, s->u_fs, sc.up,
                                s->up_fs, nf, fp, s->d_err, st);
            launch_densify(I0, I1, lv, s->pyr_fs, sc.up, s->up_fs, Ucur, s->u_fs, nf, fp, st);
            // the coarser flow is consumed by the search: its buffer is free
            float *Utmp = (Ucur == sc.Ua) ? sc.Ub : sc.Ua;
            const CUtensorMap *cmap =
                sc.cmaps && sc.cmaps->ok[l] ? &sc.cmaps->map[l] : nullptr;
            Ucur = launch_variational(I0, I0x, I0y, I1, lv, s->pyr_fs, Ucur, Utmp, s->u_fs,
                                      sc.work, s->work_fs, nf, fp, cmap, s->d_err, st);
            Uc = Ucur;
            lvc = &lv;
        }
        tl_level = -1;
        if (via_args)
            launch_flow_out_ptr(Ucur, W, H, s->pitch0, s->u_fs, d_flows + ff, nf, st);
        else
            launch_flow_out(Ucur, W, H, s->pitch0, s->u_fs, d_flow + (size_t)ff * flow_frame,
                            nf, st);
    }
    if (!via_args) {
        if (geo.levels == 0)
            cudaMemsetAsync(d_flow, 0, sizeof(float) * flow_frame * n, st);
        else if (ff == 1)
            cudaMemsetAsync(d_flow, 0, sizeof(float) * flow_frame, st);
    }
}

// Copies the descriptors and flow destinations of n windows to s->d_call.
void stage_call(ebof_stream *s, int n, const ebof_window_desc *wins, float *const *flows,
                cudaStream_t st)
{
    const int B = s->p.max_batch;
    ebof_window_desc *hw = (ebof_window_desc *)s->h_call.data();
    float **hf = (float **)(s->h_call.data() + sizeof(ebof_window_desc) * B);
    for (int k = 0; k < n; ++k) {
        hw[k] = wins[k];
        hf[k] = flows[k];
    }
    cudaMemcpyAsync(s->d_call, s->h_call.data(), s->h_call.size(), cudaMemcpyHostToDevice, st);
}

// Captures enqueue(via_args) of n windows (current ones from slot cur_first,
// previous from prev_first) into an executable graph on s->cap, after work
// already queued on st.  Returns nullptr on failure; *kernels gets the number
// of kernels in the graph.
cudaGraphExec_t capture(ebof_stream *s, int n, int cur_first, int prev_first, cudaStream_t st,
                        long long *kernels, int parts = kPartAll, char *pyr = nullptr,
                        const ebof_window_desc *d_wins = nullptr, float *const *d_flows = nullptr,
                        const FlowScratch *scratch = nullptr)
{
    cudaEvent_t ready;
    cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
    cudaEventRecord(ready, st);
    cudaStreamWaitEvent(s->cap, ready, 0);
    cudaEventDestroy(ready);
    const unsigned long long before = g_launches.load();
    cudaGraph_t gr = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        Profiler *keep = tl_prof;
        tl_prof = nullptr;
        enqueue(s, n, nullptr, nullptr, nullptr, 0, 0, 0, nullptr, nullptr, nullptr, nullptr,
                nullptr, true, cur_first, prev_first, true, s->cap, parts, pyr, d_wins, d_flows,
                scratch);
        tl_prof = keep;
        cudaStreamEndCapture(s->cap, &gr);
    }
    if (gr && cudaGraphInstantiate(&ge, gr, 0) != cudaSuccess) ge = nullptr;
    if (gr) cudaGraphDestroy(gr);
    *kernels = (long long)(g_launches.load() - before);
    g_launches.fetch_sub((unsigned long long)*kernels);
    if (!ge) cudaGetLastError();
    return ge;
}

// A list call: n windows of arbitrary extents.  With a previous window, that
// window's pyramid is moved to slot 0 (if it is not there) and the current
// windows go to slots 1..n, so the enqueued sequence depends on n alone and is
// replayed from list_graph[n].
void pipeline_leave(ebof_stream *s, cudaStream_t st);

ebof_status run_list(ebof_stream *s, int n, const ebof_window_desc *wins, float *const *flows,
                     cudaStream_t st)
{
    ProfScope prof_scope(&s->prof);
    cudaGetLastError();
    pipeline_leave(s, st);
    if (s->have_last && s->last_stream != st) cudaStreamWaitEvent(st, s->done, 0);
    const bool had_prev = s->has_prev;
    if (had_prev && s->head != 0)
        cudaMemcpyAsync(s->pyr, s->pyr + (size_t)s->head * s->pyr_fs * s->es, s->pyr_fs * s->es,
                        cudaMemcpyDeviceToDevice, st);
    s->head = 0;
    stage_call(s, n, wins, flows, st);
    const size_t flow_bytes = sizeof(float) * 2 * (size_t)s->p.width * s->p.height;
    if (had_prev && !s->prof.on && s->geo.levels > 0) {
        if (!s->list_graph[n]) {
            s->list_graph[n] = capture(s, n, 1, 0, st, &s->list_graph_kernels[n]);
            if (!s->list_graph[n]) return EBOF_ERR_CUDA;
        }
        if (cudaGraphLaunch(s->list_graph[n], st) != cudaSuccess) return EBOF_ERR_CUDA;
        g_launches.fetch_add((unsigned long long)s->list_graph_kernels[n]);
    } else {
        enqueue(s, n, nullptr, nullptr, nullptr, 0, 0, 0, nullptr, nullptr, nullptr, nullptr,
                nullptr, true, 1, had_prev ? 0 : 1, had_prev, st);
        for (int k = 0; k < n; ++k)
            if (s->geo.levels == 0 || (k == 0 && !had_prev))
                cudaMemsetAsync(flows[k], 0, flow_bytes, st);
    }
    s->head = n;
    s->has_prev = true;
    s->last_n = n;
    s->last_had_prev = had_prev;
    s->last_list = true;
    s->last_events = 0;
    for (int k = 0; k < n; ++k) {
        s->last_win_events[k] = wins[k].n_events;
        s->last_events += wins[k].n_events;
    }
    cudaEventRecord(s->done, st);
    s->last_stream = st;
    s->have_last = true;
    if (cudaGetLastError() != cudaSuccess) return EBOF_ERR_CUDA;
    return had_prev ? EBOF_OK : EBOF_NO_PREVIOUS;
}

// One call: slot bookkeeping, then either a graph replay (single window in
// steady state) or an eager enqueue.
ebof_status run(ebof_stream *s, int n, const uint16_t *x, const uint16_t *y, const int64_t *t,
                int64_t nev, int64_t t_begin, int64_t dt, const float *surface_in,
                float *d_flow, uint8_t *d_edge, int32_t *d_edt, float *d_surface,
                cudaStream_t st)
{
    ProfScope prof_scope(&s->prof);
    cudaGetLastError();  // start from a clean error state
    pipeline_leave(s, st);
    if (s->have_last && s->last_stream != st) cudaStreamWaitEvent(st, s->done, 0);

    if (n > 1 && s->head + n >= s->nslots) {
        if (s->has_prev && s->head != 0)
            cudaMemcpyAsync(s->pyr, s->pyr + (size_t)s->head * s->pyr_fs * s->es,
                            s->pyr_fs * s->es, cudaMemcpyDeviceToDevice, st);
        s->head = 0;
    }
    const bool had_prev = s->has_prev;
    const int cur_first = n == 1 ? (s->head + 1) % s->nslots : s->head + 1;
    const int prev_first = n == 1 ? s->head : s->head + (had_prev ? 0 : 1);
    const bool graph = n == 1 && had_prev && !surface_in && !d_edge && !d_edt && !d_surface &&
                       !s->prof.on && s->nslots == 2 && s->geo.levels > 0;
    if (graph) {
        const int b = s->head;
        ebof_window_desc w;
        w.x = x;
        w.y = y;
        w.t = t;
        w.n_events = nev;
        w.t_begin = t_begin;
        w.t_end = t_begin + dt;
        stage_call(s, 1, &w, &d_flow, st);
        if (!s->graph[b]) {
            s->graph[b] = capture(s, 1, cur_first, prev_first, st, &s->graph_kernels[b]);
            if (!s->graph[b]) return EBOF_ERR_CUDA;
        }
        if (cudaGraphLaunch(s->graph[b], st) != cudaSuccess) return EBOF_ERR_CUDA;
        g_launches.fetch_add((unsigned long long)s->graph_kernels[b]);
    } else {
        enqueue(s, n, x, y, t, nev, t_begin, dt, surface_in, d_flow, d_edge, d_edt, d_surface,
                false, cur_first, prev_first, had_prev, st);
    }

    s->head = n == 1 ? cur_first : s->head + n;
    s->has_prev = true;
    s->last_list = false;
    s->last_n = n;
    s->last_events = nev;
    s->last_had_prev = had_prev;
    cudaEventRecord(s->done, st);
    s->last_stream = st;
    s->have_last = true;
    if (cudaGetLastError() != cudaSuccess) return EBOF_ERR_CUDA;
    return had_prev ? EBOF_OK : EBOF_NO_PREVIOUS;
}

// ----------------------------------------------------------------- pipelined calls
constexpr int kPipeSlots = ebof_stream::Pipeline::kSlots;
constexpr int kPipeFlows = ebof_stream::Pipeline::kFlows;
constexpr size_t kPipeCallBytes = 128;  // per slot: one ebof_window_desc, one float *

ebof_window_desc *pipe_wins(ebof_stream *s, int j)
{
    return (ebof_window_desc *)(s->pl.call + (size_t)j * kPipeCallBytes);
}

float **pipe_flows(ebof_stream *s, int j)
{
    return (float **)(s->pl.call + (size_t)j * kPipeCallBytes + 64);
}

// Releases what pipeline_ready made (after a failure there).
void pipeline_release(ebof_stream *s)
{
    auto &L = s->pl;
    for (int j = 0; j < kPipeSlots; ++j) {
        if (L.front_done[j]) cudaEventDestroy(L.front_done[j]);
        if (L.flow_done[j]) cudaEventDestroy(L.flow_done[j]);
        L.front_done[j] = L.flow_done[j] = nullptr;
    }
    if (L.inputs) cudaEventDestroy(L.inputs);
    L.inputs = nullptr;
    if (L.front) cudaStreamDestroy(L.front);
    L.front = nullptr;
    for (cudaStream_t &f : L.flow) {
        if (f) cudaStreamDestroy(f);
        f = nullptr;
    }
    for (char **b : {&L.pyr, &L.call}) {
        cudaFree(*b);
        *b = nullptr;
    }
    for (int f = 0; f < kPipeFlows; ++f)
        for (float **b : {&L.up[f], &L.Ua[f], &L.Ub[f], &L.work[f]}) {
            cudaFree(*b);
            *b = nullptr;
        }
}

// Streams, events, slots, descriptor blocks and the extra scratch sets of
// the pipelined calls, made on first use.
ebof_status pipeline_ready(ebof_stream *s)
{
    auto &L = s->pl;
    if (L.ready) return EBOF_OK;
    static_assert(sizeof(ebof_window_desc) <= 64, "descriptor block");
    bool ok = cudaStreamCreateWithFlags(&L.front, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&L.inputs, cudaEventDisableTiming) == cudaSuccess;
    for (int f = 0; f < kPipeFlows && ok; ++f)
        ok = cudaStreamCreateWithFlags(&L.flow[f], cudaStreamNonBlocking) == cudaSuccess;
    for (int j = 0; j < kPipeSlots && ok; ++j)
        ok = cudaEventCreateWithFlags(&L.front_done[j], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&L.flow_done[j], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && dmalloc(&L.pyr, s->es * s->pyr_fs * kPipeSlots) == cudaSuccess &&
         dmalloc(&L.call, kPipeSlots * kPipeCallBytes) == cudaSuccess;
    for (int f = 1; f < kPipeFlows && ok; ++f)
        ok = dmalloc(&L.up[f], sizeof(float) * s->up_fs) == cudaSuccess &&
             dmalloc(&L.Ua[f], sizeof(float) * s->u_fs) == cudaSuccess &&
             dmalloc(&L.Ub[f], sizeof(float) * s->u_fs) == cudaSuccess &&
             dmalloc(&L.work[f], sizeof(float) * s->work_fs) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        pipeline_release(s);
        return EBOF_ERR_OOM;
    }
    L.h_call.assign(kPipeSlots * kPipeCallBytes, 0);
    L.ready = true;
    return EBOF_OK;
}

// The ordinary calls and the pipelined ones keep their own pyramid slots;
// the newest window's pyramid moves over, with one copy, when the kind of
// call changes (after the work that wrote it).
void pipeline_enter(ebof_stream *s)
{
    auto &L = s->pl;
    if (L.latest) return;
    L.has_prev = s->has_prev;
    if (s->has_prev) {
        if (s->have_last) cudaStreamWaitEvent(L.front, s->done, 0);
        const size_t slot = s->pyr_fs * s->es;
        cudaMemcpyAsync(L.pyr + (size_t)L.head * slot, s->pyr + (size_t)s->head * slot, slot,
                        cudaMemcpyDeviceToDevice, L.front);
    }
    L.latest = true;
}

void pipeline_leave(ebof_stream *s, cudaStream_t st)
{
    auto &L = s->pl;
    if (!L.latest) return;
    if (s->have_last && s->last_stream != st) cudaStreamWaitEvent(st, s->done, 0);
    s->has_prev = L.has_prev;
    if (L.has_prev) {
        const size_t slot = s->pyr_fs * s->es;
        cudaMemcpyAsync(s->pyr + (size_t)s->head * slot, L.pyr + (size_t)L.head * slot, slot,
                        cudaMemcpyDeviceToDevice, st);
    }
    L.latest = false;
}

// One pipelined window in slot j = head + 1 (mod kSlots).  The caller has
// made L.front wait for the window's inputs (and every flow stream for
// d_flow to be free, if it reuses it).  The front end goes to L.front after
// the flows that last read slot j and its descriptor block (kSlots - 1 and
// kSlots calls back: their current slots are j + 1 and j); the flow goes to
// flow[j % kFlows], whose scratch set it uses, after the front end.  s->done
// then follows every flow stream.
ebof_status run_pipelined(ebof_stream *s, const uint16_t *x, const uint16_t *y, const int64_t *t,
                          int64_t nev, int64_t t_begin, int64_t dt, float *d_flow)
{
    auto &L = s->pl;
    ProfScope prof_scope(&s->prof);
    pipeline_enter(s);
    const int j = (L.head + 1) % kPipeSlots, prev = L.head;
    const bool had_prev = L.has_prev;
    for (int c : {(j + 1) % kPipeSlots, j})
        if (L.flow_used[c]) cudaStreamWaitEvent(L.front, L.flow_done[c], 0);
    ebof_window_desc w;
    w.x = x;
    w.y = y;
    w.t = t;
    w.n_events = nev;
    w.t_begin = t_begin;
    w.t_end = t_begin + dt;
    char *hc = L.h_call.data() + (size_t)j * kPipeCallBytes;
    std::memcpy(hc, &w, sizeof(w));
    std::memcpy(hc + 64, &d_flow, sizeof(d_flow));
    cudaMemcpyAsync(L.call + (size_t)j * kPipeCallBytes, hc, kPipeCallBytes,
                    cudaMemcpyHostToDevice, L.front);
    const bool graphs = !s->prof.on;
    // slot j's flow stream and scratch set (kSlots is a multiple of kFlows,
    // so consecutive windows take consecutive sets)
    const int f = j % kPipeFlows;
    const FlowScratch setf = {L.up[f], L.Ua[f], L.Ub[f], L.work[f], nullptr};
    const FlowScratch *sc = f ? &setf : nullptr;  // set 0: the stream's own buffers
    cudaStream_t fl = L.flow[f];
    if (graphs) {
        if (!L.front_graph[j]) {
            L.front_graph[j] = capture(s, 1, j, prev, L.front, &L.front_k[j], kPartFront, L.pyr,
                                       pipe_wins(s, j), pipe_flows(s, j));
            if (!L.front_graph[j]) return EBOF_ERR_CUDA;
        }
        if (cudaGraphLaunch(L.front_graph[j], L.front) != cudaSuccess) return EBOF_ERR_CUDA;
        g_launches.fetch_add((unsigned long long)L.front_k[j]);
    } else {
        enqueue(s, 1, nullptr, nullptr, nullptr, 0, 0, 0, nullptr, nullptr, nullptr, nullptr,
                nullptr, true, j, prev, had_prev, L.front, kPartFront, L.pyr, pipe_wins(s, j),
                pipe_flows(s, j));
    }
    cudaEventRecord(L.front_done[j], L.front);
    cudaStreamWaitEvent(fl, L.front_done[j], 0);
    // windows in flight that write the same flow destination write it in
    // call order
    for (int c = 0; c < kPipeSlots; ++c)
        if (c != j && L.flow_used[c] && L.dflow[c] == d_flow)
            cudaStreamWaitEvent(fl, L.flow_done[c], 0);
    L.dflow[j] = d_flow;
    if (had_prev && s->geo.levels > 0) {
        if (graphs) {
            if (!L.flow_graph[j]) {
                L.flow_graph[j] = capture(s, 1, j, prev, fl, &L.flow_k[j], kPartFlow, L.pyr,
                                          pipe_wins(s, j), pipe_flows(s, j), sc);
                if (!L.flow_graph[j]) return EBOF_ERR_CUDA;
            }
            if (cudaGraphLaunch(L.flow_graph[j], fl) != cudaSuccess) return EBOF_ERR_CUDA;
            g_launches.fetch_add((unsigned long long)L.flow_k[j]);
        } else {
            enqueue(s, 1, nullptr, nullptr, nullptr, 0, 0, 0, nullptr, nullptr, nullptr, nullptr,
                    nullptr, true, j, prev, true, fl, kPartFlow, L.pyr, pipe_wins(s, j),
                    pipe_flows(s, j), sc);
        }
    } else {
        cudaMemsetAsync(d_flow, 0, sizeof(float) * 2 * (size_t)s->p.width * s->p.height, fl);
    }
    cudaEventRecord(L.flow_done[j], fl);
    L.flow_used[j] = true;
    // s->done: after this flow and the previous windows' (on the other streams)
    for (int b = 1; b < kPipeFlows; ++b) {
        const int c = (j + kPipeSlots - b) % kPipeSlots;
        if (L.flow_used[c]) cudaStreamWaitEvent(fl, L.flow_done[c], 0);
    }
    cudaEventRecord(s->done, fl);
    L.head = j;
    L.has_prev = true;
    s->last_list = false;
    s->last_n = 1;
    s->last_events = nev;
    s->last_had_prev = had_prev;
    s->last_stream = fl;
    s->have_last = true;
    if (cudaGetLastError() != cudaSuccess) return EBOF_ERR_CUDA;
    return had_prev ? EBOF_OK : EBOF_NO_PREVIOUS;
}

void free_group(ebof_group *g)
{
    for (int b = 0; b < 2; ++b)
        if (g->graph[b]) cudaGraphExecDestroy(g->graph[b]);
    cudaFree(g->E); cudaFree(g->Ed); cudaFree(g->Edf); cudaFree(g->g); cudaFree(g->pyr);
    cudaFree(g->up); cudaFree(g->Ua); cudaFree(g->Ub); cudaFree(g->work); cudaFree(g->flow);
    cudaFree(g->dstats); cudaFree(g->d_dropped_time); cudaFree(g->d_err); cudaFree(g->d_desc);
    delete[] g->h_events;
    if (g->cap) cudaStreamDestroy(g->cap);
    if (g->done) cudaEventDestroy(g->done);
}

// One lockstep step of a group: every stage once for its n streams.  The
// current windows go to bank `parity`, the previous ones are in the other
// bank.  Enqueued on `st`; nothing here depends on host values that change
// between steps of the same parity, so the sequence can be captured.
void run_group_flow(ebof_group *g, bool with_flow, cudaStream_t st);

void run_group(ebof_group *g, bool with_flow, cudaStream_t st)
{
    const ebof_params &p = g->p;
    const Geometry &geo = g->geo;
    const int W = p.width, H = p.height, n = g->n;
    const bool half = p.storage == EBOF_STORAGE_FP16;
    const size_t es = g->es;
    char *cur = g->pyr + (size_t)g->parity * n * g->pyr_fs * es;
    tl_level = -1;
    cudaMemsetAsync(g->dstats, 0, sizeof(DevStats) * n, st);
    cudaMemsetAsync(g->d_dropped_time, 0, sizeof(unsigned long long), st);
    cudaMemsetAsync(g->E, 0, g->e_fs * n, st);
    launch_scatter_desc(g->d_desc, n, W, H, g->pitch0, g->E, g->e_fs, g->dstats,
                        g->d_dropped_time, st);
    launch_denoise_fill(g->E, g->Ed, g->Edf, W, H, g->pitch0, g->e_fs, n, p.connectivity, p.n_d,
                        p.n_f, nullptr, g->dstats, st);
    launch_edt_columns(g->Edf, g->pitch0, g->e_fs, W, H, g->g, g->pitch0, g->g_fs, n, st);
    launch_edt_rows_surface(g->g, g->pitch0, g->g_fs, W, H, surface_map(p), nullptr, nullptr, cur,
                            g->pitch0, g->pyr_fs, n, half, st);
    tl_level = 0;
    launch_pyramid(cur, geo, g->pyr_fs, n, half, st);
    run_group_flow(g, with_flow, st);
}

// The flow part of a group step (A6-A9), after its pyramid.
void run_group_flow(ebof_group *g, bool with_flow, cudaStream_t st)
{
    const ebof_params &p = g->p;
    const Geometry &geo = g->geo;
    const int W = p.width, H = p.height, n = g->n;
    const size_t es = g->es;
    char *cur = g->pyr + (size_t)g->parity * n * g->pyr_fs * es;
    char *prv = g->pyr + (size_t)(g->parity ^ 1) * n * g->pyr_fs * es;
    const size_t flow_frame = (size_t)2 * W * H;
    if (with_flow && geo.levels > 0) {
        const FlowParams fp = flow_params(p);
        float *Ucur = nullptr, *Uc = nullptr;
        const Level *lvc = nullptr;
        for (int l = geo.levels - 1; l >= 0; --l) {
            tl_level = l;
            const Level &lv = geo.lv[l];
            const char *I0 = prv + geo.pyr_off[l] * es;
            const char *I1 = cur + geo.pyr_off[l] * es;
            const char *I0x = I0 + lv.plane * es, *I0y = I0 + 2 * lv.plane * es;
            Ucur = (Uc == g->Ua) ? g->Ub : g->Ua;
            launch_patch_search(I0, I0x, I0y, I1, lv, g->pyr_fs, Uc, lvc, g->u_fs, g->up,
                                g->up_fs, n, fp, g->d_err, st);
            launch_densify(I0, I1, lv, g->pyr_fs, g->up, g->up_fs, Ucur, g->u_fs, n, fp, st);
            float *Utmp = (Ucur == g->Ua) ? g->Ub : g->Ua;
            Ucur = launch_variational(I0, I0x, I0y, I1, lv, g->pyr_fs, Ucur, Utmp, g->u_fs,
                                      g->work, g->work_fs, n, fp,
                                      g->cmaps.ok[l] ? &g->cmaps.map[l] : nullptr, g->d_err, st);
            Uc = Ucur;
            lvc = &lv;
        }
        tl_level = -1;
        launch_flow_out(Ucur, W, H, g->pitch0, g->u_fs, g->flow, n, st);
    } else {
        cudaMemsetAsync(g->flow, 0, sizeof(float) * flow_frame * n, st);
    }
}

// ----------------------------------------------------------------- fused steps
// Adds one operation per table of `segs` (a segment and its block count
// each; at most kMaxSeg segments per table) that calls
// `launch(table, blocks, stream)`; the table travels by value.
template <class A, class L>
void emit_seg(FusedPlan &P, const std::vector<std::pair<A, int>> &segs, L launch)
{
    for (size_t i = 0; i < segs.size(); i += kMaxSeg) {
        SegTable<A> t;
        std::memset(&t, 0, sizeof(t));
        int blocks = 0;
        for (size_t j = i; j < std::min(segs.size(), i + kMaxSeg); ++j) {
            if (segs[j].second <= 0) continue;
            t.first[t.n] = blocks;
            t.a[t.n] = segs[j].first;
            blocks += segs[j].second;
            ++t.n;
        }
        t.first[t.n] = blocks;
        if (blocks == 0) continue;
        P.ops.push_back([t, blocks, launch](cudaStream_t st) { launch(t, blocks, st); });
    }
}

// Segments sorted by a kernel-instance key: one emit per distinct key.
template <class A, class L>
void emit_keyed(FusedPlan &P, const std::vector<std::pair<long long, std::pair<A, int>>> &segs,
                L launch_for_key)
{
    std::vector<long long> keys;
    for (const auto &s : segs)
        if (std::find(keys.begin(), keys.end(), s.first) == keys.end()) keys.push_back(s.first);
    for (long long k : keys) {
        std::vector<std::pair<A, int>> sub;
        for (const auto &s : segs)
            if (s.first == k) sub.push_back(s.second);
        emit_seg(P, sub, launch_for_key(k));
    }
}

// Can the fused launches run group g?  The fused pyramid kernel builds at
// most seg_max_levels() levels; the fused SOR is the register-strip region
// kernel, which needs var_fused_supported(var_sor).
bool fused_supported(const ebof_group *g, int mode)
{
    return g->geo.levels <= seg_max_levels() &&
           (mode == 2 || var_fused_supported(g->p.var_sor));
}

// The plan of one steady-state step of multigroup m (every group has a
// previous window; parities as the groups hold them now): the stages of
// run_group in the same order, each stage one launch over all groups (one
// per kernel instance where groups differ in storage, patch size or lane
// layout).  Pyramid levels are aligned at the coarsest level (below).
// Results are those of run_group bit for bit: every kernel body is the
// group kernel's, and every layout that differs (EDT rows of one warp, the
// tile form of the coefficients, the even-halo SOR regions) gives the same
// values.
void build_fused_plan(ebof_multigroup *m, FusedPlan &P, int mode)
{
    const int nsm = [] {
        int d = 0, n = 0;
        cudaGetDevice(&d);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
        return n > 0 ? n : 152;
    }();
    FusedPlan *pp = &P;
    // per-group banks of this step
    struct GS {
        ebof_group *g;
        char *cur, *prv;
        float *U;  // result of the last level done (null before the first)
        const Level *lvc;
    };
    std::vector<GS> gs;
    for (ebof_group *g : m->groups) {
        const size_t bank = (size_t)g->n * g->pyr_fs * g->es;
        gs.push_back({g, g->pyr + (size_t)g->parity * bank, g->pyr + (size_t)(g->parity ^ 1) * bank,
                      nullptr, nullptr});
    }
    // counters of this step
    for (GS &x : gs) {
        ebof_group *g = x.g;
        P.ops.push_back([g](cudaStream_t st) {
            cudaMemsetAsync(g->dstats, 0, sizeof(DevStats) * g->n, st);
            cudaMemsetAsync(g->d_dropped_time, 0, sizeof(unsigned long long), st);
            cudaMemsetAsync(g->E, 0, g->e_fs * g->n, st);
        });
    }
    // A1: the work list of all windows
    {
        std::vector<ScatterWin> wins;
        for (GS &x : gs) {
            ebof_group *g = x.g;
            for (int k = 0; k < g->n; ++k)
                wins.push_back({g->d_desc + k, g->E + (size_t)k * g->e_fs, g->dstats + k,
                                g->d_dropped_time, g->p.width, g->p.height, g->pitch0});
        }
        for (size_t i = 0; i < wins.size(); i += kScatterListMax) {
            const int nw = (int)std::min(wins.size() - i, (size_t)kScatterListMax);
            const size_t off = P.add(wins.data() + i, sizeof(ScatterWin) * nw);
            const int blocks = 4 * nsm;
            P.ops.push_back([pp, off, nw, blocks](cudaStream_t st) {
                launch_seg_scatter(reinterpret_cast<const ScatterWin *>(pp->dev + off), nw,
                                   blocks, st);
            });
        }
    }
    // A2
    {
        std::vector<std::pair<SegDenoise, int>> segs;
        for (GS &x : gs) {
            ebof_group *g = x.g;
            const ebof_params &p = g->p;
            SegDenoise a = {};
            a.E = g->E;
            a.Edf = g->Edf;
            a.stats = g->dstats;
            a.fs = g->e_fs;
            a.W = p.width;
            a.H = p.height;
            a.pitch = g->pitch0;
            a.conn = p.connectivity;
            a.n_d = p.n_d;
            a.n_f = p.n_f;
            a.gx = (p.width + 31) / 32;
            a.gy = (p.height + 7) / 8;
            segs.push_back({a, a.gx * a.gy * g->n});
        }
        emit_seg(P, segs, launch_seg_denoise_fill);
    }
    // A3
    {
        std::vector<std::pair<SegEdtCols, int>> segs;
        int nch_max = 1;
        for (GS &x : gs) {
            ebof_group *g = x.g;
            SegEdtCols a = {};
            a.E = g->Edf;
            a.g = g->g;
            a.efs = g->e_fs;
            a.gfs = g->g_fs;
            a.epitch = a.gpitch = g->pitch0;
            a.W = g->p.width;
            a.H = g->p.height;
            edt_cols_chunks(a.H, a.CH, a.nch);
            a.gx = (a.W + 31) / 32;
            nch_max = std::max(nch_max, a.nch);
            segs.push_back({a, a.gx * g->n});
        }
        emit_seg(P, segs, [nch_max](const SegTable<SegEdtCols> &t, int b, cudaStream_t st) {
            launch_seg_edt_cols(t, b, nch_max, st);
        });
    }
    // A4 (keyed by storage): rows of one warp
    {
        std::vector<std::pair<long long, std::pair<SegEdtRows, int>>> segs;
        int rows_max = 1;
        size_t smem = 0;
        for (GS &x : gs) {
            ebof_group *g = x.g;
            SegEdtRows a = {};
            a.g = g->g;
            a.I0 = x.cur;
            a.gfs = g->g_fs;
            a.ifs = g->pyr_fs;
            a.sm = surface_map(g->p);
            a.gpitch = a.ipitch = g->pitch0;
            a.W = g->p.width;
            a.H = g->p.height;
            a.rows = edt_rows_block_rows(a.W);
            a.gx = (a.H + a.rows - 1) / a.rows;
            rows_max = std::max(rows_max, a.rows);
            smem = std::max(smem, edt_rows_smem(a.W, a.rows));
            segs.push_back({g->p.storage == EBOF_STORAGE_FP16, {a, a.gx * g->n}});
        }
        emit_keyed(P, segs, [rows_max, smem](long long half) {
            return [rows_max, smem, half](const SegTable<SegEdtRows> &t, int b, cudaStream_t st) {
                launch_seg_edt_rows(t, b, rows_max, smem, half != 0, st);
            };
        });
    }
    // A5 (keyed by storage): box means, then gradients
    {
        std::vector<std::pair<long long, std::pair<SegPyr, int>>> means, grads;
        for (GS &x : gs) {
            ebof_group *g = x.g;
            SegPyr a = {};
            a.slots = x.cur;
            a.fs = g->pyr_fs;
            a.d = make_pyr_desc(g->geo);
            const long long half = g->p.storage == EBOF_STORAGE_FP16;
            if (a.d.levels > 1) {
                a.gx = (a.d.w[0] + 63) / 64;  // 64 x 64 regions of level 0
                a.gy = (a.d.h[0] + 63) / 64;
                means.push_back({half, {a, a.gx * a.gy * g->n}});
            }
            a.gx = a.d.blk0[a.d.levels] - a.d.gb0;
            a.gy = 1;
            grads.push_back({half, {a, a.gx * g->n}});
        }
        emit_keyed(P, means, [](long long half) {
            return [half](const SegTable<SegPyr> &t, int b, cudaStream_t st) {
                launch_seg_pyr_means(t, b, half != 0, st);
            };
        });
        emit_keyed(P, grads, [](long long half) {
            return [half](const SegTable<SegPyr> &t, int b, cudaStream_t st) {
                launch_seg_pyr_grads(t, b, half != 0, st);
            };
        });
    }
    if (mode == 2) {
        // the flow of each group as one branch, forked from and joined into
        // the step's stream: the latency-bound levels of the groups overlap
        P.ops.push_back([m](cudaStream_t st) {
            cudaEventRecord(m->fork[0], st);
            for (size_t i = 0; i < m->groups.size(); ++i) {
                ebof_group *g = m->groups[i];
                cudaStreamWaitEvent(g->cap, m->fork[0], 0);
                run_group_flow(g, true, g->cap);
                cudaEventRecord(m->fork[1 + i], g->cap);
                cudaStreamWaitEvent(st, m->fork[1 + i], 0);
            }
        });
        return;
    }
    // A6-A8 per level.  The levels are aligned at the coarsest one: step j
    // runs level L - 1 - j of every group with L > j levels, so the small
    // levels of a large resolution, which leave most SMs idle, share their
    // launches with the larger levels of a small one.  A step with one group
    // left runs that group's own launches (with its own layouts).
    int Lmax = 0;
    for (GS &x : gs) Lmax = std::max(Lmax, x.g->geo.levels);
    int cax = 32, cay = 12;
    coeff_tile_shape(cax, cay);
    for (int j = 0; j < Lmax; ++j) {
        int active = 0;
        for (GS &x : gs) active += j < x.g->geo.levels;
        if (active == 1) {
            for (GS &x : gs) {
                ebof_group *g = x.g;
                if (j >= g->geo.levels) continue;
                const int l = g->geo.levels - 1 - j;
                const Level *lv = &g->geo.lv[l];
                const size_t es = g->es;
                const char *I0 = x.prv + g->geo.pyr_off[l] * es;
                const char *I1 = x.cur + g->geo.pyr_off[l] * es;
                const char *I0x = I0 + lv->plane * es, *I0y = I0 + 2 * lv->plane * es;
                float *Ucur = (x.U == g->Ua) ? g->Ub : g->Ua;
                float *Utmp = (Ucur == g->Ua) ? g->Ub : g->Ua;
                const FlowParams fp = flow_params(g->p);
                const float *Uc = x.U;
                const Level *lvc = x.lvc;
                const CUtensorMap *cmap = g->cmaps.ok[l] ? &g->cmaps.map[l] : nullptr;
                P.ops.push_back([=](cudaStream_t st) {
                    tl_level = l;
                    launch_patch_search(I0, I0x, I0y, I1, *lv, g->pyr_fs, Uc, lvc, g->u_fs, g->up,
                                        g->up_fs, g->n, fp, g->d_err, st);
                    launch_densify(I0, I1, *lv, g->pyr_fs, g->up, g->up_fs, Ucur, g->u_fs, g->n,
                                   fp, st);
                    launch_variational(I0, I0x, I0y, I1, *lv, g->pyr_fs, Ucur, Utmp, g->u_fs,
                                       g->work, g->work_fs, g->n, fp, cmap, g->d_err, st);
                    tl_level = -1;
                });
                // where launch_variational leaves the result
                x.U = (fp.var_outer > 0 && (fp.var_outer & 1)) ? Utmp : Ucur;
                x.lvc = lv;
            }
            continue;
        }
        std::vector<std::pair<long long, std::pair<SegSearch, int>>> search;
        std::vector<std::pair<long long, std::pair<SegDensify, int>>> dense;
        struct VarSeg {
            GS *x;
            const Level *lv;
            const char *I0, *I0x, *I0y, *I1;
            float *a, *b;
        };
        std::vector<VarSeg> var;
        for (GS &x : gs) {
            ebof_group *g = x.g;
            if (j >= g->geo.levels) continue;
            const int l = g->geo.levels - 1 - j;
            const ebof_params &p = g->p;
            const Level &lv = g->geo.lv[l];
            const size_t es = g->es;
            const char *I0 = x.prv + g->geo.pyr_off[l] * es;
            const char *I1 = x.cur + g->geo.pyr_off[l] * es;
            const char *I0x = I0 + lv.plane * es, *I0y = I0 + 2 * lv.plane * es;
            float *Ucur = (x.U == g->Ua) ? g->Ub : g->Ua;
            const long long half = p.storage == EBOF_STORAGE_FP16;
            const int np = lv.npx * lv.npy;
            if (np > 0) {
                const bool wide = search_wide(np);
                SegSearch a = {};
                a.I0 = I0;
                a.I0x = I0x;
                a.I0y = I0y;
                a.I1 = I1;
                a.Uc = x.U;
                a.up = g->up;
                a.err = g->d_err;
                a.pfs = g->pyr_fs;
                a.plane_c = x.lvc ? x.lvc->plane : 0;
                a.ucfs = g->u_fs;
                a.upfs = g->up_fs;
                a.w = lv.w;
                a.h = lv.h;
                a.pitch = lv.pitch;
                a.npx = lv.npx;
                a.npy = lv.npy;
                a.wc = x.lvc ? x.lvc->w : 0;
                a.hc = x.lvc ? x.lvc->h : 0;
                a.pitch_c = x.lvc ? x.lvc->pitch : 0;
                a.stride = p.stride;
                a.iters = p.gn_iters;
                a.kappa = p.gn_damping;
                const int ppb = search_patches_per_block(p.patch, wide);
                a.gx = (np + ppb - 1) / ppb;
                search.push_back({(half << 40) | ((long long)p.patch << 8) | (wide ? 1 : 0),
                                  {a, a.gx * g->n}});
            }
            {
                SegDensify a = {};
                a.I0 = I0;
                a.I1 = I1;
                a.up = g->up;
                a.U = Ucur;
                a.pfs = g->pyr_fs;
                a.upfs = g->up_fs;
                a.ufs = g->u_fs;
                a.plane = lv.plane;
                a.w = lv.w;
                a.h = lv.h;
                a.pitch = lv.pitch;
                a.npx = lv.npx;
                a.npy = lv.npy;
                a.ps = p.patch;
                a.stride = p.stride;
                a.gx = (lv.w + 31) / 32;
                a.gy = (lv.h + 7) / 8;
                const int nc = (p.patch + p.stride - 1) / p.stride;
                const long long nck = (nc >= 2 && nc <= 4) ? nc : 0;
                dense.push_back({(half << 40) | nck, {a, a.gx * a.gy * g->n}});
            }
            float *Utmp = (Ucur == g->Ua) ? g->Ub : g->Ua;
            var.push_back({&x, &lv, I0, I0x, I0y, I1, Ucur, Utmp});
            x.U = Ucur;  // the densified flow; the variational steps move it
            x.lvc = &lv;
        }
        emit_keyed(P, search, [](long long k) {
            const bool half = (k >> 40) != 0, wide = (k & 1) != 0;
            const int ps = (int)((k >> 8) & 0xff);
            return [half, wide, ps](const SegTable<SegSearch> &t, int b, cudaStream_t st) {
                launch_seg_search(t, b, ps, wide, half, st);
            };
        });
        emit_keyed(P, dense, [](long long k) {
            const bool half = (k >> 40) != 0;
            const int nc = (int)(k & 0xff);
            return [half, nc](const SegTable<SegDensify> &t, int b, cudaStream_t st) {
                launch_seg_densify(t, b, nc, half, st);
            };
        });
        // A8: outer iteration k of every group that has it: coefficients,
        // then SOR, a and b swapping as in launch_variational
        int outer_max = 0;
        for (const VarSeg &v : var) outer_max = std::max(outer_max, v.x->g->p.var_outer);
        for (int k = 0; k < outer_max; ++k) {
            std::vector<std::pair<long long, std::pair<SegCoeff, int>>> coeff;
            std::vector<std::pair<SegSor, int>> sor;
            for (VarSeg &v : var) {
                const ebof_params &p = v.x->g->p;
                if (k >= p.var_outer) continue;
                const FlowParams fp = flow_params(p);
                const Level &lv = *v.lv;
                const size_t cfs = (size_t)coeff_planes() * lv.plane;
                SegCoeff c = {};
                c.I0 = v.I0;
                c.I0x = v.I0x;
                c.I0y = v.I0y;
                c.I1 = v.I1;
                c.U = v.a;
                c.coef = v.x->g->work;
                c.pfs = v.x->g->pyr_fs;
                c.ufs = v.x->g->u_fs;
                c.plane = lv.plane;
                c.cfs = cfs;
                c.w = lv.w;
                c.h = lv.h;
                c.pitch = lv.pitch;
                c.gx = (lv.w + cax - 1) / cax;
                c.gy = (lv.h + cay - 1) / cay;
                c.delta = fp.delta;
                c.gamma = fp.gamma;
                c.alpha_s = fp.alpha_s;
                c.omega = fp.omega;
                coeff.push_back({fp.half ? 1 : 0, {c, c.gx * c.gy * v.x->g->n}});
                const int n_half = 2 * fp.var_sor;
                SegSor r = {};
                r.Uin = v.a;
                r.Uout = v.b;
                r.coef = v.x->g->work;
                r.ufs = v.x->g->u_fs;
                r.plane = lv.plane;
                r.cfs = cfs;
                r.w = lv.w;
                r.h = lv.h;
                r.pitch = lv.pitch;
                r.R = n_half > 0 ? n_half - 1 : 0;
                r.n_half = n_half;
                r.omega = fp.omega;
                r.gx = (lv.w + sor_tile_x(r.R) - 1) / sor_tile_x(r.R);
                r.gy = (lv.h + sor_tile_y(r.R) - 1) / sor_tile_y(r.R);
                sor.push_back({r, r.gx * r.gy * v.x->g->n});
                std::swap(v.a, v.b);
                v.x->U = v.a;
            }
            emit_keyed(P, coeff, [](long long half) {
                return [half](const SegTable<SegCoeff> &t, int b, cudaStream_t st) {
                    launch_seg_coeff(t, b, half != 0, st);
                };
            });
            emit_seg(P, sor, launch_seg_sor);
        }
    }
    // A9: each group's level-0 flow into its flow buffer
    {
        std::vector<std::pair<SegFlowOut, int>> segs;
        for (GS &x : gs) {
            ebof_group *g = x.g;
            const int W = g->p.width, H = g->p.height;
            if (g->geo.levels == 0) {
                P.ops.push_back([g, W, H](cudaStream_t st) {
                    cudaMemsetAsync(g->flow, 0, sizeof(float) * 2 * (size_t)W * H * g->n, st);
                });
                continue;
            }
            SegFlowOut a = {};
            a.U = x.U;
            a.flow = g->flow;
            a.ufs = g->u_fs;
            a.plane = (size_t)g->pitch0 * H;
            a.W = W;
            a.H = H;
            a.pitch = g->pitch0;
            a.gx = (W + 255) / 256;
            segs.push_back({a, a.gx * H * g->n});
        }
        emit_seg(P, segs, launch_seg_flow_out);
    }
}

bool events_ok(const void *x, const void *y, const void *t, int64_t n)
{
    return n >= 0 && (n == 0 || (x && y && t));
}

}  // namespace

extern "C" {

void ebof_default_params(ebof_params *p, int32_t width, int32_t height)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->struct_size = sizeof(ebof_params);
    p->width = width;
    p->height = height;
    p->connectivity = 8;
    p->n_d = 1;
    p->n_f = 9;
    p->alpha = 1.08f;
    const bool hr = width >= 640;
    p->levels = hr ? 5 : 3;
    p->patch = hr ? 12 : 8;
    p->stride = 4;
    p->gn_iters = 12;
    p->gn_damping = 0.1f;
    p->var_outer = 5;
    p->var_sor = 5;
    p->var_delta = 5.0f;
    p->var_gamma = 10.0f;
    p->var_alpha = 20.0f;
    p->sor_omega = 1.6f;
    p->max_batch = 1;
    p->storage = EBOF_STORAGE_FP32;
    p->surface = EBOF_SURFACE_EXP;
    p->d_sat = 6.0f;
    p->coeff_cw_min_width = 1024;
    // the copy-ahead SOR kernel: 1280 x 720 batches of 40 windows ran 3 %
    // faster without it (same flow); 346 x 260 groups slightly faster with it
    p->sor_tma_min_per_sm = width >= 1024 ? (1 << 20) : 4;
    p->sor_row_waves = 1;
    // the cluster-resident refinement of small levels gives the same flow but
    // measured no faster inside a graph (1544 vs 1573 frames/s at 1280 x 720):
    // off unless chosen (the autotuner tries it for groups)
    p->var_cluster_max = 0;
    p->coeff_cw_rows = 8;
}

float ebof_alpha_from_dsat(float d_sat) { return d_sat / std::log(255.0f); }

ebof_status ebof_stream_create(const ebof_params *p, int device, ebof_stream **out)
{
    if (!out) return EBOF_ERR_INVALID_ARG;
    *out = nullptr;
    const ebof_status ps = check_params(p);
    if (ps != EBOF_OK) return ps;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return device < 0 ? EBOF_ERR_INVALID_ARG : EBOF_ERR_CUDA;
    DeviceGuard dg(device);
    if (!dg.ok) return EBOF_ERR_CUDA;
    ebof_stream *s = new (std::nothrow) ebof_stream();
    if (!s) return EBOF_ERR_OOM;
    s->p = *p;
    s->device = device;
    s->geo = make_geometry(p->width, p->height, p->levels, p->patch, p->stride);
    const Geometry &geo = s->geo;
    const int B = p->max_batch;
    s->pitch0 = geo.lv[0].pitch;
    const size_t plane0 = geo.lv[0].plane;
    s->e_fs = plane0;
    s->g_fs = plane0;
    s->pyr_fs = geo.pyr_floats;
    s->up_fs = (size_t)2 * std::max(geo.max_patches, 1);
    s->u_fs = 2 * plane0;
    s->work_fs = 9 * plane0;
    s->nslots = B + 1;
    bool ok = true;
    ok &= dmalloc(&s->E, s->e_fs * B) == cudaSuccess;
    ok &= dmalloc(&s->Ed, s->e_fs * B) == cudaSuccess;
    ok &= dmalloc(&s->Edf, s->e_fs * B) == cudaSuccess;
    ok &= dmalloc(&s->g, sizeof(int32_t) * s->g_fs * B) == cudaSuccess;
    s->es = p->storage == EBOF_STORAGE_FP16 ? 2 : 4;
    ok &= dmalloc(&s->pyr, s->es * s->pyr_fs * s->nslots) == cudaSuccess;
    ok &= dmalloc(&s->up, sizeof(float) * s->up_fs * B) == cudaSuccess;
    ok &= dmalloc(&s->Ua, sizeof(float) * s->u_fs * B) == cudaSuccess;
    ok &= dmalloc(&s->Ub, sizeof(float) * s->u_fs * B) == cudaSuccess;
    ok &= dmalloc(&s->work, sizeof(float) * s->work_fs * B) == cudaSuccess;
    ok &= dmalloc(&s->dstats, sizeof(DevStats) * B) == cudaSuccess;
    ok &= dmalloc(&s->d_dropped_time, sizeof(unsigned long long)) == cudaSuccess;
    ok &= dmalloc(&s->d_err, sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&s->flow_stage, sizeof(float) * 2 * (size_t)p->width * p->height) == cudaSuccess;
    ok &= cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming) == cudaSuccess;
    const size_t call_bytes = (sizeof(ebof_window_desc) + sizeof(float *)) * B;
    ok &= dmalloc(&s->d_call, call_bytes) == cudaSuccess;
    s->d_wins = (ebof_window_desc *)s->d_call;
    s->d_flows = (float **)(s->d_call + sizeof(ebof_window_desc) * B);
    s->h_call.assign(call_bytes, 0);
    s->list_graph.assign(B + 1, nullptr);
    s->list_graph_kernels.assign(B + 1, 0);
    s->last_win_events.assign(B, 0);
    ok &= cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_all(s);
        delete s;
        return EBOF_ERR_OOM;
    }
    cudaMemset(s->d_err, 0, sizeof(int));
    cudaMemset(s->dstats, 0, sizeof(DevStats) * B);
    make_coef_maps(s->work, s->geo, B, &s->cmaps);
    cudaMemset(s->d_dropped_time, 0, sizeof(unsigned long long));
    if (cudaDeviceSynchronize() != cudaSuccess) {
        free_all(s);
        delete s;
        return EBOF_ERR_CUDA;
    }
    *out = s;
    return EBOF_OK;
}

int64_t ebof_stream_device_bytes(const ebof_params *p)
{
    if (check_params(p) != EBOF_OK) return -1;
    const Geometry geo = make_geometry(p->width, p->height, p->levels, p->patch, p->stride);
    const size_t B = (size_t)p->max_batch, plane0 = geo.lv[0].plane;
    const size_t es = p->storage == EBOF_STORAGE_FP16 ? 2 : 4;
    auto r = [](size_t b) { return std::max<size_t>(b, 256); };
    size_t total = 3 * r(plane0 * B) + r(4 * plane0 * B) + r(es * geo.pyr_floats * (B + 1));
    total += r(4 * 2 * (size_t)std::max(geo.max_patches, 1) * B);
    total += 2 * r(4 * 2 * plane0 * B) + r(4 * 9 * plane0 * B);
    total += r(sizeof(DevStats) * B) + 2 * 256 + r(4 * 2 * (size_t)p->width * p->height) +
             r((sizeof(ebof_window_desc) + sizeof(float *)) * B);
    return (int64_t)total;
}

ebof_status ebof_stream_destroy(ebof_stream *s)
{
    if (!s) return EBOF_OK;
    DeviceGuard dg(s->device);
    if (s->have_last) cudaEventSynchronize(s->done);
    free_all(s);
    delete s;
    return EBOF_OK;
}

ebof_status ebof_stream_reset(ebof_stream *s)
{
    if (!s) return EBOF_ERR_INVALID_ARG;
    BusyGuard bg(s->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    DeviceGuard dg(s->device);
    if (s->have_last && cudaEventSynchronize(s->done) != cudaSuccess) return EBOF_ERR_CUDA;
    s->has_prev = false;
    s->head = 0;
    s->pl.has_prev = false;
    s->pl.latest = false;
    return EBOF_OK;
}

ebof_status ebof_process_window(ebof_stream *s, const uint16_t *d_x, const uint16_t *d_y,
                                const int64_t *d_t, const int8_t *d_p, int64_t n_events,
                                int64_t t_begin, int64_t t_end, float *d_flow, uint8_t *d_edge,
                                int32_t *d_edt, float *d_surface, void *cuda_stream)
{
    (void)d_p;  // polarity is not used (§III-A)
    if (!s || !d_flow || !events_ok(d_x, d_y, d_t, n_events) || t_end < t_begin)
        return EBOF_ERR_INVALID_ARG;
    BusyGuard bg(s->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    DeviceGuard dg(s->device);
    if (!dg.ok) return EBOF_ERR_CUDA;
    return run(s, 1, d_x, d_y, d_t, n_events, t_begin, t_end - t_begin, nullptr, d_flow, d_edge,
               d_edt, d_surface, (cudaStream_t)cuda_stream);
}

ebof_status ebof_process_windows(ebof_stream *s, int32_t n_windows, const uint16_t *d_x,
                                 const uint16_t *d_y, const int64_t *d_t, const int8_t *d_p,
                                 int64_t n_events, int64_t t_begin, int64_t dt, float *d_flow,
                                 uint8_t *d_edge, int32_t *d_edt, float *d_surface,
                                 void *cuda_stream)
{
    (void)d_p;
    if (!s || !d_flow || !events_ok(d_x, d_y, d_t, n_events) || dt < 0) return EBOF_ERR_INVALID_ARG;
    if (n_windows < 1 || n_windows > s->p.max_batch) return EBOF_ERR_INVALID_ARG;
    BusyGuard bg(s->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    DeviceGuard dg(s->device);
    if (!dg.ok) return EBOF_ERR_CUDA;
    return run(s, n_windows, d_x, d_y, d_t, n_events, t_begin, dt, nullptr, d_flow, d_edge,
               d_edt, d_surface, (cudaStream_t)cuda_stream);
}

ebof_status ebof_process_window_list(ebof_stream *s, int32_t n_windows,
                                     const ebof_window_desc *windows, float *const *d_flows,
                                     void *cuda_stream)
{
    if (!s || !windows || !d_flows || n_windows < 1 || n_windows > s->p.max_batch)
        return EBOF_ERR_INVALID_ARG;
    for (int k = 0; k < n_windows; ++k) {
        const ebof_window_desc &w = windows[k];
        if (!d_flows[k] || !events_ok(w.x, w.y, w.t, w.n_events) || w.t_end < w.t_begin)
            return EBOF_ERR_INVALID_ARG;
    }
    BusyGuard bg(s->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    DeviceGuard dg(s->device);
    if (!dg.ok) return EBOF_ERR_CUDA;
    return run_list(s, n_windows, windows, d_flows, (cudaStream_t)cuda_stream);
}

ebof_status ebof_process_surface(ebof_stream *s, const float *d_surface, float *d_flow,
                                 void *cuda_stream)
{
    if (!s || !d_surface || !d_flow) return EBOF_ERR_INVALID_ARG;
    BusyGuard bg(s->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    DeviceGuard dg(s->device);
    if (!dg.ok) return EBOF_ERR_CUDA;
    return run(s, 1, nullptr, nullptr, nullptr, 0, 0, 0, d_surface, d_flow, nullptr, nullptr,
               nullptr, (cudaStream_t)cuda_stream);
}

ebof_status ebof_stream_get_pyramid(ebof_stream *s, int32_t level, float *d_I, float *d_Ix,
                                    float *d_Iy, void *cuda_stream)
{
    if (!s || level < 0 || level >= s->geo.levels) return EBOF_ERR_INVALID_ARG;
    BusyGuard bg(s->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    DeviceGuard dg(s->device);
    if (!dg.ok) return EBOF_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaGetLastError();
    // the newest window's pyramid into the ordinary slots (after the work
    // that wrote it), as before an ordinary call
    pipeline_leave(s, st);
    if (!s->has_prev) return EBOF_NO_PREVIOUS;
    if (s->have_last && s->last_stream != st) cudaStreamWaitEvent(st, s->done, 0);
    const Level &lv = s->geo.lv[level];
    const char *I = s->pyr + ((size_t)s->head * s->pyr_fs + s->geo.pyr_off[level]) * s->es;
    const bool half = s->es == 2;
    float *dst[3] = {d_I, d_Ix, d_Iy};
    for (int k = 0; k < 3; ++k)
        if (dst[k])
            launch_pyramid_export(I + (size_t)k * lv.plane * s->es, half, lv.w, lv.h, lv.pitch,
                                  dst[k], st);
    // later calls write this slot only after the copies
    cudaEventRecord(s->done, st);
    s->last_stream = st;
    s->have_last = true;
    return cudaGetLastError() == cudaSuccess ? EBOF_OK : EBOF_ERR_CUDA;
}

typedef CUresult (*PointerAttrFn)(void *, CUpointer_attribute, CUdeviceptr);

static PointerAttrFn pointer_attr_fn()
{
    static std::atomic<PointerAttrFn> fn{nullptr};
    static std::atomic<int> tried{0};
    if (!tried.exchange(1)) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn.store((PointerAttrFn)p);
        cudaGetLastError();
    }
    return fn.load();
}

// A host buffer of `bytes` bytes that the current device can address at the
// same virtual address: page-locked memory registered with CUDA under unified
// addressing, the whole extent inside one registered range (a buffer that
// starts in a page-locked range and runs past its end is not).  Pageable
// memory is not addressable either; the caller stages it.
static bool device_addressable(const void *h, size_t bytes)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type != cudaMemoryTypeHost || a.devicePointer != h) return false;
    PointerAttrFn fn = pointer_attr_fn();
    if (!fn) return false;
    CUdeviceptr start = 0;
    size_t size = 0;
    if (fn(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, (CUdeviceptr)h) != CUDA_SUCCESS ||
        fn(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, (CUdeviceptr)h) != CUDA_SUCCESS)
        return false;
    const uintptr_t b = (uintptr_t)h, s0 = (uintptr_t)start;
    return b >= s0 && bytes <= size && b - s0 <= size - bytes;
}

ebof_status ebof_process_window_host(ebof_stream *s, const uint16_t *h_x, const uint16_t *h_y,
                                     const int64_t *h_t, int64_t n_events, int64_t t_begin,
                                     int64_t t_end, float *h_flow, void *cuda_stream)
{
    if (!s || !h_flow || !events_ok(h_x, h_y, h_t, n_events) || t_end < t_begin)
        return EBOF_ERR_INVALID_ARG;
    BusyGuard bg(s->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    DeviceGuard dg(s->device);
    if (!dg.ok) return EBOF_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t n = (size_t)n_events;
    // page-locked buffers of a window with a previous one: the kernels read
    // the events and write the flow in place over the host link, with no
    // staging copies (the first window, whose flow is cleared with a memset,
    // and pageable buffers take the staged path below)
    const size_t flow_bytes = sizeof(float) * 2 * (size_t)s->p.width * s->p.height;
    if (s->has_prev && s->geo.levels > 0 && device_addressable(h_flow, flow_bytes) &&
        (n == 0 || (device_addressable(h_x, 2 * n) && device_addressable(h_y, 2 * n) &&
                    device_addressable(h_t, 8 * n)))) {
        const ebof_status r = run(s, 1, h_x, h_y, h_t, n_events, t_begin, t_end - t_begin,
                                  nullptr, h_flow, nullptr, nullptr, nullptr, st);
        if (r < 0) return r;
        if (cudaStreamSynchronize(st) != cudaSuccess) return EBOF_ERR_CUDA;
        return r;
    }
    const size_t bx = ((2 * n + 255) / 256) * 256;
    const size_t need = 2 * bx + 8 * n;
    if (need > s->ev_stage_bytes) {
        if (s->have_last) cudaEventSynchronize(s->done);
        cudaFree(s->ev_stage);
        s->ev_stage = nullptr;
        s->ev_stage_bytes = 0;
        if (dmalloc(&s->ev_stage, std::max<size_t>(need, 1 << 20)) != cudaSuccess) {
            cudaGetLastError();
            return EBOF_ERR_OOM;
        }
        s->ev_stage_bytes = std::max<size_t>(need, 1 << 20);
    }
    char *base = (char *)s->ev_stage;
    uint16_t *dx = (uint16_t *)base;
    uint16_t *dy = (uint16_t *)(base + bx);
    int64_t *dt = (int64_t *)(base + 2 * bx);
    if (s->have_last && s->last_stream != st) cudaStreamWaitEvent(st, s->done, 0);
    if (n) {
        cudaMemcpyAsync(dx, h_x, 2 * n, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dy, h_y, 2 * n, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dt, h_t, 8 * n, cudaMemcpyHostToDevice, st);
    }
    ebof_status r = run(s, 1, dx, dy, dt, n_events, t_begin, t_end - t_begin, nullptr,
                        s->flow_stage, nullptr, nullptr, nullptr, st);
    if (r < 0) return r;
    cudaMemcpyAsync(h_flow, s->flow_stage, flow_bytes, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return EBOF_ERR_CUDA;
    return r;
}

ebof_status ebof_process_window_async(ebof_stream *s, const uint16_t *d_x, const uint16_t *d_y,
                                      const int64_t *d_t, const int8_t *d_p, int64_t n_events,
                                      int64_t t_begin, int64_t t_end, float *d_flow,
                                      void *cuda_stream)
{
    (void)d_p;  // polarity is not used (§III-A)
    if (!s || !d_flow || !events_ok(d_x, d_y, d_t, n_events) || t_end < t_begin)
        return EBOF_ERR_INVALID_ARG;
    BusyGuard bg(s->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    DeviceGuard dg(s->device);
    if (!dg.ok) return EBOF_ERR_CUDA;
    cudaGetLastError();
    const ebof_status rp = pipeline_ready(s);
    if (rp < 0) return rp;
    auto &L = s->pl;
    // the window's inputs: the caller's work on its stream so far
    cudaEventRecord(L.inputs, (cudaStream_t)cuda_stream);
    cudaStreamWaitEvent(L.front, L.inputs, 0);
    // d_flow: the caller's stream may read what an earlier call wrote there
    for (cudaStream_t f : L.flow) cudaStreamWaitEvent(f, L.inputs, 0);
    return run_pipelined(s, d_x, d_y, d_t, n_events, t_begin, t_end - t_begin, d_flow);
}

ebof_status ebof_process_window_host_async(ebof_stream *s, const uint16_t *h_x,
                                           const uint16_t *h_y, const int64_t *h_t,
                                           int64_t n_events, int64_t t_begin, int64_t t_end,
                                           float *h_flow, void *cuda_stream)
{
    (void)cuda_stream;  // every step runs on the stream's own streams
    if (!s || !h_flow || !events_ok(h_x, h_y, h_t, n_events) || t_end < t_begin)
        return EBOF_ERR_INVALID_ARG;
    const size_t n = (size_t)n_events;
    const size_t flow_bytes = sizeof(float) * 2 * (size_t)s->p.width * s->p.height;
    bool pinned;
    {
        DeviceGuard dg(s->device);
        if (!dg.ok) return EBOF_ERR_CUDA;
        pinned = device_addressable(h_flow, flow_bytes) &&
                 (n == 0 || (device_addressable(h_x, 2 * n) && device_addressable(h_y, 2 * n) &&
                             device_addressable(h_t, 8 * n)));
    }
    // pageable buffers: the synchronous staged call
    if (!pinned)
        return ebof_process_window_host(s, h_x, h_y, h_t, n_events, t_begin, t_end, h_flow,
                                        cuda_stream);
    BusyGuard bg(s->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    DeviceGuard dg(s->device);
    if (!dg.ok) return EBOF_ERR_CUDA;
    cudaGetLastError();
    ebof_status rp = pipeline_ready(s);
    if (rp < 0) return rp;
    auto &L = s->pl;
    auto &q = s->pipe;
    if (!q.ready) {
        bool ok = cudaStreamCreateWithFlags(&q.h2d, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&q.d2h, cudaStreamNonBlocking) == cudaSuccess;
        for (int j = 0; j < ebof_stream::HostPipe::kSlots && ok; ++j) {
            ok &= cudaEventCreateWithFlags(&q.in_done[j], cudaEventDisableTiming) == cudaSuccess;
            ok &= cudaEventCreateWithFlags(&q.run_done[j], cudaEventDisableTiming) == cudaSuccess;
            ok &= cudaEventCreateWithFlags(&q.out_done[j], cudaEventDisableTiming) == cudaSuccess;
            ok &= dmalloc(&q.flow[j], flow_bytes) == cudaSuccess;
        }
        if (!ok) {
            cudaGetLastError();
            // undo, so that a later call starts again from nothing
            for (int k = 0; k < ebof_stream::HostPipe::kSlots; ++k) {
                cudaFree(q.flow[k]);
                q.flow[k] = nullptr;
                for (cudaEvent_t *e : {&q.in_done[k], &q.run_done[k], &q.out_done[k]})
                    if (*e) {
                        cudaEventDestroy(*e);
                        *e = nullptr;
                    }
            }
            for (cudaStream_t *x : {&q.h2d, &q.d2h})
                if (*x) {
                    cudaStreamDestroy(*x);
                    *x = nullptr;
                }
            return EBOF_ERR_OOM;
        }
        q.ready = true;
    }
    const int j = q.slot;
    // the slot's events buffer: the front end kSlots calls back must have read it
    const size_t bx = ((2 * n + 255) / 256) * 256;
    const size_t need = 2 * bx + 8 * n;
    if (need > q.ev_bytes[j]) {
        if (q.used[j]) cudaEventSynchronize(q.run_done[j]);
        cudaFree(q.ev[j]);
        q.ev[j] = nullptr;
        q.ev_bytes[j] = 0;
        const size_t bytes = std::max<size_t>(need, 1 << 20);
        if (dmalloc(&q.ev[j], bytes) != cudaSuccess) {
            cudaGetLastError();
            return EBOF_ERR_OOM;
        }
        q.ev_bytes[j] = bytes;
    }
    char *base = (char *)q.ev[j];
    uint16_t *dx = (uint16_t *)base;
    uint16_t *dy = (uint16_t *)(base + bx);
    int64_t *dt = (int64_t *)(base + 2 * bx);
    // events in, after the front end that last read this slot
    if (q.used[j]) cudaStreamWaitEvent(q.h2d, q.run_done[j], 0);
    if (n) {
        cudaMemcpyAsync(dx, h_x, 2 * n, cudaMemcpyHostToDevice, q.h2d);
        cudaMemcpyAsync(dy, h_y, 2 * n, cudaMemcpyHostToDevice, q.h2d);
        cudaMemcpyAsync(dt, h_t, 8 * n, cudaMemcpyHostToDevice, q.h2d);
    }
    cudaEventRecord(q.in_done[j], q.h2d);
    cudaStreamWaitEvent(L.front, q.in_done[j], 0);
    // the flow staging slot: after the copy out kSlots calls back
    if (q.used[j])
        for (cudaStream_t f : L.flow) cudaStreamWaitEvent(f, q.out_done[j], 0);
    const ebof_status r = run_pipelined(s, dx, dy, dt, n_events, t_begin, t_end - t_begin,
                                        q.flow[j]);
    if (r < 0) return r;
    cudaEventRecord(q.run_done[j], L.front);  // the front end has read the events
    // flow out, overlapping the next windows' kernels
    cudaStreamWaitEvent(q.d2h, s->done, 0);
    cudaMemcpyAsync(h_flow, q.flow[j], flow_bytes, cudaMemcpyDeviceToHost, q.d2h);
    cudaEventRecord(q.out_done[j], q.d2h);
    q.used[j] = true;
    q.slot = (j + 1) % ebof_stream::HostPipe::kSlots;
    if (cudaGetLastError() != cudaSuccess) return EBOF_ERR_CUDA;
    return r;
}

ebof_status ebof_stream_join(ebof_stream *s, void *cuda_stream)
{
    if (!s) return EBOF_ERR_INVALID_ARG;
    BusyGuard bg(s->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    DeviceGuard dg(s->device);
    if (!dg.ok) return EBOF_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (s->have_last) cudaStreamWaitEvent(st, s->done, 0);
    for (int j = 0; j < ebof_stream::HostPipe::kSlots; ++j)
        if (s->pipe.used[j]) cudaStreamWaitEvent(st, s->pipe.out_done[j], 0);
    return cudaGetLastError() == cudaSuccess ? EBOF_OK : EBOF_ERR_CUDA;
}

ebof_status ebof_stream_set_wait_limit(ebof_stream *s, int64_t iterations)
{
    if (!s) return EBOF_ERR_INVALID_ARG;
    BusyGuard bg(s->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    s->wait_limit = iterations < 0 ? kWaitLimitDefault : (long long)iterations;
    return EBOF_OK;
}

void ebof_debug_fail_allocation(int32_t n) { g_alloc_fail_after.store(n < 0 ? -1 : n); }

ebof_status ebof_stream_sync(ebof_stream *s, ebof_window_stats *out, int32_t n_out)
{
    if (!s || n_out < 0 || (n_out > 0 && !out)) return EBOF_ERR_INVALID_ARG;
    BusyGuard bg(s->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    DeviceGuard dg(s->device);
    if (!dg.ok) return EBOF_ERR_CUDA;
    if (s->have_last && cudaEventSynchronize(s->done) != cudaSuccess) return EBOF_ERR_CUDA;
    for (int j = 0; j < ebof_stream::HostPipe::kSlots; ++j)
        if (s->pipe.used[j] && cudaEventSynchronize(s->pipe.out_done[j]) != cudaSuccess)
            return EBOF_ERR_CUDA;
    int err = 0;
    if (cudaMemcpy(&err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return EBOF_ERR_CUDA;
    const int n = std::min<int>(n_out, s->last_n);
    if (n > 0) {
        DevStats hs[64];
        unsigned long long dropped_time = 0;
        cudaMemcpy(&dropped_time, s->d_dropped_time, sizeof(dropped_time),
                   cudaMemcpyDeviceToHost);
        for (int k0 = 0; k0 < n; k0 += 64) {
            const int m = std::min(64, n - k0);
            if (cudaMemcpy(hs, s->dstats + k0, sizeof(DevStats) * m, cudaMemcpyDeviceToHost) !=
                cudaSuccess)
                return EBOF_ERR_CUDA;
            for (int k = 0; k < m; ++k) {
                ebof_window_stats &o = out[k0 + k];
                o.events = s->last_list ? s->last_win_events[k0 + k] : s->last_events;
                o.in_window = (int64_t)hs[k].in_window;
                o.dropped_time = (int64_t)dropped_time;
                o.dropped_oob = (int64_t)hs[k].dropped_oob;
                o.edge_px = (int64_t)hs[k].edge_px;
                const bool hf = (k0 + k) > 0 || s->last_had_prev;
                o.has_flow = hf ? 1 : 0;
                o.levels_used = hf ? s->geo.levels : 0;
            }
        }
    }
    if (err) {
        cudaMemset(s->d_err, 0, sizeof(int));
        return (err & kErrTimeout) ? EBOF_ERR_TIMEOUT : EBOF_ERR_DEVICE_BOUNDS;
    }
    return EBOF_OK;
}

ebof_status ebof_edt(const uint8_t *d_edge, int32_t width, int32_t height, int32_t *d_scratch,
                     int32_t *d_edt, float *d_surface, float alpha, void *cuda_stream)
{
    if (!d_edge || !d_scratch || !d_edt || width < 1 || height < 1 || width > kMaxDim ||
        height > kMaxDim || !(std::isfinite(alpha) && alpha > 0.0f))
        return EBOF_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EBOF_ERR_CUDA;
    DeviceGuard dg(dev);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaGetLastError();
    const size_t plane = (size_t)width * height;
    launch_edt_columns(d_edge, width, plane, width, height, d_scratch, width, plane, 1, st);
    launch_edt_rows_surface(d_scratch, width, plane, width, height, alpha, d_edt, d_surface,
                            nullptr, width, plane, 1, false, st);
    return cudaGetLastError() == cudaSuccess ? EBOF_OK : EBOF_ERR_CUDA;
}

ebof_status ebof_group_create(const ebof_params *p, int32_t n_streams, int device,
                              ebof_group **out)
{
    if (!out) return EBOF_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_streams < 1 || n_streams > 4096) return EBOF_ERR_INVALID_ARG;
    ebof_params q;
    if (p) {
        q = *p;
        q.max_batch = 1;  // not used by groups; keeps the parameter check happy
    }
    const ebof_status ps = check_params(p ? &q : nullptr);
    if (ps != EBOF_OK) return ps;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return device < 0 ? EBOF_ERR_INVALID_ARG : EBOF_ERR_CUDA;
    DeviceGuard dg(device);
    if (!dg.ok) return EBOF_ERR_CUDA;
    ebof_group *g = new (std::nothrow) ebof_group();
    if (!g) return EBOF_ERR_OOM;
    g->p = q;
    g->device = device;
    g->n = n_streams;
    g->geo = make_geometry(q.width, q.height, q.levels, q.patch, q.stride);
    const Geometry &geo = g->geo;
    const int n = n_streams;
    g->pitch0 = geo.lv[0].pitch;
    const size_t plane0 = geo.lv[0].plane;
    g->e_fs = plane0;
    g->g_fs = plane0;
    g->pyr_fs = geo.pyr_floats;
    g->up_fs = (size_t)2 * std::max(geo.max_patches, 1);
    g->u_fs = 2 * plane0;
    g->work_fs = 9 * plane0;
    g->es = q.storage == EBOF_STORAGE_FP16 ? 2 : 4;
    g->h_events = new (std::nothrow) int64_t[n];
    bool ok = g->h_events != nullptr;
    ok &= dmalloc(&g->E, g->e_fs * n) == cudaSuccess;
    ok &= dmalloc(&g->Ed, g->e_fs * n) == cudaSuccess;
    ok &= dmalloc(&g->Edf, g->e_fs * n) == cudaSuccess;
    ok &= dmalloc(&g->g, sizeof(int32_t) * g->g_fs * n) == cudaSuccess;
    ok &= dmalloc(&g->pyr, g->es * g->pyr_fs * n * 2) == cudaSuccess;
    ok &= dmalloc(&g->up, sizeof(float) * g->up_fs * n) == cudaSuccess;
    ok &= dmalloc(&g->Ua, sizeof(float) * g->u_fs * n) == cudaSuccess;
    ok &= dmalloc(&g->Ub, sizeof(float) * g->u_fs * n) == cudaSuccess;
    ok &= dmalloc(&g->work, sizeof(float) * g->work_fs * n) == cudaSuccess;
    ok &= dmalloc(&g->flow, sizeof(float) * 2 * (size_t)q.width * q.height * n) == cudaSuccess;
    ok &= dmalloc(&g->dstats, sizeof(DevStats) * n) == cudaSuccess;
    ok &= dmalloc(&g->d_dropped_time, sizeof(unsigned long long)) == cudaSuccess;
    ok &= dmalloc(&g->d_err, sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&g->d_desc, sizeof(ebof_window_desc) * n) == cudaSuccess;
    ok &= cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking) == cudaSuccess;
    ok &= cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_group(g);
        delete g;
        return EBOF_ERR_OOM;
    }
    cudaMemset(g->d_err, 0, sizeof(int));
    cudaMemset(g->flow, 0, sizeof(float) * 2 * (size_t)q.width * q.height * n);
    make_coef_maps(g->work, g->geo, n, &g->cmaps);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        free_group(g);
        delete g;
        return EBOF_ERR_CUDA;
    }
    *out = g;
    return EBOF_OK;
}

ebof_status ebof_group_destroy(ebof_group *g)
{
    if (!g) return EBOF_OK;
    DeviceGuard dg(g->device);
    if (g->have_last) cudaEventSynchronize(g->done);
    free_group(g);
    delete g;
    return EBOF_OK;
}

ebof_status ebof_group_reset(ebof_group *g)
{
    if (!g) return EBOF_ERR_INVALID_ARG;
    BusyGuard bg(g->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    DeviceGuard dg(g->device);
    if (g->have_last && cudaEventSynchronize(g->done) != cudaSuccess) return EBOF_ERR_CUDA;
    g->has_prev = false;
    g->parity = 0;
    return EBOF_OK;
}

ebof_status ebof_group_process(ebof_group *g, const ebof_window_desc *h_desc, float *d_flow,
                               void *cuda_stream)
{
    if (!g || !h_desc) return EBOF_ERR_INVALID_ARG;
    for (int k = 0; k < g->n; ++k)
        if (!events_ok(h_desc[k].x, h_desc[k].y, h_desc[k].t, h_desc[k].n_events) ||
            h_desc[k].t_end < h_desc[k].t_begin)
            return EBOF_ERR_INVALID_ARG;
    BusyGuard bg(g->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    DeviceGuard dg(g->device);
    if (!dg.ok) return EBOF_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaGetLastError();
    if (g->have_last && g->last_stream != st) cudaStreamWaitEvent(st, g->done, 0);
    for (int k = 0; k < g->n; ++k) g->h_events[k] = h_desc[k].n_events;
    cudaMemcpyAsync(g->d_desc, h_desc, sizeof(ebof_window_desc) * g->n, cudaMemcpyHostToDevice,
                    st);
    const bool had_prev = g->has_prev;
    ProfScope prof_scope(&g->prof);
    if (!had_prev || g->prof.on) {
        run_group(g, had_prev, st);  // first step, or timed stage by stage: no graph
    } else {
        const int b = g->parity;
        if (!g->graph[b]) {
            // capture this parity's step once; the capture stream starts after `st`
            cudaEvent_t ready;
            cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
            cudaEventRecord(ready, st);
            cudaStreamWaitEvent(g->cap, ready, 0);
            cudaEventDestroy(ready);
            const unsigned long long before = g_launches.load();
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                tl_prof = nullptr;  // no event records inside a graph
                run_group(g, true, g->cap);
                cudaStreamEndCapture(g->cap, &graph);
            }
            if (graph && cudaGraphInstantiate(&g->graph[b], graph, 0) != cudaSuccess)
                g->graph[b] = nullptr;
            if (graph) cudaGraphDestroy(graph);
            g->graph_kernels[b] = (long long)(g_launches.load() - before);
            g_launches.fetch_sub((unsigned long long)g->graph_kernels[b]);
            if (!g->graph[b]) {
                cudaGetLastError();
                return EBOF_ERR_CUDA;
            }
        }
        if (cudaGraphLaunch(g->graph[b], st) != cudaSuccess) return EBOF_ERR_CUDA;
        g_launches.fetch_add((unsigned long long)g->graph_kernels[b]);
    }
    if (d_flow)
        cudaMemcpyAsync(d_flow, g->flow, sizeof(float) * 2 * (size_t)g->p.width * g->p.height * g->n,
                        cudaMemcpyDeviceToDevice, st);
    g->parity ^= 1;
    g->has_prev = true;
    g->last_had_prev = had_prev;
    cudaEventRecord(g->done, st);
    g->last_stream = st;
    g->have_last = true;
    if (cudaGetLastError() != cudaSuccess) return EBOF_ERR_CUDA;
    return had_prev ? EBOF_OK : EBOF_NO_PREVIOUS;
}

ebof_status ebof_multigroup_create(ebof_group *const *groups, int32_t n_groups,
                                   ebof_multigroup **out)
{
    if (!out) return EBOF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!groups || n_groups < 1 || n_groups > 64) return EBOF_ERR_INVALID_ARG;
    for (int i = 0; i < n_groups; ++i) {
        if (!groups[i] || groups[i]->device != groups[0]->device) return EBOF_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (groups[j] == groups[i]) return EBOF_ERR_INVALID_ARG;
    }
    DeviceGuard dg(groups[0]->device);
    if (!dg.ok) return EBOF_ERR_CUDA;
    ebof_multigroup *m = new (std::nothrow) ebof_multigroup();
    if (!m) return EBOF_ERR_OOM;
    m->groups.assign(groups, groups + n_groups);
    m->device = groups[0]->device;
    bool ok = cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking) == cudaSuccess;
    m->fork.assign(n_groups + 1, nullptr);
    for (auto &e : m->fork)
        ok &= cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        ebof_multigroup_destroy(m);
        return EBOF_ERR_OOM;
    }
    *out = m;
    return EBOF_OK;
}

ebof_status ebof_multigroup_destroy(ebof_multigroup *m)
{
    if (!m) return EBOF_OK;
    DeviceGuard dg(m->device);
    for (ebof_group *g : m->groups)
        if (g->have_last) cudaEventSynchronize(g->done);
    for (auto &pg : m->graphs)
        if (pg.second) cudaGraphExecDestroy(pg.second);
    for (cudaEvent_t e : m->fork)
        if (e) cudaEventDestroy(e);
    if (m->cap) cudaStreamDestroy(m->cap);
    delete m;
    return EBOF_OK;
}

ebof_status ebof_multigroup_set_fused(ebof_multigroup *m, int32_t fused)
{
    if (!m || fused < 0 || fused > 2) return EBOF_ERR_INVALID_ARG;
    if (fused)
        for (const ebof_group *g : m->groups)
            if (!fused_supported(g, fused)) return EBOF_ERR_UNSUPPORTED;
    if (m->fused == fused) return EBOF_OK;
    std::vector<std::unique_ptr<BusyGuard>> guards;
    for (ebof_group *g : m->groups) {
        guards.emplace_back(new (std::nothrow) BusyGuard(g->busy));
        if (!guards.back()) return EBOF_ERR_OOM;
        if (!guards.back()->ok) return EBOF_ERR_BUSY;
    }
    DeviceGuard dg(m->device);
    if (!dg.ok) return EBOF_ERR_CUDA;
    // graphs in flight may still read their tables
    for (ebof_group *g : m->groups)
        if (g->have_last) cudaEventSynchronize(g->done);
    for (auto &pg : m->graphs)
        if (pg.second) cudaGraphExecDestroy(pg.second);
    m->graphs.clear();
    m->graph_kernels.clear();
    m->plans.clear();
    m->fused = fused;
    return EBOF_OK;
}

ebof_status ebof_multigroup_process(ebof_multigroup *m, const ebof_window_desc *const *h_descs,
                                    void *cuda_stream)
{
    if (!m || !h_descs) return EBOF_ERR_INVALID_ARG;
    const int ng = (int)m->groups.size();
    for (int i = 0; i < ng; ++i) {
        const ebof_group *g = m->groups[i];
        if (!h_descs[i]) return EBOF_ERR_INVALID_ARG;
        for (int k = 0; k < g->n; ++k) {
            const ebof_window_desc &w = h_descs[i][k];
            if (!events_ok(w.x, w.y, w.t, w.n_events) || w.t_end < w.t_begin)
                return EBOF_ERR_INVALID_ARG;
        }
    }
    // every group is claimed for the call (released when the guards go)
    std::vector<std::unique_ptr<BusyGuard>> guards;
    for (ebof_group *g : m->groups) {
        guards.emplace_back(new (std::nothrow) BusyGuard(g->busy));
        if (!guards.back()) return EBOF_ERR_OOM;
        if (!guards.back()->ok) return EBOF_ERR_BUSY;
    }
    DeviceGuard dg(m->device);
    if (!dg.ok) return EBOF_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaGetLastError();
    bool all_prev = true, any_prof = false;
    unsigned long long key = 0;
    for (int i = 0; i < ng; ++i) {
        ebof_group *g = m->groups[i];
        if (g->have_last && g->last_stream != st) cudaStreamWaitEvent(st, g->done, 0);
        for (int k = 0; k < g->n; ++k) g->h_events[k] = h_descs[i][k].n_events;
        cudaMemcpyAsync(g->d_desc, h_descs[i], sizeof(ebof_window_desc) * g->n,
                        cudaMemcpyHostToDevice, st);
        all_prev &= g->has_prev;
        any_prof |= g->prof.on;
        key |= (unsigned long long)g->parity << i;
    }
    if (!all_prev || any_prof) {
        // first step of some group, or stage timing: each group's step eagerly
        for (ebof_group *g : m->groups) {
            ProfScope prof_scope(&g->prof);
            run_group(g, g->has_prev, st);
        }
    } else {
        size_t slot = m->graphs.size();
        for (size_t j = 0; j < m->graphs.size(); ++j)
            if (m->graphs[j].first == key) slot = j;
        if (slot == m->graphs.size()) {
            // capture the step once for this parity pattern: every group's
            // step as one branch of the graph, forked from and joined into
            // the capture stream, which itself starts after `st`
            cudaEventRecord(m->fork[0], st);
            cudaStreamWaitEvent(m->cap, m->fork[0], 0);
            const unsigned long long before = g_launches.load();
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t ge = nullptr;
            std::unique_ptr<FusedPlan> plan;
            if (m->fused) {
                // the fused launches' tables, copied to the device once
                plan.reset(new (std::nothrow) FusedPlan());
                if (!plan) return EBOF_ERR_OOM;
                build_fused_plan(m, *plan, m->fused);
                if (dmalloc(&plan->dev, plan->host.size()) != cudaSuccess) {
                    cudaGetLastError();
                    return EBOF_ERR_OOM;
                }
                if (cudaMemcpyAsync(plan->dev, plan->host.data(), plan->host.size(),
                                    cudaMemcpyHostToDevice, m->cap) != cudaSuccess ||
                    cudaStreamSynchronize(m->cap) != cudaSuccess) {
                    cudaGetLastError();
                    return EBOF_ERR_CUDA;
                }
            }
            if (cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                tl_prof = nullptr;
                if (plan) {
                    for (auto &op : plan->ops) op(m->cap);
                } else {
                    cudaEventRecord(m->fork[0], m->cap);
                    for (int i = 0; i < ng; ++i) {
                        ebof_group *g = m->groups[i];
                        cudaStreamWaitEvent(g->cap, m->fork[0], 0);
                        run_group(g, true, g->cap);
                        cudaEventRecord(m->fork[1 + i], g->cap);
                        cudaStreamWaitEvent(m->cap, m->fork[1 + i], 0);
                    }
                }
                cudaStreamEndCapture(m->cap, &graph);
            }
            if (graph && cudaGraphInstantiate(&ge, graph, 0) != cudaSuccess) ge = nullptr;
            if (graph) cudaGraphDestroy(graph);
            const long long kernels = (long long)(g_launches.load() - before);
            g_launches.fetch_sub((unsigned long long)kernels);
            if (!ge) {
                cudaGetLastError();
                return EBOF_ERR_CUDA;
            }
            m->graphs.emplace_back(key, ge);
            m->graph_kernels.push_back(kernels);
            m->plans.push_back(std::move(plan));
        }
        if (cudaGraphLaunch(m->graphs[slot].second, st) != cudaSuccess) return EBOF_ERR_CUDA;
        g_launches.fetch_add((unsigned long long)m->graph_kernels[slot]);
    }
    ebof_status ret = EBOF_OK;
    for (ebof_group *g : m->groups) {
        if (!g->has_prev) ret = EBOF_NO_PREVIOUS;
        g->last_had_prev = g->has_prev;
        g->parity ^= 1;
        g->has_prev = true;
        cudaEventRecord(g->done, st);
        g->last_stream = st;
        g->have_last = true;
    }
    if (cudaGetLastError() != cudaSuccess) return EBOF_ERR_CUDA;
    return ret;
}

const float *ebof_group_flow(const ebof_group *g, int32_t k)
{
    if (!g || k < 0 || k >= g->n) return nullptr;
    return g->flow + (size_t)k * 2 * g->p.width * g->p.height;
}

ebof_status ebof_group_sync(ebof_group *g, ebof_window_stats *out, int32_t n_out)
{
    if (!g || n_out < 0 || (n_out > 0 && !out)) return EBOF_ERR_INVALID_ARG;
    BusyGuard bg(g->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    DeviceGuard dg(g->device);
    if (!dg.ok) return EBOF_ERR_CUDA;
    if (g->have_last && cudaEventSynchronize(g->done) != cudaSuccess) return EBOF_ERR_CUDA;
    int err = 0;
    if (cudaMemcpy(&err, g->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return EBOF_ERR_CUDA;
    const int n = std::min<int>(n_out, g->n);
    if (n > 0) {
        DevStats hs[64];
        unsigned long long dropped_time = 0;
        cudaMemcpy(&dropped_time, g->d_dropped_time, sizeof(dropped_time),
                   cudaMemcpyDeviceToHost);
        for (int k0 = 0; k0 < n; k0 += 64) {
            const int m = std::min(64, n - k0);
            if (cudaMemcpy(hs, g->dstats + k0, sizeof(DevStats) * m, cudaMemcpyDeviceToHost) !=
                cudaSuccess)
                return EBOF_ERR_CUDA;
            for (int k = 0; k < m; ++k) {
                ebof_window_stats &o = out[k0 + k];
                o.events = g->h_events[k0 + k];
                o.in_window = (int64_t)hs[k].in_window;
                o.dropped_time = (int64_t)dropped_time;
                o.dropped_oob = (int64_t)hs[k].dropped_oob;
                o.edge_px = (int64_t)hs[k].edge_px;
                o.has_flow = g->last_had_prev ? 1 : 0;
                o.levels_used = g->last_had_prev ? g->geo.levels : 0;
            }
        }
    }
    if (err) {
        cudaMemset(g->d_err, 0, sizeof(int));
        return (err & kErrTimeout) ? EBOF_ERR_TIMEOUT : EBOF_ERR_DEVICE_BOUNDS;
    }
    return EBOF_OK;
}

ebof_status ebof_stream_set_profiling(ebof_stream *s, int32_t enable)
{
    if (!s) return EBOF_ERR_INVALID_ARG;
    BusyGuard bg(s->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    DeviceGuard dg(s->device);
    s->prof.reset();
    s->prof.on = enable != 0;
    if (s->prof.on) {
        // create the events up front so that timed regions never create any
        while (s->prof.pool.size() < 65536) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreate(&e) != cudaSuccess) break;
            s->prof.pool.push_back(e);
        }
    }
    return EBOF_OK;
}

ebof_status ebof_stream_get_profile(ebof_stream *s, double *ms, int64_t *launches, int32_t n)
{
    if (!s || n < 0 || n > EBOF_STAGE_COUNT) return EBOF_ERR_INVALID_ARG;
    BusyGuard bg(s->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    DeviceGuard dg(s->device);
    s->prof.flush();
    for (int i = 0; i < n; ++i) {
        double t = 0.0;
        long long c = 0;
        for (int l = 0; l < kProfLevels; ++l) { t += s->prof.ms[i][l]; c += s->prof.launches[i][l]; }
        if (ms) ms[i] = t;
        if (launches) launches[i] = c;
    }
    return EBOF_OK;
}

ebof_status ebof_stream_get_profile_level(ebof_stream *s, int32_t level, double *ms,
                                          int64_t *launches, int32_t n)
{
    if (!s || n < 0 || n > EBOF_STAGE_COUNT || level < -1 || level >= kProfLevels - 1)
        return EBOF_ERR_INVALID_ARG;
    BusyGuard bg(s->busy);
    if (!bg.ok) return EBOF_ERR_BUSY;
    DeviceGuard dg(s->device);
    s->prof.flush();
    const int l = level < 0 ? kProfLevels - 1 : level;
    for (int i = 0; i < n; ++i) {
        if (ms) ms[i] = s->prof.ms[i][l];
        if (launches) launches[i] = s->prof.launches[i][l];
    }
    return EBOF_OK;
}

const char *ebof_stage_name(int32_t stage) { return stage_name(stage); }

uint64_t ebof_kernel_launches(void) { return g_launches.load(); }

const char *ebof_status_string(ebof_status st)
{
    switch (st) {
    case EBOF_OK: return "ok";
    case EBOF_NO_PREVIOUS: return "first window: no previous surface, flow zero";
    case EBOF_ERR_INVALID_ARG: return "invalid argument";
    case EBOF_ERR_OOM: return "out of device memory";
    case EBOF_ERR_CUDA: return "CUDA error";
    case EBOF_ERR_TIMEOUT: return "device wait timed out";
    case EBOF_ERR_DEVICE_BOUNDS: return "device bounds check failed";
    case EBOF_ERR_UNSUPPORTED: return "unsupported parameter";
    case EBOF_ERR_BUSY: return "stream in use by another thread";
    case EBOF_QUEUED: return "waiting for memory to be admitted";
    case EBOF_ERR_CANCELLED: return "cancelled before it ran";
    }
    return "unknown status";
}

}  // extern "C"
