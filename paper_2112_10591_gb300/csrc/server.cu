// server.cu -- ebof_server_* of include/ebof.h: the request loop of
// serve_core.h on a CUDA backend.  Each worker is a non-blocking CUDA stream
// with one completion event; a batch is one ebof_process_window_list call on
// the worker's stream followed by an event record.
#include "ebof.h"
#include "serve_core.h"

#include <cuda_runtime.h>

#include <new>

namespace {

class CudaBackend : public ebof_serve::Backend {
public:
    CudaBackend(int device, int n_workers) : device_(device), st_(n_workers), ev_(n_workers) {}

    bool init()
    {
        if (cudaSetDevice(device_) != cudaSuccess) return false;
        for (size_t w = 0; w < st_.size(); ++w) {
            if (cudaStreamCreateWithFlags(&st_[w], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev_[w], cudaEventDisableTiming) != cudaSuccess)
                return false;
        }
        return true;
    }

    ~CudaBackend() override
    {
        cudaSetDevice(device_);
        for (size_t w = 0; w < st_.size(); ++w) {
            if (st_[w]) cudaStreamSynchronize(st_[w]);
            if (ev_[w]) cudaEventDestroy(ev_[w]);
            if (st_[w]) cudaStreamDestroy(st_[w]);
        }
    }

    int64_t stream_bytes(const ebof_params &p) override { return ebof_stream_device_bytes(&p); }

    int create_stream(const ebof_params &p, void **handle) override
    {
        ebof_stream *s = nullptr;
        const ebof_status r = ebof_stream_create(&p, device_, &s);
        *handle = s;
        return r;
    }

    void destroy_stream(void *handle) override { ebof_stream_destroy((ebof_stream *)handle); }

    int launch(int w, void *handle, int n, const ebof_window_desc *wins,
               float *const *flows) override
    {
        const ebof_status r =
            ebof_process_window_list((ebof_stream *)handle, n, wins, flows, st_[w]);
        cudaEventRecord(ev_[w], st_[w]);
        return r;
    }

    int query(int w) override
    {
        const cudaError_t e = cudaEventQuery(ev_[w]);
        if (e == cudaSuccess) return 0;
        if (e == cudaErrorNotReady) return 1;
        return EBOF_ERR_CUDA;
    }

    void bind_thread() override { cudaSetDevice(device_); }

private:
    int device_;
    std::vector<cudaStream_t> st_;
    std::vector<cudaEvent_t> ev_;
};

}  // namespace

struct ebof_server {
    ebof_serve::Server *core = nullptr;
};

extern "C" {

int64_t ebof_now_ns(void) { return ebof_serve::now_ns(); }

void ebof_server_default_config(ebof_server_config *c)
{
    if (!c) return;
    c->struct_size = (int32_t)sizeof(ebof_server_config);
    c->device = 0;
    c->memory_budget = 40000000000LL;
    c->n_workers = 8;
}

ebof_status ebof_server_create(const ebof_server_config *c, ebof_server **out)
{
    if (!out) return EBOF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!c || c->struct_size != (int32_t)sizeof(ebof_server_config) || c->memory_budget <= 0 ||
        c->n_workers < 1 || c->n_workers > 64 || c->device < 0)
        return EBOF_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c->device >= ndev) return EBOF_ERR_CUDA;
    int prev = -1;
    cudaGetDevice(&prev);
    CudaBackend *be = new (std::nothrow) CudaBackend(c->device, c->n_workers);
    if (!be) return EBOF_ERR_OOM;
    const bool ok = be->init();
    if (prev >= 0) cudaSetDevice(prev);
    if (!ok) {
        delete be;
        cudaGetLastError();
        return EBOF_ERR_CUDA;
    }
    ebof_server *v = new (std::nothrow) ebof_server();
    if (!v) {
        delete be;
        return EBOF_ERR_OOM;
    }
    v->core = new (std::nothrow)
        ebof_serve::Server(std::unique_ptr<ebof_serve::Backend>(be), c->memory_budget,
                           c->n_workers);
    if (!v->core) {
        delete v;
        return EBOF_ERR_OOM;
    }
    *out = v;
    return EBOF_OK;
}

ebof_status ebof_server_destroy(ebof_server *v)
{
    if (!v) return EBOF_OK;
    delete v->core;
    delete v;
    return EBOF_OK;
}

ebof_status ebof_server_open_stream(ebof_server *v, const ebof_params *p, int32_t *id)
{
    if (!v || !p || !id) return EBOF_ERR_INVALID_ARG;
    return (ebof_status)v->core->open_stream(*p, id);
}

ebof_status ebof_server_close_stream(ebof_server *v, int32_t id)
{
    if (!v) return EBOF_ERR_INVALID_ARG;
    return (ebof_status)v->core->close_stream(id);
}

ebof_status ebof_server_submit(ebof_server *v, int32_t id, const ebof_window_desc *w,
                               float *d_flow, uint64_t tag, int64_t arrival_ns)
{
    if (!v || !w || !d_flow || w->n_events < 0 || w->t_end < w->t_begin ||
        (w->n_events > 0 && (!w->x || !w->y || !w->t)))
        return EBOF_ERR_INVALID_ARG;
    return (ebof_status)v->core->submit(id, *w, d_flow, tag, arrival_ns);
}

int32_t ebof_server_poll(ebof_server *v, ebof_completion *out, int32_t max_out, int32_t wait_us)
{
    if (!v || max_out < 0 || (max_out > 0 && !out)) return EBOF_ERR_INVALID_ARG;
    return v->core->poll(out, max_out, wait_us);
}

ebof_status ebof_server_drain(ebof_server *v, int32_t timeout_ms)
{
    if (!v || timeout_ms < 0) return EBOF_ERR_INVALID_ARG;
    return (ebof_status)v->core->drain(timeout_ms);
}

ebof_status ebof_server_get_info(ebof_server *v, ebof_server_info *out)
{
    if (!v || !out) return EBOF_ERR_INVALID_ARG;
    v->core->info(out);
    return EBOF_OK;
}

}  // extern "C"
