// Host-only checks of the server's scheduling core (serve_core.h) against a
// fake backend whose batches take a fixed wall time.  Built and run by
// tests/test_serve_core.py; prints one "PASS name" or "FAIL name: why" line
// per scenario and exits non-zero on any failure.
#include "serve_core.h"

#include <atomic>
#include <cstdio>
#include <map>
#include <string>

using ebof_serve::now_ns;

namespace {

struct FakeStream {
    int id;
    bool busy = false, has_prev = false;
};

struct Launch {
    int worker, stream, n;
    std::vector<int64_t> tags;
};

class FakeBackend : public ebof_serve::Backend {
public:
    FakeBackend(int n_workers, int64_t batch_us, std::atomic<int> *violations)
        : end_(n_workers, 0), owner_(n_workers, nullptr), batch_us_(batch_us), viol_(violations)
    {
    }
    // the fake's "device bytes" of a stream are its width
    int64_t stream_bytes(const ebof_params &p) override { return p.width; }
    int create_stream(const ebof_params &p, void **h) override
    {
        if (p.height == 13) return EBOF_ERR_OOM;  // a stream whose allocation fails
        std::lock_guard<std::mutex> lk(mu);
        FakeStream *s = new FakeStream();
        s->id = p.levels;  // the scenario's name for the stream
        created.push_back(s->id);
        *h = s;
        return EBOF_OK;
    }
    void destroy_stream(void *h) override
    {
        std::lock_guard<std::mutex> lk(mu);
        FakeStream *s = (FakeStream *)h;
        if (s->busy) ++*viol_;
        destroyed.push_back(s->id);
        delete s;
    }
    int launch(int w, void *h, int n, const ebof_window_desc *wins, float *const *) override
    {
        std::lock_guard<std::mutex> lk(mu);
        FakeStream *s = (FakeStream *)h;
        if (s->busy || owner_[w]) ++*viol_;  // stream or worker already busy
        s->busy = true;
        owner_[w] = s;
        end_[w] = now_ns() + batch_us_ * 1000;
        Launch L{w, s->id, n, {}};
        for (int k = 0; k < n; ++k) L.tags.push_back(wins[k].t_begin);
        launches.push_back(L);
        if (s->id == 99) return EBOF_ERR_CUDA;  // a stream whose launches fail
        const int r = s->has_prev ? EBOF_OK : EBOF_NO_PREVIOUS;
        s->has_prev = true;
        return r;
    }
    int query(int w) override
    {
        std::lock_guard<std::mutex> lk(mu);
        if (now_ns() < end_[w]) return 1;
        if (owner_[w]) owner_[w]->busy = false;
        owner_[w] = nullptr;
        return 0;
    }
    std::mutex mu;
    std::vector<int> created, destroyed;
    std::vector<Launch> launches;

private:
    std::vector<int64_t> end_;
    std::vector<FakeStream *> owner_;
    int64_t batch_us_;
    std::atomic<int> *viol_;
};

ebof_params params(int name, int bytes, int max_batch)
{
    ebof_params p{};
    p.width = bytes;
    p.height = 8;
    p.levels = name;
    p.max_batch = max_batch;
    return p;
}

ebof_window_desc win(int64_t tag)
{
    ebof_window_desc w{};
    w.t_begin = tag;
    w.t_end = tag + 1;
    return w;
}

float g_flow[1];
int g_fail = 0;

void check(bool ok, const char *name, const std::string &why)
{
    if (ok) {
        std::printf("PASS %s\n", name);
    } else {
        std::printf("FAIL %s: %s\n", name, why.c_str());
        ++g_fail;
    }
}

// Waits until the fake has seen n launches.
bool wait_launches(FakeBackend *be, size_t n, int timeout_ms = 5000)
{
    const int64_t t_end = now_ns() + (int64_t)timeout_ms * 1000000;
    while (now_ns() < t_end) {
        {
            std::lock_guard<std::mutex> lk(be->mu);
            if (be->launches.size() >= n) return true;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    return false;
}

std::vector<ebof_completion> collect(ebof_serve::Server &srv, size_t n, int timeout_ms = 5000)
{
    std::vector<ebof_completion> out;
    const int64_t t_end = now_ns() + (int64_t)timeout_ms * 1000000;
    ebof_completion buf[64];
    while (out.size() < n && now_ns() < t_end) {
        const int k = srv.poll(buf, 64, 2000);
        out.insert(out.end(), buf, buf + k);
    }
    return out;
}

// Streams are admitted in order while they fit; a later small stream does
// not overtake a waiting large one; closing frees memory and admits waiters.
void admission()
{
    std::atomic<int> viol{0};
    auto *be = new FakeBackend(2, 200, &viol);
    ebof_serve::Server srv(std::unique_ptr<ebof_serve::Backend>(be), 100, 2);
    int32_t a, b, c, d, e;
    bool ok = srv.open_stream(params(1, 40, 4), &a) == EBOF_OK;
    ok &= srv.open_stream(params(2, 40, 4), &b) == EBOF_OK;
    ok &= srv.open_stream(params(3, 40, 4), &c) == EBOF_QUEUED;
    ok &= srv.open_stream(params(4, 10, 4), &d) == EBOF_QUEUED;  // fits, but waits its turn
    ok &= srv.open_stream(params(5, 101, 4), &e) == EBOF_ERR_OOM;
    ebof_server_info in{};
    srv.info(&in);
    ok &= in.streams_admitted == 2 && in.streams_waiting == 2 && in.memory_in_use == 80;
    for (int k = 0; k < 3; ++k) {
        ok &= srv.submit(a, win(100 + k), g_flow, 100 + k, 0) == EBOF_OK;
        ok &= srv.submit(c, win(300 + k), g_flow, 300 + k, 0) == EBOF_OK;
        ok &= srv.submit(d, win(400 + k), g_flow, 400 + k, 0) == EBOF_OK;
    }
    auto got = collect(srv, 3);  // only stream a's windows can run
    ok &= got.size() == 3;
    for (auto &x : got) ok &= x.stream_id == a;
    srv.info(&in);
    ok &= in.streams_waiting == 2;
    ok &= srv.close_stream(a) == EBOF_OK;
    ok &= srv.submit(a, win(1), g_flow, 1, 0) == EBOF_ERR_INVALID_ARG;
    got = collect(srv, 6);
    ok &= got.size() == 6 && srv.drain(2000) == EBOF_OK;
    srv.info(&in);
    ok &= in.streams_admitted == 3 && in.streams_waiting == 0 && in.memory_in_use == 90;
    {
        std::lock_guard<std::mutex> lk(be->mu);
        ok &= be->created == std::vector<int>({1, 2, 3, 4});
        ok &= be->destroyed == std::vector<int>({1});
    }
    check(ok && viol == 0, "admission", "admission order, budget or retirement wrong");
}

// A stream's windows complete in submission order, in batches no larger than
// its limit, never two batches of one stream at once; the first window of a
// stream reports NO_PREVIOUS.
void fifo_and_batches()
{
    std::atomic<int> viol{0};
    auto *be = new FakeBackend(4, 300, &viol);
    ebof_serve::Server srv(std::unique_ptr<ebof_serve::Backend>(be), 1000, 4);
    int32_t s1, s2;
    bool ok = srv.open_stream(params(1, 10, 3), &s1) == EBOF_OK;
    ok &= srv.open_stream(params(2, 10, 5), &s2) == EBOF_OK;
    const int N = 40;
    for (int k = 0; k < N; ++k) {
        srv.submit(s1, win(k), g_flow, k, 0);
        srv.submit(s2, win(1000 + k), g_flow, 1000 + k, 0);
        if (k % 7 == 0) std::this_thread::sleep_for(std::chrono::microseconds(500));
    }
    auto got = collect(srv, 2 * N);
    ok &= got.size() == (size_t)(2 * N);
    std::map<int, int64_t> next = {{s1, 0}, {s2, 1000}};
    for (auto &x : got) {
        ok &= (int64_t)x.tag == next[x.stream_id];
        next[x.stream_id]++;
        const bool first = x.tag == 0 || x.tag == 1000;
        ok &= x.status == (first ? EBOF_NO_PREVIOUS : EBOF_OK);
        ok &= x.batch >= 1 && x.batch <= (x.stream_id == s1 ? 3 : 5);
        ok &= x.done_ns >= x.launch_ns && x.launch_ns >= x.arrival_ns;
    }
    int maxb1 = 0;
    {
        std::lock_guard<std::mutex> lk(be->mu);
        for (auto &L : be->launches)
            if (L.stream == 1) maxb1 = std::max(maxb1, L.n);
    }
    check(ok && viol == 0 && maxb1 == 3, "fifo_and_batches",
          "order, status, batch limit or exclusivity violated");
}

// With one worker busy, the backlog of a stream is launched as one batch.
void continuous_batching()
{
    std::atomic<int> viol{0};
    auto *be = new FakeBackend(1, 20000, &viol);
    ebof_serve::Server srv(std::unique_ptr<ebof_serve::Backend>(be), 1000, 1);
    int32_t s;
    bool ok = srv.open_stream(params(1, 10, 8), &s) == EBOF_OK;
    srv.submit(s, win(0), g_flow, 0, 0);
    ok &= wait_launches(be, 1);  // the first window runs alone
    for (int k = 1; k < 20; ++k) srv.submit(s, win(k), g_flow, k, 0);
    auto got = collect(srv, 20);
    ok &= got.size() == 20;
    std::vector<int> sizes;
    {
        std::lock_guard<std::mutex> lk(be->mu);
        for (auto &L : be->launches) sizes.push_back(L.n);
    }
    ok &= sizes == std::vector<int>({1, 8, 8, 3});
    ebof_server_info in{};
    srv.info(&in);
    ok &= in.batches_launched == 4 && in.max_batch_seen == 8 && in.windows_completed == 20;
    check(ok && viol == 0, "continuous_batching", "batches did not follow the backlog");
}

// When a worker frees up, the stream whose oldest window arrived first goes.
void oldest_first()
{
    std::atomic<int> viol{0};
    auto *be = new FakeBackend(1, 20000, &viol);
    ebof_serve::Server srv(std::unique_ptr<ebof_serve::Backend>(be), 1000, 1);
    int32_t z, x, y;
    bool ok = srv.open_stream(params(7, 10, 1), &z) == EBOF_OK;
    ok &= srv.open_stream(params(8, 10, 1), &x) == EBOF_OK;
    ok &= srv.open_stream(params(9, 10, 1), &y) == EBOF_OK;
    srv.submit(z, win(0), g_flow, 0, 0);  // occupies the only worker
    ok &= wait_launches(be, 1);
    const int64_t t0 = now_ns();
    srv.submit(x, win(1), g_flow, 1, t0 + 200);  // submitted first, arrived later
    srv.submit(y, win(2), g_flow, 2, t0 + 100);
    auto got = collect(srv, 3);
    ok &= got.size() == 3;
    std::vector<int> order;
    {
        std::lock_guard<std::mutex> lk(be->mu);
        for (auto &L : be->launches) order.push_back(L.stream);
    }
    check(ok && viol == 0 && order == std::vector<int>({7, 9, 8}), "oldest_first",
          "launch order did not follow arrival times");
}

// Closing a waiting stream cancels its windows; failed allocations and
// failed launches are reported per window; destroy with a backlog returns.
void errors_and_cancel()
{
    std::atomic<int> viol{0};
    auto *be = new FakeBackend(2, 200, &viol);
    bool ok = true;
    {
        ebof_serve::Server srv(std::unique_ptr<ebof_serve::Backend>(be), 50, 2);
        int32_t a, w, bad, oom;
        ok &= srv.open_stream(params(1, 30, 2), &a) == EBOF_OK;
        ok &= srv.open_stream(params(2, 30, 2), &w) == EBOF_QUEUED;
        for (int k = 0; k < 4; ++k) srv.submit(w, win(k), g_flow, k, 0);
        ok &= srv.close_stream(w) == EBOF_OK;
        auto got = collect(srv, 4);
        ok &= got.size() == 4;
        for (auto &x : got) ok &= x.status == EBOF_ERR_CANCELLED && x.stream_id == w;
        ok &= srv.open_stream(params(99, 10, 2), &bad) == EBOF_OK;
        for (int k = 0; k < 3; ++k) srv.submit(bad, win(k), g_flow, k, 0);
        got = collect(srv, 3);
        ok &= got.size() == 3;
        for (auto &x : got) ok &= x.status == EBOF_ERR_CUDA;
        ebof_params p = params(3, 5, 2);
        p.height = 13;  // the fake fails this allocation
        ok &= srv.open_stream(p, &oom) == EBOF_ERR_OOM;
        ok &= srv.submit(12345, win(0), g_flow, 0, 0) == EBOF_ERR_INVALID_ARG;
        for (int k = 0; k < 50; ++k) srv.submit(a, win(k), g_flow, k, 0);
    }  // destroyed with windows still queued
    check(ok && viol == 0, "errors_and_cancel", "cancellation or error reporting wrong");
}

}  // namespace

int main()
{
    admission();
    fifo_and_batches();
    continuous_batching();
    oldest_first();
    errors_and_cancel();
    return g_fail ? 1 : 0;
}
