// serve_core.h -- the request loop behind ebof_server_* (include/ebof.h),
// written without CUDA so that its scheduling can be exercised on a host with
// a fake backend.
//
// A server holds camera streams, each with its own flow state (previous
// window, pyramids, buffers).  Streams are admitted in arrival order while
// the sum of their device-state sizes stays within a byte budget; a stream
// that does not fit waits until closed streams free enough memory.  Windows
// submitted to a stream wait in that stream's FIFO.  One dispatcher thread
// keeps up to n_workers batches in flight: whenever a worker is free it takes
// the stream whose oldest queued window arrived first (and that has no batch
// in flight, so a stream's windows run in order) and launches all of that
// stream's queued windows up to its batch limit as one batch.  Batches
// therefore grow with the backlog and shrink again when the queues empty
// (continuous batching).  The device work goes through Backend.
#pragma once

#include "ebof.h"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace ebof_serve {

inline int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// The device side of the server.  Worker w is one queue of device work (a
// CUDA stream); launch() is called only for a worker whose previous batch has
// completed, and only from the dispatcher thread.
class Backend {
public:
    virtual ~Backend() = default;
    virtual int64_t stream_bytes(const ebof_params &p) = 0;          // -1: invalid
    virtual int create_stream(const ebof_params &p, void **handle) = 0;  // ebof_status
    virtual void destroy_stream(void *handle) = 0;
    // n windows of one stream on worker w; returns the call's ebof_status.
    virtual int launch(int w, void *handle, int n, const ebof_window_desc *wins,
                       float *const *flows) = 0;
    // 1 while worker w's batch runs, 0 once it completed, < 0 an ebof_status.
    virtual int query(int w) = 0;
    virtual void bind_thread() {}  // called once on the dispatcher thread
};

class Server {
public:
    Server(std::unique_ptr<Backend> be, int64_t budget, int n_workers)
        : be_(std::move(be)), budget_(budget), workers_(n_workers)
    {
        thread_ = std::thread([this] { loop(); });
    }

    // Stops the dispatcher: queued windows are dropped, batches in flight
    // complete, then every stream's state is freed.
    ~Server()
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stopping_ = true;
            for (auto &s : streams_) {
                outstanding_ -= (int64_t)s->queue.size();
                s->queue.clear();
            }
        }
        cv_work_.notify_all();
        thread_.join();
        for (auto &s : streams_)
            if (s->handle) be_->destroy_stream(s->handle);
    }

    int open_stream(const ebof_params &p, int32_t *id)
    {
        const int64_t bytes = be_->stream_bytes(p);
        if (bytes < 0) return EBOF_ERR_INVALID_ARG;
        if (bytes > budget_) return EBOF_ERR_OOM;
        std::unique_lock<std::mutex> lk(mu_);
        if (stopping_) return EBOF_ERR_INVALID_ARG;
        auto s = std::make_unique<Stream>();
        s->p = p;
        s->bytes = bytes;
        Stream *sp = s.get();
        const int32_t sid = (int32_t)streams_.size();
        if (waiting_.empty() && used_ + bytes <= budget_) {
            used_ += bytes;
            sp->state = kCreating;
            streams_.push_back(std::move(s));
            lk.unlock();
            void *h = nullptr;
            const int r = be_->create_stream(p, &h);
            lk.lock();
            if (r < 0) {
                used_ -= bytes;
                sp->state = kClosed;
                return r;
            }
            sp->handle = h;
            sp->state = kAdmitted;
            *id = sid;
            lk.unlock();
            cv_work_.notify_all();
            return EBOF_OK;
        }
        sp->state = kWaiting;
        streams_.push_back(std::move(s));
        waiting_.push_back(sid);
        *id = sid;
        return EBOF_QUEUED;
    }

    // No further submissions; queued windows of an admitted stream still run,
    // then its state is freed and waiting streams are admitted.  A stream
    // still waiting for admission is dropped with its windows cancelled.
    int close_stream(int32_t id)
    {
        std::unique_lock<std::mutex> lk(mu_);
        Stream *s = get(id);
        if (!s || s->closing || s->state == kCreating) return EBOF_ERR_INVALID_ARG;
        s->closing = true;
        if (s->state == kWaiting) {
            waiting_.erase(std::find(waiting_.begin(), waiting_.end(), id));
            cancel(id, *s, EBOF_ERR_CANCELLED);
            s->state = kClosed;
            lk.unlock();
            cv_done_.notify_all();
            cv_work_.notify_all();  // the next waiting stream may fit now
            return EBOF_OK;
        }
        lk.unlock();
        cv_work_.notify_all();
        return EBOF_OK;
    }

    int submit(int32_t id, const ebof_window_desc &w, float *flow, uint64_t tag,
               int64_t arrival_ns)
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            Stream *s = get(id);
            if (!s || s->closing || stopping_) return EBOF_ERR_INVALID_ARG;
            Pending q;
            q.win = w;
            q.flow = flow;
            q.tag = tag;
            q.arrival = arrival_ns > 0 ? arrival_ns : now_ns();
            s->queue.push_back(q);
            ++outstanding_;
            ++submitted_;
        }
        cv_work_.notify_all();
        return EBOF_OK;
    }

    // Moves up to max_out completions to out, waiting up to wait_us for the
    // first one; returns how many.
    int poll(ebof_completion *out, int max_out, int wait_us)
    {
        std::unique_lock<std::mutex> lk(mu_);
        if (done_.empty() && wait_us > 0)
            cv_done_.wait_for(lk, std::chrono::microseconds(wait_us),
                              [this] { return !done_.empty(); });
        int n = 0;
        while (n < max_out && !done_.empty()) {
            out[n++] = done_.front();
            done_.pop_front();
        }
        return n;
    }

    // Waits until every submitted window has completed or been cancelled.
    int drain(int timeout_ms)
    {
        std::unique_lock<std::mutex> lk(mu_);
        const bool ok = cv_done_.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                          [this] { return outstanding_ == 0; });
        return ok ? EBOF_OK : EBOF_ERR_TIMEOUT;
    }

    void info(ebof_server_info *o)
    {
        std::lock_guard<std::mutex> lk(mu_);
        o->streams_admitted = 0;
        o->streams_waiting = (int32_t)waiting_.size();
        for (auto &s : streams_)
            if (s->state == kAdmitted) ++o->streams_admitted;
        o->memory_budget = budget_;
        o->memory_in_use = used_;
        o->windows_submitted = submitted_;
        o->windows_completed = completed_;
        o->batches_launched = batches_;
        o->batches_in_flight = in_flight_;
        o->max_batch_seen = max_batch_seen_;
    }

private:
    enum State { kWaiting, kCreating, kAdmitted, kClosed };
    struct Pending {
        ebof_window_desc win;
        float *flow;
        uint64_t tag;
        int64_t arrival;
    };
    struct Stream {
        ebof_params p;
        int64_t bytes = 0;
        void *handle = nullptr;
        State state = kWaiting;
        bool closing = false, busy = false;
        std::deque<Pending> queue;
    };
    struct Worker {
        int32_t sid = -1;  // stream of the batch in flight, -1 = free
        bool launching = false;
        int status = EBOF_OK;
        int64_t launch_ns = 0;
        std::vector<Pending> batch;
    };

    Stream *get(int32_t id)
    {
        if (id < 0 || id >= (int32_t)streams_.size()) return nullptr;
        Stream *s = streams_[id].get();
        return s->state == kClosed ? nullptr : s;
    }

    void cancel(int32_t id, Stream &s, int status)
    {
        const int64_t t = now_ns();
        for (const Pending &q : s.queue) {
            ebof_completion c{};
            c.stream_id = id;
            c.status = status;
            c.tag = q.tag;
            c.arrival_ns = q.arrival;
            c.launch_ns = t;
            c.done_ns = t;
            done_.push_back(c);
        }
        outstanding_ -= (int64_t)s.queue.size();
        s.queue.clear();
    }

    // Frees a closed stream's state and admits waiting streams that now fit
    // (in arrival order, no overtaking).  Called with the lock held; drops it
    // around backend calls.
    void retire(int32_t id, std::unique_lock<std::mutex> &lk)
    {
        Stream &s = *streams_[id];
        void *h = s.handle;
        s.handle = nullptr;
        s.state = kClosed;
        lk.unlock();
        be_->destroy_stream(h);
        lk.lock();
        used_ -= s.bytes;
        admit_waiting(lk);
    }

    void admit_waiting(std::unique_lock<std::mutex> &lk)
    {
        while (!waiting_.empty() && !stopping_) {
            const int32_t id = waiting_.front();
            Stream &s = *streams_[id];
            if (used_ + s.bytes > budget_) break;
            waiting_.pop_front();
            used_ += s.bytes;
            s.state = kCreating;
            lk.unlock();
            void *h = nullptr;
            const int r = be_->create_stream(s.p, &h);
            lk.lock();
            if (r < 0) {
                used_ -= s.bytes;
                cancel(id, s, r);
                s.state = kClosed;
                cv_done_.notify_all();
                continue;
            }
            s.handle = h;
            s.state = kAdmitted;
            if (s.closing && s.queue.empty()) retire(id, lk);
        }
    }

    // Admitted stream with queued windows, no batch in flight, and the
    // earliest-arrived head window; -1 if none.
    int32_t pick() const
    {
        int32_t best = -1;
        int64_t t = 0;
        for (int32_t i = 0; i < (int32_t)streams_.size(); ++i) {
            const Stream &s = *streams_[i];
            if (s.state != kAdmitted || s.busy || s.queue.empty()) continue;
            if (best < 0 || s.queue.front().arrival < t) {
                best = i;
                t = s.queue.front().arrival;
            }
        }
        return best;
    }

    void finish(int w, int q, std::unique_lock<std::mutex> &lk)
    {
        Worker &wk = workers_[w];
        const int64_t t = now_ns();
        const int n = (int)wk.batch.size();
        for (int k = 0; k < n; ++k) {
            ebof_completion c{};
            c.stream_id = wk.sid;
            if (q < 0) c.status = q;
            else if (wk.status < 0) c.status = wk.status;
            else c.status = (k == 0 && wk.status == EBOF_NO_PREVIOUS) ? EBOF_NO_PREVIOUS : EBOF_OK;
            c.tag = wk.batch[k].tag;
            c.arrival_ns = wk.batch[k].arrival;
            c.launch_ns = wk.launch_ns;
            c.done_ns = t;
            c.batch = n;
            c.index = k;
            done_.push_back(c);
        }
        completed_ += n;
        outstanding_ -= n;
        --in_flight_;
        const int32_t sid = wk.sid;
        Stream &s = *streams_[sid];
        s.busy = false;
        wk.sid = -1;
        wk.batch.clear();
        cv_done_.notify_all();
        if (s.closing && s.queue.empty()) retire(sid, lk);
    }

    void loop()
    {
        be_->bind_thread();
        std::vector<ebof_window_desc> wins;
        std::vector<float *> flows;
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            bool progress = false;
            for (int w = 0; w < (int)workers_.size(); ++w) {
                Worker &wk = workers_[w];
                if (wk.sid < 0) continue;
                const int q = be_->query(w);
                if (q == 1) continue;
                finish(w, q, lk);
                progress = true;
            }
            // streams closed while idle, and admissions they make possible
            for (int32_t i = 0; i < (int32_t)streams_.size(); ++i) {
                Stream &s = *streams_[i];
                if (s.state == kAdmitted && s.closing && !s.busy && s.queue.empty()) {
                    retire(i, lk);
                    progress = true;
                }
            }
            if (!waiting_.empty()) admit_waiting(lk);
            for (int w = 0; w < (int)workers_.size() && !stopping_; ++w) {
                Worker &wk = workers_[w];
                if (wk.sid >= 0) continue;
                const int32_t sid = pick();
                if (sid < 0) break;
                Stream &s = *streams_[sid];
                const int n = std::min<int>((int)s.queue.size(), std::max(s.p.max_batch, 1));
                wk.batch.assign(s.queue.begin(), s.queue.begin() + n);
                s.queue.erase(s.queue.begin(), s.queue.begin() + n);
                s.busy = true;
                wk.sid = sid;
                ++in_flight_;
                ++batches_;
                max_batch_seen_ = std::max(max_batch_seen_, n);
                void *h = s.handle;
                wins.resize(n);
                flows.resize(n);
                for (int k = 0; k < n; ++k) {
                    wins[k] = wk.batch[k].win;
                    flows[k] = wk.batch[k].flow;
                }
                wk.launch_ns = now_ns();
                lk.unlock();
                const int r = be_->launch(w, h, n, wins.data(), flows.data());
                lk.lock();
                wk.status = r;
                progress = true;
            }
            if (stopping_ && in_flight_ == 0) break;
            if (!progress) {
                if (in_flight_ > 0) {
                    lk.unlock();
                    std::this_thread::yield();
                    lk.lock();
                } else {
                    cv_work_.wait(lk);
                }
            }
        }
    }

    std::unique_ptr<Backend> be_;
    const int64_t budget_;
    std::vector<Worker> workers_;
    std::vector<std::unique_ptr<Stream>> streams_;
    std::deque<int32_t> waiting_;
    std::deque<ebof_completion> done_;
    int64_t used_ = 0, outstanding_ = 0, submitted_ = 0, completed_ = 0, batches_ = 0;
    int32_t in_flight_ = 0, max_batch_seen_ = 0;
    bool stopping_ = false;
    std::mutex mu_;
    std::condition_variable cv_work_, cv_done_;
    std::thread thread_;  // last member: starts after the others exist
};

}  // namespace ebof_serve
