// profiler.cuh -- per-stage CUDA-event timing and kernel launch counting.
// Timing is off unless a stream enables it; launch counting is always on.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <vector>

namespace ebof {

enum Stage {
    kStScatter = 0,
    kStDenoiseFill,
    kStEdtCols,
    kStEdtRows,
    kStPyramid,
    kStSearch,
    kStDensify,
    kStVarWarp,
    kStVarCoeff,
    kStVarSor,
    kStVarAdd,
    kStFlowOut,
    kNumStages
};

const char *stage_name(int s);

struct Profiler {
    bool on = false;
    struct Rec {
        int stage;
        int launches;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<Rec> recs;
    double ms[kNumStages] = {};
    long long launches[kNumStages] = {};
    ~Profiler();
    cudaEvent_t get();
    void flush();   // waits for recorded events, accumulates, recycles them
    void reset();
};

// The profiler of the stream whose call is running on this host thread.
extern thread_local Profiler *tl_prof;
extern std::atomic<unsigned long long> g_launches;

// Brackets one stage's launches on `st` (no-ops when timing is off).
struct StageScope {
    Profiler *p;
    int stage, n;
    cudaStream_t st;
    cudaEvent_t b = nullptr;
    StageScope(int stage_, int n_launches, cudaStream_t st_)
        : p(tl_prof), stage(stage_), n(n_launches), st(st_)
    {
        g_launches.fetch_add((unsigned long long)n_launches, std::memory_order_relaxed);
        if (p && p->on) {
            cudaEvent_t a = p->get();
            b = p->get();
            cudaEventRecord(a, st);
            p->recs.push_back({stage, n, a, b});
        }
    }
    ~StageScope()
    {
        if (b) cudaEventRecord(b, st);
    }
};

}  // namespace ebof
