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

constexpr int kProfLevels = 9;  // pyramid levels 0..7, and 8 = not level-specific

struct Profiler {
    bool on = false;
    struct Rec {
        int stage;
        int level;
        int launches;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<Rec> recs;
    double ms[kNumStages][kProfLevels] = {};
    long long launches[kNumStages][kProfLevels] = {};
    ~Profiler();
    cudaEvent_t get();
    void flush();   // waits for recorded events, accumulates, recycles them
    void reset();
};

// The profiler of the stream whose call is running on this host thread, and
// the pyramid level its launches belong to (-1: not level-specific).
extern thread_local Profiler *tl_prof;
extern thread_local int tl_level;
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
            const int lv = (tl_level >= 0 && tl_level < kProfLevels - 1) ? tl_level : kProfLevels - 1;
            p->recs.push_back({stage, lv, n, a, b});
        }
    }
    ~StageScope()
    {
        if (b) cudaEventRecord(b, st);
    }
};

}  // namespace ebof
