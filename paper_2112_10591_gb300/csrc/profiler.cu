// profiler.cu -- see profiler.cuh.
#include "profiler.cuh"

namespace ebof {

thread_local Profiler *tl_prof = nullptr;
thread_local int tl_level = -1;
std::atomic<unsigned long long> g_launches{0};

const char *stage_name(int s)
{
    static const char *names[kNumStages] = {
        "scatter", "denoise_fill", "edt_cols", "edt_rows_surface", "pyramid", "patch_search",
        "densify", "var_warp", "var_coeff", "var_sor", "var_add", "flow_out"};
    return (s >= 0 && s < kNumStages) ? names[s] : "?";
}

Profiler::~Profiler()
{
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

cudaEvent_t Profiler::get()
{
    if (used == pool.size()) {
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        pool.push_back(e);
    }
    return pool[used++];
}

void Profiler::flush()
{
    for (const Rec &r : recs) {
        float t = 0.0f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            ms[r.stage][r.level] += t;
            launches[r.stage][r.level] += r.launches;
        }
    }
    recs.clear();
    used = 0;
}

void Profiler::reset()
{
    flush();
    for (int i = 0; i < kNumStages; ++i)
        for (int l = 0; l < kProfLevels; ++l) { ms[i][l] = 0.0; launches[i][l] = 0; }
}

}  // namespace ebof
