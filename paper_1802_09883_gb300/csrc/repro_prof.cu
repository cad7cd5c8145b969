// repro_prof.cu -- optional CUDA-event timing of the library's kernels and
// a count of its launches (profiling aids; no effect on results).
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "repro.h"
#include "repro_internal.h"

namespace rp {

namespace {
struct Pending {
    cudaEvent_t a, b;
};
std::mutex g_mu;
std::atomic<int> g_on{0};
std::atomic<long long> g_launches{0};
std::vector<Pending> g_pending[PROF_COUNT];
Pending g_open[PROF_COUNT];
bool g_is_open[PROF_COUNT] = {};
const char* kNames[PROF_COUNT] = {"window", "accum", "fused", "partition", "merge", "finalize", "fp64", "fp32"};
}  // namespace

void prof_begin(ProfKernel k, cudaStream_t s) {
    if (!g_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lock(g_mu);
    Pending p;
    if (cudaEventCreate(&p.a) != cudaSuccess) return;
    if (cudaEventCreate(&p.b) != cudaSuccess) {
        cudaEventDestroy(p.a);
        return;
    }
    cudaEventRecord(p.a, s);
    g_open[k] = p;
    g_is_open[k] = true;
}

void prof_end(ProfKernel k, cudaStream_t s) {
    if (!g_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_is_open[k]) return;
    cudaEventRecord(g_open[k].b, s);
    g_pending[k].push_back(g_open[k]);
    g_is_open[k] = false;
}

void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

}  // namespace rp

extern "C" {

void repro_profile_enable(int on) { rp::g_on.store(on ? 1 : 0); }

repro_status repro_profile_read(const char* kernel, double* total_ms, int64_t* launches) {
    using namespace rp;
    if (!kernel) return REPRO_EINVAL;
    int k = -1;
    for (int i = 0; i < PROF_COUNT; ++i)
        if (std::strcmp(kernel, kNames[i]) == 0) k = i;
    if (k < 0) return REPRO_EINVAL;
    std::vector<Pending> mine;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        mine.swap(g_pending[k]);
    }
    double sum = 0;
    repro_status st = REPRO_OK;
    for (auto& p : mine) {
        float ms = 0;
        if (cudaEventSynchronize(p.b) != cudaSuccess || cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess)
            st = REPRO_ECUDA;
        sum += ms;
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    if (total_ms) *total_ms = sum;
    if (launches) *launches = (int64_t)mine.size();
    return st;
}

int64_t repro_launch_count(void) { return (int64_t)rp::g_launches.load(); }

}  // extern "C"
