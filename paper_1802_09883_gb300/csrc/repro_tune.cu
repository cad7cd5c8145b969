// repro_tune.cu -- measured configuration choices (repro_tune_* in
// include/repro.h).
//
// The paper tunes its partitioning fan-out and buffer sizes offline for its
// CPUs and notes that the best values depend on the group count (Sec. V-C,
// VI).  Here the choices are the single-pass kernel's configuration (stages,
// rows per tile, consumer warps, CTAs per SM, table copies) and the
// partition width of the partitioned path.  repro_tune_groupby times every
// candidate that fits on the caller's own data and records the fastest per
// (dtype, L, group count rounded up to a power of two); later calls with a
// group count in the same bucket use it.  Choices never change a result:
// every candidate computes the same exact bins.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "repro.h"
#include "multi_types.h"
#include "repro_internal.h"

namespace rp {
namespace {

using Key = std::tuple<int, int, int>;  // dtype, L, ceil(log2 G)

std::mutex g_mu;
std::map<Key, FusedPlanConfig> g_fused;
// A partitioned choice: width, passes (0 = the rule's) and, when measured,
// the aggregation kernel's configuration (S == 0: the rule's).
struct PartTuned {
    int shift, levels;
    FusedPlanConfig cfg;
    int ipc;  // work items per CTA, 0: the built-in default
};
std::map<Key, PartTuned> g_shift;

thread_local const FusedPlanConfig* t_force_fused = nullptr;
thread_local int t_force_shift = 0;
thread_local int t_force_levels = 0;
thread_local bool t_ignore_cache = false;

int gbucket(long long G) {
    int b = 0;
    while (b < 40 && (1ll << b) < G) ++b;
    return b;
}

Key key_of(int dtype, int L, long long G) { return Key{dtype, L, gbucket(G)}; }

// Median of `reps` timed calls of run() on s (after one untimed call).
double time_median(const std::function<cudaError_t()>& run, cudaStream_t s, int reps, cudaError_t& err) {
    cudaEvent_t a = nullptr, b = nullptr;
    err = cudaEventCreate(&a);
    if (err == cudaSuccess) err = cudaEventCreate(&b);
    std::vector<float> t;
    if (err == cudaSuccess) err = run();
    for (int i = 0; i < reps && err == cudaSuccess; ++i) {
        err = cudaEventRecord(a, s);
        if (err == cudaSuccess) err = run();
        if (err == cudaSuccess) err = cudaEventRecord(b, s);
        if (err == cudaSuccess) err = cudaEventSynchronize(b);
        float ms = 0;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, a, b);
        t.push_back(ms);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (err != cudaSuccess || t.empty()) return 0.0;
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

// RAII: force a choice on this thread while a candidate is timed.
struct Force {
    Force(const FusedPlanConfig* f, int shift, bool ignore_cache, int levels = 0) {
        t_force_fused = f;
        t_force_shift = shift;
        t_force_levels = levels;
        t_ignore_cache = ignore_cache;
    }
    ~Force() {
        t_force_fused = nullptr;
        t_force_shift = 0;
        t_force_levels = 0;
        t_ignore_cache = false;
    }
};

repro_status status_of(cudaError_t e) {
    return e == cudaSuccess ? REPRO_OK : e == cudaErrorMemoryAllocation ? REPRO_ENOMEM : REPRO_ECUDA;
}

}  // namespace

bool tune_lookup_fused(int dtype, int L, long long G, FusedPlanConfig& cfg) {
    if (t_ignore_cache) return false;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_fused.find(key_of(dtype, L, G));
    if (it == g_fused.end()) return false;
    cfg = it->second;
    return true;
}

bool tune_lookup_shift(int dtype, int L, long long G, int& shift, int& levels, FusedPlanConfig& cfg, int& ipc) {
    if (t_ignore_cache) return false;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_shift.find(key_of(dtype, L, G));
    if (it == g_shift.end()) return false;
    shift = it->second.shift;
    levels = it->second.levels;
    cfg = it->second.cfg;
    ipc = it->second.ipc;
    return true;
}

const FusedPlanConfig* tune_forced_fused() { return t_force_fused; }
int tune_forced_shift() { return t_force_shift; }
int tune_forced_levels() { return t_force_levels; }

}  // namespace rp

using namespace rp;

extern "C" {

repro_status repro_tune_groupby(const int32_t* keys, const void* values, int64_t n, repro_dtype dtype, int L,
                                int64_t num_groups, void* stream, repro_tune_result* out) {
    if (!out || n <= 0 || !keys || !values || (dtype != REPRO_F64 && dtype != REPRO_F32) || L < 1 || L > 4 ||
        num_groups < 1 || num_groups > INT32_MAX)
        return REPRO_EINVAL;
    std::memset(out, 0, sizeof(*out));
    cudaStream_t s = (cudaStream_t)stream;
    const long long G = num_groups;
    const size_t sbytes = repro_state_bytes(dtype, L, G);
    cudaError_t err = cudaSuccess;
    void* state = nullptr;
    void* scratch = nullptr;
    auto cleanup = [&]() {
        if (state) cudaFree(state);
        if (scratch) cudaFree(scratch);
    };
    if (fused_supported(dtype, L, G, keys, values, true)) {
        out->path = 0;
        std::vector<FusedPlanConfig> cands;
        // S = 1: a single stage per CTA (its tile loads while the SM's other
        // CTAs compute), which leaves room for larger tiles at 3 CTAs per SM
        for (int S : {1, 2, 3, 4})
            for (int R : {1024, 2048, 3072, 3968, 4096, 6144, 7936})
                for (int ncw : {8, 16, 24, 31})
                    for (int cps : {1, 2, 3, 4})
                        for (int copies : {1, 32}) {
                            const FusedPlanConfig c{S, R, ncw, cps, copies};
                            if (S == 1 && R == 1024) continue;
                            if (fused_config_fits(dtype, L, (int)G, 0, c, true)) cands.push_back(c);
                        }
        FusedPlanConfig def{};
        {
            Force f(nullptr, 0, true);
            if (!fused_plan_config(dtype, L, (int)G, 0, def, true)) return REPRO_ERANGE;
        }
        size_t need = 16;
        for (const FusedPlanConfig& c : cands) need = std::max(need, fused_scratch_bytes(c, L, G, n));
        err = cudaMalloc(&state, sbytes);
        if (err == cudaSuccess) err = cudaMalloc(&scratch, need);
        if (err != cudaSuccess) {
            cleanup();
            return status_of(err);
        }
        double best = 0;
        FusedPlanConfig pick = def;
        for (const FusedPlanConfig& c : cands) {
            auto run = [&]() -> cudaError_t {
                cudaError_t e = launch_init_state(state, dtype, L, G, s);
                return e == cudaSuccess ? launch_groupby_fused(keys, values, n, dtype, L, G, c, state, scratch, s)
                                        : e;
            };
            const double ms = time_median(run, s, 3, err);
            if (err != cudaSuccess) break;
            ++out->candidates;
            if (c.S == def.S && c.R == def.R && c.ncw == def.ncw && c.ctas_per_sm == def.ctas_per_sm &&
                c.copies == def.copies)
                out->default_ms = ms;
            if (best == 0 || ms < best) {
                best = ms;
                pick = c;
            }
        }
        cleanup();
        if (err != cudaSuccess) return status_of(err);
        out->best_ms = best;
        out->stages = pick.S;
        out->tile_rows = pick.R;
        out->consumer_warps = pick.ncw;
        out->ctas_per_sm = pick.ctas_per_sm;
        out->table_copies = pick.copies;
        std::lock_guard<std::mutex> lk(g_mu);
        g_fused[key_of(dtype, L, G)] = pick;
        return REPRO_OK;
    }
    if (partitioned_supported(dtype, L, G, n, keys, values)) {
        out->path = 1;
        PartChoice def{};
        {
            Force f(nullptr, 0, true);
            if (!partition_choose(dtype, L, G, def)) return REPRO_ERANGE;
        }
        // every width, each with one and with two partition passes where
        // partition_choose allows that many
        std::vector<PartChoice> cands;
        auto levels_of = [](const PartChoice& pc) { return pc.shift1 > pc.shift ? 2 : 1; };
        for (int shift = 6; shift <= 12; ++shift)
            for (int levels = 1; levels <= 2; ++levels) {
                Force f(nullptr, shift, true, levels);
                PartChoice pc{};
                if (partition_choose(dtype, L, G, pc) && pc.shift == shift && levels_of(pc) == levels)
                    cands.push_back(pc);
            }
        size_t need = 16;
        for (const PartChoice& pc : cands) need = std::max(need, partitioned_scratch_bytes(pc, dtype, L, G, n));
        err = cudaMalloc(&state, sbytes);
        if (err == cudaSuccess) err = cudaMalloc(&scratch, need);
        if (err != cudaSuccess) {
            cleanup();
            return status_of(err);
        }
        double best = 0;
        PartChoice pick = def;
        auto time_choice = [&](const PartChoice& pc) -> double {
            auto run = [&]() -> cudaError_t {
                cudaError_t e = launch_init_state(state, dtype, L, G, s);
                return e == cudaSuccess
                           ? launch_groupby_partitioned(keys, values, n, dtype, L, G, pc, state, scratch, s)
                           : e;
            };
            const double ms = time_median(run, s, 3, err);
            if (err == cudaSuccess) {
                ++out->candidates;
                if (best == 0 || ms < best) {
                    best = ms;
                    pick = pc;
                }
            }
            return ms;
        };
        // the partitioning first (with the rule's aggregation configuration)
        for (const PartChoice& pc : cands) {
            const double ms = time_choice(pc);
            if (err != cudaSuccess) break;
            if (pc.shift == def.shift && pc.shift1 == def.shift1) out->default_ms = ms;
        }
        // then the aggregation kernel's configuration for the chosen width
        bool cfg_tuned = false;
        std::vector<PartChoice> cfgs;
        const PartChoice base = pick;
        for (int S : {1, 2, 3, 4})
            for (int R : {1024, 2048})
                for (int ncw : {8, 16})
                    for (int cps : {1, 2, 3, 4}) {
                        if (S == 1 && R == 1024) continue;
                        const FusedPlanConfig c{S, R, ncw, cps, 1};
                        if (c.S == base.cfg.S && c.R == base.cfg.R && c.ncw == base.cfg.ncw &&
                            c.ctas_per_sm == base.cfg.ctas_per_sm && c.copies == base.cfg.copies)
                            continue;
                        if (!fused_config_fits(dtype, L, 1 << base.shift, kMetaSmemBytes, c)) continue;
                        PartChoice pc = base;
                        pc.cfg = c;
                        cfgs.push_back(pc);
                    }
        size_t need2 = need;
        for (const PartChoice& pc : cfgs) need2 = std::max(need2, partitioned_scratch_bytes(pc, dtype, L, G, n));
        if (err == cudaSuccess && need2 > need) {
            cudaFree(scratch);
            scratch = nullptr;
            err = cudaMalloc(&scratch, need2);
        }
        for (const PartChoice& pc : cfgs) {
            if (err != cudaSuccess) break;
            const double before = best;
            time_choice(pc);
            if (best < before) cfg_tuned = true;
        }
        // then the work items per CTA for the chosen width and configuration
        bool ipc_tuned = false;
        {
            const PartChoice base2 = pick;
            for (int ipc : {1, 4, 8}) {
                if (err != cudaSuccess) break;
                PartChoice pc = base2;
                pc.ipc = ipc;
                const size_t nb = partitioned_scratch_bytes(pc, dtype, L, G, n);
                if (nb > need2) {
                    cudaFree(scratch);
                    scratch = nullptr;
                    if ((err = cudaMalloc(&scratch, nb)) != cudaSuccess) break;
                    need2 = nb;
                }
                const double before = best;
                time_choice(pc);
                if (best < before) ipc_tuned = true;
            }
        }
        cleanup();
        if (err != cudaSuccess) return status_of(err);
        out->best_ms = best;
        out->partition_shift = pick.shift;
        out->partition_levels = levels_of(pick);
        out->stages = pick.cfg.S;
        out->tile_rows = pick.cfg.R;
        out->consumer_warps = pick.cfg.ncw;
        out->ctas_per_sm = pick.cfg.ctas_per_sm;
        out->table_copies = pick.cfg.copies;
        out->partition_items_per_cta = pick.ipc;
        std::lock_guard<std::mutex> lk(g_mu);
        g_shift[key_of(dtype, L, G)] = PartTuned{pick.shift, levels_of(pick),
                                                 cfg_tuned || ipc_tuned ? pick.cfg : FusedPlanConfig{},
                                                 ipc_tuned ? pick.ipc : 0};
        return REPRO_OK;
    }
    out->path = 2;  // two-pass path: nothing to choose
    return REPRO_OK;
}

repro_status repro_tune_save(const char* path) {
    if (!path) return REPRO_EINVAL;
    FILE* f = fopen(path, "w");
    if (!f) return REPRO_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    fprintf(f, "# repro tune cache v1: kind dtype L log2G values (part: shift levels [S R ncw cps copies [ipc]])\n");
    for (const auto& kv : g_fused) {
        const FusedPlanConfig& c = kv.second;
        fprintf(f, "fused %d %d %d %d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first),
                std::get<2>(kv.first), c.S, c.R, c.ncw, c.ctas_per_sm, c.copies);
    }
    for (const auto& kv : g_shift) {
        const PartTuned& t = kv.second;
        fprintf(f, "part %d %d %d %d %d", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                t.shift, t.levels);
        if (t.cfg.S) fprintf(f, " %d %d %d %d %d", t.cfg.S, t.cfg.R, t.cfg.ncw, t.cfg.ctas_per_sm, t.cfg.copies);
        if (t.cfg.S && t.ipc) fprintf(f, " %d", t.ipc);
        fprintf(f, "\n");
    }
    return fclose(f) == 0 ? REPRO_OK : REPRO_EINVAL;
}

repro_status repro_tune_load(const char* path) {
    if (!path) return REPRO_EINVAL;
    FILE* f = fopen(path, "r");
    if (!f) return REPRO_EINVAL;
    std::map<Key, FusedPlanConfig> fused;
    std::map<Key, PartTuned> shift;
    char line[256];
    bool ok = true;
    while (ok && fgets(line, sizeof line, f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        char kind[16] = {};
        int d, L, gb, a[7];
        if (sscanf(line, "%15s", kind) != 1) continue;
        if (!strcmp(kind, "fused")) {
            ok = sscanf(line, "%*s %d %d %d %d %d %d %d %d", &d, &L, &gb, &a[0], &a[1], &a[2], &a[3], &a[4]) == 8;
            if (ok) fused[Key{d, L, gb}] = FusedPlanConfig{a[0], a[1], a[2], a[3], a[4]};
        } else if (!strcmp(kind, "part")) {
            // shift [levels (0 = the rule's) [S R ncw cps copies [items per CTA]]]
            int c[5] = {0, 0, 0, 0, 0};
            int ipc = 0;
            a[1] = 0;
            const int got = sscanf(line, "%*s %d %d %d %d %d %d %d %d %d %d %d", &d, &L, &gb, &a[0], &a[1], &c[0],
                                   &c[1], &c[2], &c[3], &c[4], &ipc);
            ok = (got == 4 || got == 5 || got == 10 || got == 11) && a[0] >= 6 && a[0] <= 12 && a[1] >= 0 &&
                 a[1] <= 2;
            if (ok && got >= 10) ok = c[0] >= 1 && c[1] >= 1 && c[2] >= 1 && c[3] >= 1 && c[4] >= 1;
            if (ok && got == 11) ok = ipc >= 1 && ipc <= 64;
            if (ok) shift[Key{d, L, gb}] = PartTuned{a[0], a[1], FusedPlanConfig{c[0], c[1], c[2], c[3], c[4]}, ipc};
        } else {
            ok = false;
        }
    }
    fclose(f);
    if (!ok) return REPRO_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto& kv : fused) g_fused[kv.first] = kv.second;
    for (const auto& kv : shift) g_shift[kv.first] = kv.second;
    return REPRO_OK;
}

void repro_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_fused.clear();
    g_shift.clear();
}

}  // extern "C"
