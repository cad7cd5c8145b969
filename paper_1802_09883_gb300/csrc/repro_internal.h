// repro_internal.h -- host-side interface between the C ABI (repro_api.cu)
// and the kernel launchers (repro_kernels.cu).  Not installed.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <functional>
#include <vector>

namespace rp {

struct DeviceInfo {
    int device;
    int sms;            // multiprocessors
    size_t smem_optin;  // opt-in shared memory per block, bytes
    size_t smem_per_sm; // shared memory per multiprocessor, bytes
};

// Properties of the current device (queried once per device).
const DeviceInfo& device_info();

// The library's stream-ordered memory pool on the current device (cached:
// freed blocks stay with the pool until repro_release_cached_memory).
cudaMemPool_t library_pool(cudaError_t& err);

// One accumulation into a state: the single-pass path when its table fits,
// else the partitioned path, else the two-pass path (returns a repro_status).
int groupby_dispatch(const int32_t* keys, const void* values, long long n, int dtype, int L, long long num_groups,
                     void* state, cudaStream_t s);

// CTAs of `kern` (threads per CTA, dynamic shared memory) that fit on one SM
// at once (opts the kernel into that much shared memory first); 0 if none.
int resident_ctas(const void* kern, int threads, size_t smem);

// Profiling hooks (repro_profile_enable / repro_profile_read) and the launch
// counter (repro_launch_count).
enum ProfKernel { PROF_WINDOW, PROF_ACCUM, PROF_FUSED, PROF_PARTITION, PROF_MERGE, PROF_FINALIZE, PROF_FP64,
                  PROF_FP32, PROF_COUNT };
void prof_begin(ProfKernel k, cudaStream_t s);
void prof_end(ProfKernel k, cudaStream_t s);
void count_launches(int k);

cudaError_t launch_init_state(void* state, int dtype, int L, long long G, cudaStream_t s);

size_t two_pass_scratch_bytes(long long G);
cudaError_t launch_groupby_two_pass(const int32_t* keys, const void* vals, long long n, int dtype, int L,
                                    long long G, void* state, void* scratch, cudaStream_t s);

// Single-pass fused path (shared-memory group tables, TMA-staged tiles).
struct FusedPlanConfig {
    int S, R, ncw, ctas_per_sm, copies;  // stages, rows per tile, consumer warps, CTAs per SM, table copies
};
// The configuration for a group table of G groups (extra_smem bytes reserved
// on top of the kernel's layout): the tuner's forced choice on this thread,
// else REPRO_FUSED_CFG, else the tuned cache, else the built-in rule -- the
// first that fits; false if none fits.  Callers choose once per call and pass
// the configuration on, so scratch sizing and launch always agree.
// pad (single): configurations of the single-task kernel, which also has
// 24- and 31-warp variants; false: the multi-task kernel's.
bool fused_plan_config(int dtype, int L, int G, size_t extra_smem, FusedPlanConfig& cfg, bool pad = false);
bool fused_config_fits(int dtype, int L, int G, size_t extra_smem, const FusedPlanConfig& cfg, bool pad = false);
size_t fused_plan_smem(int dtype, int L, int G, const FusedPlanConfig& cfg);
bool fused_supported(int dtype, int L, long long G, const void* keys, const void* vals, bool pad = false);
size_t fused_scratch_bytes(const FusedPlanConfig& cfg, int L, long long G, long long n);
// max_ctas > 0 caps the number of CTAs (and so the partial tables in scratch);
// square: sum RN(x*x) instead of x; G_hdr > 0: the state holds G_hdr >= G
// groups and every key is below G (only its first G records are touched).
cudaError_t launch_groupby_fused(const int32_t* keys, const void* vals, long long n, int dtype, int L, long long G,
                                 const FusedPlanConfig& cfg, void* state, void* scratch, cudaStream_t s,
                                 int max_ctas = 0, bool square = false, long long G_hdr = 0);

// Large group counts: partition by key range, then the multi-task kernel
// over the partitions (repro_partition.cu).  A choice fixes the partition
// width 2^shift, the coarse width 2^shift1 of a first pass (0: one pass),
// the multi-task kernel's configuration and the work items per CTA it aims
// at (0: the built-in default).  More items balance the CTAs' ends better;
// fewer restart each CTA's table (and its windows) less often.
struct PartChoice {
    int shift = 0;
    int shift1 = 0;
    FusedPlanConfig cfg{};
    int ipc = 0;
    bool measured = false;  // from the tuner (forced or cached), not the rule
};
bool partition_choose(int dtype, int L, long long G, PartChoice& pc);
// A choice of width 2^shift with `levels` partition passes and the rule's
// aggregation configuration; false where that width or depth is not usable.
bool partition_with(int dtype, int L, long long G, int shift, int levels, PartChoice& pc);
bool partitioned_supported(int dtype, int L, long long G, long long n, const void* keys, const void* vals);
size_t partitioned_scratch_bytes(const PartChoice& pc, int dtype, int L, long long G, long long n);
// The key range and the final partitions' row counts read by the first
// partition pass's histogram, for a caller that may drop the call when
// another plan suits the keys better: dev points to {min, max} (preset to
// {INT32_MAX, INT32_MIN}); once the histogram and the partition totals are
// known the stream is synchronised and keep(min, max, totals) decides; when
// it returns false the call returns at once with abandoned set (nothing has
// been written to the state: only keys outside [0, G) would have flagged
// it, and keep must return true for those).
struct PartProbe {
    int* dev = nullptr;
    std::function<bool(int, int, const std::vector<long long>&)> keep;
    bool abandoned = false;
};

// G_hdr > 0: the state holds G_hdr >= G groups and every key is below G.
cudaError_t launch_groupby_partitioned(const int32_t* keys, const void* vals, long long n, int dtype, int L,
                                       long long G, const PartChoice& pc, void* state, void* scratch, cudaStream_t s,
                                       long long G_hdr = 0, PartProbe* probe = nullptr);


// A value column and its square over one key column in one pass
// (repro_cols.cu): NV = 2 and square only (vals[0], two states).  Supported
// only where the two tables leave three CTAs per SM.
bool cols_supported(int dtype, int L, long long G, int NV, const int32_t* keys, const void* const* vals);
size_t cols_scratch_bytes(int dtype, int L, long long G, int NV, long long n);
cudaError_t launch_groupby_cols(const int32_t* keys, const void* const* vals, int NV, bool square, long long n,
                                int dtype, int L, long long G, void* const* states, void* scratch, cudaStream_t s);

// Many inputs partitioned in one pass and aggregated by one multi-task
// launch (a batch's large-group tasks; repro_partition.cu).  plan() builds
// the chunk list and tables on the host (false if the inputs do not qualify:
// 16-byte aligned columns, at most 64 partitions per input), upload() copies
// them into scratch (synchronous), launch() only enqueues kernels.
struct BatchPartInput {
    const int32_t* keys;
    const void* vals;
    long long n;
    int G;
    unsigned char* state;
};
struct BatchPartition {
    struct Impl;
    Impl* impl;
    BatchPartition();
    ~BatchPartition();
    BatchPartition(const BatchPartition&) = delete;
    BatchPartition& operator=(const BatchPartition&) = delete;
    bool plan(int dtype, int L, const std::vector<BatchPartInput>& in);
    size_t scratch_bytes() const;
    // the host-built tables are the scratch's first table_bytes() bytes
    size_t table_bytes() const;
    void pack_tables(void* host) const;
    cudaError_t upload(void* scratch) const;
    // pack into page-locked `pinned` (table_bytes() long, alive until the copy ran) and copy on s
    cudaError_t upload_async(void* scratch, void* pinned, cudaStream_t s) const;
    cudaError_t launch(void* scratch, cudaStream_t s) const;
};

// Measured choices (repro_tune.cu).  The cache holds, per (dtype, L, group
// count rounded up to a power of two), a single-pass configuration and a
// partition width with its number of partition passes (levels: 1 or 2, 0 =
// the rule's); the tuner forces candidates on its own thread while it times
// them.
bool tune_lookup_fused(int dtype, int L, long long G, FusedPlanConfig& cfg);
// cfg.S == 0: no measured aggregation configuration for that width; ipc 0:
// no measured items per CTA
bool tune_lookup_shift(int dtype, int L, long long G, int& shift, int& levels, FusedPlanConfig& cfg, int& ipc);
const FusedPlanConfig* tune_forced_fused();
int tune_forced_shift();   // 0: none
int tune_forced_levels();  // 0: the rule's

// Multi-task single-pass kernel and its partial merge (repro_batch.cu); the
// task / item / merge-block arrays are laid out as in multi_types.h.
cudaError_t launch_multi(int dtype, int L, const FusedPlanConfig& cfg, int gcap, const void* tasks, const void* items,
                         int nitems, const int* nitems_ptr, int* counter, void* partials, int ctas, cudaStream_t s);
cudaError_t launch_merge_items(int L, int dtype, const void* tasks, const void* blks, int nblks, const int* nblks_ptr,
                               const void* partials, cudaStream_t s);

cudaError_t launch_merge(void* dst, const void* src, int dtype, int L, long long G, cudaStream_t s);
// dst += src over G bare records (no headers).
cudaError_t launch_merge_records(void* dst, const void* src, int L, long long G, cudaStream_t s);
// state += C partial record arrays of G records each (parts[c * G + g]).
cudaError_t launch_merge_partials(const void* parts, int C, long long G, void* state, int dtype, int L,
                                  cudaStream_t s);
cudaError_t launch_finalize(const void* state, int dtype, int L, long long G, void* out, cudaStream_t s);

// The conventional floating-point GroupBy; mode < 0: the built-in choice
// (or REPRO_FP_MODE), else one of the table strategies 0..4 of
// repro_kernels.cu (fp_mode_supported tells which fit).
cudaError_t launch_groupby_fp64(const int32_t* keys, const double* vals, long long n, long long G, double* out,
                                cudaStream_t s, int mode = -1);
cudaError_t launch_groupby_fp32(const int32_t* keys, const float* vals, long long n, long long G, float* out,
                                cudaStream_t s, int mode = -1);
bool fp_mode_supported(int dtype, int mode, long long G);

}  // namespace rp
