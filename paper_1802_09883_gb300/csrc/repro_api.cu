// repro_api.cu -- the C ABI of librepro.so (declared in include/repro.h).
//
// Each entry point validates its arguments on the host, takes stream-ordered
// scratch from the device's default memory pool when it needs any, and
// enqueues the kernels of repro_kernels.cu on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <map>
#include <mutex>
#include <vector>
#include <tuple>

#include "repro.h"
#include "repro_internal.h"

namespace rp {

const DeviceInfo& device_info() {
    static DeviceInfo cache[64];
    static bool have[64] = {};
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (!have[dev]) {
        DeviceInfo d{dev, 1, 48 * 1024, 48 * 1024};
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess && v > 0)
            d.smem_per_sm = (size_t)v;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) d.sms = v;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess && v > 0)
            d.smem_optin = (size_t)v;
        cache[dev] = d;
        have[dev] = true;
    }
    return cache[dev];
}

int resident_ctas(const void* kern, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void*, int, size_t>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, kern, threads, smem);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int nb = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        nb = 0;
    }
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = nb;
    return nb;
}

static bool valid_dtype(int t) { return t == REPRO_F64 || t == REPRO_F32; }
static bool valid_shape(int L, int64_t G) { return L >= 1 && L <= 4 && G >= 1 && G <= INT32_MAX; }

static repro_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return REPRO_OK;
    if (e == cudaErrorMemoryAllocation) return REPRO_ENOMEM;
    return REPRO_ECUDA;
}

// The library's own memory pool on the current device: scratch returns to
// it on free and stays cached (release threshold = unlimited), so repeated
// calls do not map and unmap multi-gigabyte scratch from the driver.
// repro_release_cached_memory() hands the cached bytes back.
cudaMemPool_t library_pool(cudaError_t& err) {
    static cudaMemPool_t pools[64] = {};
    static std::mutex mu;
    int dev = 0;
    err = cudaGetDevice(&dev);
    if (err != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        err = cudaMemPoolCreate(&p, &props);
        if (err != cudaSuccess) return nullptr;
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
        pools[dev] = p;
    }
    return pools[dev];
}

// Stream-ordered scratch from the library pool, freed on scope exit.
struct Scratch {
    void* p = nullptr;
    cudaStream_t s;
    cudaError_t err = cudaSuccess;
    Scratch(size_t bytes, cudaStream_t st) : s(st) {
        if (!bytes) return;
        cudaMemPool_t pool = library_pool(err);
        if (pool) err = cudaMallocFromPoolAsync(&p, bytes, pool, s);
    }
    ~Scratch() {
        if (p) cudaFreeAsync(p, s);
    }
};

// Composite group id from two uint8 key columns: gid = k1 * card2 + k2, or -1
// (an invalid key) when it falls outside [0, G).  Four rows per thread.
__global__ void k_composite_keys(const uint8_t* __restrict__ k1, const uint8_t* __restrict__ k2, int card2,
                                 long long n, long long G, int32_t* __restrict__ gid) {
    const long long stride = 4ll * gridDim.x * blockDim.x;
    for (long long i = 4ll * (blockIdx.x * (long long)blockDim.x + threadIdx.x); i < n; i += stride) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (i + j < n) {
                const long long g = (long long)k1[i + j] * card2 + k2[i + j];
                gid[i + j] = g < G ? (int32_t)g : -1;
            }
    }
}


}  // namespace rp

using namespace rp;

namespace rp {

// The adaptive entry point's skew test: the fullest partition above this
// many times the mean row count of the partitions the keys reach.
constexpr double kAdaptiveSkewRatio = 4.0;

// Rows per staged chunk of repro_groupby_sum_host (two chunks in flight);
// REPRO_HOST_CHUNK_ROWS (2^20 to 2^27) overrides it.
constexpr long long kHostChunkRows = 1ll << 24;

static long long host_chunk_rows() {
    static const long long v = [] {
        const char* e = getenv("REPRO_HOST_CHUNK_ROWS");
        const long long x = e ? atoll(e) : 0;
        return x >= (1ll << 20) && x <= (1ll << 27) ? (x & ~255ll) : kHostChunkRows;
    }();
    return v;
}

// A library stream per device for host-to-device copies.
static cudaStream_t copy_stream(cudaError_t& err) {
    static cudaStream_t streams[64] = {};
    static std::mutex mu;
    int dev = 0;
    err = cudaGetDevice(&dev);
    if (err != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!streams[dev]) err = cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
    return err == cudaSuccess ? streams[dev] : nullptr;
}

int groupby_dispatch(const int32_t* keys, const void* values, long long n, int dtype, int L, long long num_groups,
                     void* state, cudaStream_t s) {
    // each path's configuration is chosen once and passed on, so the scratch
    // size and the launch agree even if the tuned cache changes meanwhile
    FusedPlanConfig cfg;
    if (n > 0 && fused_supported(dtype, L, num_groups, keys, values, true) &&
        fused_plan_config(dtype, L, (int)num_groups, 0, cfg, true)) {
        Scratch scratch(fused_scratch_bytes(cfg, L, num_groups, n), s);
        if (scratch.err != cudaSuccess) return from_cuda(scratch.err);
        return from_cuda(launch_groupby_fused(keys, values, n, dtype, L, num_groups, cfg, state, scratch.p, s));
    }
    PartChoice pc;
    if (n > 0 && partitioned_supported(dtype, L, num_groups, n, keys, values) &&
        partition_choose(dtype, L, num_groups, pc)) {
        Scratch scratch(partitioned_scratch_bytes(pc, dtype, L, num_groups, n), s);
        if (scratch.err != cudaSuccess) return from_cuda(scratch.err);
        return from_cuda(launch_groupby_partitioned(keys, values, n, dtype, L, num_groups, pc, state, scratch.p, s));
    }
    Scratch scratch(two_pass_scratch_bytes(num_groups), s);
    if (scratch.err != cudaSuccess) return from_cuda(scratch.err);
    return from_cuda(launch_groupby_two_pass(keys, values, n, dtype, L, num_groups, state, scratch.p, s));
}

}  // namespace rp

extern "C" {

size_t repro_state_bytes(repro_dtype dtype, int L, int64_t num_groups) {
    if (!valid_dtype(dtype) || !valid_shape(L, num_groups)) return 0;
    return sizeof(repro_state_header) + (size_t)num_groups * (8 + 16 * (size_t)L);
}

repro_status repro_state_init(void* state, repro_dtype dtype, int L, int64_t num_groups, void* stream) {
    if (!state || !valid_dtype(dtype) || !valid_shape(L, num_groups)) return REPRO_EINVAL;
    if ((uintptr_t)state % 16) return REPRO_EINVAL;
    return from_cuda(launch_init_state(state, dtype, L, num_groups, (cudaStream_t)stream));
}

repro_status repro_groupby_sum(const int32_t* keys, const void* values, int64_t n, repro_dtype dtype, int L,
                               int64_t num_groups, void* state, void* stream) {
    if (!state || !valid_dtype(dtype) || !valid_shape(L, num_groups) || n < 0) return REPRO_EINVAL;
    if (n > 0 && (!keys || !values)) return REPRO_EINVAL;
    if ((uintptr_t)state % 16 || (uintptr_t)keys % 4 || (uintptr_t)values % (dtype == REPRO_F64 ? 8 : 4))
        return REPRO_EINVAL;
    return (repro_status)groupby_dispatch(keys, values, n, dtype, L, num_groups, state, (cudaStream_t)stream);
}

repro_status repro_groupby_sum_adaptive(const int32_t* keys, const void* values, int64_t n, repro_dtype dtype, int L,
                                        int64_t num_groups, void* state, int* depth_out, void* stream) {
    if (depth_out) *depth_out = -1;
    if (!state || !valid_dtype(dtype) || !valid_shape(L, num_groups) || n < 0) return REPRO_EINVAL;
    if (n > 0 && (!keys || !values)) return REPRO_EINVAL;
    if ((uintptr_t)state % 16 || (uintptr_t)keys % 4 || (uintptr_t)values % (dtype == REPRO_F64 ? 8 : 4))
        return REPRO_EINVAL;
    if (n == 0) return REPRO_OK;
    cudaStream_t s = (cudaStream_t)stream;
    FusedPlanConfig cfg;
    if (fused_supported(dtype, L, num_groups, keys, values, true) &&
        fused_plan_config(dtype, L, (int)num_groups, 0, cfg, true)) {  // one table holds every group anyway
        if (depth_out) *depth_out = 0;
        return (repro_status)groupby_dispatch(keys, values, n, dtype, L, num_groups, state, s);
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    PartChoice pc;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone ||
        !partitioned_supported(dtype, L, num_groups, n, keys, values) ||
        !partition_choose(dtype, L, num_groups, pc))
        return (repro_status)groupby_dispatch(keys, values, n, dtype, L, num_groups, state, s);
    // the partitioned path planned for num_groups reads the key range and the
    // partitions' row counts in its first pass; it goes on when the groups
    // the keys reach, max + 1, and their skew call for the same plan, else it
    // stops there and the call is planned again
    Scratch rng(2 * sizeof(int), s);
    if (rng.err != cudaSuccess) return from_cuda(rng.err);
    const int init[2] = {INT32_MAX, INT32_MIN};
    cudaError_t e = cudaMemcpyAsync(rng.p, init, sizeof(init), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return from_cuda(e);
    long long Gk = num_groups;
    bool single = false;
    PartChoice pk;
    PartProbe probe;
    probe.dev = (int*)rng.p;
    probe.keep = [&](int kmin, int kmax, const std::vector<long long>& tot) {
        if (kmin < 0 || (long long)kmax >= num_groups) return true;  // bad keys: this path flags them
        Gk = (long long)kmax + 1;
        FusedPlanConfig c;
        if (fused_supported(dtype, L, Gk, keys, values, true) && fused_plan_config(dtype, L, (int)Gk, 0, c, true)) {
            single = true;
            return false;
        }
        if (!partition_choose(dtype, L, Gk, pk)) return true;
        // skewed keys (the fullest partition the keys reach above
        // kAdaptiveSkewRatio x their mean), unless the choice was measured:
        // one pass into partitions small enough for lane-private table
        // copies (a hot key's rows then never meet on one word within a
        // warp), where at most 2048 partitions cover the groups; else one
        // wide pass instead of two.  Both are what the tuner measured best
        // on Zipf keys (2^16 groups: 2^7 or 2^6 groups per partition; 2^20:
        // one pass into 1024 partitions)
        const long long Fk = std::min<long long>((long long)tot.size(), ((Gk - 1) >> pc.shift) + 1);
        long long hot = 0;
        for (long long p = 0; p < Fk; ++p) hot = std::max(hot, tot[(size_t)p]);
        const bool skewed = (double)hot * (double)Fk > kAdaptiveSkewRatio * (double)n;
        if (skewed && !pk.measured) {
            PartChoice t;
            bool found = false;
            for (int sh = pk.shift; sh >= 6 && !found; --sh)
                if (partition_with(dtype, L, Gk, sh, 1, t) && t.cfg.copies == 32) {
                    pk = t;
                    found = true;
                }
            // else one pass where at most 1024 partitions cover the groups
            // (a single pass into 2048 scatters slower than into 1024), at
            // the rule's width or twice it
            if (!found && (pk.shift1 > pk.shift || ((Gk - 1) >> pk.shift) + 1 > 1024))
                for (int sh = pk.shift; sh <= pk.shift + 1 && !found; ++sh)
                    if (((Gk - 1) >> sh) + 1 <= 1024 && partition_with(dtype, L, Gk, sh, 1, t)) {
                        pk = t;
                        found = true;
                    }
        }
        return pk.shift == pc.shift && (pk.shift1 > pk.shift) == (pc.shift1 > pc.shift) &&
               pk.cfg.copies == pc.cfg.copies;
    };
    {
        Scratch scratch(partitioned_scratch_bytes(pc, dtype, L, num_groups, n), s);
        if (scratch.err != cudaSuccess) return from_cuda(scratch.err);
        e = launch_groupby_partitioned(keys, values, n, dtype, L, num_groups, pc, state, scratch.p, s, 0, &probe);
        if (e != cudaSuccess) return from_cuda(e);
        if (!probe.abandoned) {
            if (depth_out) *depth_out = pc.shift1 > pc.shift ? 2 : 1;
            return REPRO_OK;
        }
    }
    // another plan for the Gk <= num_groups groups the keys reach: none, one
    // or two passes (records [0, Gk) of the state; the header keeps num_groups)
    if (single) {
        if (!fused_plan_config(dtype, L, (int)Gk, 0, cfg, true))  // not expected: the probe just saw it fit
            return (repro_status)groupby_dispatch(keys, values, n, dtype, L, num_groups, state, s);
        Scratch scratch(fused_scratch_bytes(cfg, L, Gk, n), s);
        if (scratch.err != cudaSuccess) return from_cuda(scratch.err);
        if (depth_out) *depth_out = 0;
        return from_cuda(launch_groupby_fused(keys, values, n, dtype, L, Gk, cfg, state, scratch.p, s, 0, false,
                                              num_groups));
    }
    Scratch scratch(partitioned_scratch_bytes(pk, dtype, L, Gk, n), s);
    if (scratch.err != cudaSuccess) return from_cuda(scratch.err);
    if (depth_out) *depth_out = pk.shift1 > pk.shift ? 2 : 1;
    return from_cuda(launch_groupby_partitioned(keys, values, n, dtype, L, Gk, pk, state, scratch.p, s, num_groups));
}

repro_status repro_groupby_sum_cols(const uint8_t* key1, const uint8_t* key2, int card2, const void* const* cols,
                                    int ncols, int64_t n, repro_dtype dtype, int L, int64_t num_groups,
                                    void* const* states, void* stream) {
    if (!cols || !states || ncols < 1 || card2 < 1 || n < 0 || !valid_dtype(dtype) || !valid_shape(L, num_groups))
        return REPRO_EINVAL;
    if (n > 0 && (!key1 || !key2)) return REPRO_EINVAL;
    for (int c = 0; c < ncols; ++c) {
        if (!states[c] || (uintptr_t)states[c] % 16) return REPRO_EINVAL;
        if (n > 0 && (!cols[c] || (uintptr_t)cols[c] % (dtype == REPRO_F64 ? 8 : 4))) return REPRO_EINVAL;
    }
    if (n == 0) return REPRO_OK;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch gid(sizeof(int32_t) * (size_t)n, s);
    if (gid.err != cudaSuccess) return from_cuda(gid.err);
    const int th = 256;
    long long blocks = (n + 4ll * th - 1) / (4ll * th);
    if (blocks > (long long)device_info().sms * 8) blocks = (long long)device_info().sms * 8;
    k_composite_keys<<<(int)blocks, th, 0, s>>>(key1, key2, card2, n, num_groups, (int32_t*)gid.p);
    count_launches(1);
    if (cudaGetLastError() != cudaSuccess) return REPRO_ECUDA;
    // one single pass per column over the shared group ids (measured: with
    // the single-pass kernel's contiguous loads and cheaper digits, four
    // float columns over 4 groups take 0.96 ms this way against 1.09 ms for
    // the four-column kernel of repro_cols.cu, which now only serves the
    // statistics' x and x*x)
    const int32_t* g = (const int32_t*)gid.p;
    for (int c = 0; c < ncols; ++c) {
        const repro_status st = (repro_status)groupby_dispatch(g, cols[c], n, dtype, L, num_groups, states[c], s);
        if (st != REPRO_OK) return st;
    }
    return REPRO_OK;
}

repro_status repro_sum(const void* values, int64_t n, repro_dtype dtype, int L, void* state, void* stream) {
    if (!state || (uintptr_t)state % 16 || n < 0 || !valid_dtype(dtype) || !valid_shape(L, 1)) return REPRO_EINVAL;
    if (n > 0 && (!values || (uintptr_t)values % (dtype == REPRO_F64 ? 8 : 4))) return REPRO_EINVAL;
    if (n == 0) return REPRO_OK;
    cudaStream_t s = (cudaStream_t)stream;
    FusedPlanConfig cfg;
    if (fused_supported(dtype, L, 1, nullptr, values, true) && fused_plan_config(dtype, L, 1, 0, cfg, true)) {
        Scratch scratch(fused_scratch_bytes(cfg, L, 1, n), s);
        if (scratch.err != cudaSuccess) return from_cuda(scratch.err);
        return from_cuda(launch_groupby_fused(nullptr, values, n, dtype, L, 1, cfg, state, scratch.p, s));
    }
    // values not 16-byte aligned: the grouped path with an all-zero key column
    Scratch keys(4 * (size_t)n, s);
    if (keys.err != cudaSuccess) return from_cuda(keys.err);
    cudaError_t e = cudaMemsetAsync(keys.p, 0, 4 * (size_t)n, s);
    if (e != cudaSuccess) return from_cuda(e);
    return (repro_status)groupby_dispatch((const int32_t*)keys.p, values, n, dtype, L, 1, state, s);
}

repro_status repro_groupby_sum_host(const int32_t* keys, const void* values, int64_t n, repro_dtype dtype, int L,
                                    int64_t num_groups, void* state, void* stream) {
    if (!state || (uintptr_t)state % 16 || n < 0 || !valid_dtype(dtype) || !valid_shape(L, num_groups))
        return REPRO_EINVAL;
    if (n == 0) return REPRO_OK;
    if (!keys || !values) return REPRO_EINVAL;
    for (const void* p : {(const void*)keys, values}) {  // page-locked host memory only: copies stay asynchronous
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess || a.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            return REPRO_EINVAL;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vs = dtype == REPRO_F64 ? 8 : 4;
    const long long chunk = std::min<long long>(n, host_chunk_rows());
    cudaError_t e = cudaSuccess;
    cudaStream_t cs = copy_stream(e);
    if (!cs) return from_cuda(e);
    // two staging buffers (keys then values, 16-byte aligned) in stream order on s
    const size_t kbytes = ((size_t)chunk * 4 + 255) & ~(size_t)255;
    Scratch buf0(kbytes + (size_t)chunk * vs, s), buf1(kbytes + (size_t)chunk * vs, s);
    if (buf0.err != cudaSuccess) return from_cuda(buf0.err);
    if (buf1.err != cudaSuccess) return from_cuda(buf1.err);
    unsigned char* buf[2] = {(unsigned char*)buf0.p, (unsigned char*)buf1.p};
    cudaEvent_t ready[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&ready[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&freed[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(freed[i], s);  // the buffers exist from here on s
    }
    repro_status st = from_cuda(e);
    for (long long r0 = 0, i = 0; st == REPRO_OK && r0 < n; r0 += chunk, ++i) {
        const int b = (int)(i & 1);
        const long long rows = std::min<long long>(chunk, n - r0);
        e = cudaStreamWaitEvent(cs, freed[b], 0);  // the chunk two back has been aggregated
        if (e == cudaSuccess) e = cudaMemcpyAsync(buf[b], keys + r0, (size_t)rows * 4, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(buf[b] + kbytes, (const unsigned char*)values + (size_t)r0 * vs, (size_t)rows * vs,
                                cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ready[b], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ready[b], 0);
        st = from_cuda(e);
        if (st == REPRO_OK)
            st = (repro_status)groupby_dispatch((const int32_t*)buf[b], buf[b] + kbytes, rows, dtype, L, num_groups,
                                                state, s);
        if (st == REPRO_OK) st = from_cuda(cudaEventRecord(freed[b], s));
    }
    for (int i = 0; i < 2; ++i) {
        if (ready[i]) cudaEventDestroy(ready[i]);
        if (freed[i]) cudaEventDestroy(freed[i]);
    }
    return st;  // the staging buffers return to the pool in stream order on s
}

repro_status repro_merge(void* dst, const void* src, repro_dtype dtype, int L, int64_t num_groups, void* stream) {
    if (!dst || !src || !valid_dtype(dtype) || !valid_shape(L, num_groups)) return REPRO_EINVAL;
    if (dst == src || (uintptr_t)dst % 16 || (uintptr_t)src % 16) return REPRO_EINVAL;
    const size_t bytes = repro_state_bytes(dtype, L, num_groups);
    const char* a = (const char*)dst;
    const char* b = (const char*)src;
    if (a < b + bytes && b < a + bytes) return REPRO_EINVAL;
    return from_cuda(launch_merge(dst, src, dtype, L, num_groups, (cudaStream_t)stream));
}

repro_status repro_merge_records(void* dst, const void* src, int L, int64_t num_records, void* stream) {
    if (!dst || !src || L < 1 || L > 4 || num_records < 0) return REPRO_EINVAL;
    if (dst == src || (uintptr_t)dst % 8 || (uintptr_t)src % 8) return REPRO_EINVAL;
    const size_t bytes = (size_t)num_records * (8 + 16 * (size_t)L);
    const char* a = (const char*)dst;
    const char* b = (const char*)src;
    if (num_records > 0 && a < b + bytes && b < a + bytes) return REPRO_EINVAL;
    if (num_records == 0) return REPRO_OK;
    return from_cuda(launch_merge_records(dst, src, L, num_records, (cudaStream_t)stream));
}

repro_status repro_finalize(const void* state, repro_dtype dtype, int L, int64_t num_groups, void* out,
                            void* stream) {
    if (!state || !out || !valid_dtype(dtype) || !valid_shape(L, num_groups)) return REPRO_EINVAL;
    if ((uintptr_t)state % 16 || (uintptr_t)out % (dtype == REPRO_F64 ? 8 : 4)) return REPRO_EINVAL;
    return from_cuda(launch_finalize(state, dtype, L, num_groups, out, (cudaStream_t)stream));
}

repro_status repro_state_check(const void* state, uint32_t* errors_out, void* stream) {
    if (!state) return REPRO_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, &((const repro_state_header*)state)->errors, sizeof(err),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    if (errors_out) *errors_out = err;
    if (err & REPRO_ERR_KEY) return REPRO_EKEY;
    if (err & REPRO_ERR_TIMEOUT) return REPRO_ETIMEOUT;
    if (err & REPRO_ERR_LAYOUT) return REPRO_ELAYOUT;
    return REPRO_OK;
}

repro_status groupby_sum_fp64(const int32_t* keys, const double* values, int64_t n, int64_t num_groups,
                              double* out, void* stream) {
    if (!out || n < 0 || num_groups < 1 || num_groups > INT32_MAX) return REPRO_EINVAL;
    if (n > 0 && (!keys || !values)) return REPRO_EINVAL;
    return from_cuda(launch_groupby_fp64(keys, values, n, num_groups, out, (cudaStream_t)stream));
}

repro_status groupby_sum_fp32(const int32_t* keys, const float* values, int64_t n, int64_t num_groups,
                              float* out, void* stream) {
    if (!out || n < 0 || num_groups < 1 || num_groups > INT32_MAX) return REPRO_EINVAL;
    if (n > 0 && (!keys || !values)) return REPRO_EINVAL;
    return from_cuda(launch_groupby_fp32(keys, values, n, num_groups, out, (cudaStream_t)stream));
}

repro_status groupby_sum_fp_mode(const int32_t* keys, const void* values, int64_t n, repro_dtype dtype,
                                 int64_t num_groups, int mode, void* out, void* stream) {
    if (!out || n < 0 || num_groups < 1 || num_groups > INT32_MAX || !valid_dtype(dtype)) return REPRO_EINVAL;
    if (n > 0 && (!keys || !values)) return REPRO_EINVAL;
    if (mode < 0 || mode > 4) return REPRO_EINVAL;
    if (!fp_mode_supported(dtype, mode, num_groups)) return REPRO_ERANGE;
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == REPRO_F64)
        return from_cuda(launch_groupby_fp64(keys, (const double*)values, n, num_groups, (double*)out, s, mode));
    return from_cuda(launch_groupby_fp32(keys, (const float*)values, n, num_groups, (float*)out, s, mode));
}

const char* repro_strerror(repro_status status) {
    switch (status) {
        case REPRO_OK: return "ok";
        case REPRO_EINVAL: return "invalid argument";
        case REPRO_EKEY: return "a key outside [0, num_groups) was seen";
        case REPRO_ERANGE: return "size beyond the supported maximum";
        case REPRO_ENOMEM: return "scratch memory could not be allocated";
        case REPRO_ECUDA: return "CUDA error";
        case REPRO_ETIMEOUT: return "a bounded device wait gave up";
        case REPRO_ELAYOUT: return "state header does not match dtype / L / num_groups";
    }
    return "unknown status";
}

int repro_version(void) { return 100; }

repro_status repro_release_cached_memory(void) {
    cudaError_t e;
    cudaMemPool_t pool = library_pool(e);
    if (!pool) return from_cuda(e);
    e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
    return from_cuda(e);
}

}  // extern "C"
