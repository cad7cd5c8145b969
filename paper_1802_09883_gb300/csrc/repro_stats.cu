// repro_stats.cu -- SQL aggregates built on the reproducible SUM
// (repro_stats_* in include/repro.h).
//
// The paper notes that once SUM is reproducible every SQL aggregate can be
// made reproducible: COUNT needs no floating point, AVG / VARIANCE / STDDEV
// are functions of SUM(x) and SUM(x^2) (Sec. I).  A stats state is
//   [repro state of x][repro state of x*x][uint64 count[G]]
// (each part 16-byte aligned).  When the group table fits the single-pass
// layout, the two SUMs run in one pass of the two-column kernel
// (repro_cols.cu; each x*x rounded to nearest in T, formed in shared
// memory) and k_count counts rows per group (exact integers, so atomics in
// any order agree).  Otherwise k_square_count writes x*x to scratch and
// counts, and the two SUMs go through the regular dispatcher.
// k_stats_finalize evaluates the aggregates per group in a fixed order of
// IEEE operations, so they are as reproducible as the sums they read.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "repro.h"
#include "repro_device.cuh"
#include "repro_internal.h"

namespace rp {
namespace {

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

struct StatsLayout {
    size_t sq, count, total;  // byte offsets of the x^2 state and the counts; total size
};

StatsLayout stats_layout(int dtype, int L, long long G) {
    const size_t one = align16(repro_state_bytes((repro_dtype)dtype, L, G));
    return StatsLayout{one, 2 * one, 2 * one + align16(8 * (size_t)G)};
}

// Shared-memory counters when the group count allows, else global atomics.
constexpr int kCountSmemGroups = 8192;

template <typename T>
__global__ void __launch_bounds__(256) k_square_count(const int32_t* __restrict__ keys, const T* __restrict__ vals,
                                                      long long n, int G, T* __restrict__ sq,
                                                      unsigned long long* __restrict__ count) {
    __shared__ unsigned s_cnt[kCountSmemGroups];
    const bool smem = G <= kCountSmemGroups;
    if (smem) {
        for (int g = threadIdx.x; g < G; g += blockDim.x) s_cnt[g] = 0;
        __syncthreads();
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const T x = vals[i];
        sq[i] = x * x;  // one rounding to nearest (no contraction: built with -fmad=false)
        const int g = keys[i];
        if ((unsigned)g < (unsigned)G) {
            if (smem)
                atomicAdd(&s_cnt[g], 1u);
            else
                atomicAdd(&count[g], 1ull);
        }
    }
    if (smem) {
        __syncthreads();
        for (int g = threadIdx.x; g < G; g += blockDim.x)
            if (s_cnt[g]) atomicAdd(&count[g], (unsigned long long)s_cnt[g]);
    }
}

// Rows per group only (the sums run in the two-column single pass).
__global__ void __launch_bounds__(256) k_count(const int32_t* __restrict__ keys, long long n, int G,
                                               unsigned long long* __restrict__ count) {
    __shared__ unsigned s_cnt[kCountSmemGroups];
    const bool smem = G <= kCountSmemGroups;
    if (smem) {
        for (int g = threadIdx.x; g < G; g += blockDim.x) s_cnt[g] = 0;
        __syncthreads();
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int g = keys[i];
        if ((unsigned)g < (unsigned)G) {
            if (smem)
                atomicAdd(&s_cnt[g], 1u);
            else
                atomicAdd(&count[g], 1ull);
        }
    }
    if (smem) {
        __syncthreads();
        for (int g = threadIdx.x; g < G; g += blockDim.x)
            if (s_cnt[g]) atomicAdd(&count[g], (unsigned long long)s_cnt[g]);
    }
}

__global__ void k_add_counts(unsigned long long* __restrict__ dst, const unsigned long long* __restrict__ src,
                             long long G) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G; g += (long long)gridDim.x * blockDim.x)
        dst[g] += src[g];
}

// Per group: COUNT, SUM, AVG = SUM / COUNT, and with D = SUMSQ - SUM*SUM/COUNT
// (each operation rounded to nearest in T, in this order, D clamped at 0),
// VAR_SAMP = D / (COUNT - 1), VAR_POP = D / COUNT and their square roots.
// Empty groups give NaN for AVG and the variances; a single row gives NaN for
// the sample variance (SQL's NULL).
template <typename T>
__global__ void k_stats_finalize(const unsigned char* __restrict__ st, StatsLayout ly, int dtype, int L, long long G,
                                 repro_stats_out out) {
    const StateView sx{const_cast<unsigned char*>(st), L, G};
    const StateView sq{const_cast<unsigned char*>(st) + ly.sq, L, G};
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        s_ok = header_ok(sx, dtype) && header_ok(sq, dtype);
        if (!s_ok) atomicOr(&sx.header()->errors, REPRO_ERR_LAYOUT);
    }
    __syncthreads();
    if (!s_ok) return;
    const unsigned long long* cnt = reinterpret_cast<const unsigned long long*>(st + ly.count);
    const T nan = quiet_nan<T>();
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G; g += (long long)gridDim.x * blockDim.x) {
        const unsigned long long c = cnt[g];
        const T S = state_finalize_group<T>(sx, g);
        const T Q = state_finalize_group<T>(sq, g);
        const T n = (T)c;  // exact for counts below 2^53 (2^24 in float)
        T mean = nan, vs = nan, vp = nan;
        if (c > 0) {
            mean = S / n;
            T D = Q - (S * S) / n;
            if (D < (T)0) D = (T)0;  // rounding can leave a tiny negative
            vp = D / n;
            if (c > 1) vs = D / (n - (T)1);
        }
        if (out.count) out.count[g] = (int64_t)c;
        if (out.sum) static_cast<T*>(out.sum)[g] = S;
        if (out.mean) static_cast<T*>(out.mean)[g] = mean;
        if (out.var_samp) static_cast<T*>(out.var_samp)[g] = vs;
        if (out.var_pop) static_cast<T*>(out.var_pop)[g] = vp;
        if (out.stddev_samp) static_cast<T*>(out.stddev_samp)[g] = sqrt(vs);
        if (out.stddev_pop) static_cast<T*>(out.stddev_pop)[g] = sqrt(vp);
    }
}

bool valid(int dtype, int L, int64_t G) {
    return (dtype == REPRO_F64 || dtype == REPRO_F32) && L >= 1 && L <= 4 && G >= 1 && G <= INT32_MAX;
}

repro_status from_cuda(cudaError_t e) {
    return e == cudaSuccess ? REPRO_OK : e == cudaErrorMemoryAllocation ? REPRO_ENOMEM : REPRO_ECUDA;
}

}  // namespace
}  // namespace rp

using namespace rp;

extern "C" {

size_t repro_stats_state_bytes(repro_dtype dtype, int L, int64_t num_groups) {
    if (!valid(dtype, L, num_groups)) return 0;
    return stats_layout(dtype, L, num_groups).total;
}

repro_status repro_stats_init(void* state, repro_dtype dtype, int L, int64_t num_groups, void* stream) {
    if (!state || (uintptr_t)state % 16 || !valid(dtype, L, num_groups)) return REPRO_EINVAL;
    const StatsLayout ly = stats_layout(dtype, L, num_groups);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* b = (unsigned char*)state;
    cudaError_t e = launch_init_state(b, dtype, L, num_groups, s);
    if (e == cudaSuccess) e = launch_init_state(b + ly.sq, dtype, L, num_groups, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b + ly.count, 0, 8 * (size_t)num_groups, s);
    return from_cuda(e);
}

repro_status repro_groupby_stats(const int32_t* keys, const void* values, int64_t n, repro_dtype dtype, int L,
                                 int64_t num_groups, void* state, void* stream) {
    if (!state || (uintptr_t)state % 16 || n < 0 || !valid(dtype, L, num_groups)) return REPRO_EINVAL;
    if (n > 0 && (!keys || !values || (uintptr_t)keys % 4 || (uintptr_t)values % (dtype == REPRO_F64 ? 8 : 4)))
        return REPRO_EINVAL;
    if (n == 0) return REPRO_OK;
    const StatsLayout ly = stats_layout(dtype, L, num_groups);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* b = (unsigned char*)state;
    const size_t vs = dtype == REPRO_F64 ? 8 : 4;
    cudaError_t err = cudaSuccess;
    unsigned long long* counts = reinterpret_cast<unsigned long long*>(b + ly.count);
    const void* xv[2] = {values, values};
    if (cols_supported(dtype, L, num_groups, 2, keys, xv)) {
        // one pass for the sums of x and x*x (squares formed in shared memory), one for the counts
        cudaMemPool_t pool0 = library_pool(err);
        if (!pool0) return from_cuda(err);
        void* part = nullptr;
        err = cudaMallocFromPoolAsync(&part, std::max<size_t>(16, cols_scratch_bytes(dtype, L, num_groups, 2, n)),
                                      pool0, s);
        if (err != cudaSuccess) return from_cuda(err);
        void* states[2] = {b, b + ly.sq};
        err = launch_groupby_cols(keys, xv, 2, true, n, dtype, L, num_groups, states, part, s);
        cudaFreeAsync(part, s);
        if (err != cudaSuccess) return from_cuda(err);
        k_count<<<device_info().sms * 8, 256, 0, s>>>(keys, n, (int)num_groups, counts);
        count_launches(1);
        return from_cuda(cudaGetLastError());
    }
    FusedPlanConfig cfg;
    if (fused_supported(dtype, L, num_groups, keys, values, true) &&
        fused_plan_config(dtype, L, (int)num_groups, 0, cfg, true)) {
        // two single passes over the same columns, the second squaring each
        // staged value in place (no x*x column in memory), and the counts
        cudaMemPool_t pool0 = library_pool(err);
        if (!pool0) return from_cuda(err);
        void* part = nullptr;
        err = cudaMallocFromPoolAsync(&part, std::max<size_t>(16, fused_scratch_bytes(cfg, L, num_groups, n)), pool0,
                                      s);
        if (err != cudaSuccess) return from_cuda(err);
        err = launch_groupby_fused(keys, values, n, dtype, L, num_groups, cfg, b, part, s);
        if (err == cudaSuccess)
            err = launch_groupby_fused(keys, values, n, dtype, L, num_groups, cfg, b + ly.sq, part, s, 0, true);
        cudaFreeAsync(part, s);
        if (err != cudaSuccess) return from_cuda(err);
        k_count<<<device_info().sms * 8, 256, 0, s>>>(keys, n, (int)num_groups, counts);
        count_launches(1);
        return from_cuda(cudaGetLastError());
    }
    cudaMemPool_t pool = library_pool(err);
    if (!pool) return from_cuda(err);
    void* sq = nullptr;
    err = cudaMallocFromPoolAsync(&sq, align16(vs * (size_t)n), pool, s);
    if (err != cudaSuccess) return from_cuda(err);
    const int grid = device_info().sms * 8;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(b + ly.count);
    if (dtype == REPRO_F64)
        k_square_count<double><<<grid, 256, 0, s>>>(keys, (const double*)values, n, (int)num_groups, (double*)sq, cnt);
    else
        k_square_count<float><<<grid, 256, 0, s>>>(keys, (const float*)values, n, (int)num_groups, (float*)sq, cnt);
    count_launches(1);
    err = cudaGetLastError();
    repro_status st = from_cuda(err);
    if (st == REPRO_OK) st = (repro_status)groupby_dispatch(keys, values, n, dtype, L, num_groups, b, s);
    if (st == REPRO_OK) st = (repro_status)groupby_dispatch(keys, sq, n, dtype, L, num_groups, b + ly.sq, s);
    cudaFreeAsync(sq, s);
    return st;
}

repro_status repro_stats_merge(void* dst, const void* src, repro_dtype dtype, int L, int64_t num_groups,
                               void* stream) {
    if (!dst || !src || dst == src || (uintptr_t)dst % 16 || (uintptr_t)src % 16 || !valid(dtype, L, num_groups))
        return REPRO_EINVAL;
    const StatsLayout ly = stats_layout(dtype, L, num_groups);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* d = (unsigned char*)dst;
    const unsigned char* c = (const unsigned char*)src;
    if (d < c + ly.total && c < d + ly.total) return REPRO_EINVAL;
    repro_status st = repro_merge(d, c, dtype, L, num_groups, stream);
    if (st == REPRO_OK) st = repro_merge(d + ly.sq, c + ly.sq, dtype, L, num_groups, stream);
    if (st != REPRO_OK) return st;
    k_add_counts<<<device_info().sms * 4, 256, 0, s>>>(reinterpret_cast<unsigned long long*>(d + ly.count),
                                                        reinterpret_cast<const unsigned long long*>(c + ly.count),
                                                        num_groups);
    count_launches(1);
    return from_cuda(cudaGetLastError());
}

repro_status repro_stats_finalize(const void* state, repro_dtype dtype, int L, int64_t num_groups,
                                  const repro_stats_out* out, void* stream) {
    if (!state || !out || (uintptr_t)state % 16 || !valid(dtype, L, num_groups)) return REPRO_EINVAL;
    const StatsLayout ly = stats_layout(dtype, L, num_groups);
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = device_info().sms * 4;
    if (dtype == REPRO_F64)
        k_stats_finalize<double><<<grid, 256, 0, s>>>((const unsigned char*)state, ly, dtype, L, num_groups, *out);
    else
        k_stats_finalize<float><<<grid, 256, 0, s>>>((const unsigned char*)state, ly, dtype, L, num_groups, *out);
    count_launches(1);
    return from_cuda(cudaGetLastError());
}

}  // extern "C"
