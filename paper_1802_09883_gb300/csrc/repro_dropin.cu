// repro_dropin.cu -- the unbuffered drop-in accumulator (repro_accum.cuh)
// used as a library routine, and the DECIMAL fixed-point baseline: the two
// extra comparison points of the paper's evaluation (the naive repro type,
// Sec. IV / VI; exact fixed-point DECIMAL sums, Sec. VI).
//
// repro_sum_unbuffered: every thread adds its strided rows into its own
// repro_accum, one value at a time; the CTA merges its threads' accumulators
// in shared memory and writes one partial record; the partials are merged
// into the caller's one-group state.  Same bits as repro_sum.
//
// groupby_sum_decimal64: SUM of int64 values (a DECIMAL column as scaled
// integers) per group, exact (two's-complement wrap-around on overflow):
// shared-memory 64-bit atomics per CTA when the groups fit, else global.
#include <cuda_runtime.h>

#include <cstdint>

#include "repro.h"
#include "repro_accum.cuh"
#include "repro_internal.h"

namespace rp {
namespace {

constexpr int kDropThreads = 256;

template <typename T, int L>
__global__ void __launch_bounds__(kDropThreads) k_sum_unbuffered(const T* __restrict__ vals, long long n,
                                                                 unsigned char* __restrict__ parts) {
    __shared__ repro_accum<T, L> s_acc[kDropThreads];
    repro_accum<T, L> a;
    a.init();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a.add(vals[i]);
    s_acc[threadIdx.x] = a;
    __syncthreads();
    for (int w = kDropThreads / 2; w > 0; w >>= 1) {  // merges commute: any tree gives the same state
        if ((int)threadIdx.x < w) s_acc[threadIdx.x].merge(s_acc[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) s_acc[0].store(parts + (size_t)blockIdx.x * (8 + 16 * L));
}

template <typename T>
cudaError_t launch_unbuffered(const T* vals, long long n, int L, unsigned char* parts, int grid, cudaStream_t s) {
    switch (L) {
        case 1: k_sum_unbuffered<T, 1><<<grid, kDropThreads, 0, s>>>(vals, n, parts); break;
        case 2: k_sum_unbuffered<T, 2><<<grid, kDropThreads, 0, s>>>(vals, n, parts); break;
        case 3: k_sum_unbuffered<T, 3><<<grid, kDropThreads, 0, s>>>(vals, n, parts); break;
        default: k_sum_unbuffered<T, 4><<<grid, kDropThreads, 0, s>>>(vals, n, parts); break;
    }
    count_launches(1);
    return cudaGetLastError();
}

constexpr int kDecimalSmemGroups = 4096;

__global__ void __launch_bounds__(256) k_groupby_decimal(const int32_t* __restrict__ keys,
                                                         const long long* __restrict__ vals, long long n, int G,
                                                         unsigned long long* __restrict__ out) {
    __shared__ unsigned long long s_sum[kDecimalSmemGroups];
    const bool smem = G <= kDecimalSmemGroups;
    if (smem) {
        for (int g = threadIdx.x; g < G; g += blockDim.x) s_sum[g] = 0;
        __syncthreads();
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int g = keys[i];
        if ((unsigned)g >= (unsigned)G) continue;
        const unsigned long long v = (unsigned long long)vals[i];
        if (smem)
            atomicAdd(&s_sum[g], v);
        else
            atomicAdd(&out[g], v);
    }
    if (smem) {
        __syncthreads();
        for (int g = threadIdx.x; g < G; g += blockDim.x)
            if (s_sum[g]) atomicAdd(&out[g], s_sum[g]);
    }
}

}  // namespace
}  // namespace rp

using namespace rp;

extern "C" {

repro_status repro_sum_unbuffered(const void* values, int64_t n, repro_dtype dtype, int L, void* state,
                                  void* stream) {
    if (!state || (uintptr_t)state % 16 || n < 0 || (dtype != REPRO_F64 && dtype != REPRO_F32) || L < 1 || L > 4)
        return REPRO_EINVAL;
    if (n > 0 && (!values || (uintptr_t)values % (dtype == REPRO_F64 ? 8 : 4))) return REPRO_EINVAL;
    if (n == 0) return REPRO_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = device_info().sms * 4;
    cudaError_t e = cudaSuccess;
    cudaMemPool_t pool = library_pool(e);
    if (!pool) return e == cudaErrorMemoryAllocation ? REPRO_ENOMEM : REPRO_ECUDA;
    void* parts = nullptr;
    e = cudaMallocFromPoolAsync(&parts, (size_t)grid * (8 + 16 * (size_t)L), pool, s);
    if (e == cudaSuccess)
        e = dtype == REPRO_F64 ? launch_unbuffered<double>((const double*)values, n, L, (unsigned char*)parts, grid, s)
                               : launch_unbuffered<float>((const float*)values, n, L, (unsigned char*)parts, grid, s);
    if (e == cudaSuccess) e = launch_merge_partials(parts, grid, 1, state, dtype, L, s);
    if (parts) cudaFreeAsync(parts, s);
    return e == cudaSuccess ? REPRO_OK : e == cudaErrorMemoryAllocation ? REPRO_ENOMEM : REPRO_ECUDA;
}

repro_status groupby_sum_decimal64(const int32_t* keys, const int64_t* values, int64_t n, int64_t num_groups,
                                   int64_t* out, void* stream) {
    if (!out || n < 0 || num_groups < 1 || num_groups > INT32_MAX) return REPRO_EINVAL;
    if (n > 0 && (!keys || !values)) return REPRO_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int64_t) * (size_t)num_groups, s);
    if (e != cudaSuccess || n == 0) return e == cudaSuccess ? REPRO_OK : REPRO_ECUDA;
    k_groupby_decimal<<<device_info().sms * 8, 256, 0, s>>>(keys, (const long long*)values, n, (int)num_groups,
                                                             (unsigned long long*)out);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? REPRO_OK : REPRO_ECUDA;
}

}  // extern "C"
