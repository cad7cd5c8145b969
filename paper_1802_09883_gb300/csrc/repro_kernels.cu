// repro_kernels.cu -- CUDA kernels (sm_103a) of the reproducible grouped SUM.
//
// Two-pass path, any group count:
//   k_window    per-group top grid index K and flags (max-abs pre-pass:
//               Algorithm 2's "check extractor validity" taken over the whole
//               input instead of value by value)
//   k_rebase    raise each group's stored window to the new K, dropping
//               levels that fall off the bottom (operator+=(repro) alignment)
//   k_accum_*   extract every value's digits in its group's window and add
//               them exactly: shared-memory int64 bins flushed into the
//               state's 128-bit bins (small G), or 128-bit global atomics
// and per group: k_merge (operator+=(repro)), k_finalize (eq. (1)), plus the
// conventional floating-point atomic GroupBy used as the baseline.
#include <cuda_runtime.h>

#include <cstdint>

#include "repro_device.cuh"
#include "repro_internal.h"

namespace rp {

// ------------------------------------------------------------------- kernels

// Every record starts all zero (K = 0, no flags, zero level sums), so the
// record area is cleared as one flat byte range with coalesced 16-byte stores
// (the state is 16-byte aligned and the header 64 bytes); the header is
// written by thread 0.
__global__ void k_init_state(unsigned char* base, int dtype, int L, long long G) {
    StateView st{base, L, G};
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    if (tid == 0) state_init_header(st, dtype);
    const unsigned long long bytes = (unsigned long long)G * (8ull + 16ull * (unsigned long long)L);
    uint4* rec = reinterpret_cast<uint4*>(base + sizeof(repro_state_header));
    const long long n16 = (long long)(bytes / 16);
    for (long long i = tid; i < n16; i += nth) rec[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0 && (bytes & 15))  // G odd: one 8-byte word left
        *reinterpret_cast<unsigned long long*>(base + sizeof(repro_state_header) + bytes - 8) = 0ull;
}

// Max-abs pre-pass.  Kmax[g] (zeroed by the caller) receives max K(b) over
// the group's finite in-range values and fl[g] the OR of the value flags.
// Shared-memory tables when G <= smem_groups, else global atomics.
template <typename T>
__global__ void k_window(const int32_t* __restrict__ keys, const T* __restrict__ vals, long long n, int G,
                         int smem_groups, int* __restrict__ Kmax, unsigned* __restrict__ fl,
                         unsigned* __restrict__ errors) {
    extern __shared__ int s_win[];
    const bool use_smem = G <= smem_groups;
    int* sK = s_win;
    unsigned* sF = reinterpret_cast<unsigned*>(s_win + (use_smem ? G : 0));
    if (use_smem) {
        for (int g = threadIdx.x; g < G; g += blockDim.x) {
            sK[g] = 0;
            sF[g] = 0;
        }
        __syncthreads();
    }
    bool bad_key = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int g = keys[i];
        if ((unsigned)g >= (unsigned)G) {
            bad_key = true;
            continue;
        }
        const Split s = split_value(vals[i]);
        int* pk = use_smem ? &sK[g] : &Kmax[g];
        unsigned* pf = use_smem ? &sF[g] : &fl[g];
        if (s.flag) {
            atomicOr(pf, s.flag);
        } else if (s.kb > *(volatile int*)pk) {
            atomicMax(pk, s.kb);
        }
    }
    if (__any_sync(0xffffffffu, bad_key) && (threadIdx.x & 31) == 0) atomicOr(errors, REPRO_ERR_KEY);
    if (use_smem) {
        __syncthreads();
        for (int g = threadIdx.x; g < G; g += blockDim.x) {
            if (sK[g] > 0) atomicMax(&Kmax[g], sK[g]);
            if (sF[g]) atomicOr(&fl[g], sF[g]);
        }
    }
}

// Raise each group's window to max(K, Kmax[g]) and OR in the new flags.
__global__ void k_rebase(unsigned char* base, int dtype, int L, long long G, const int* __restrict__ Kmax,
                         const unsigned* __restrict__ fl) {
    StateView st{base, L, G};
    if (!cta_header_ok(st, dtype)) return;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G;
         g += (long long)gridDim.x * blockDim.x) {
        if (fl[g]) *st.flags(g) |= fl[g];
        const int K0 = *st.K(g);
        const int K1 = max(K0, Kmax[g]);
        if (K1 == K0) continue;
        const int d = K1 - K0;
        for (int j = L - 1; j >= 0; --j) {  // new level j <- old level j - d
            __int128 v = 0;
            if (j - d >= 0) v = bin_read(st.lo(g, j - d), st.hi(g, j - d));
            bin_write(st.lo(g, j), st.hi(g, j), v);
        }
        *st.K(g) = K1;
    }
}

// Accumulate with per-CTA shared-memory int64 bins.  Each CTA takes a
// contiguous chunk of at most 2^23 rows, so no int64 bin can overflow
// (|digit| <= 2^39) before it is flushed into the state's 128-bit bins.
template <typename T>
__global__ void k_accum_smem(const int32_t* __restrict__ keys, const T* __restrict__ vals, long long n,
                             long long chunk, unsigned char* base, int dtype, int L, int G) {
    StateView st{base, L, G};
    if (!cta_header_ok(st, dtype)) return;
    extern __shared__ long long s_acc[];
    long long* sbin = s_acc;                                  // [G][L]
    int* sK = reinterpret_cast<int*>(s_acc + (size_t)G * L);  // [G]
    for (int i = threadIdx.x; i < G * L; i += blockDim.x) sbin[i] = 0;
    for (int g = threadIdx.x; g < G; g += blockDim.x) sK[g] = *st.K(g);
    __syncthreads();
    const long long beg = blockIdx.x * chunk;
    const long long end = min(n, beg + chunk);
    for (long long i = beg + threadIdx.x; i < end; i += blockDim.x) {
        const int g = keys[i];
        if ((unsigned)g >= (unsigned)G) continue;
        const Split s = split_value(vals[i]);
        if (s.flag) continue;
        long long* row = &sbin[g * L];
        for_each_digit<T>(s, sK[g], L, [&](int j, long long d) {
            atomicAdd(reinterpret_cast<unsigned long long*>(&row[j]), (unsigned long long)d);
        });
    }
    __syncthreads();
    for (int i = threadIdx.x; i < G * L; i += blockDim.x) {
        const long long v = sbin[i];
        if (v != 0) add128_atomic(st.lo(i / L, i % L), st.hi(i / L, i % L), v);
    }
}

// Accumulate straight into the state's 128-bit bins with global atomics.
template <typename T>
__global__ void k_accum_global(const int32_t* __restrict__ keys, const T* __restrict__ vals, long long n,
                               unsigned char* base, int dtype, int L, long long G) {
    StateView st{base, L, G};
    if (!cta_header_ok(st, dtype)) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int g = keys[i];
        if ((unsigned)g >= (unsigned long long)G) continue;
        const Split s = split_value(vals[i]);
        if (s.flag) continue;
        for_each_digit<T>(s, *st.K(g), L, [&](int j, long long d) { add128_atomic(st.lo(g, j), st.hi(g, j), d); });
    }
}

// dst += src (operator+=(repro), Sec. V-B): align to the larger window,
// drop the levels below it, add bins, OR flags.
__global__ void k_merge(unsigned char* dst, const unsigned char* src, int dtype, int L, long long G) {
    StateView d{dst, L, G};
    StateView s{const_cast<unsigned char*>(src), L, G};
    if (!cta_header_ok(d, dtype, &s)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned e = s.header()->errors;
        if (e) atomicOr(&d.header()->errors, e);
    }
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G;
         g += (long long)gridDim.x * blockDim.x) {
        const int Kd = *d.K(g), Ks = *s.K(g);
        const int K = max(Kd, Ks);
        __int128 acc[4];
        for (int j = 0; j < L; ++j) {
            __int128 v = 0;
            if (j - (K - Kd) >= 0) v += bin_read(d.lo(g, j - (K - Kd)), d.hi(g, j - (K - Kd)));
            if (j - (K - Ks) >= 0) v += bin_read(s.lo(g, j - (K - Ks)), s.hi(g, j - (K - Ks)));
            acc[j] = v;
        }
        for (int j = 0; j < L; ++j) bin_write(d.lo(g, j), d.hi(g, j), acc[j]);
        *d.K(g) = K;
        *d.flags(g) |= *s.flags(g);
    }
}

// Eq. (1): V_j = RN_T(T_j u(K - j)), folded from the lowest level up.
template <typename T>
__global__ void k_finalize(const unsigned char* base, int dtype, int L, long long G, T* __restrict__ out) {
    StateView st{const_cast<unsigned char*>(base), L, G};
    if (!cta_header_ok(st, dtype)) return;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G;
         g += (long long)gridDim.x * blockDim.x)
        out[g] = state_finalize_group<T>(st, g);
}

// Conventional floating-point GroupBy (non-reproducible baseline).
template <typename T>
__global__ void k_groupby_float(const int32_t* __restrict__ keys, const T* __restrict__ vals, long long n,
                                int G, int smem_groups, T* __restrict__ out) {
    extern __shared__ unsigned char s_raw[];
    T* sacc = reinterpret_cast<T*>(s_raw);
    const bool use_smem = G <= smem_groups;
    if (use_smem) {
        for (int g = threadIdx.x; g < G; g += blockDim.x) sacc[g] = (T)0;
        __syncthreads();
    }
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int g = keys[i];
        if ((unsigned)g >= (unsigned)G) continue;
        atomicAdd(use_smem ? &sacc[g] : &out[g], vals[i]);
    }
    if (use_smem) {
        __syncthreads();
        for (int g = threadIdx.x; g < G; g += blockDim.x)
            if (sacc[g] != (T)0) atomicAdd(&out[g], sacc[g]);
    }
}

// ------------------------------------------------------------------ launchers

// Kernels taking more than 48 KB of dynamic shared memory must opt in.
template <typename K>
static cudaError_t allow_smem(K* kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static int grid_for(long long work, int threads, int max_blocks) {
    long long b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)(b < max_blocks ? b : max_blocks);
}

cudaError_t launch_init_state(void* state, int dtype, int L, long long G, cudaStream_t s) {
    const int th = 256;
    const long long words = G * (8 + 16ll * L) / 16 + 1;
    k_init_state<<<grid_for(words, th, device_info().sms * 4), th, 0, s>>>((unsigned char*)state, dtype, L, G);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_groupby_two_pass_t(const int32_t* keys, const T* vals, long long n, int dtype, int L,
                                             long long G, void* state, void* scratch, cudaStream_t s) {
    const DeviceInfo& di = device_info();
    int* Kmax = reinterpret_cast<int*>(scratch);
    unsigned* fl = reinterpret_cast<unsigned*>(Kmax + G);
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int) * 2 * (size_t)G, s);
    if (e != cudaSuccess) return e;
    unsigned* errors = &reinterpret_cast<repro_state_header*>(state)->errors;
    const int th = 256;
    // pass 1: window
    const int win_smem_groups = 8192;
    const size_t win_smem = G <= win_smem_groups ? 8 * (size_t)G : 0;
    if (n > 0) {
        if ((e = allow_smem(k_window<T>, win_smem)) != cudaSuccess) return e;
        prof_begin(PROF_WINDOW, s);
        k_window<T><<<grid_for(n, th, di.sms * 8), th, win_smem, s>>>(keys, vals, n, (int)G, win_smem_groups,
                                                                       Kmax, fl, errors);
        prof_end(PROF_WINDOW, s);
        count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_rebase<<<grid_for(G, th, di.sms * 8), th, 0, s>>>((unsigned char*)state, dtype, L, G, Kmax, fl);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    // pass 2: digits
    const size_t acc_smem = (size_t)G * L * 8 + (size_t)G * 4;
    if (acc_smem <= di.smem_optin - 1024) {
        if ((e = allow_smem(k_accum_smem<T>, acc_smem)) != cudaSuccess) return e;
        const int th2 = 512;
        const long long per_cta_max = 1ll << 23;
        long long blocks = (long long)di.sms * 2;
        if (blocks * per_cta_max < n) blocks = (n + per_cta_max - 1) / per_cta_max;
        if (blocks > n) blocks = n;
        const long long chunk = (n + blocks - 1) / blocks;
        blocks = (n + chunk - 1) / chunk;
        prof_begin(PROF_ACCUM, s);
        k_accum_smem<T><<<(int)blocks, th2, acc_smem, s>>>(keys, vals, n, chunk, (unsigned char*)state, dtype,
                                                           L, (int)G);
        prof_end(PROF_ACCUM, s);
    } else {
        prof_begin(PROF_ACCUM, s);
        k_accum_global<T><<<grid_for(n, th, di.sms * 8), th, 0, s>>>(keys, vals, n, (unsigned char*)state,
                                                                      dtype, L, G);
        prof_end(PROF_ACCUM, s);
    }
    count_launches(1);
    return cudaGetLastError();
}

size_t two_pass_scratch_bytes(long long G) { return sizeof(int) * 2 * (size_t)G; }

cudaError_t launch_groupby_two_pass(const int32_t* keys, const void* vals, long long n, int dtype, int L,
                                    long long G, void* state, void* scratch, cudaStream_t s) {
    if (dtype == REPRO_F64)
        return launch_groupby_two_pass_t<double>(keys, (const double*)vals, n, dtype, L, G, state, scratch, s);
    return launch_groupby_two_pass_t<float>(keys, (const float*)vals, n, dtype, L, G, state, scratch, s);
}

cudaError_t launch_merge(void* dst, const void* src, int dtype, int L, long long G, cudaStream_t s) {
    const int th = 256;
    prof_begin(PROF_MERGE, s);
    k_merge<<<grid_for(G, th, device_info().sms * 8), th, 0, s>>>((unsigned char*)dst, (const unsigned char*)src,
                                                                   dtype, L, G);
    prof_end(PROF_MERGE, s);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const void* state, int dtype, int L, long long G, void* out, cudaStream_t s) {
    const int th = 256;
    const int b = grid_for(G, th, device_info().sms * 8);
    prof_begin(PROF_FINALIZE, s);
    if (dtype == REPRO_F64)
        k_finalize<double><<<b, th, 0, s>>>((const unsigned char*)state, dtype, L, G, (double*)out);
    else
        k_finalize<float><<<b, th, 0, s>>>((const unsigned char*)state, dtype, L, G, (float*)out);
    prof_end(PROF_FINALIZE, s);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_groupby_float_t(const int32_t* keys, const T* vals, long long n, long long G, T* out,
                                          cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(T) * (size_t)G, s);
    if (e != cudaSuccess || n == 0) return e;
    const int smem_groups = 12288;
    const size_t smem = G <= smem_groups ? sizeof(T) * (size_t)G : 0;
    if ((e = allow_smem(k_groupby_float<T>, smem)) != cudaSuccess) return e;
    const int th = 256;
    const ProfKernel pk = sizeof(T) == 8 ? PROF_FP64 : PROF_FP32;
    prof_begin(pk, s);
    k_groupby_float<T><<<grid_for(n, th, device_info().sms * 8), th, smem, s>>>(keys, vals, n, (int)G,
                                                                                 smem_groups, out);
    prof_end(pk, s);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_groupby_fp64(const int32_t* keys, const double* vals, long long n, long long G, double* out,
                                cudaStream_t s) {
    return launch_groupby_float_t<double>(keys, vals, n, G, out, s);
}

cudaError_t launch_groupby_fp32(const int32_t* keys, const float* vals, long long n, long long G, float* out,
                                cudaStream_t s) {
    return launch_groupby_float_t<float>(keys, vals, n, G, out, s);
}

}  // namespace rp
