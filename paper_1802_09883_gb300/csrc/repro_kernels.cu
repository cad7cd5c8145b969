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

#include <algorithm>
#include <cstdint>
#include <cstdlib>

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

// dst += src over bare record arrays (no headers): the same per-group
// merge as k_merge, for blocks of records exchanged between ranks.
__global__ void k_merge_records(unsigned char* dst, const unsigned char* src, int L, long long G) {
    const size_t rec = 8 + 16 * (size_t)L;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G;
         g += (long long)gridDim.x * blockDim.x) {
        unsigned char* d = dst + (size_t)g * rec;
        const unsigned char* s = src + (size_t)g * rec;
        const int Kd = *reinterpret_cast<const int*>(d), Ks = *reinterpret_cast<const int*>(s);
        const int K = max(Kd, Ks);
        long long* db = reinterpret_cast<long long*>(d + 8);
        const long long* sb = reinterpret_cast<const long long*>(s + 8);
        __int128 acc[4];
        for (int j = 0; j < L; ++j) {
            __int128 v = 0;
            if (j - (K - Kd) >= 0) v += bin_read(&db[2 * (j - (K - Kd))], &db[2 * (j - (K - Kd)) + 1]);
            if (j - (K - Ks) >= 0) v += bin_read(&sb[2 * (j - (K - Ks))], &sb[2 * (j - (K - Ks)) + 1]);
            acc[j] = v;
        }
        for (int j = 0; j < L; ++j) bin_write(&db[2 * j], &db[2 * j + 1], acc[j]);
        *reinterpret_cast<int*>(d) = K;
        *reinterpret_cast<unsigned*>(d + 4) |= *reinterpret_cast<const unsigned*>(s + 4);
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

// ------------------------------------- conventional GroupBy (the baseline)
//
// SUM(value) GROUP BY key with built-in floating-point adds in whatever order
// the hardware takes them: the non-reproducible reference point the paper
// measures its types against (Sec. VI-C, aggregation without summation
// buffers).  Built for speed, with the same input handling as the
// reproducible kernels -- 16-byte vector loads, two quads of rows in flight
// per thread, a persistent grid -- and one of five table strategies:
//   FP_SMEM    one shared-memory table per CTA (C = 32: one copy per lane,
//              so a warp's adds never meet on an address), atomicAdd;
//   FP_MATCH   one shared table, rows of equal key within a warp combined by
//              __match_any_sync + shuffles first (skewed keys), one atomic
//              per distinct key;
//   FP_WARP    one table per warp: after the same combining the leaders'
//              keys are distinct, so they add with plain loads and stores;
//   FP_GLOBAL  atomicAdd straight into the result (L2 atomics);
//   FP_GMATCH  the same after combining equal keys within the warp.
// The launcher picks by group count, or a caller (the benchmark) times them
// all and keeps the fastest.
enum FpMode { FP_SMEM = 0, FP_MATCH = 1, FP_WARP = 2, FP_GLOBAL = 3, FP_GMATCH = 4, FP_MODES = 5 };

template <typename T>
struct FpQuad;
template <>
struct FpQuad<double> {
    static __device__ __forceinline__ void load(const double* v, long long q, double x[4]) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(v) + 2 * q);
        const double2 b = __ldg(reinterpret_cast<const double2*>(v) + 2 * q + 1);
        x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
    }
};
template <>
struct FpQuad<float> {
    static __device__ __forceinline__ void load(const float* v, long long q, float x[4]) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(v) + q);
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    }
};

// Combine the values of lanes holding the same key (all 32 lanes call it;
// invalid rows pass a key no other lane has).  Returns true in the lane that
// adds the combined sum (the lowest of its peers).
template <typename T>
__device__ __forceinline__ bool fp_combine(int key, T& v) {
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    unsigned others = lane == leader ? peers & ~(1u << lane) : 0u;
    const int iters = __reduce_max_sync(0xffffffffu, __popc(others));
    T sum = v;
    for (int i = 0; i < iters; ++i) {
        const int src = others ? __ffs(others) - 1 : lane;
        const T x = __shfl_sync(0xffffffffu, v, src);
        if (others) {
            sum += x;
            others &= others - 1;
        }
    }
    v = sum;
    return lane == leader;
}

template <typename T, int MODE>
__device__ __forceinline__ void fp_add_row(int g, T v, int G, T* tab, int C, T* out) {
    const int lane = threadIdx.x & 31;
    const bool ok = (unsigned)g < (unsigned)G;
    if (MODE == FP_SMEM) {
        if (ok) atomicAdd(&tab[(size_t)g * C + (lane & (C - 1))], v);
    } else if (MODE == FP_GLOBAL) {
        if (ok) atomicAdd(&out[g], v);
    } else {
        const int key = ok ? g : -1 - lane;
        const bool lead = fp_combine(key, v);
        if (lead && ok) {
            if (MODE == FP_MATCH) atomicAdd(&tab[g], v);
            else if (MODE == FP_GMATCH) atomicAdd(&out[g], v);
            else tab[g] += v;  // FP_WARP: this warp's own table, distinct keys
        }
    }
}

// VEC: keys and values 16-byte aligned (quads by vector loads); the rows
// past the last whole quad, and every row when !VEC, by scalar loads.
template <typename T, int MODE, bool VEC>
__global__ void __launch_bounds__(512) k_groupby_fp(const int32_t* __restrict__ keys, const T* __restrict__ vals,
                                                    long long n, int G, int C, T* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    T* stab = reinterpret_cast<T*>(s_raw);
    const bool smem = MODE == FP_SMEM || MODE == FP_MATCH || MODE == FP_WARP;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int words = MODE == FP_WARP ? G * nw : G * C;
    T* tab = MODE == FP_WARP ? stab + (size_t)warp * G : stab;
    if (smem) {
        for (int i = threadIdx.x; i < words; i += blockDim.x) stab[i] = (T)0;
        __syncthreads();
    }
    const long long gw = (long long)blockIdx.x * nw + warp, nwarps = (long long)gridDim.x * nw;
    const long long nq = VEC ? n / 4 : 0;
    // two chunks of 32 quads per warp in flight; the loop bound is warp-uniform
    for (long long c = gw; c * 32 < nq; c += 2 * nwarps) {
        const long long q0 = c * 32 + lane, q1 = (c + nwarps) * 32 + lane;
        const bool v0 = q0 < nq, v1 = q1 < nq;
        int4 k0 = make_int4(-1, -1, -1, -1), k1 = make_int4(-1, -1, -1, -1);
        T x0[4] = {0, 0, 0, 0}, x1[4] = {0, 0, 0, 0};
        if (v0) {
            k0 = __ldg(reinterpret_cast<const int4*>(keys) + q0);
            FpQuad<T>::load(vals, q0, x0);
        }
        if (v1) {
            k1 = __ldg(reinterpret_cast<const int4*>(keys) + q1);
            FpQuad<T>::load(vals, q1, x1);
        }
        fp_add_row<T, MODE>(k0.x, x0[0], G, tab, C, out);
        fp_add_row<T, MODE>(k0.y, x0[1], G, tab, C, out);
        fp_add_row<T, MODE>(k0.z, x0[2], G, tab, C, out);
        fp_add_row<T, MODE>(k0.w, x0[3], G, tab, C, out);
        fp_add_row<T, MODE>(k1.x, x1[0], G, tab, C, out);
        fp_add_row<T, MODE>(k1.y, x1[1], G, tab, C, out);
        fp_add_row<T, MODE>(k1.z, x1[2], G, tab, C, out);
        fp_add_row<T, MODE>(k1.w, x1[3], G, tab, C, out);
    }
    // scalar rows (all of them when the columns are not 16-byte aligned)
    for (long long r0 = 4 * nq + gw * 32; r0 < n; r0 += nwarps * 32) {
        const long long r = r0 + lane;
        const bool v = r < n;
        fp_add_row<T, MODE>(v ? keys[r] : -1, v ? vals[r] : (T)0, G, tab, C, out);
    }
    if (smem) {
        __syncthreads();
        for (int g = threadIdx.x; g < G; g += blockDim.x) {
            T acc = (T)0;
            if (MODE == FP_WARP) {
                for (int w = 0; w < nw; ++w) acc += stab[(size_t)w * G + g];
            } else {
                for (int c = 0; c < C; ++c) acc += stab[(size_t)g * C + c];
            }
            if (acc != (T)0) atomicAdd(&out[g], acc);
        }
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

cudaError_t launch_merge_records(void* dst, const void* src, int L, long long G, cudaStream_t s) {
    const int th = 256;
    prof_begin(PROF_MERGE, s);
    k_merge_records<<<grid_for(G, th, device_info().sms * 8), th, 0, s>>>((unsigned char*)dst,
                                                                           (const unsigned char*)src, L, G);
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

// Shared-memory words each strategy needs for G groups (0: not applicable).
template <typename T>
static size_t fp_smem_bytes(int mode, long long G, int threads, int& C) {
    const size_t cap = 200 * 1024;
    C = 1;
    switch (mode) {
        case FP_SMEM:
            if ((size_t)G * 32 * sizeof(T) <= 64 * 1024) C = 32;  // one copy per lane
            return (size_t)G * C * sizeof(T) <= cap ? (size_t)G * C * sizeof(T) : 0;
        case FP_MATCH: return (size_t)G * sizeof(T) <= cap ? (size_t)G * sizeof(T) : 0;
        case FP_WARP: return (size_t)G * (threads / 32) * sizeof(T) <= cap ? (size_t)G * (threads / 32) * sizeof(T) : 0;
        default: return 0;
    }
}

// The built-in choice: lane-private copies for small tables, one shared
// table with within-warp combining up to the shared-memory limit, global
// atomics with combining beyond.
template <typename T>
static int fp_rule(long long G) {
    int C;
    if ((size_t)G * 32 * sizeof(T) <= 64 * 1024) return FP_SMEM;
    if (fp_smem_bytes<T>(FP_MATCH, G, 512, C)) return FP_MATCH;
    return FP_GMATCH;
}

template <typename T, int MODE, bool VEC>
static cudaError_t launch_fp_mode(const int32_t* keys, const T* vals, long long n, int G, int C, size_t smem,
                                  T* out, cudaStream_t s) {
    auto kern = k_groupby_fp<T, MODE, VEC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int th = 512;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, th, smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long work = (n + 4ll * th - 1) / (4ll * th);
    const int blocks = (int)std::max(1ll, std::min<long long>(work, (long long)device_info().sms * per_sm));
    kern<<<blocks, th, smem, s>>>(keys, vals, n, G, C, out);
    return cudaGetLastError();
}

template <typename T, int MODE>
static cudaError_t launch_fp_vec(bool vec, const int32_t* keys, const T* vals, long long n, int G, int C, size_t smem,
                                 T* out, cudaStream_t s) {
    return vec ? launch_fp_mode<T, MODE, true>(keys, vals, n, G, C, smem, out, s)
               : launch_fp_mode<T, MODE, false>(keys, vals, n, G, C, smem, out, s);
}

static int env_fp_mode() {
    static const int v = [] {
        const char* e = getenv("REPRO_FP_MODE");
        return e ? atoi(e) : -1;
    }();
    return v;
}

template <typename T>
static cudaError_t launch_groupby_float_t(const int32_t* keys, const T* vals, long long n, long long G, T* out,
                                          cudaStream_t s, int mode) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(T) * (size_t)G, s);
    if (e != cudaSuccess || n == 0) return e;
    if (mode < 0) mode = env_fp_mode();
    if (mode < 0 || mode >= FP_MODES) mode = fp_rule<T>(G);
    int C = 1;
    const size_t smem = fp_smem_bytes<T>(mode, G, 512, C);
    if ((mode == FP_SMEM || mode == FP_MATCH || mode == FP_WARP) && smem == 0) return cudaErrorInvalidValue;
    const bool vec = (uintptr_t)keys % 16 == 0 && (uintptr_t)vals % 16 == 0;
    const ProfKernel pk = sizeof(T) == 8 ? PROF_FP64 : PROF_FP32;
    prof_begin(pk, s);
    switch (mode) {
        case FP_SMEM: e = launch_fp_vec<T, FP_SMEM>(vec, keys, vals, n, (int)G, C, smem, out, s); break;
        case FP_MATCH: e = launch_fp_vec<T, FP_MATCH>(vec, keys, vals, n, (int)G, C, smem, out, s); break;
        case FP_WARP: e = launch_fp_vec<T, FP_WARP>(vec, keys, vals, n, (int)G, C, smem, out, s); break;
        case FP_GLOBAL: e = launch_fp_vec<T, FP_GLOBAL>(vec, keys, vals, n, (int)G, C, smem, out, s); break;
        default: e = launch_fp_vec<T, FP_GMATCH>(vec, keys, vals, n, (int)G, C, smem, out, s); break;
    }
    prof_end(pk, s);
    count_launches(1);
    return e;
}

bool fp_mode_supported(int dtype, int mode, long long G) {
    if (mode < 0 || mode >= FP_MODES || G < 1 || G > INT32_MAX) return false;
    if (mode == FP_GLOBAL || mode == FP_GMATCH) return true;
    int C;
    return (dtype == REPRO_F64 ? fp_smem_bytes<double>(mode, G, 512, C) : fp_smem_bytes<float>(mode, G, 512, C)) != 0;
}

cudaError_t launch_groupby_fp64(const int32_t* keys, const double* vals, long long n, long long G, double* out,
                                cudaStream_t s, int mode) {
    return launch_groupby_float_t<double>(keys, vals, n, G, out, s, mode);
}

cudaError_t launch_groupby_fp32(const int32_t* keys, const float* vals, long long n, long long G, float* out,
                                cudaStream_t s, int mode) {
    return launch_groupby_float_t<float>(keys, vals, n, G, out, s, mode);
}

}  // namespace rp
