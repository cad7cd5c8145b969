/*
 * repro_accum.cuh -- the reproducible accumulator repro<T,L> as a drop-in
 * device type (the paper's unbuffered data type, Sec. IV).
 *
 * A user kernel that sums with a `double` accumulator can sum with a
 * repro_accum<double, L> instead: add() one value at a time, merge() two
 * accumulators, value() the result.  Every add does the whole per-value work
 * of Algorithm 2 on its own -- classify the value, raise the window when
 * the value is above it (the level sums shift down, low levels drop), add
 * its balanced digits to the exact level sums -- so the type costs several
 * times a plain floating-point add (the paper measures the same "naive"
 * slowdown on CPUs); the library's grouped kernels amortise that work over
 * shared-memory tables instead.  Results are bit-identical to the library's
 * (and to any order or split of the adds): the state is canonical.
 *
 * Layout of the value: window K (top level's grid index; -1 before the first
 * finite nonzero value), flags (REPRO_FLAG_*), L exact 128-bit level sums,
 * level j in units u(K - j) = 2^(g_min + (K - j) W).  store() writes it as a
 * state record of include/repro.h (int32 K, uint32 flags, {lo, hi}[L]).
 *
 * Device-only; include with the library's device sources on the include
 * path (-I include -I paper_1802_09883_gb300/csrc) and compile with
 * -fmad=false like the library.
 */
#pragma once

#include "repro.h"
#include "repro_device.cuh"

template <typename T, int L>
struct repro_accum {
    static_assert(L >= 1 && L <= 4, "L must be in 1..4");
    int K;
    unsigned flags;
    __int128 bins[L];

    __device__ __forceinline__ void init() {
        K = -1;
        flags = 0;
#pragma unroll
        for (int j = 0; j < L; ++j) bins[j] = 0;
    }

    // v[j] <- v[j - d] (zero where j < d), d >= 0, one level per step: the
    // indices stay fixed, so the levels stay in registers.
    __device__ __forceinline__ static void shift_down(__int128 (&v)[L], int d) {
        for (int s = 0; s < d && s < L; ++s) {
#pragma unroll
            for (int j = L - 1; j > 0; --j) v[j] = v[j - 1];
            v[0] = 0;
        }
    }

    // Move the window up to grid index k: level j takes the old level j - d.
    __device__ __forceinline__ void raise(int k) {
        shift_down(bins, k - K);
        K = k;
    }

    __device__ __forceinline__ void add(T x) {
        const rp::Split s = rp::split_value(x);
        if (s.flag) {
            flags |= s.flag;
            return;
        }
        if (s.mant == 0) return;
        if (s.kb > K) raise(s.kb);
        long long top, mid, low;
        rp::digits3<T>(s, top, mid, low);
        // the digits at levels j, j + 1, j + 2 (j = K - K(b), the level of
        // the top digit; grid indices below 0 and levels past L - 1 drop out)
        __int128 a[L];
#pragma unroll
        for (int i = 0; i < L; ++i) a[i] = 0;
        a[0] = top;
        if (L > 1 && s.kb >= 1) a[L > 1 ? 1 : 0] = mid;
        if (L > 2 && s.kb >= 2) a[L > 2 ? 2 : 0] = low;
        shift_down(a, K - s.kb);
#pragma unroll
        for (int i = 0; i < L; ++i) bins[i] += a[i];
    }

    __device__ __forceinline__ void merge(const repro_accum& o) {
        flags |= o.flags;
        if (o.K < 0) return;
        if (o.K > K) raise(o.K);
        __int128 ob[L];
#pragma unroll
        for (int j = 0; j < L; ++j) ob[j] = o.bins[j];
        shift_down(ob, K - o.K);
#pragma unroll
        for (int j = 0; j < L; ++j) bins[j] += ob[j];
    }

    // Eq. (1): the level values rounded once each, folded from the lowest up.
    __device__ __forceinline__ T value() const {
        if ((flags & (REPRO_FLAG_NAN | REPRO_FLAG_RANGE)) ||
            ((flags & REPRO_FLAG_POS_INF) && (flags & REPRO_FLAG_NEG_INF)))
            return rp::quiet_nan<T>();
        if (flags & REPRO_FLAG_POS_INF) return rp::inf_of<T>(false);
        if (flags & REPRO_FLAG_NEG_INF) return rp::inf_of<T>(true);
        T q = (T)0;
        bool first = true;
#pragma unroll
        for (int j = L - 1; j >= 0; --j) {
            if (K - j < 0) continue;
            const __int128 t = bins[j];
            const bool neg = t < 0;
            const unsigned __int128 mag = neg ? (unsigned __int128)(-t) : (unsigned __int128)t;
            const T v = rp::round_scaled<T>(neg, mag, rp::Traits<T>::GMIN + (K - j) * rp::Traits<T>::W);
            q = first ? v : rp::t_add(q, v);
            first = false;
        }
        return q;
    }

    // As a state record (8 + 16 L bytes, 8-byte aligned).
    __device__ __forceinline__ void store(unsigned char* rec) const {
        *reinterpret_cast<int*>(rec) = K;
        *reinterpret_cast<unsigned*>(rec + 4) = flags;
        long long* b = reinterpret_cast<long long*>(rec + 8);
#pragma unroll
        for (int j = 0; j < L; ++j) rp::bin_write(&b[2 * j], &b[2 * j + 1], bins[j]);
    }
};
