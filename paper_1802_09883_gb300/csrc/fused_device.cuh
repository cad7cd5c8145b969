// fused_device.cuh -- device code shared by the single-pass kernels
// (repro_fused.cu: one aggregation; repro_batch.cu: a list of them): the
// shared-memory layout, the CTA table of 32-bit LO/HI word pairs, the
// per-row and per-quad consumers, the per-tile window raise and the flush
// of a CTA table into a partial or final state record array.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "ptx.cuh"
#include "repro_device.cuh"

namespace rp {

constexpr uint64_t kWaitNs = 2000000000ull;  // every mbarrier wait gives up after 2 s

struct FusedSmem {
    // byte offsets into dynamic shared memory
    size_t bars, ctl, keys, vals, bins, K, Kp, F, dlist, slist, rlist, total;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The table is padded: two spare levels after each group's L levels and one
// spare group after the last, so that a row's three digit adds always have
// table words at fixed offsets from its group's window level (digits past
// the window land in the spare levels, rows with nothing to add in the
// spare group; neither is ever read back, so they are never cleared).
template <typename T>
__host__ __device__ inline FusedSmem fused_layout(int S, int R, int G, int L, int C) {
    FusedSmem m;
    size_t o = 0;
    m.bars = o;
    o += 16 * (size_t)S;  // full[S], empty[S]
    m.ctl = o;
    o += 64;  // counters[3][2], abort, pad, slow-list counters[3]
    o = align_up(o, 128);
    m.keys = o;
    o += (size_t)S * R * 4;
    o = align_up(o, 128);
    m.vals = o;
    o += (size_t)S * R * sizeof(T);
    o = align_up(o, 16);
    m.bins = o;  // LO[G + 1][L + 2][C] (uint32) then HI[G + 1][L + 2][C] (int32)
    o += (size_t)(G + 1) * (L + 2) * C * 8;
    m.K = o;
    o += (size_t)G * 4;
    m.Kp = o;
    o += (size_t)G * 4;
    m.F = o;
    o += (size_t)G * 4;
    m.dlist = o;
    o += (size_t)R * 2;
    m.slist = o;
    o += (size_t)R * 2;
    o = align_up(o, 4);
    m.rlist = o;
    o += (size_t)(R < G ? R : G) * 4;
    m.total = align_up(o, 16);
    return m;
}




// The CTA table holds each bin of each group as a 64-bit value
// HI * 2^32 + LO with LO unsigned and HI signed, both 32-bit words in shared
// memory: 32-bit shared atomics run far faster than 64-bit ones.  A digit d
// is added to LO as its low 32 bits; the value LO held before (returned by
// the atomic) tells whether LO wrapped, and HI takes d's high part plus that
// carry, skipped when zero.  Every add is exact and adds commute, so the
// result is independent of their order.  With C copies, lane l uses copy
// l mod C (C = 32: conflict-free, and skewed keys never collide in a warp).
struct Table {
    unsigned* lo;
    int* hi;
    int L, C;
    __device__ __forceinline__ size_t at(int g, int j, int copy) const {
        return ((size_t)g * L + j) * C + copy;
    }
};

__device__ __forceinline__ void add_digit(const Table& t, size_t i, long long d) {
    const unsigned lo = (unsigned)(unsigned long long)d;
    const unsigned old = atomicAdd(&t.lo[i], lo);
    const int carry = (unsigned)(old + lo) < old;
    const int hi = (int)(d >> 32) + carry;
    if (hi != 0) atomicAdd(&t.hi[i], hi);
}

__device__ __forceinline__ long long table_value(const Table& t, size_t i) {
    return (long long)(((unsigned long long)(long long)t.hi[i] << 32) + (unsigned long long)t.lo[i]);
}

// Add one row's digits into the CTA table (its window must hold the value).
template <typename T, int L>
__device__ __forceinline__ void add_row(const Split& s, int K, const Table& t, int g, int copy) {
    long long top, mid, low;
    digits3<T>(s, top, mid, low);
    const int j = K - s.kb;  // level of the value's top digit
    if (j < L && top != 0) add_digit(t, t.at(g, j, copy), top);
    if (j + 1 < L && s.kb >= 1 && mid != 0) add_digit(t, t.at(g, j + 1, copy), mid);
    if (j + 2 < L && s.kb >= 2 && low != 0) add_digit(t, t.at(g, j + 2, copy), low);
}

// CTA-table window of a group no row has reached yet (its bins are zero).
constexpr int kNoWindow = -1;
// Bit of a group's flag word: the group is on this tile's raise list.
constexpr unsigned kQueued = 0x80000000u;

// Phase A for one row: add it, flag it, or defer it until its group's window
// is raised.  The first row of a group claims the window with one
// compare-and-swap (no raise is needed while the bins are zero); a row above
// an established window is deferred, and the first such row of the tile puts
// the group on the raise list.  Within phase A a window changes only from
// kNoWindow, so every add lands at the window the tile ends with.
template <typename T, int L>
__device__ __forceinline__ void consume_row(int g, T b, int idx, int G, const Table& t, int copy, int* sK,
                                            int* sKp, unsigned* sF, unsigned short* dlist, int* rlist, int* cnt,
                                            bool& bad_key) {
    if ((unsigned)g >= (unsigned)G) {
        bad_key = true;
        return;
    }
    const Split s = split_value(b);
    if (s.flag) {
        atomicOr(&sF[g], s.flag);
        return;
    }
    if (s.mant == 0) return;
    int K = sK[g];
    if (K < 0) {
        const int old = atomicCAS(&sK[g], kNoWindow, s.kb);
        K = old < 0 ? s.kb : old;
    }
    if (s.kb <= K) {
        add_row<T, L>(s, K, t, g, copy);
        return;
    }
    dlist[atomicAdd(&cnt[0], 1)] = (unsigned short)idx;
    atomicMax(&sKp[g], s.kb);
    if (!(atomicOr(&sF[g], kQueued) & kQueued)) rlist[atomicAdd(&cnt[1], 1)] = g;
}

// Shared-window addresses of the hot loop's arrays.
struct SAddr {
    uint32_t keys, vals;  // stage s starts at keys + 4 R s, vals + sizeof(T) R s
    uint32_t K;           // int K[G]
    uint32_t lo, hi;      // table words [(g LP + j) C + copy], LP = L + 2 levels per group
};

// Value bit-words of two consecutive rows: (hi, lo) per row for double, the
// single word for float.
template <typename T>
struct PairWords;
template <>
struct PairWords<double> {
    static __device__ __forceinline__ void load(const double* v, uint32_t& h0, uint32_t& l0, uint32_t& h1,
                                                uint32_t& l1) {
        const uint4 p = *reinterpret_cast<const uint4*>(v);
        l0 = p.x;
        h0 = p.y;
        l1 = p.z;
        h1 = p.w;
    }
};
template <>
struct PairWords<float> {
    static __device__ __forceinline__ void load(const float* v, uint32_t& h0, uint32_t& l0, uint32_t& h1,
                                                uint32_t& l1) {
        const uint2 p = *reinterpret_cast<const uint2*>(v);
        h0 = p.x;
        h1 = p.y;
        l0 = l1 = 0u;
    }
};

// The two halves of adding digit (lo, hi) to a table word pair: a shared
// atomic on the LO word returns its old value; hi plus the carry out of
// old + lo then goes to the HI word with a reduction.  Unconditional (a
// digit that must not be added arrives as zero, at a word of its own group),
// so no predicate is needed.  Split in two so that a row's three atomics are
// in flight together before their carries are needed; the asm blocks are
// ordered among themselves (volatile), and the phases around them are
// separated by barriers.
__device__ __forceinline__ unsigned table_add_lo(uint32_t lo_addr, unsigned lo) {
    unsigned old;
    asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(lo_addr), "r"(lo));
    return old;
}

__device__ __forceinline__ void table_add_hi(uint32_t hi_addr, unsigned old, unsigned lo, int hi) {
    int h;
    asm("{\n\t.reg .u32 t;\n\t"
        "add.cc.u32 t, %1, %2;\n\t"
        "addc.s32 %0, %3, 0;\n\t}"
        : "=r"(h)
        : "r"(old), "r"(lo), "r"(hi));
    asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(hi_addr), "r"(h));
}

// Biased exponent E and t = E + (fraction bits); K(b) = floor(t / W) by
// multiply-shift.  E == 0 (zero, subnormal) and E all ones (Inf, NaN) are
// left to the caller's checks: an all-ones E gives K(b) = KMAX + 1.
template <typename T>
struct Expo;
template <>
struct Expo<double> {
    static __device__ __forceinline__ void get(uint32_t vhi, int& E, int& t, int& kb) {
        E = (int)((vhi >> 20) & 0x7ffu);
        t = E + 52;
        // t / 40 as the high word of t * ceil(2^32 / 40): exact for t < 2^12
        kb = (int)__umulhi((unsigned)t, 107374183u);
    }
};
template <>
struct Expo<float> {
    static __device__ __forceinline__ void get(uint32_t bits, int& E, int& t, int& kb) {
        E = (int)((bits >> 23) & 0xffu);
        t = E + 23;
        // t / 18 as the high word of t * ceil(2^32 / 18): exact for t < 2^12
        kb = (int)__umulhi((unsigned)t, 238609295u);
    }
};

// Phase A for four consecutive rows of a staged tile, row by row and
// without branches on the common path (the table is the padded layout of
// fused_layout; the copy count CC is fixed at compile time): a row whose key
// is good, whose value is normal and inside its group's window adds its
// three signed digits (Signed<T>) at fixed offsets from its top level; a
// zero with a good key adds nothing (into the spare group); every other row
// -- a bad key, a special or subnormal value, a group without a window yet,
// a value above its group's window -- is put on the tile's slow list (its
// counter at scnt_addr) for consume_row after the tile.  The digits of such
// rows are computed too, from whatever their words hold, and added to the
// spare group, which keeps the four rows' work straight-line.
// The four rows are r0, r0 + 1, r0 + H and r0 + H + 1.  H = 2 takes four
// consecutive rows; H = 64 with r0 = (128-row block) + 2 lane makes each of
// a warp's shared loads of keys and values one contiguous run (no bank
// conflicts: 16-byte loads at a 32-byte lane stride took two wavefronts per
// 128 bytes).
template <typename T, int L, int CC, int H>
__device__ __forceinline__ void consume_quad_fast(const SAddr& sa, const int32_t* tk, const T* tv, const int* sK,
                                                  int r0, int G, int spare, int copy, unsigned short* slist,
                                                  uint32_t scnt_addr) {
    constexpr uint32_t LP = L + 2;  // levels per group in the padded table
    // plain loads (the staged tile and the windows do not change during
    // this phase), so that the compiler may start the next row's loads
    // while this row's atomics are in flight
    int gq[4];
    if (H == 2) {
        const int4 k4 = *reinterpret_cast<const int4*>(tk + r0);
        gq[0] = k4.x;
        gq[1] = k4.y;
        gq[2] = k4.z;
        gq[3] = k4.w;
    } else {
        const int2 ka = *reinterpret_cast<const int2*>(tk + r0);
        const int2 kc = *reinterpret_cast<const int2*>(tk + r0 + H);
        gq[0] = ka.x;
        gq[1] = ka.y;
        gq[2] = kc.x;
        gq[3] = kc.y;
    }
    uint32_t vhi[4], vlo[4];
    PairWords<T>::load(tv + r0, vhi[0], vlo[0], vhi[1], vlo[1]);
    PairWords<T>::load(tv + r0 + H, vhi[2], vlo[2], vhi[3], vlo[3]);
    const uint32_t hi_off = sa.hi - sa.lo;
    unsigned okm = 0;  // bit q: row q added its digits
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int E, t, kb;
        Expo<T>::get(vhi[q], E, t, kb);
        const bool key_ok = (unsigned)gq[q] < (unsigned)G;
        const unsigned gc = min((unsigned)gq[q], (unsigned)(G - 1));
        const int K = sK[gc];
        const bool ok = key_ok && E != 0 && kb <= K;
        unsigned lo[3];
        int hi[3];
        Signed<T>::digits(vhi[q], vlo[q], t, kb, lo, hi);
        // the top digit's word: level K - kb of the row's group, or the spare
        // group for a row with nothing to add (including a value so far below
        // its window, K - kb >= L, that all its digits drop out); the other
        // digits follow at fixed offsets (past the window: spare levels)
        const bool adds = ok && K - kb < L;
        const uint32_t tg = adds ? (uint32_t)gq[q] * LP + (uint32_t)(K - kb) : (uint32_t)spare * LP;
        const uint32_t a = sa.lo + 4u * (tg * CC + (uint32_t)copy);
        constexpr int ND = L < 3 ? L : 3;
        unsigned old[ND];
#pragma unroll
        for (int k = 0; k < ND; ++k) old[k] = table_add_lo(a + 4u * CC * k, lo[k]);
#pragma unroll
        for (int k = 0; k < ND; ++k) table_add_hi(a + hi_off + 4u * CC * k, old[k], lo[k], hi[k]);
        okm |= (unsigned)ok << q;
    }
    if (okm != 0xfu) {  // rare: a row that did not add; a zero with a good key needs nothing more
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (!(okm & (1u << q)) && !((unsigned)gq[q] < (unsigned)G && Lean<T>::is_zero(vhi[q], vlo[q]))) {
                uint32_t idx;
                asm volatile("atom.shared.add.u32 %0, [%1], 1;" : "=r"(idx) : "r"(scnt_addr) : "memory");
                slist[idx] = (unsigned short)(r0 + (q & 1) + (q >> 1) * H);
            }
    }
}

// After phase A: raise the windows collected in rlist (dropping low levels)
// and add the deferred rows.  Consumer-uniform; uses named barrier 1.
template <typename T, int L>
__device__ __forceinline__ void raise_and_add(int nr, int nd, const int32_t* tk, const T* tv, const Table& t,
                                              int* sK, const int* sKp, unsigned* sF, const unsigned short* dlist,
                                              const int* rlist, int ctid, int NC) {
    for (int i = ctid; i < nr * t.C; i += NC) {
        const int g = rlist[i / t.C];
        const int copy = i % t.C;
        const int d = sKp[g] - sK[g];
#pragma unroll
        for (int j = L - 1; j >= 0; --j) {
            const size_t dst = t.at(g, j, copy);
            if (j - d >= 0) {
                const size_t src = t.at(g, j - d, copy);
                t.lo[dst] = t.lo[src];
                t.hi[dst] = t.hi[src];
            } else {
                t.lo[dst] = 0;
                t.hi[dst] = 0;
            }
        }
    }
    named_bar_sync(1, NC);
    for (int i = ctid; i < nr; i += NC) {
        sK[rlist[i]] = sKp[rlist[i]];
        sF[rlist[i]] &= ~kQueued;
    }
    named_bar_sync(1, NC);
    for (int i = ctid; i < nd; i += NC) {
        const int r = dlist[i];
        const int g = tk[r];
        const Split s = split_value(tv[r]);
        add_row<T, L>(s, sK[g], t, g, (ctid & 31) & (t.C - 1));
    }
}

// Write (first) or add (later) the CTA table into this CTA's partial record
// array, then clear the table's bins.  Consumer threads only.
template <int L>
__device__ void flush_partial(unsigned char* part, int G, const Table& t, const int* sK, const unsigned* sF,
                              bool first, int ctid, int NC) {
    constexpr size_t rec = 8 + 16 * L;
    for (int g = ctid; g < G; g += NC) {
        unsigned char* r = part + (size_t)g * rec;
        int* pK = reinterpret_cast<int*>(r);
        unsigned* pF = reinterpret_cast<unsigned*>(r + 4);
        long long* pb = reinterpret_cast<long long*>(r + 8);
        const int K = sK[g];
        __int128 acc[L];
#pragma unroll
        for (int j = 0; j < L; ++j) {
            acc[j] = 0;
            for (int c = 0; c < t.C; ++c) {
                const size_t i = t.at(g, j, c);
                acc[j] += (__int128)table_value(t, i);
                t.lo[i] = 0;
                t.hi[i] = 0;
            }
        }
        if (first) {
            *pK = K;
            *pF = sF[g] & ~kQueued;
        } else {
            const int d = K - *pK;  // the CTA window only rises
#pragma unroll
            for (int j = L - 1; j >= 0; --j)
                if (j - d >= 0) acc[j] += bin_read(&pb[2 * (j - d)], &pb[2 * (j - d) + 1]);
            *pK = K;
            *pF |= sF[g] & ~kQueued;
        }
#pragma unroll
        for (int j = 0; j < L; ++j) bin_write(&pb[2 * j], &pb[2 * j + 1], acc[j]);
    }
}

// An empty record for every group (window kNoWindow, no flags, zero bins):
// what a CTA that gave up on a wait leaves as its partial, so that the merge
// adds nothing.  Consumer threads only.
template <int L>
__device__ void write_empty_partial(unsigned char* part, int G, int ctid, int NC) {
    constexpr size_t rec = 8 + 16 * L;
    for (int g = ctid; g < G; g += NC) {
        unsigned char* r = part + (size_t)g * rec;
        *reinterpret_cast<int*>(r) = kNoWindow;
        *reinterpret_cast<unsigned*>(r + 4) = 0u;
        long long* pb = reinterpret_cast<long long*>(r + 8);
#pragma unroll
        for (int j = 0; j < 2 * L; ++j) pb[j] = 0;
    }
}

}  // namespace rp
