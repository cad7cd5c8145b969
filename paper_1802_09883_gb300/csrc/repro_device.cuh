// repro_device.cuh -- device-side arithmetic of the reproducible grouped SUM.
//
// The paper's repro<T,L> (Sec. III-C, Sec. IV) keeps, per level, a running
// sum S in [1.5, 1.75) ufp(S) and a carry count C; ulp(S) is the level's
// unit.  Here each level is held directly as the exact integer
// T = (S - 1.5 ufp(S)) / ulp(S) + C 2^(m-2): the same value, without the
// floating-point container.  Everything in this file is integer arithmetic
// except the final rounding to T (eq. (1)).
//
// The grid: level units are u(k) = 2^(g_min + k W), g_min = -1074 (double)
// or -149 (float), so every finite value is an integer multiple of u(0).
// A value b = mant * 2^p * u(0) needs the top grid index
//   K(b) = min{K >= 0 : |b| < 2^(W-1) u(K)}          (Algorithm 2's raise test)
// and its digit at grid index k is
//   d_k(b) = RNE(b / u(k)) - 2^W RNE(b / u(k+1)),    |d_k| <= 2^(W-1),
// which is the contribution q / u of Algorithm 2's transform against the
// constant extractor 1.5 ufp(S) (ties to even).  d_k does not depend on the
// window the value is extracted in, which is what lets partial states with
// different windows merge exactly.
#pragma once

#include <cstdint>

#include "repro.h"

namespace rp {

template <typename T>
struct Traits;

template <>
struct Traits<double> {
    static constexpr int W = 40;       // bits between levels (Sec. III-C)
    static constexpr int M = 52;       // fraction bits
    static constexpr int KMAX = 51;    // top grid index with a finite S
    static constexpr int GMIN = -1074; // exponent of u(0)
    static constexpr int BIAS = 1023;
    static constexpr int EMIN = -1022;
    static constexpr int EMAX = 1023;
};

template <>
struct Traits<float> {
    static constexpr int W = 18;
    static constexpr int M = 23;
    static constexpr int KMAX = 14;
    static constexpr int GMIN = -149;
    static constexpr int BIAS = 127;
    static constexpr int EMIN = -126;
    static constexpr int EMAX = 127;
};

// A value split into sign, integer significand and grid position.
struct Split {
    uint64_t mant;  // |b| = mant * 2^p * u(0)
    int p;
    int kb;         // K(b)
    uint32_t flag;  // REPRO_FLAG_* for NaN / Inf / out of range; 0 otherwise
    bool neg;
};

__device__ __forceinline__ Split split_value(double b) {
    const uint64_t bits = (uint64_t)__double_as_longlong(b);
    Split s;
    s.neg = (bits >> 63) != 0;
    const uint32_t E = (uint32_t)(bits >> 52) & 0x7ffu;
    const uint64_t F = bits & ((1ull << 52) - 1);
    s.flag = 0;
    if (E == 0x7ffu) {
        s.flag = F ? REPRO_FLAG_NAN : (s.neg ? REPRO_FLAG_NEG_INF : REPRO_FLAG_POS_INF);
        s.mant = 0; s.p = 0; s.kb = 0;
        return s;
    }
    if (E == 0) {  // subnormal or zero: top bit at t = 63 - clz, K = (t + 1) / W
        s.mant = F;
        s.p = 0;
        s.kb = F ? (64 - __clzll((long long)F)) / 40 : 0;
    } else {       // normal: top bit at t = E + 51, K = (t + 1) / W
        s.mant = F | (1ull << 52);
        s.p = (int)E - 1;
        s.kb = ((int)E + 52) / 40;
    }
    if (s.kb > Traits<double>::KMAX) s.flag = REPRO_FLAG_RANGE;
    return s;
}

__device__ __forceinline__ Split split_value(float b) {
    const uint32_t bits = (uint32_t)__float_as_int(b);
    Split s;
    s.neg = (bits >> 31) != 0;
    const uint32_t E = (bits >> 23) & 0xffu;
    const uint32_t F = bits & ((1u << 23) - 1);
    s.flag = 0;
    if (E == 0xffu) {
        s.flag = F ? REPRO_FLAG_NAN : (s.neg ? REPRO_FLAG_NEG_INF : REPRO_FLAG_POS_INF);
        s.mant = 0; s.p = 0; s.kb = 0;
        return s;
    }
    if (E == 0) {  // top bit at t = 31 - clz
        s.mant = F;
        s.p = 0;
        s.kb = F ? (32 - __clz((int)F)) / 18 : 0;
    } else {       // top bit at t = E + 22
        s.mant = F | (1u << 23);
        s.p = (int)E - 1;
        s.kb = ((int)E + 23) / 18;
    }
    if (s.kb > Traits<float>::KMAX) s.flag = REPRO_FLAG_RANGE;
    return s;
}

// Low 64 bits of RNE(mant * 2^s), ties to even; mant < 2^53.
__device__ __forceinline__ uint64_t rne_scaled(uint64_t mant, int s) {
    if (s >= 0) return s < 64 ? (mant << s) : 0ull;
    const int r = -s;
    if (r >= 64) return 0ull;
    const uint64_t q = mant >> r;
    const uint64_t rem = mant - (q << r);
    const uint64_t half = 1ull << (r - 1);
    return q + (uint64_t)((rem > half) | ((rem == half) & (uint32_t)(q & 1)));
}

// The (at most three) nonzero digits of a split value in the window with top
// grid index K and L levels: grid indices max(K(b) - 2, K - L + 1, 0) ..
// min(K(b), K).  A value's bits span at most three W-bit levels (53 bits
// over W = 40, 24 bits over W = 18), so lower digits vanish.
// Calls f(level, digit) for each, level j = K - k (0 = top of the window).
template <typename T, typename F>
__device__ __forceinline__ void for_each_digit(const Split& s, int K, int L, F&& f) {
    constexpr int W = Traits<T>::W;
    const int khi = min(s.kb, K);
    const int klo = max(max(s.kb - 2, K - L + 1), 0);
    if (s.mant == 0 || khi < klo) return;
    uint64_t r_up = rne_scaled(s.mant, s.p - W * (khi + 1));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int k = khi - i;
        if (k >= klo) {
            const uint64_t r = rne_scaled(s.mant, s.p - W * k);
            const long long d = (long long)(r - (r_up << W));
            if (d != 0) f(K - k, s.neg ? -d : d);
            r_up = r;
        }
    }
}

// Digits of a finite nonzero split value at grid indices kb, kb - 1 and
// kb - 2 (its top, middle and low levels), without rounding steps per level:
// X = |b| / u(kb - 2) is an exact integer below 2^(3W - 1) (the value's
// bits all sit at or above u(kb - 2)), cut into W-bit pieces x2:x1:x0, and
// the round-to-nearest-even carries c1 = [RNE(X / 2^W) > floor(X / 2^W)],
// c2 = [RNE(X / 2^2W) > floor(X / 2^2W)] turn them into balanced digits
//   low = x0 - c1 2^W,  mid = x1 + c1 - c2 2^W,  top = x2 + c2,
// i.e. d_k = RNE(X / 2^(W i)) - 2^W RNE(X / 2^(W (i + 1))) for i = 0, 1, 2.
// If the window drops the low level (or low and middle), the kept digits are
// still right: c1 (c2) carries the rounding of the dropped part.
// Levels below grid index 0 get zero digits.
template <typename T>
__device__ __forceinline__ void digits3(const Split& s, long long& top, long long& mid, long long& low);

template <>
__device__ __forceinline__ void digits3<double>(const Split& s, long long& top, long long& mid, long long& low) {
    constexpr uint64_t M = (1ull << 40) - 1, H = 1ull << 39;
    const int s2 = s.p - 40 * s.kb + 80;  // mant's lowest bit in units of u(kb - 2): 27..80
    const unsigned __int128 X = (unsigned __int128)s.mant << s2;  // below 2^119
    const uint64_t x0 = (uint64_t)X & M;
    const uint64_t x1 = (uint64_t)(X >> 40) & M;
    const uint64_t x2 = (uint64_t)(X >> 80);
    const uint64_t c1 = (uint64_t)((x0 > H) | ((x0 == H) & (uint32_t)(x1 & 1)));
    const uint64_t c2 = (uint64_t)((x1 > H) | ((x1 == H) & ((x0 != 0) | (uint32_t)(x2 & 1))));
    low = (long long)x0 - (long long)(c1 << 40);
    mid = (long long)(x1 + c1) - (long long)(c2 << 40);
    top = (long long)(x2 + c2);
    if (s.neg) {
        top = -top;
        mid = -mid;
        low = -low;
    }
}

template <>
__device__ __forceinline__ void digits3<float>(const Split& s, long long& top, long long& mid, long long& low) {
    constexpr uint64_t M = (1ull << 18) - 1, H = 1ull << 17;
    const int s2 = s.p - 18 * s.kb + 36;  // 12..36
    const uint64_t X = s.mant << s2;      // below 2^60
    const uint64_t x0 = X & M, x1 = (X >> 18) & M, x2 = X >> 36;
    const uint64_t c1 = (uint64_t)((x0 > H) | ((x0 == H) & (uint32_t)(x1 & 1)));
    const uint64_t c2 = (uint64_t)((x1 > H) | ((x1 == H) & ((x0 != 0) | (uint32_t)(x2 & 1))));
    low = (long long)x0 - (long long)(c1 << 18);
    mid = (long long)(x1 + c1) - (long long)(c2 << 18);
    top = (long long)(x2 + c2);
    if (s.neg) {
        top = -top;
        mid = -mid;
        low = -low;
    }
}

// Zero test on a value's bit words (hi, lo) for double, the single word for
// float: +0 and -0 add nothing.
template <typename T>
struct Lean;

template <>
struct Lean<double> {
    static __device__ __forceinline__ bool is_zero(uint32_t vhi, uint32_t vlo) {
        return ((vhi << 1) | vlo) == 0u;
    }
};

template <>
struct Lean<float> {
    static __device__ __forceinline__ bool is_zero(uint32_t bits, uint32_t) { return (bits << 1) == 0u; }
};

// ------------------------------------------ signed digits for the hot loop
//
// The same digits once more, with fewer operations: the sign is applied to
// the significand before the shift (X is the two's complement of +-|b| /
// u(kb - 2)), and the pieces and round-to-nearest-even carries are taken on
// that signed X.  Rounding to nearest with ties to even is symmetric
// (RNE(-x) = -RNE(x)), and on a two's complement X the floor-based pieces
// with carry c = [rest > half, or rest == half and the part above is odd]
// compute exactly RNE of the signed quotient, so the digits come out
// negated for negative values without negating three digits afterwards.
// Inputs: the value's words, t = E + 52 (double) / E + 23 (float) for its
// biased exponent E >= 1, and kb = floor(t / W); the value must be normal.
template <typename T>
struct Signed;

template <>
struct Signed<double> {
    static __device__ __forceinline__ void digits(uint32_t vhi, uint32_t vlo, int t, int kb, unsigned lo[3],
                                                  int hi[3]) {
        const uint32_t S = (uint32_t)((int)vhi >> 31);  // 0 or all ones
        const uint32_t mh = (vhi & 0xfffffu) | 0x100000u;
        uint32_t sl, sh;  // the significand with the value's sign, two's complement
        asm("{\n\t.reg .u32 a, b;\n\t"
            "xor.b32 a, %2, %4;\n\t"
            "xor.b32 b, %3, %4;\n\t"
            "sub.cc.u32 %0, a, %4;\n\t"
            "subc.u32 %1, b, %4;\n\t}"
            : "=r"(sl), "=r"(sh)
            : "r"(vlo), "r"(mh), "r"(S));
        // X = significand * 2^s, s = E + 79 - 40 kb in [27, 66], has at least
        // 27 zero bits at the bottom; the words hold X' = X / 2^8, the signed
        // significand shifted by s - 8 in [19, 58] = r within a word and q =
        // 0 or 1 whole words (X' < 2^111 in magnitude), so that X's 40-bit
        // field [40, 80) is word 1 plus the low byte of word 2
        const int s8 = t + 19 - 40 * kb;
        const int r = s8 & 31;
        const bool q = s8 >= 32;
        const uint32_t v0 = sl << r;
        const uint32_t v1 = __funnelshift_l(sl, sh, r);
        const uint32_t v2 = __funnelshift_l(sh, S, r);
        const uint32_t w0 = q ? 0u : v0;
        const uint32_t w1 = q ? v0 : v1;
        const uint32_t w2 = q ? v1 : v2;
        const uint32_t w3 = q ? v2 : S;
        // fields of X: x0 = w0 2^8 (bits [0, 40)), x1 = w1 + 2^32 (w2 & 0xff),
        // x2 = (w3:w2) >> 8 (signed)
        const uint32_t x1h = w2 & 0xffu;
        const uint32_t x2l = __funnelshift_r(w2, w3, 8);
        const int x2h = (int)w3 >> 8;
        // carries at bits 40 and 80, round to nearest even: at 40,
        // [x0 + 2^39 - 1 + (x1 & 1) >= 2^40] = [w0 + (w1 & 1) > 2^31] (x0's
        // low byte is zero); at 80, [x1 + 2^39 - 1 + tie >= 2^40] with tie =
        // [x0 != 0] | (x2 & 1), x1's low word folded into the carry-in
        const uint32_t c1 = (uint32_t)(((unsigned long long)w0 + (w1 & 1u) + 0x7fffffffull) >> 32);
        const uint32_t z2 = w1 | w0 | (w2 & 0x100u);
        const uint32_t c2 = (x1h + 0x7fu + (uint32_t)(((unsigned long long)z2 + 0xffffffffull) >> 32)) >> 8;
        lo[0] = x2l + c2;
        hi[0] = x2h + (int)(lo[0] < c2);
        lo[1] = w1 + c1;
        hi[1] = (int)x1h + (int)(lo[1] < c1) - 256 * (int)c2;
        lo[2] = w0 << 8;
        hi[2] = (int)(w0 >> 24) - 256 * (int)c1;
    }
};

template <>
struct Signed<float> {
    static __device__ __forceinline__ void digits(uint32_t bits, uint32_t, int t, int kb, unsigned lo[3], int hi[3]) {
        const int M = (int)((bits & 0x7fffffu) | 0x800000u);
        const int Ms = (int)bits < 0 ? -M : M;
        const int s = t + 12 - 18 * kb;  // E + 35 - 18 kb in [12, 29]
        const long long X = (long long)Ms << s;  // |X| < 2^53
        const uint32_t xl = (uint32_t)X, xh = (uint32_t)((unsigned long long)X >> 32);
        const int x0 = (int)(xl & 0x3ffffu);
        const int x1 = (int)(__funnelshift_r(xl, xh, 18) & 0x3ffffu);
        const int x2 = (int)xh >> 4;  // signed part above bit 36
        const int c1 = (x0 + 0x1ffff + (x1 & 1)) >> 18;
        const int c2 = (x1 + 0x1ffff + ((x0 != 0) | (x2 & 1))) >> 18;
        const int d0 = x2 + c2, d1 = x1 + c1 - (c2 << 18), d2 = x0 - (c1 << 18);
        lo[0] = (unsigned)d0;
        hi[0] = d0 >> 31;
        lo[1] = (unsigned)d1;
        hi[1] = d1 >> 31;
        lo[2] = (unsigned)d2;
        hi[2] = d2 >> 31;
    }
};

// ---------------------------------------------------------------- state view

struct StateView {
    unsigned char* base;
    int L;
    long long G;

    __device__ __forceinline__ repro_state_header* header() const {
        return reinterpret_cast<repro_state_header*>(base);
    }
    __device__ __forceinline__ size_t stride() const { return 8 + 16 * (size_t)L; }
    __device__ __forceinline__ int* K(long long g) const {
        return reinterpret_cast<int*>(base + sizeof(repro_state_header) + (size_t)g * stride());
    }
    __device__ __forceinline__ unsigned* flags(long long g) const {
        return reinterpret_cast<unsigned*>(K(g) + 1);
    }
    __device__ __forceinline__ long long* lo(long long g, int j) const {
        return reinterpret_cast<long long*>(base + sizeof(repro_state_header) + (size_t)g * stride() + 8 +
                                            16 * (size_t)j);
    }
    __device__ __forceinline__ long long* hi(long long g, int j) const { return lo(g, j) + 1; }
};

// Add a signed 64-bit amount to a 128-bit bin held as hi 2^64 + lo (both
// halves signed): lo takes the add, and the rare signed overflow of lo,
// detected from the value the atomic returns, moves one unit into hi.
// Adds commute, so the final (lo, hi) do not depend on their order.
__device__ __forceinline__ void add128_atomic(long long* lo, long long* hi, long long d) {
    const unsigned long long old = atomicAdd(reinterpret_cast<unsigned long long*>(lo),
                                             (unsigned long long)d);
    const long long o = (long long)old;
    const long long nw = (long long)(old + (unsigned long long)d);
    if (((o >= 0) == (d >= 0)) && ((nw >= 0) != (d >= 0)))
        atomicAdd(reinterpret_cast<unsigned long long*>(hi), d >= 0 ? 1ull : ~0ull);
}

__device__ __forceinline__ __int128 bin_read(const long long* lo, const long long* hi) {
    return (((__int128)*hi) << 64) + (__int128)*lo;
}

__device__ __forceinline__ void bin_write(long long* lo, long long* hi, __int128 v) {
    const long long l = (long long)(unsigned long long)v;
    *lo = l;
    *hi = (long long)((v - (__int128)l) >> 64);
}

// ----------------------------------------------------------------- finalize

// RN_T(+-mag * 2^e2), round to nearest even, gradual underflow, overflow to
// infinity; e2 >= g_min so results below the normal range are exact.
template <typename T>
__device__ __forceinline__ T round_scaled(bool neg, unsigned __int128 mag, int e2);

template <>
__device__ __forceinline__ double round_scaled<double>(bool neg, unsigned __int128 mag, int e2) {
    if (mag == 0) return 0.0;
    const uint64_t mh = (uint64_t)(mag >> 64), ml = (uint64_t)mag;
    const int nb = mh ? 128 - __clzll((long long)mh) : 64 - __clzll((long long)ml);
    int E = nb - 1 + e2;
    uint64_t bits;
    if (E < -1022) {
        bits = (uint64_t)(mag << (e2 + 1074));  // exact: below 2^52 units of 2^-1074
    } else {
        const int sh = nb - 53;
        uint64_t q;
        if (sh <= 0) {
            q = ml << (-sh);
        } else {
            q = (uint64_t)(mag >> sh);
            const unsigned __int128 rem = mag - ((unsigned __int128)q << sh);
            const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
            if (rem > half || (rem == half && (q & 1))) ++q;
            if (q == (1ull << 53)) { q >>= 1; ++E; }
        }
        if (E > 1023) return neg ? -__longlong_as_double(0x7ff0000000000000ll)
                                 : __longlong_as_double(0x7ff0000000000000ll);
        bits = ((uint64_t)(E + 1023) << 52) | (q & ((1ull << 52) - 1));
    }
    if (neg) bits |= 1ull << 63;
    return __longlong_as_double((long long)bits);
}

template <>
__device__ __forceinline__ float round_scaled<float>(bool neg, unsigned __int128 mag, int e2) {
    if (mag == 0) return 0.0f;
    const uint64_t mh = (uint64_t)(mag >> 64), ml = (uint64_t)mag;
    const int nb = mh ? 128 - __clzll((long long)mh) : 64 - __clzll((long long)ml);
    int E = nb - 1 + e2;
    uint32_t bits;
    if (E < -126) {
        bits = (uint32_t)(mag << (e2 + 149));
    } else {
        const int sh = nb - 24;
        uint64_t q;
        if (sh <= 0) {
            q = ml << (-sh);
        } else {
            q = (uint64_t)(mag >> sh);
            const unsigned __int128 rem = mag - ((unsigned __int128)q << sh);
            const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
            if (rem > half || (rem == half && (q & 1))) ++q;
            if (q == (1ull << 24)) { q >>= 1; ++E; }
        }
        if (E > 127) return neg ? -__int_as_float(0x7f800000) : __int_as_float(0x7f800000);
        bits = ((uint32_t)(E + 127) << 23) | ((uint32_t)q & ((1u << 23) - 1));
    }
    if (neg) bits |= 1u << 31;
    return __int_as_float((int)bits);
}

__device__ __forceinline__ double t_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float t_add(float a, float b) { return __fadd_rn(a, b); }

template <typename T>
__device__ __forceinline__ T quiet_nan();
template <>
__device__ __forceinline__ double quiet_nan<double>() { return __longlong_as_double(0x7ff8000000000000ll); }
template <>
__device__ __forceinline__ float quiet_nan<float>() { return __int_as_float(0x7fc00000); }

template <typename T>
__device__ __forceinline__ T inf_of(bool neg);
template <>
__device__ __forceinline__ double inf_of<double>(bool neg) {
    return __longlong_as_double(neg ? (long long)0xfff0000000000000ull : 0x7ff0000000000000ll);
}
template <>
__device__ __forceinline__ float inf_of<float>(bool neg) {
    return __int_as_float(neg ? (int)0xff800000u : 0x7f800000);
}

// ------------------------------------------------- per-group state helpers

__device__ __forceinline__ bool header_ok(const StateView& st, int dtype) {
    const repro_state_header* h = st.header();
    return h->magic == REPRO_STATE_MAGIC && h->dtype == (uint32_t)dtype && h->L == (uint32_t)st.L &&
           h->num_groups == st.G;
}

// One thread per CTA checks the header(s); a mismatch marks the state and
// makes every thread of the CTA return.
__device__ __forceinline__ bool cta_header_ok(const StateView& a, int dtype, const StateView* b = nullptr) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = header_ok(a, dtype);
        if (b && !header_ok(*b, dtype)) ok = 0;
        if (!ok) atomicOr(&a.header()->errors, REPRO_ERR_LAYOUT);
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ void state_init_header(const StateView& st, int dtype) {
    repro_state_header* h = st.header();
    h->magic = REPRO_STATE_MAGIC;
    h->dtype = (uint32_t)dtype;
    h->L = (uint32_t)st.L;
    h->errors = 0;
    h->num_groups = st.G;
    for (int i = 0; i < 40; ++i) h->reserved[i] = 0;
}

// The result of one group (eq. (1)): the special values first, else
// V_j = RN(T_j u_j) folded from the lowest level up, left-associative.
template <typename T>
__device__ __forceinline__ T state_finalize_group(const StateView& st, long long g) {
    constexpr int W = Traits<T>::W, GMIN = Traits<T>::GMIN;
    const unsigned f = *st.flags(g);
    if ((f & (REPRO_FLAG_NAN | REPRO_FLAG_RANGE)) || ((f & REPRO_FLAG_POS_INF) && (f & REPRO_FLAG_NEG_INF)))
        return quiet_nan<T>();
    if (f & REPRO_FLAG_POS_INF) return inf_of<T>(false);
    if (f & REPRO_FLAG_NEG_INF) return inf_of<T>(true);
    const int K = *st.K(g);
    bool first = true;
    T q = (T)0;
    for (int j = st.L - 1; j >= 0; --j) {
        if (K - j < 0) continue;
        const __int128 t = bin_read(st.lo(g, j), st.hi(g, j));
        const bool neg = t < 0;
        const unsigned __int128 mag = neg ? (unsigned __int128)(-t) : (unsigned __int128)t;
        const T v = round_scaled<T>(neg, mag, GMIN + (K - j) * W);
        q = first ? v : t_add(q, v);
        first = false;
    }
    return q;
}

}  // namespace rp
