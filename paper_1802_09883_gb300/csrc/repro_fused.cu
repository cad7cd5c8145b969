// repro_fused.cu -- single-pass reproducible grouped SUM for group tables
// that fit in shared memory.
//
// One read of the rows.  Each persistent CTA owns a contiguous range of
// tiles; a producer warp streams key/value tiles into a ring of shared-memory
// stages with 1-D TMA bulk copies (cp.async.bulk + mbarrier), and the
// consumer warps turn every row into at most three integer digits added with
// shared-memory atomics into a CTA-private table repro<T,L>[G].
//
// Windows are CTA-local (Algorithm 2's level raising, done per tile): a row
// whose top grid index K(b) exceeds its group's current CTA window is
// deferred; after the tile the CTA raises the windows of those groups
// (shifting their bins, dropping levels that fall off the bottom) and adds
// the deferred rows.  Digits are the same in every window that can hold the
// value, so rows added before a raise stay correct.  At the end each CTA
// writes its table as a partial state; k_merge_partials aligns and adds the
// partials into the caller's state (operator+=(repro), Algorithm 4's merge).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "fused_device.cuh"
#include "repro_internal.h"

namespace rp {

namespace {

struct FusedArgs {
    const int32_t* keys;
    const void* vals;
    long long n;
    int G;
    int R;             // rows per tile
    int S;             // stages
    int C;             // copies of the table (1, or 32 for lane-private copies)
    long long ntiles;  // full tiles (n / R)
    int tiles_per_cta;
    long long flush_rows;     // flush the int64 table into the partial before this many rows
    unsigned char* partials;  // [gridDim.x][G] records of 8 + 16 L bytes
    unsigned* errors;         // state header error word
    unsigned long long wait_ns;  // limit of every mbarrier wait
    int stall_tile;           // failure injection: the producer issues no tile from this index on (-1: off)
};

}  // namespace

// SQ: sum x*x instead of x (each staged value squared in place, RN in T, by
// the thread that consumes it; the sums behind VARIANCE / STDDEV).
// CC: copies of the table (a.C), fixed at compile time for the hot loop.
template <typename T, int L, int NCW, bool SQ, int CC>
__global__ void __launch_bounds__(32 * (NCW + 1), NCW == 8 ? 4 : (NCW == 16 ? 2 : 1)) k_fused(FusedArgs a) {
    constexpr int NC = 32 * NCW;
    extern __shared__ __align__(128) unsigned char smem[];
    const FusedSmem m = fused_layout<T>(a.S, a.R, a.G, L, a.C);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + m.bars);
    uint64_t* empty = full + a.S;
    int* ctl = reinterpret_cast<int*>(smem + m.ctl);  // cnt[3][2] at 0..5, abort at 6, slow counts[3] at 8..10
    int32_t* skeys = reinterpret_cast<int32_t*>(smem + m.keys);
    T* svals = reinterpret_cast<T*>(smem + m.vals);
    Table tab;
    tab.lo = reinterpret_cast<unsigned*>(smem + m.bins);
    tab.hi = reinterpret_cast<int*>(tab.lo + (size_t)(a.G + 1) * (L + 2) * a.C);
    tab.L = L + 2;  // level stride of the padded table (levels L, L + 1 and group G are spare)
    tab.C = a.C;
    int* sK = reinterpret_cast<int*>(smem + m.K);
    int* sKp = reinterpret_cast<int*>(smem + m.Kp);
    unsigned* sF = reinterpret_cast<unsigned*>(smem + m.F);
    unsigned short* dlist = reinterpret_cast<unsigned short*>(smem + m.dlist);
    unsigned short* slist = reinterpret_cast<unsigned short*>(smem + m.slist);
    int* rlist = reinterpret_cast<int*>(smem + m.rlist);
    volatile int* abort_flag = &ctl[6];  // consumers only

    const int tid = threadIdx.x;
    const int G = a.G, R = a.R, S = a.S;
    for (int i = tid; i < (G + 1) * (L + 2) * a.C; i += blockDim.x) {
        tab.lo[i] = 0;
        tab.hi[i] = 0;
    }
    for (int g = tid; g < G; g += blockDim.x) {
        sK[g] = kNoWindow;
        sKp[g] = kNoWindow;
        sF[g] = 0;
    }
    if (tid < 16) ctl[tid] = 0;
    // without a key column every row belongs to group 0: the key ring holds
    // zeros and the producer never copies into it
    const bool keyless = a.keys == nullptr;
    if (keyless)
        for (int i = tid; i < S * R; i += blockDim.x) skeys[i] = 0;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        fence_barrier_init();
    }
    __syncthreads();

    const long long t0 = (long long)blockIdx.x * a.tiles_per_cta;
    const long long t1 = min(a.ntiles, t0 + a.tiles_per_cta);
    const int ntile = (int)max(0ll, t1 - t0);
    const T* vals = reinterpret_cast<const T*>(a.vals);

    if (tid >= NC) {
        // ---------------------------------------------------------- producer
        if (tid == NC) {
            const uint32_t kb = keyless ? 0u : (uint32_t)R * 4, vb = (uint32_t)R * sizeof(T);
            int issued = 0;
            int s = 0;         // stage of tile i (i mod S, kept without a division)
            uint32_t par = 0;  // parity of the ring round i / S
            for (int i = 0; i < ntile; ++i) {
                if (i == a.stall_tile) break;  // injected failure: the consumers' waits run out
                if (i >= S && !mbar_wait_bounded(&empty[s], par ^ 1u, a.wait_ns)) {
                    // consumers will time out on the stages never filled
                    atomicOr(a.errors, REPRO_ERR_TIMEOUT);
                    break;
                }
                const long long row0 = (t0 + i) * (long long)R;
                mbar_arrive_expect_tx(&full[s], kb + vb);
                if (!keyless) bulk_g2s(skeys + (size_t)s * R, a.keys + row0, kb, &full[s]);
                bulk_g2s(svals + (size_t)s * R, vals + row0, vb, &full[s]);
                ++issued;
                if (++s == S) {
                    s = 0;
                    par ^= 1u;
                }
            }
            // never leave with a copy in flight
            for (int i = max(0, issued - S); i < issued; ++i)
                if (!mbar_wait_bounded(&full[i % S], (i / S) & 1, a.wait_ns)) break;
        }
        return;
    }

    // -------------------------------------------------------------- consumers
    const int ctid = tid;
    const int copy = (ctid & 31) & (a.C - 1);
    SAddr sa;
    sa.K = smem_addr(sK);
    sa.lo = smem_addr(tab.lo);
    sa.hi = smem_addr(tab.hi);
    bool bad_key = false;
    bool first_flush = true;
    long long rows_since_flush = 0;
    int tcount = 0;  // tiles processed
    int c3 = 0;      // tcount mod 3: the counter buffer of this tile
    int s = 0;       // stage of tile i and the parity of its ring round, kept without divisions
    uint32_t par = 0;
    for (int i = 0; i < ntile; ++i) {
        if (rows_since_flush + R > a.flush_rows) {
            named_bar_sync(1, NC);
            flush_partial<L>(a.partials + (size_t)blockIdx.x * G * (8 + 16 * L), G, tab, sK, sF, first_flush,
                             ctid, NC);
            first_flush = false;
            rows_since_flush = 0;
            named_bar_sync(1, NC);
        }
        const bool ok = mbar_wait_bounded(&full[s], par, a.wait_ns);
        int* cnt = &ctl[2 * c3];
        int* scnt = &ctl[8 + c3];
        const int32_t* tk = skeys + (size_t)s * R;
        const T* tv = svals + (size_t)s * R;
        if (ok) {
            sa.keys = smem_addr(tk);
            sa.vals = smem_addr(tv);
            if (SQ) {  // this thread's quads, squared where they lie (read only after the barrier by others)
                T* w = svals + (size_t)s * R;
                for (int b = 128 * (ctid >> 5) + 2 * (ctid & 31); b < R; b += 128 * NCW)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int r = b + (q & 1) + (q >> 1) * 64;
                        w[r] = w[r] * w[r];
                    }
                asm volatile("" ::: "memory");  // the stores stay ahead of the quads' shared loads
            }
            // each warp takes 128-row blocks (R is a multiple of 128 NCW),
            // each lane rows 2 lane + {0, 1, 64, 65} of a block
            for (int b = 128 * (ctid >> 5) + 2 * (ctid & 31); b < R; b += 128 * NCW)
                consume_quad_fast<T, L, CC, 64>(sa, tk, tv, sK, b, G, G, copy, slist, smem_addr(scnt));
        } else {
            *abort_flag = 1;  // written before the barrier, read after it: uniform
            atomicOr(a.errors, REPRO_ERR_TIMEOUT);
        }
        named_bar_sync(1, NC);
        if (ctid == 0) {  // the counters of the tile before are no longer read
            const int p = c3 == 0 ? 2 : c3 - 1;
            ctl[2 * p] = 0;
            ctl[2 * p + 1] = 0;
            ctl[8 + p] = 0;
        }
        if (*abort_flag) break;
        const int ns = *scnt;
        if (ns > 0) {  // the tile's unusual rows, one by one (claims, flags, deferrals)
            for (int i2 = ctid; i2 < ns; i2 += NC) {
                const int r = slist[i2];
                consume_row<T, L>(tk[r], tv[r], r, G, tab, copy, sK, sKp, sF, dlist, rlist, cnt, bad_key);
            }
            named_bar_sync(1, NC);
        }
        const int nd = cnt[0], nr = cnt[1];
        if (nr > 0) {
            raise_and_add<T, L>(nr, nd, tk, tv, tab, sK, sKp, sF, dlist, rlist, ctid, NC);
            named_bar_sync(1, NC);
        }
        if (SQ) fence_proxy_async_smem();  // the squares written here before the next TMA write
        __syncwarp();
        if ((ctid & 31) == 0) mbar_arrive(&empty[s]);
        rows_since_flush += R;
        ++tcount;
        c3 = c3 == 2 ? 0 : c3 + 1;
        if (++s == S) {
            s = 0;
            par ^= 1u;
        }
    }

    // ragged tail (n mod R rows), read straight from global memory by the last CTA
    const long long tail0 = a.ntiles * (long long)R;
    if (!*abort_flag && blockIdx.x == gridDim.x - 1 && tail0 < a.n) {
        const int rows = (int)(a.n - tail0);
        if (rows_since_flush + rows > a.flush_rows) {
            named_bar_sync(1, NC);
            flush_partial<L>(a.partials + (size_t)blockIdx.x * G * (8 + 16 * L), G, tab, sK, sF, first_flush,
                             ctid, NC);
            first_flush = false;
            named_bar_sync(1, NC);
        }
        int* cnt = &ctl[2 * c3];
        const int32_t* tk = keyless ? skeys : a.keys + tail0;  // fewer than R tail rows
        const T* tv = vals + tail0;
        if (SQ) {  // the tail's squares in the (now idle) first stage
            for (int r = ctid; r < rows; r += NC) svals[r] = tv[r] * tv[r];
            named_bar_sync(1, NC);
            tv = svals;
        }
        for (int r = ctid; r < rows; r += NC)
            consume_row<T, L>(tk[r], tv[r], r, G, tab, copy, sK, sKp, sF, dlist, rlist, cnt, bad_key);
        named_bar_sync(1, NC);
        const int nd = cnt[0], nr = cnt[1];
        if (nr > 0) {
            raise_and_add<T, L>(nr, nd, tk, tv, tab, sK, sKp, sF, dlist, rlist, ctid, NC);
        }
    }
    if (__any_sync(0xffffffffu, bad_key) && (ctid & 31) == 0) atomicOr(a.errors, REPRO_ERR_KEY);
    named_bar_sync(1, NC);
    if (*abort_flag) {
        // the state is flagged; this CTA's partial adds nothing to it (rows
        // flushed before the time-out included), so the merge leaves the
        // state's bins as they were
        write_empty_partial<L>(a.partials + (size_t)blockIdx.x * G * (8 + 16 * L), G, ctid, NC);
        return;
    }
    flush_partial<L>(a.partials + (size_t)blockIdx.x * G * (8 + 16 * L), G, tab, sK, sF, first_flush, ctid, NC);
}

// state += sum of C partial tables (one record per group each), aligned to
// the largest window.  Block = 32 groups x NW warps; warps split the partials.
// G_hdr: the group count the state's header must show (the partials may
// cover only its first G groups).
template <int L>
__global__ void __launch_bounds__(256) k_merge_partials(const unsigned char* __restrict__ parts, int C, int G,
                                                        unsigned char* base, int dtype, long long G_hdr) {
    constexpr int NW = 8;
    constexpr size_t rec = 8 + 16 * L;
    StateView st{base, L, G};
    __shared__ int s_ok;
    __shared__ int sKw[NW][32];
    __shared__ unsigned sFw[NW][32];
    __shared__ long long sAcc[NW][32][L][2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        const repro_state_header* h = st.header();
        s_ok = h->magic == REPRO_STATE_MAGIC && h->dtype == (uint32_t)dtype && h->L == (uint32_t)L &&
               h->num_groups == G_hdr;
        if (!s_ok) atomicOr(&st.header()->errors, REPRO_ERR_LAYOUT);
    }
    __syncthreads();
    if (!s_ok) return;
    const long long g = (long long)blockIdx.x * 32 + lane;
    const bool valid = g < G;
    int K = 0;
    unsigned fl = 0;
    if (valid)
        for (int c = w; c < C; c += NW) {
            const unsigned char* r = parts + ((size_t)c * G + g) * rec;
            K = max(K, *reinterpret_cast<const int*>(r));
            fl |= *reinterpret_cast<const unsigned*>(r + 4);
        }
    sKw[w][lane] = K;
    sFw[w][lane] = fl;
    __syncthreads();
    int Kg = valid ? *st.K(g) : 0;
#pragma unroll
    for (int i = 0; i < NW; ++i) Kg = max(Kg, sKw[i][lane]);
    __int128 acc[L];
#pragma unroll
    for (int j = 0; j < L; ++j) acc[j] = 0;
    if (valid)
        for (int c = w; c < C; c += NW) {
            const unsigned char* r = parts + ((size_t)c * G + g) * rec;
            const int d = Kg - *reinterpret_cast<const int*>(r);
            const long long* b = reinterpret_cast<const long long*>(r + 8);
#pragma unroll
            for (int j = 0; j < L; ++j)
                if (j - d >= 0) acc[j] += bin_read(&b[2 * (j - d)], &b[2 * (j - d) + 1]);
        }
#pragma unroll
    for (int j = 0; j < L; ++j) {
        sAcc[w][lane][j][0] = (long long)(unsigned long long)acc[j];
        sAcc[w][lane][j][1] = (long long)(acc[j] >> 64);
    }
    __syncthreads();
    if (w == 0 && valid) {
        const int d = Kg - *st.K(g);
        __int128 tot[L];
#pragma unroll
        for (int j = 0; j < L; ++j) {
            tot[j] = (j - d >= 0) ? bin_read(st.lo(g, j - d), st.hi(g, j - d)) : 0;
#pragma unroll
            for (int i = 0; i < NW; ++i)
                tot[j] += (((__int128)sAcc[i][lane][j][1]) << 64) + (__int128)(unsigned long long)sAcc[i][lane][j][0];
        }
        unsigned f = *st.flags(g);
#pragma unroll
        for (int i = 0; i < NW; ++i) f |= sFw[i][lane];
#pragma unroll
        for (int j = 0; j < L; ++j) bin_write(st.lo(g, j), st.hi(g, j), tot[j]);
        *st.K(g) = Kg;
        *st.flags(g) = f;
    }
}

// ------------------------------------------------------------------ launcher

namespace {

// Whether a configuration is well formed and its layout (plus extra bytes)
// fits ctas_per_sm times into one SM's shared memory.
template <typename T>
bool config_fits(const FusedPlanConfig& c, int G, int L, const DeviceInfo& di, size_t extra, bool pad) {
    // 24 and 31 consumer warps only in the single-task kernel (pad)
    if (c.S < 1 || c.S > 8 || c.R < 1024 || c.R > 8192 || c.R % (128 * c.ncw) ||
        (c.ncw != 8 && c.ncw != 16 && !(pad && (c.ncw == 24 || c.ncw == 31))))
        return false;
    if (c.ctas_per_sm < 1 || c.ctas_per_sm > 4 || (c.copies != 1 && c.copies != 32)) return false;
    const size_t bytes = fused_layout<T>(c.S, c.R, G, L, c.copies).total + extra;
    return bytes * c.ctas_per_sm + 1024 * c.ctas_per_sm <= di.smem_per_sm && bytes <= di.smem_optin;
}

// The built-in rule: for the single-task kernel first the configuration
// the tuner measured best on most sweep cells that it fits (two stages of
// 6144 rows, 24 consumer warps, one CTA per SM: 16 and 1024 groups, L = 2
// and 3, 10-18 % faster than the next rule); else prefer two CTAs per SM
// (barrier bubbles of one hide behind the other), then one CTA with deeper
// staging; lane-private table copies when the 32 copies fit next to the
// stages.
template <typename T>
bool rule_config(int G, int L, const DeviceInfo& di, FusedPlanConfig& cfg, size_t extra, bool pad) {
    const FusedPlanConfig cands[] = {{2, 6144, 24, 1, 0}, {3, 2048, 8, 2, 0}, {2, 2048, 8, 2, 0}, {3, 4096, 16, 1, 0},
                                     {4, 1024, 8, 2, 0},  {4, 2048, 16, 1, 0}, {3, 2048, 16, 1, 0}, {2, 2048, 16, 1, 0},
                                     {2, 1024, 16, 1, 0}};
    for (int copies : {32, 1}) {
        if (copies == 32 && G > 256) continue;
        for (FusedPlanConfig c : cands) {
            c.copies = copies;
            if (config_fits<T>(c, G, L, di, extra, pad)) {
                cfg = c;
                return true;
            }
        }
    }
    return false;
}

const FusedPlanConfig* env_config() {
    static FusedPlanConfig forced{0, 0, 0, 0, 0};
    static std::once_flag once;
    std::call_once(once, [] {  // tuning aid: REPRO_FUSED_CFG="S,R,ncw,ctas_per_sm[,copies]"
        const char* e = getenv("REPRO_FUSED_CFG");
        if (e) {
            FusedPlanConfig c{0, 0, 0, 0, 1};
            if (sscanf(e, "%d,%d,%d,%d,%d", &c.S, &c.R, &c.ncw, &c.ctas_per_sm, &c.copies) >= 4) forced = c;
        }
    });
    return forced.S ? &forced : nullptr;
}

// forced by the tuner (this thread) > REPRO_FUSED_CFG > tuned cache > rule;
// each only if it fits.
template <typename T>
bool pick_config(int dtype, int G, int L, const DeviceInfo& di, FusedPlanConfig& cfg, size_t extra, bool pad) {
    if (const FusedPlanConfig* f = tune_forced_fused())
        if (config_fits<T>(*f, G, L, di, extra, pad)) {
            cfg = *f;
            return true;
        }
    if (const FusedPlanConfig* f = env_config())
        if (config_fits<T>(*f, G, L, di, extra, pad)) {
            cfg = *f;
            return true;
        }
    FusedPlanConfig t;
    if (tune_lookup_fused(dtype, L, G, t) && config_fits<T>(t, G, L, di, extra, pad)) {
        cfg = t;
        return true;
    }
    return rule_config<T>(G, L, di, cfg, extra, pad);
}

long long env_flush_rows() {
    static long long v = -2;
    if (v == -2) {
        const char* e = getenv("REPRO_FLUSH_ROWS");
        v = e ? atoll(e) : -1;
    }
    return v;
}

// Test aids, read once per process: REPRO_FUSED_CTAS caps the grid (so that
// one CTA takes many rows); REPRO_WAIT_NS shortens every bounded wait and
// REPRO_STALL_TILE makes each CTA's producer stop issuing at that tile, so a
// test can make the consumers' waits run out and check REPRO_ETIMEOUT.
long long env_ll(const char* name, long long dflt) {
    const char* e = getenv(name);
    return e ? atoll(e) : dflt;
}

int env_max_ctas() {
    static const int v = (int)env_ll("REPRO_FUSED_CTAS", 0);
    return v;
}

unsigned long long env_wait_ns() {
    static const long long v = env_ll("REPRO_WAIT_NS", 0);
    return v > 0 ? (unsigned long long)v : kWaitNs;
}

// the stall applies to the first REPRO_STALL_LAUNCHES launches (default 1)
int env_stall_tile() {
    static const int v = (int)env_ll("REPRO_STALL_TILE", -1);
    static std::atomic<long long> left{env_ll("REPRO_STALL_LAUNCHES", 1)};
    if (v < 0) return -1;
    return left.fetch_sub(1) > 0 ? v : -1;
}

template <typename T, int L, int NCW, bool SQ, int CC>
cudaError_t launch_fused_t(const FusedArgs& a0, int ctas, size_t smem, cudaStream_t s) {
    auto kern = k_fused<T, L, NCW, SQ, CC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    prof_begin(PROF_FUSED, s);
    kern<<<ctas, 32 * (NCW + 1), smem, s>>>(a0);
    prof_end(PROF_FUSED, s);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T, int L, bool SQ, int CC>
cudaError_t dispatch_ncw_cc(int ncw, const FusedArgs& a, int ctas, size_t smem, cudaStream_t s) {
    if (ncw == 8) return launch_fused_t<T, L, 8, SQ, CC>(a, ctas, smem, s);
    if (ncw == 16) return launch_fused_t<T, L, 16, SQ, CC>(a, ctas, smem, s);
    if (ncw == 24) return launch_fused_t<T, L, 24, SQ, CC>(a, ctas, smem, s);
    return launch_fused_t<T, L, 31, SQ, CC>(a, ctas, smem, s);
}

template <typename T, int L, bool SQ>
cudaError_t dispatch_ncw(int ncw, const FusedArgs& a, int ctas, size_t smem, cudaStream_t s) {
    return a.C == 32 ? dispatch_ncw_cc<T, L, SQ, 32>(ncw, a, ctas, smem, s)
                     : dispatch_ncw_cc<T, L, SQ, 1>(ncw, a, ctas, smem, s);
}

template <typename T, int L, bool SQ, int CC>
const void* kernel_ncw_cc(int ncw) {
    if (ncw == 8) return (const void*)k_fused<T, L, 8, SQ, CC>;
    if (ncw == 16) return (const void*)k_fused<T, L, 16, SQ, CC>;
    if (ncw == 24) return (const void*)k_fused<T, L, 24, SQ, CC>;
    return (const void*)k_fused<T, L, 31, SQ, CC>;
}

template <typename T, int L, bool SQ>
const void* kernel_ncw(int ncw, int C) {
    return C == 32 ? kernel_ncw_cc<T, L, SQ, 32>(ncw) : kernel_ncw_cc<T, L, SQ, 1>(ncw);
}

template <typename T, bool SQ>
const void* kernel_of_sq(int L, int ncw, int C) {
    switch (L) {
        case 1: return kernel_ncw<T, 1, SQ>(ncw, C);
        case 2: return kernel_ncw<T, 2, SQ>(ncw, C);
        case 3: return kernel_ncw<T, 3, SQ>(ncw, C);
        default: return kernel_ncw<T, 4, SQ>(ncw, C);
    }
}

template <typename T>
const void* kernel_of(int L, int ncw, int C, bool square = false) {
    return square ? kernel_of_sq<T, true>(L, ncw, C) : kernel_of_sq<T, false>(L, ncw, C);
}

template <typename T, bool SQ>
cudaError_t dispatch_L_sq(int L, int ncw, const FusedArgs& a, int ctas, size_t smem, cudaStream_t s) {
    switch (L) {
        case 1: return dispatch_ncw<T, 1, SQ>(ncw, a, ctas, smem, s);
        case 2: return dispatch_ncw<T, 2, SQ>(ncw, a, ctas, smem, s);
        case 3: return dispatch_ncw<T, 3, SQ>(ncw, a, ctas, smem, s);
        default: return dispatch_ncw<T, 4, SQ>(ncw, a, ctas, smem, s);
    }
}

template <typename T>
cudaError_t dispatch_L(int L, int ncw, const FusedArgs& a, int ctas, size_t smem, cudaStream_t s,
                       bool square = false) {
    return square ? dispatch_L_sq<T, true>(L, ncw, a, ctas, smem, s) : dispatch_L_sq<T, false>(L, ncw, a, ctas, smem, s);
}

}  // namespace

bool fused_plan_config(int dtype, int L, int G, size_t extra_smem, FusedPlanConfig& cfg, bool pad) {
    return dtype == REPRO_F64 ? pick_config<double>(dtype, G, L, device_info(), cfg, extra_smem, pad)
                              : pick_config<float>(dtype, G, L, device_info(), cfg, extra_smem, pad);
}

bool fused_config_fits(int dtype, int L, int G, size_t extra_smem, const FusedPlanConfig& cfg, bool pad) {
    return dtype == REPRO_F64 ? config_fits<double>(cfg, G, L, device_info(), extra_smem, pad)
                              : config_fits<float>(cfg, G, L, device_info(), extra_smem, pad);
}

size_t fused_plan_smem(int dtype, int L, int G, const FusedPlanConfig& c) {
    return dtype == REPRO_F64 ? fused_layout<double>(c.S, c.R, G, L, c.copies).total
                              : fused_layout<float>(c.S, c.R, G, L, c.copies).total;
}

bool fused_supported(int dtype, int L, long long G, const void* keys, const void* vals, bool pad) {
    if (G > 65535) return false;
    if ((uintptr_t)keys % 16 || (uintptr_t)vals % 16) return false;
    FusedPlanConfig cfg;
    return fused_plan_config(dtype, L, (int)G, 0, cfg, pad);
}

static int fused_ctas(long long ntiles, const FusedPlanConfig& cfg, const DeviceInfo& di) {
    // at least ~16 tiles per CTA keeps the partial tables small next to the input
    long long c = (long long)di.sms * cfg.ctas_per_sm;
    const long long by_work = (ntiles + 15) / 16;
    if (by_work < c) c = by_work;
    if (c < 1) c = 1;
    return (int)c;
}

size_t fused_scratch_bytes(const FusedPlanConfig& cfg, int L, long long G, long long n) {
    const long long ntiles = n / cfg.R;
    return (size_t)fused_ctas(ntiles, cfg, device_info()) * (size_t)G * (8 + 16 * (size_t)L);
}

cudaError_t launch_groupby_fused(const int32_t* keys, const void* vals, long long n, int dtype, int L, long long G,
                                 const FusedPlanConfig& cfg, void* state, void* scratch, cudaStream_t s,
                                 int max_ctas, bool square, long long G_hdr) {
    if (G_hdr <= 0) G_hdr = G;
    const DeviceInfo& di = device_info();
    if (!fused_config_fits(dtype, L, (int)G, 0, cfg, true)) return cudaErrorInvalidValue;
    FusedArgs a;
    a.keys = keys;
    a.vals = vals;
    a.n = n;
    a.G = (int)G;
    a.R = cfg.R;
    a.S = cfg.S;
    a.C = cfg.copies;
    a.ntiles = n / cfg.R;
    const size_t smem = dtype == REPRO_F64 ? fused_layout<double>(cfg.S, cfg.R, (int)G, L, cfg.copies).total
                                           : fused_layout<float>(cfg.S, cfg.R, (int)G, L, cfg.copies).total;
    // a persistent grid must be resident at once: never more CTAs per SM than
    // registers and shared memory allow
    const void* kern =
        dtype == REPRO_F64 ? kernel_of<double>(L, cfg.ncw, cfg.copies, square) : kernel_of<float>(L, cfg.ncw, cfg.copies, square);
    const int occ = resident_ctas(kern, 32 * (cfg.ncw + 1), smem);
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int ctas = fused_ctas(a.ntiles, cfg, di);
    ctas = std::min(ctas, di.sms * std::min(occ, cfg.ctas_per_sm));
    if (max_ctas > 0 && ctas > max_ctas) ctas = max_ctas;
    if (env_max_ctas() > 0 && ctas > env_max_ctas()) ctas = env_max_ctas();
    a.tiles_per_cta = (int)((a.ntiles + ctas - 1) / ctas);
    const long long fr = env_flush_rows();
    a.flush_rows = fr > 0 ? fr : (1ll << 23);
    a.partials = (unsigned char*)scratch;
    a.errors = &reinterpret_cast<repro_state_header*>(state)->errors;
    a.wait_ns = env_wait_ns();
    a.stall_tile = env_stall_tile();
    cudaError_t e = dtype == REPRO_F64 ? dispatch_L<double>(L, cfg.ncw, a, ctas, smem, s, square)
                                       : dispatch_L<float>(L, cfg.ncw, a, ctas, smem, s, square);
    if (e != cudaSuccess) return e;
    const int blocks = (int)((G + 31) / 32);
    prof_begin(PROF_MERGE, s);
    switch (L) {
        case 1: k_merge_partials<1><<<blocks, 256, 0, s>>>(a.partials, ctas, (int)G, (unsigned char*)state, dtype, G_hdr); break;
        case 2: k_merge_partials<2><<<blocks, 256, 0, s>>>(a.partials, ctas, (int)G, (unsigned char*)state, dtype, G_hdr); break;
        case 3: k_merge_partials<3><<<blocks, 256, 0, s>>>(a.partials, ctas, (int)G, (unsigned char*)state, dtype, G_hdr); break;
        default: k_merge_partials<4><<<blocks, 256, 0, s>>>(a.partials, ctas, (int)G, (unsigned char*)state, dtype, G_hdr); break;
    }
    prof_end(PROF_MERGE, s);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_merge_partials(const void* parts, int C, long long G, void* state, int dtype, int L,
                                  cudaStream_t s) {
    const int blocks = (int)((G + 31) / 32);
    const unsigned char* p = (const unsigned char*)parts;
    unsigned char* st = (unsigned char*)state;
    prof_begin(PROF_MERGE, s);
    switch (L) {
        case 1: k_merge_partials<1><<<blocks, 256, 0, s>>>(p, C, (int)G, st, dtype, G); break;
        case 2: k_merge_partials<2><<<blocks, 256, 0, s>>>(p, C, (int)G, st, dtype, G); break;
        case 3: k_merge_partials<3><<<blocks, 256, 0, s>>>(p, C, (int)G, st, dtype, G); break;
        default: k_merge_partials<4><<<blocks, 256, 0, s>>>(p, C, (int)G, st, dtype, G); break;
    }
    prof_end(PROF_MERGE, s);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace rp

// ------------------------------------------- entry point without allocation
//
// Some callers cannot allocate device memory while they aggregate: a host
// that has reserved all of the GPU's memory for its own buffer manager, a
// process whose allocator is owned by another runtime, or a latency-bound
// request path that must never wait on (or fail in) an allocation.  For
// them repro_groupby_sum_noalloc runs the single-pass fused path with its
// per-CTA partial tables in the fixed array below instead of pool memory.
// The array belongs to the library: every GPU that loads it keeps these
// bytes until the process exits.  Calls share it, so calls that overlap on
// the GPU (different streams, or the same array used from two threads)
// race; each call fully rewrites the part it reads, so nothing needs
// clearing between calls.

namespace rp {

constexpr size_t kStaticPartialBytes = 16u << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_static_partials[kStaticPartialBytes];

// Host-side device address of g_static_partials -- the symbol itself is
// only a host stand-in.  Looked up with the device current on every call
// that is not being captured into a CUDA graph (a new context after
// cudaDeviceReset gets a fresh address); a call under stream capture uses
// the address an earlier uncaptured call on that device looked up, and
// fails with REPRO_ECUDA if there was none.
static void* static_partials_address(cudaStream_t stream, cudaError_t& err) {
    static void* addr[64] = {};
    static std::mutex mu;
    int dev = 0;
    err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= 64) {
        err = cudaErrorInvalidDevice;
        return nullptr;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    err = cudaStreamIsCapturing(stream, &cap);
    if (err != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        err = cudaGetSymbolAddress(&p, g_static_partials);
        if (err != cudaSuccess) return nullptr;
        addr[dev] = p;
    } else if (!addr[dev]) {
        err = cudaErrorStreamCaptureUnsupported;
        return nullptr;
    }
    err = cudaSuccess;
    return addr[dev];
}

}  // namespace rp

extern "C" repro_status repro_groupby_sum_noalloc(const int32_t* keys, const void* values, int64_t n,
                                                  repro_dtype dtype, int L, int64_t num_groups, void* state,
                                                  void* stream) {
    using namespace rp;
    if (!state || (dtype != REPRO_F64 && dtype != REPRO_F32) || L < 1 || L > 4 || num_groups < 1 ||
        num_groups > INT32_MAX || n < 0)
        return REPRO_EINVAL;
    if (n > 0 && (!keys || !values)) return REPRO_EINVAL;
    if ((uintptr_t)state % 16) return REPRO_EINVAL;
    if (n == 0) return REPRO_OK;
    // only the fused path runs here: aligned inputs and a table that fits
    FusedPlanConfig cfg;
    if (!fused_supported(dtype, L, num_groups, keys, values, true) ||
        !fused_plan_config(dtype, L, (int)num_groups, 0, cfg, true))
        return REPRO_ERANGE;
    const size_t per_cta = (size_t)num_groups * (8 + 16 * (size_t)L);
    const long long max_ctas = (long long)(kStaticPartialBytes / per_cta);
    if (max_ctas < 1) return REPRO_ERANGE;
    cudaError_t e;
    void* scratch = static_partials_address((cudaStream_t)stream, e);
    if (!scratch) return REPRO_ECUDA;
    e = launch_groupby_fused(keys, values, n, dtype, L, num_groups, cfg, state, scratch, (cudaStream_t)stream,
                             (int)(max_ctas < 65535 ? max_ctas : 65535));
    return e == cudaSuccess ? REPRO_OK : REPRO_ECUDA;
}
