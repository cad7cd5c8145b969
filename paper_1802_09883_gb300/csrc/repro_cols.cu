// repro_cols.cu -- a value column and its square over one key stream in one
// pass.
//
// k_fused_cols is the single-pass kernel of repro_fused.cu for NV value
// columns that share one key column; it is built for one column and its
// square (the sums of x and x*x behind VARIANCE / STDDEV, Sec. I).  (Built
// for four plain columns -- the few-group multi-column aggregate of the
// paper's TPC-H Q1 experiment, Sec. VI -- it measured slower than one
// single pass per column: 1.09 vs 0.96 ms for four float columns over 4
// groups.)  The producer warp stages a tile of keys and
// of every column; the consumers walk the tile once per column, each column
// with its own table, windows and raise list (Algorithm 2 per column, exact
// integer bins), so per tile the keys, the TMA traffic and the tile
// bookkeeping are shared.  With SQUARE the second ring is filled by the
// consumers: each thread squares exactly the rows it will consume, so no
// barrier is needed between writing and reading them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "fused_device.cuh"
#include "repro_internal.h"

namespace rp {
namespace {

constexpr int kColsMax = 4;

struct ColsArgs {
    const int32_t* keys;
    const void* vals[kColsMax];  // SQUARE: vals[0] only
    long long n;
    int G, R, S, C;
    long long ntiles;
    int tiles_per_cta;
    long long flush_rows;
    unsigned char* partials;     // [NV][gridDim.x][G] records of 8 + 16 L bytes
    unsigned* errors[kColsMax];  // each state's header error word
};

struct ColsSmem {
    size_t bars, ctl, keys, vals, bins, K, Kp, F, dlist, slist, rlist, total;
    size_t ring, bins_col, grp_col;  // bytes of one value ring, one column's bins, one column's K (or Kp, F)
};

template <typename T>
__host__ __device__ inline ColsSmem cols_layout(int S, int R, int G, int L, int C, int NV) {
    ColsSmem m;
    size_t o = 0;
    m.bars = o;
    o += 16 * (size_t)S;
    m.ctl = o;
    o += 64;
    o = align_up(o, 128);
    m.keys = o;
    o += (size_t)S * R * 4;
    o = align_up(o, 128);
    m.ring = align_up((size_t)S * R * sizeof(T), 128);
    m.vals = o;
    o += m.ring * NV;
    m.bins_col = (size_t)(G + 1) * (L + 2) * C * 8;  // padded as the single-pass tables
    m.bins = o;
    o += m.bins_col * NV;
    m.grp_col = (size_t)G * 4;
    m.K = o;
    o += m.grp_col * NV;
    m.Kp = o;
    o += m.grp_col * NV;
    m.F = o;
    o += m.grp_col * NV;
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

// CC: copies of each column's table (a.C), fixed at compile time.
template <typename T, int L, int NCW, int NV, bool SQUARE, int CC>
__global__ void __launch_bounds__(32 * (NCW + 1)) k_fused_cols(ColsArgs a) {
    constexpr int NC = 32 * NCW;
    extern __shared__ __align__(128) unsigned char smem[];
    const ColsSmem m = cols_layout<T>(a.S, a.R, a.G, L, a.C, NV);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + m.bars);
    uint64_t* empty = full + a.S;
    int* ctl = reinterpret_cast<int*>(smem + m.ctl);  // cnt[3][2] at 0..5, abort at 6, slow counts[3] at 8..10
    int32_t* skeys = reinterpret_cast<int32_t*>(smem + m.keys);
    unsigned short* dlist = reinterpret_cast<unsigned short*>(smem + m.dlist);
    unsigned short* slist = reinterpret_cast<unsigned short*>(smem + m.slist);
    int* rlist = reinterpret_cast<int*>(smem + m.rlist);
    volatile int* abort_flag = &ctl[6];
    const int tid = threadIdx.x;
    const int G = a.G, R = a.R, S = a.S;
    auto ring = [&](int c) { return reinterpret_cast<T*>(smem + m.vals + m.ring * c); };
    auto table = [&](int c) {
        Table t;
        t.lo = reinterpret_cast<unsigned*>(smem + m.bins + m.bins_col * c);
        t.hi = reinterpret_cast<int*>(t.lo + (size_t)(G + 1) * (L + 2) * a.C);
        t.L = L + 2;  // level stride of the padded table
        t.C = a.C;
        return t;
    };
    auto colK = [&](int c) { return reinterpret_cast<int*>(smem + m.K + m.grp_col * c); };
    auto colKp = [&](int c) { return reinterpret_cast<int*>(smem + m.Kp + m.grp_col * c); };
    auto colF = [&](int c) { return reinterpret_cast<unsigned*>(smem + m.F + m.grp_col * c); };

    for (int i = tid; i < (int)(m.bins_col * NV / 4); i += blockDim.x)
        reinterpret_cast<unsigned*>(smem + m.bins)[i] = 0;
    for (int i = tid; i < G * NV; i += blockDim.x) {
        reinterpret_cast<int*>(smem + m.K)[i] = kNoWindow;
        reinterpret_cast<int*>(smem + m.Kp)[i] = kNoWindow;
        reinterpret_cast<unsigned*>(smem + m.F)[i] = 0;
    }
    if (tid < 16) ctl[tid] = 0;
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
    constexpr int NLOAD = SQUARE ? 1 : NV;  // columns the producer copies

    if (tid >= NC) {
        // ---------------------------------------------------------- producer
        if (tid == NC) {
            const uint32_t kb = (uint32_t)R * 4, vb = (uint32_t)R * sizeof(T);
            int issued = 0;
            int s = 0;  // i mod S and the parity of the ring round i / S, kept without divisions
            uint32_t par = 0;
            for (int i = 0; i < ntile; ++i) {
                if (i >= S && !mbar_wait_bounded(&empty[s], par ^ 1u, kWaitNs)) {
                    for (int c = 0; c < NV; ++c) atomicOr(a.errors[c], REPRO_ERR_TIMEOUT);
                    break;
                }
                const long long row0 = (t0 + i) * (long long)R;
                mbar_arrive_expect_tx(&full[s], kb + vb * NLOAD);
                bulk_g2s(skeys + (size_t)s * R, a.keys + row0, kb, &full[s]);
                for (int c = 0; c < NLOAD; ++c)
                    bulk_g2s(ring(c) + (size_t)s * R, static_cast<const T*>(a.vals[c]) + row0, vb, &full[s]);
                ++issued;
                if (++s == S) {
                    s = 0;
                    par ^= 1u;
                }
            }
            for (int i = max(0, issued - S); i < issued; ++i)
                if (!mbar_wait_bounded(&full[i % S], (i / S) & 1, kWaitNs)) break;
        }
        return;
    }

    // -------------------------------------------------------------- consumers
    const int ctid = tid;
    const int copy = (ctid & 31) & (a.C - 1);
    bool bad_key = false;
    bool first_flush = true;
    long long rows_since_flush = 0;
    int tcount = 0;  // column passes done (counter buffer index)
    const size_t rec = 8 + 16 * (size_t)L;
    auto flush_all = [&]() {
        named_bar_sync(1, NC);
        for (int c = 0; c < NV; ++c)
            flush_partial<L>(a.partials + ((size_t)c * gridDim.x + blockIdx.x) * G * rec, G, table(c), colK(c),
                             colF(c), first_flush, ctid, NC);
        first_flush = false;
        named_bar_sync(1, NC);
    };
    // one column over the rows of a staged tile (or the tail), then its raises
    auto column_pass = [&](int c, const int32_t* tk, const T* tv, int rows, bool staged) {
        int* cnt = &ctl[2 * (tcount % 3)];
        int* scnt = &ctl[8 + tcount % 3];
        const Table tab = table(c);
        int* sK = colK(c);
        int* sKp = colKp(c);
        unsigned* sF = colF(c);
        if (staged) {
            SAddr sa;
            sa.K = smem_addr(sK);
            sa.lo = smem_addr(tab.lo);
            sa.hi = smem_addr(tab.hi);
            sa.keys = smem_addr(tk);
            sa.vals = smem_addr(tv);
            for (int r = 4 * ctid; r < rows; r += 4 * NC)
                consume_quad_fast<T, L, CC, 2>(sa, tk, tv, sK, r, G, G, copy, slist, smem_addr(scnt));
        } else {
            for (int r = ctid; r < rows; r += NC)
                consume_row<T, L>(tk[r], tv[r], r, G, tab, copy, sK, sKp, sF, dlist, rlist, cnt, bad_key);
        }
        named_bar_sync(1, NC);
        if (ctid == 0) {  // the counters of the pass before are no longer read
            const int p = (tcount + 2) % 3;
            ctl[2 * p] = 0;
            ctl[2 * p + 1] = 0;
            ctl[8 + p] = 0;
        }
        const int ns = *scnt;
        if (ns > 0) {  // the pass's unusual rows, one by one (claims, flags, deferrals)
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
        ++tcount;
    };

    int s = 0;  // the tile's stage and the parity of its ring round, kept without divisions
    uint32_t par = 0;
    for (int i = 0; i < ntile; ++i) {
        if (rows_since_flush + R > a.flush_rows) {
            flush_all();
            rows_since_flush = 0;
        }
        const bool ok = mbar_wait_bounded(&full[s], par, kWaitNs);
        if (!ok) {
            *abort_flag = 1;
            for (int c = 0; c < NV; ++c) atomicOr(a.errors[c], REPRO_ERR_TIMEOUT);
        }
        named_bar_sync(1, NC);
        if (*abort_flag) break;
        const int32_t* tk = skeys + (size_t)s * R;
        if (SQUARE) {  // each thread squares the rows its quads will read
            const T* x = ring(0) + (size_t)s * R;
            T* x2 = ring(1) + (size_t)s * R;
            for (int r = 4 * ctid; r < R; r += 4 * NC)
#pragma unroll
                for (int q = 0; q < 4; ++q) x2[r + q] = x[r + q] * x[r + q];
        }
#pragma unroll 1
        for (int c = 0; c < NV; ++c) column_pass(c, tk, ring(c) + (size_t)s * R, R, true);
        __syncwarp();
        if ((ctid & 31) == 0) mbar_arrive(&empty[s]);
        rows_since_flush += R;
        if (++s == S) {
            s = 0;
            par ^= 1u;
        }
    }

    // ragged tail (n mod R rows), read from global memory by the last CTA
    const long long tail0 = a.ntiles * (long long)R;
    if (!*abort_flag && blockIdx.x == gridDim.x - 1 && tail0 < a.n) {
        const int rows = (int)(a.n - tail0);
        if (rows_since_flush + rows > a.flush_rows) flush_all();
        const int32_t* tk = a.keys + tail0;
        if (SQUARE) {  // the tail's squares go to the second ring's stage 0 (no stage is in flight now)
            const T* x = static_cast<const T*>(a.vals[0]) + tail0;
            T* x2 = ring(1);
            for (int r = ctid; r < rows; r += NC) x2[r] = x[r] * x[r];
            named_bar_sync(1, NC);
            column_pass(0, tk, x, rows, false);
            column_pass(1, tk, x2, rows, false);
        } else {
#pragma unroll 1
            for (int c = 0; c < NV; ++c) column_pass(c, tk, static_cast<const T*>(a.vals[c]) + tail0, rows, false);
        }
    }
    if (__any_sync(0xffffffffu, bad_key) && (ctid & 31) == 0)
        for (int c = 0; c < NV; ++c) atomicOr(a.errors[c], REPRO_ERR_KEY);
    named_bar_sync(1, NC);
    if (*abort_flag) return;
    for (int c = 0; c < NV; ++c)
        flush_partial<L>(a.partials + ((size_t)c * gridDim.x + blockIdx.x) * G * rec, G, table(c), colK(c), colF(c),
                         first_flush, ctid, NC);
}

template <typename T, int L, int NV, bool SQ>
const void* cols_kernel(int C) {
    return C == 32 ? (const void*)k_fused_cols<T, L, 8, NV, SQ, 32> : (const void*)k_fused_cols<T, L, 8, NV, SQ, 1>;
}

template <typename T, int NV, bool SQ>
const void* cols_kernel_L(int L, int C) {
    switch (L) {
        case 1: return cols_kernel<T, 1, NV, SQ>(C);
        case 2: return cols_kernel<T, 2, NV, SQ>(C);
        case 3: return cols_kernel<T, 3, NV, SQ>(C);
        default: return cols_kernel<T, 4, NV, SQ>(C);
    }
}

// The kernels built: x with x*x.
const void* cols_kernel_of(int dtype, int L, int C) {
    return dtype == REPRO_F64 ? cols_kernel_L<double, 2, true>(L, C) : cols_kernel_L<float, 2, true>(L, C);
}

size_t cols_smem(int dtype, int L, int G, int NV, const FusedPlanConfig& c) {
    return dtype == REPRO_F64 ? cols_layout<double>(c.S, c.R, G, L, c.copies, NV).total
                              : cols_layout<float>(c.S, c.R, G, L, c.copies, NV).total;
}

// Stages 2-3, tiles of 1024 or 2048 rows, 8 consumer warps; the most CTAs
// per SM whose shared memory fits, lane-private table copies when they fit.
bool cols_config(int dtype, int L, long long G, int NV, FusedPlanConfig& cfg) {
    if (G > 65535) return false;
    const DeviceInfo& di = device_info();
    bool found = false;
    for (int copies : {32, 1}) {
        if (copies == 32 && G > 256) continue;
        for (int cps = 4; cps >= 1 && !found; --cps)
            for (int R : {2048, 1024})
                for (int S : {3, 2}) {
                    if (found) break;
                    const FusedPlanConfig c{S, R, 8, cps, copies};
                    const size_t b = cols_smem(dtype, L, (int)G, NV, c);
                    if (b <= di.smem_optin && (b + 1024) * cps <= di.smem_per_sm) {
                        cfg = c;
                        found = true;
                    }
                }
        if (found) return true;
    }
    return false;
}

int cols_ctas(long long ntiles, const FusedPlanConfig& cfg, int resident) {
    long long c = (long long)device_info().sms * std::min(cfg.ctas_per_sm, resident);
    c = std::min(c, (ntiles + 15) / 16);
    return (int)std::max(1ll, c);
}

template <typename T, int L, int NV, bool SQ>
void launch_t(const ColsArgs& a, int ctas, size_t smem, cudaStream_t s) {
    if (a.C == 32) k_fused_cols<T, L, 8, NV, SQ, 32><<<ctas, 32 * 9, smem, s>>>(a);
    else k_fused_cols<T, L, 8, NV, SQ, 1><<<ctas, 32 * 9, smem, s>>>(a);
}

template <typename T, int NV, bool SQ>
void launch_L(int L, const ColsArgs& a, int ctas, size_t smem, cudaStream_t s) {
    switch (L) {
        case 1: launch_t<T, 1, NV, SQ>(a, ctas, smem, s); break;
        case 2: launch_t<T, 2, NV, SQ>(a, ctas, smem, s); break;
        case 3: launch_t<T, 3, NV, SQ>(a, ctas, smem, s); break;
        default: launch_t<T, 4, NV, SQ>(a, ctas, smem, s); break;
    }
}

template <typename T>
void launch_any(int L, const ColsArgs& a, int ctas, size_t smem, cudaStream_t s) {
    launch_L<T, 2, true>(L, a, ctas, smem, s);
}

}  // namespace

// Worth it only while the columns' tables and rings still leave three CTAs
// per SM: the per-column work is issue-bound, so occupancy matters more than
// the shared key stream (measured: two columns at one CTA per SM ran slower
// than two single-column passes).
constexpr int kColsMinCtasPerSm = 3;

bool cols_supported(int dtype, int L, long long G, int NV, const int32_t* keys, const void* const* vals) {
    if (NV != 2) return false;  // a column and its square only
    if ((uintptr_t)keys % 16) return false;
    for (int c = 0; c < NV; ++c)
        if ((uintptr_t)vals[c] % 16) return false;
    FusedPlanConfig cfg;
    return cols_config(dtype, L, G, NV, cfg) && cfg.ctas_per_sm >= kColsMinCtasPerSm;
}

size_t cols_scratch_bytes(int dtype, int L, long long G, int NV, long long n) {
    FusedPlanConfig cfg;
    if (!cols_config(dtype, L, G, NV, cfg)) return 0;
    return (size_t)NV * cols_ctas(n / cfg.R, cfg, cfg.ctas_per_sm) * (size_t)G * (8 + 16 * (size_t)L);
}

cudaError_t launch_groupby_cols(const int32_t* keys, const void* const* vals, int NV, bool square, long long n,
                                int dtype, int L, long long G, void* const* states, void* scratch, cudaStream_t s) {
    if (!square || NV != 2) return cudaErrorInvalidValue;
    const int nv = 2;
    FusedPlanConfig cfg;
    if (!cols_config(dtype, L, G, nv, cfg)) return cudaErrorInvalidValue;
    const size_t smem = cols_smem(dtype, L, (int)G, nv, cfg);
    const int resident = resident_ctas(cols_kernel_of(dtype, L, cfg.copies), 32 * 9, smem);
    if (resident < 1) return cudaErrorInvalidConfiguration;
    ColsArgs a{};
    a.keys = keys;
    a.vals[0] = vals[0];
    a.n = n;
    a.G = (int)G;
    a.R = cfg.R;
    a.S = cfg.S;
    a.C = cfg.copies;
    a.ntiles = n / cfg.R;
    const int ctas = cols_ctas(a.ntiles, cfg, resident);
    a.tiles_per_cta = (int)((a.ntiles + ctas - 1) / ctas);
    a.flush_rows = 1ll << 23;
    a.partials = (unsigned char*)scratch;
    for (int c = 0; c < nv; ++c) a.errors[c] = &reinterpret_cast<repro_state_header*>(states[c])->errors;
    prof_begin(PROF_FUSED, s);
    if (dtype == REPRO_F64) launch_any<double>(L, a, ctas, smem, s);
    else launch_any<float>(L, a, ctas, smem, s);
    prof_end(PROF_FUSED, s);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    const size_t part = (size_t)ctas * G * (8 + 16 * (size_t)L);
    for (int c = 0; c < nv && e == cudaSuccess; ++c)
        e = launch_merge_partials((unsigned char*)scratch + part * c, ctas, G, states[c], dtype, L, s);
    return e;
}

}  // namespace rp
