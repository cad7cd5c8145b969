// repro_batch.cu -- many independent reproducible grouped SUMs in one
// persistent launch.
//
// A plan (built once on the host, repro_batch_prepare) cuts every task into
// work items of whole tiles; the persistent CTAs of k_fused_multi pull items
// from a device counter, stream their tiles through the same TMA-staged
// shared-memory pipeline as the single-pass kernel, and at the end of each
// item either merge the CTA table straight into the task's state (the item
// owns the whole task) or write it as a partial that k_merge_items folds in
// afterwards (operator+=(repro), Algorithm 4's merge).  Tasks the single-pass
// table cannot hold (large G) or whose rows are not 16-byte aligned run
// through the partitioned path (or, unaligned, the two-pass path).
// repro_batch_run only launches kernels and
// copies nothing from the host, so it can be captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "batch_plan.h"
#include "fused_device.cuh"
#include "multi_types.h"
#include "repro.h"
#include "repro_internal.h"

namespace rp {

// Partial tables of one prepared plan are kept below 1 GiB where the work
// allows (larger items otherwise).
constexpr size_t kBatchPartBytes = 1ull << 30;

namespace {

__host__ __device__ constexpr size_t rec_bytes(int L) { return 8 + 16 * (size_t)L; }

__device__ __forceinline__ bool task_header_ok(const unsigned char* hdr, int dtype, int L, int G) {
    const repro_state_header* h = reinterpret_cast<const repro_state_header*>(hdr);
    return h->magic == REPRO_STATE_MAGIC && h->dtype == (uint32_t)dtype && h->L == (uint32_t)L &&
           h->num_groups == G;
}

// Deferred rows after a raise; rows at or beyond rows_tma come from global memory.
template <typename T, int L>
__device__ __forceinline__ void raise_and_add_multi(int nr, int nd, const int32_t* tk, const T* tv,
                                                    const int32_t* gk, const T* gv, int rows_tma, const Table& t,
                                                    int* sK, const int* sKp, unsigned* sF,
                                                    const unsigned short* dlist, const int* rlist, int ctid,
                                                    int NC) {
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
        const int g = r < rows_tma ? tk[r] : gk[r];
        const Split s = split_value(r < rows_tma ? tv[r] : gv[r]);
        add_row<T, L>(s, sK[g], t, g, (ctid & 31) & (t.C - 1));
    }
}

// v[j] <- v[j - d] (zero where j < d), d >= 0: one level per step with
// fixed indices, so that v stays in registers.
template <int L>
__device__ __forceinline__ void shift_levels(__int128 (&v)[L], int d) {
    for (int s = 0; s < d && s < L; ++s) {
#pragma unroll
        for (int j = L - 1; j > 0; --j) v[j] = v[j - 1];
        v[0] = 0;
    }
}

// Fold the CTA table into a record array (a partial table, or the task's
// state when the item owns the task): records are aligned to the larger
// window and their low levels dropped (operator+=(repro)); with `overwrite`
// the old content is ignored.  Clears the table for the next item.  Each
// thread takes NB groups at a time and reads their old records before it
// writes any, so that NB record reads are in flight instead of one.  With
// `hint`, every window the table reached is also raised there for the
// task's later items.
template <int L>
__device__ void flush_table(unsigned char* recs, int G, const Table& t, int* sK, int* sKp, unsigned* sF,
                            bool overwrite, int ctid, int NC, int* hint) {
    constexpr size_t rec = 8 + 16 * L;
    constexpr int NB = 2;
    for (int g0 = ctid; g0 < G; g0 += NB * NC) {
        int Ks[NB];
        unsigned Fo[NB];
        __int128 old[NB][L];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int g = g0 + b * NC;
            Ks[b] = 0;
            Fo[b] = 0;
#pragma unroll
            for (int j = 0; j < L; ++j) old[b][j] = 0;
            if (g < G && !overwrite) {
                const unsigned char* r = recs + (size_t)g * rec;
                const long long* pb = reinterpret_cast<const long long*>(r + 8);
                Ks[b] = *reinterpret_cast<const int*>(r);
                Fo[b] = *reinterpret_cast<const unsigned*>(r + 4);
#pragma unroll
                for (int j = 0; j < L; ++j) old[b][j] = bin_read(&pb[2 * j], &pb[2 * j + 1]);
            }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int g = g0 + b * NC;
            if (g >= G) continue;
            unsigned char* r = recs + (size_t)g * rec;
            long long* pb = reinterpret_cast<long long*>(r + 8);
            const int Kt = sK[g];
            if (hint && Kt >= 0) atomicMax(&hint[g], Kt);
            const int Kr = overwrite ? Kt : Ks[b];
            const int K = max(Kt, Kr);
            // table levels (all copies), aligned to K
            __int128 tab[L];
#pragma unroll
            for (int j = 0; j < L; ++j) {
                tab[j] = 0;
                for (int c = 0; c < t.C; ++c) {
                    const size_t i = t.at(g, j, c);
                    tab[j] += (__int128)table_value(t, i);
                    t.lo[i] = 0;
                    t.hi[i] = 0;
                }
            }
            // level j of the result takes level j - (K - Kt) of the table and
            // j - (K - Kr) of the old record
            shift_levels<L>(tab, K - Kt);
            shift_levels<L>(old[b], K - Kr);
            __int128 acc[L];
#pragma unroll
            for (int j = 0; j < L; ++j) acc[j] = overwrite ? tab[j] : tab[j] + old[b][j];
            const unsigned f = (sF[g] & ~kQueued) | Fo[b];
#pragma unroll
            for (int j = 0; j < L; ++j) bin_write(&pb[2 * j], &pb[2 * j + 1], acc[j]);
            *reinterpret_cast<int*>(r) = K;
            *reinterpret_cast<unsigned*>(r + 4) = f;
            sK[g] = kNoWindow;
            sKp[g] = kNoWindow;
            sF[g] = 0;
        }
    }
}

// Clear the CTA table (an item whose state header does not match is dropped).
template <int L>
__device__ void clear_table(int G, const Table& t, int* sK, int* sKp, unsigned* sF, int ctid, int NC) {
    for (int g = ctid; g < G; g += NC) {
        for (int j = 0; j < L; ++j)
            for (int c = 0; c < t.C; ++c) {
                const size_t x = t.at(g, j, c);
                t.lo[x] = 0;
                t.hi[x] = 0;
            }
        sK[g] = kNoWindow;
        sKp[g] = kNoWindow;
        sF[g] = 0;
    }
}

}  // namespace

// At most 96 registers: two 8-warp CTAs per SM, and the compiler's own
// choice for four levels otherwise grew past 110 with no gain.
// CC: copies of the table (a.C), fixed at compile time for the hot loop.
template <typename T, int L, int NCW, int CC>
__global__ void __maxnreg__(96) k_fused_multi(MultiArgs a, int dtype) {
    constexpr int NC = 32 * NCW;
    extern __shared__ __align__(128) unsigned char smem[];
    const FusedSmem m = fused_layout<T>(a.S, a.R, a.Gcap, L, a.C);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + m.bars);
    uint64_t* empty = full + a.S;
    int* ctl = reinterpret_cast<int*>(smem + m.ctl);  // cnt[3][2] at 0..5, abort at 6, slow counts[3] at 8..10
    StageMeta* meta = reinterpret_cast<StageMeta*>(smem + m.total);  // S entries
    int32_t* skeys = reinterpret_cast<int32_t*>(smem + m.keys);
    T* svals = reinterpret_cast<T*>(smem + m.vals);
    Table tab;
    tab.lo = reinterpret_cast<unsigned*>(smem + m.bins);
    tab.hi = reinterpret_cast<int*>(tab.lo + (size_t)(a.Gcap + 1) * (L + 2) * a.C);
    tab.L = L + 2;  // level stride of the padded table (levels L, L + 1 and group Gcap are spare)
    tab.C = a.C;
    int* sK = reinterpret_cast<int*>(smem + m.K);
    int* sKp = reinterpret_cast<int*>(smem + m.Kp);
    unsigned* sF = reinterpret_cast<unsigned*>(smem + m.F);
    unsigned short* dlist = reinterpret_cast<unsigned short*>(smem + m.dlist);
    unsigned short* slist = reinterpret_cast<unsigned short*>(smem + m.slist);
    int* rlist = reinterpret_cast<int*>(smem + m.rlist);
    volatile int* abort_flag = &ctl[6];

    const int tid = threadIdx.x;
    const int R = a.R, S = a.S;
    for (int i = tid; i < (a.Gcap + 1) * (L + 2) * a.C; i += blockDim.x) {
        tab.lo[i] = 0;
        tab.hi[i] = 0;
    }
    for (int g = tid; g < a.Gcap; g += blockDim.x) {
        sK[g] = kNoWindow;
        sKp[g] = kNoWindow;
        sF[g] = 0;
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

    if (tid >= NC) {
        // ------------------------------------------------------------ producer
        if (tid == NC) {
            long long i = 0;  // tiles issued by this CTA (ring position)
            int s = 0;        // i mod S and the parity of the ring round i / S, kept without divisions
            uint32_t par = 0;
            bool ok = true;
            const int nitems = a.nitems_ptr ? *a.nitems_ptr : a.nitems;
            for (;;) {
                const int w = atomicAdd(a.counter, 1);
                const bool done = w >= nitems;
                const MItem it = done ? MItem{0, 0, 0, 0, 0} : a.items[w];
                const MTask tk = a.tasks[done ? 0 : it.task];
                const long long nrows = it.row1 - it.row0;
                const long long ntile = done ? 1 : (nrows + R - 1) / R;
                for (long long t = 0; t < ntile; ++t) {
                    if (i >= S && !mbar_wait_bounded(&empty[s], par ^ 1u, kWaitNs)) {
                        ok = false;
                        break;
                    }
                    StageMeta sm;
                    if (done) {
                        sm.item = -1;
                        sm.rows = sm.rows_tma = sm.last = 0;
                        sm.row0 = 0;
                        sm.G = 0;
                        sm.first = 0;
                        sm.keys = nullptr;
                        sm.vals = nullptr;
                        sm.win = nullptr;
                        sm.hint = 0;
                    } else {
                        sm.item = w;
                        sm.row0 = it.row0 + t * R;
                        sm.rows = (int)min((long long)R, it.row1 - sm.row0);
                        sm.rows_tma = sm.rows & ~3;
                        sm.last = t == ntile - 1;
                        sm.G = tk.G;
                        sm.first = t == 0;
                        sm.keys = tk.keys + sm.row0;
                        sm.vals = reinterpret_cast<const T*>(tk.vals) + sm.row0;
                        sm.win = tk.win;
                        sm.hint = tk.hint;
                    }
                    meta[s] = sm;
                    const uint32_t kb = (uint32_t)sm.rows_tma * 4, vb = (uint32_t)sm.rows_tma * sizeof(T);
                    mbar_arrive_expect_tx(&full[s], kb + vb);
                    if (sm.rows_tma > 0) {
                        bulk_g2s(skeys + (size_t)s * R, tk.keys + sm.row0, kb, &full[s]);
                        bulk_g2s(svals + (size_t)s * R, reinterpret_cast<const T*>(tk.vals) + sm.row0, vb, &full[s]);
                    }
                    ++i;
                    if (++s == S) {
                        s = 0;
                        par ^= 1u;
                    }
                }
                if (done || !ok) break;
            }
            // never leave with a copy in flight
            for (long long k = max(0ll, i - S); k < i; ++k)
                if (!mbar_wait_bounded(&full[k % S], (uint32_t)((k / S) & 1), kWaitNs)) break;
        }
        return;
    }

    // --------------------------------------------------------------- consumers
    const int ctid = tid;
    const int copy = (ctid & 31) & (a.C - 1);
    SAddr sa;
    sa.K = smem_addr(sK);
    sa.lo = smem_addr(tab.lo);
    sa.hi = smem_addr(tab.hi);
    bool bad_key = false;
    int c3 = 0;  // the tile's counter buffer (tiles processed mod 3)
    int s = 0;   // the tile's stage and the parity of its ring round, kept without divisions
    uint32_t par = 0;
    for (;; ) {
        const bool ok = mbar_wait_bounded(&full[s], par, kWaitNs);
        if (!ok) *abort_flag = 1;  // before the barrier, read after it
        named_bar_sync(1, NC);
        if (*abort_flag) break;
        const StageMeta sm = meta[s];
        if (sm.item < 0) break;
        const int G = sm.G;
        if (sm.win && sm.first) {
            // exact windows (no row of the item raises one), or a lower bound
            // that earlier items of the task left (few rows raise one): either
            // is at most the group's final window, which is all a window
            // needs (a digit does not depend on the window it is taken in)
            if (sm.hint)
                for (int g = ctid; g < G; g += NC) sK[g] = sKp[g] = *reinterpret_cast<const volatile int*>(sm.win + g);
            else
                for (int g = ctid; g < G; g += NC) sK[g] = sKp[g] = __ldg(&sm.win[g]);
            named_bar_sync(1, NC);
        }
        int* cnt = &ctl[2 * c3];
        int* scnt = &ctl[8 + c3];
        const int32_t* tk_s = skeys + (size_t)s * R;
        const T* tv_s = svals + (size_t)s * R;
        const int32_t* gk = sm.keys;
        const T* gv = static_cast<const T*>(sm.vals);
        sa.keys = smem_addr(tk_s);
        sa.vals = smem_addr(tv_s);
        // whole 128-row blocks with a warp's loads contiguous (lane rows
        // 2 lane + {0, 1, 64, 65}), then the item's last quads
        const int full = sm.rows_tma & ~127;
        for (int b = 128 * (ctid >> 5) + 2 * (ctid & 31); b < full; b += 128 * NCW)
            consume_quad_fast<T, L, CC, 64>(sa, tk_s, tv_s, sK, b, G, a.Gcap, copy, slist, smem_addr(scnt));
        for (int r = full + 4 * ctid; r < sm.rows_tma; r += 4 * NC)
            consume_quad_fast<T, L, CC, 2>(sa, tk_s, tv_s, sK, r, G, a.Gcap, copy, slist, smem_addr(scnt));
        for (int r = sm.rows_tma + ctid; r < sm.rows; r += NC)
            consume_row<T, L>(gk[r], gv[r], r, G, tab, copy, sK, sKp, sF, dlist, rlist, cnt, bad_key);
        named_bar_sync(1, NC);
        if (ctid == 0) {  // the counters of the tile before are no longer read
            const int p = c3 == 0 ? 2 : c3 - 1;
            ctl[2 * p] = 0;
            ctl[2 * p + 1] = 0;
            ctl[8 + p] = 0;
        }
        const int ns = *scnt;
        if (ns > 0) {  // the tile's unusual staged rows, one by one (claims, flags, deferrals)
            for (int i2 = ctid; i2 < ns; i2 += NC) {
                const int r = slist[i2];
                consume_row<T, L>(tk_s[r], tv_s[r], r, G, tab, copy, sK, sKp, sF, dlist, rlist, cnt, bad_key);
            }
            named_bar_sync(1, NC);
        }
        const int nd = cnt[0], nr = cnt[1];
        if (nr > 0) {
            raise_and_add_multi<T, L>(nr, nd, tk_s, tv_s, gk, gv, sm.rows_tma, tab, sK, sKp, sF, dlist, rlist,
                                      ctid, NC);
            named_bar_sync(1, NC);
        }
        __syncwarp();
        if ((ctid & 31) == 0) mbar_arrive(&empty[s]);
        c3 = c3 == 2 ? 0 : c3 + 1;
        if (++s == S) {
            s = 0;
            par ^= 1u;
        }
        if (sm.last) {
            const MItem it = a.items[sm.item];
            const MTask tk = a.tasks[it.task];
            unsigned* errors = &reinterpret_cast<repro_state_header*>(tk.hdr)->errors;
            const bool hdr_ok = task_header_ok(tk.hdr, dtype, L, tk.G_hdr);
            if (__any_sync(0xffffffffu, bad_key) && (ctid & 31) == 0) atomicOr(errors, REPRO_ERR_KEY);
            bad_key = false;
            if (ctid == 0 && !hdr_ok) atomicOr(errors, REPRO_ERR_LAYOUT);
            unsigned char* dst = it.excl ? tk.recs : a.partials + (size_t)it.part * rec_bytes(L);
            if (hdr_ok || !it.excl)
                flush_table<L>(dst, G, tab, sK, sKp, sF, !it.excl, ctid, NC,
                               tk.hint ? const_cast<int*>(tk.win) : nullptr);
            else
                clear_table<L>(G, tab, sK, sKp, sF, ctid, NC);
            named_bar_sync(1, NC);
        }
    }
}

// state += sum of a task's partial tables; one block = 32 groups of one task,
// 8 warps splitting the partials.  Blocks at or beyond *nblks_ptr (when
// given) have nothing to do.
template <int L>
__global__ void __launch_bounds__(256) k_merge_items(const MTask* __restrict__ tasks, const MergeBlk* __restrict__ blks,
                                                     const int* nblks_ptr, const unsigned char* __restrict__ parts,
                                                     int dtype) {
    constexpr int NW = 8;
    constexpr size_t rec = 8 + 16 * L;
    __shared__ int sKw[NW][32];
    __shared__ unsigned sFw[NW][32];
    __shared__ long long sAcc[NW][32][L][2];
    if (nblks_ptr && (int)blockIdx.x >= *nblks_ptr) return;
    const MergeBlk b = blks[blockIdx.x];
    const MTask tk = tasks[b.task];
    const int G = tk.G;
    if (!task_header_ok(tk.hdr, dtype, L, tk.G_hdr)) return;  // flagged by k_fused_multi
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long g = (long long)b.g0 + lane;
    const bool valid = g < G;
    int* pK = reinterpret_cast<int*>(tk.recs + (size_t)g * rec);
    unsigned* pF = reinterpret_cast<unsigned*>(tk.recs + (size_t)g * rec + 4);
    long long* pb = reinterpret_cast<long long*>(tk.recs + (size_t)g * rec + 8);
    int K = 0;
    unsigned fl = 0;
    if (valid)
        for (int c = w; c < b.nparts; c += NW) {
            const unsigned char* r = parts + ((size_t)b.part + (size_t)c * G + g) * rec;
            K = max(K, *reinterpret_cast<const int*>(r));
            fl |= *reinterpret_cast<const unsigned*>(r + 4);
        }
    sKw[w][lane] = K;
    sFw[w][lane] = fl;
    __syncthreads();
    int Kg = valid ? *pK : 0;
#pragma unroll
    for (int i = 0; i < NW; ++i) Kg = max(Kg, sKw[i][lane]);
    __int128 acc[L];
#pragma unroll
    for (int j = 0; j < L; ++j) acc[j] = 0;
    if (valid)
        for (int c = w; c < b.nparts; c += NW) {
            const unsigned char* r = parts + ((size_t)b.part + (size_t)c * G + g) * rec;
            const int d = Kg - *reinterpret_cast<const int*>(r);
            const long long* bb = reinterpret_cast<const long long*>(r + 8);
#pragma unroll
            for (int j = 0; j < L; ++j)
                if (j - d >= 0) acc[j] += bin_read(&bb[2 * (j - d)], &bb[2 * (j - d) + 1]);
        }
#pragma unroll
    for (int j = 0; j < L; ++j) {
        sAcc[w][lane][j][0] = (long long)(unsigned long long)acc[j];
        sAcc[w][lane][j][1] = (long long)(acc[j] >> 64);
    }
    __syncthreads();
    if (w == 0 && valid) {
        const int d = Kg - *pK;
        __int128 tot[L];
#pragma unroll
        for (int j = 0; j < L; ++j) {
            tot[j] = (j - d >= 0) ? bin_read(&pb[2 * (j - d)], &pb[2 * (j - d) + 1]) : 0;
#pragma unroll
            for (int i = 0; i < NW; ++i)
                tot[j] += (((__int128)sAcc[i][lane][j][1]) << 64) + (__int128)(unsigned long long)sAcc[i][lane][j][0];
        }
        unsigned f = *pF;
#pragma unroll
        for (int i = 0; i < NW; ++i) f |= sFw[i][lane];
#pragma unroll
        for (int j = 0; j < L; ++j) bin_write(&pb[2 * j], &pb[2 * j + 1], tot[j]);
        *pK = Kg;
        *pF = f;
    }
}

// Host launchers shared with the partitioned path.
cudaError_t launch_multi(int dtype, int L, const FusedPlanConfig& cfg, int gcap, const void* tasks, const void* items,
                         int nitems, const int* nitems_ptr, int* counter, void* partials, int ctas, cudaStream_t s);
cudaError_t launch_merge_items(int L, int dtype, const void* tasks, const void* blks, int nblks, const int* nblks_ptr,
                               const void* partials, cudaStream_t s);

// ---------------------------------------------------------------------- plan

namespace {

template <typename T, int L, int NCW, int CC>
cudaError_t launch_multi_t(const MultiArgs& a, int dtype, int ctas, size_t smem, cudaStream_t s) {
    auto kern = k_fused_multi<T, L, NCW, CC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // a persistent grid must be resident at once (items come from a counter,
    // so fewer CTAs only take longer)
    const int occ = resident_ctas((const void*)kern, 32 * (NCW + 1), smem);
    if (occ < 1) return cudaErrorInvalidConfiguration;
    ctas = std::min(ctas, device_info().sms * occ);
    prof_begin(PROF_FUSED, s);
    kern<<<ctas, 32 * (NCW + 1), smem, s>>>(a, dtype);
    prof_end(PROF_FUSED, s);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T, int L>
cudaError_t launch_multi_ncw(int ncw, const MultiArgs& a, int dtype, int ctas, size_t smem, cudaStream_t s) {
    if (a.C == 32)
        return ncw == 8 ? launch_multi_t<T, L, 8, 32>(a, dtype, ctas, smem, s)
                        : launch_multi_t<T, L, 16, 32>(a, dtype, ctas, smem, s);
    return ncw == 8 ? launch_multi_t<T, L, 8, 1>(a, dtype, ctas, smem, s)
                    : launch_multi_t<T, L, 16, 1>(a, dtype, ctas, smem, s);
}

template <typename T>
cudaError_t launch_multi_L(int L, int ncw, const MultiArgs& a, int dtype, int ctas, size_t smem, cudaStream_t s) {
    switch (L) {
        case 1: return launch_multi_ncw<T, 1>(ncw, a, dtype, ctas, smem, s);
        case 2: return launch_multi_ncw<T, 2>(ncw, a, dtype, ctas, smem, s);
        case 3: return launch_multi_ncw<T, 3>(ncw, a, dtype, ctas, smem, s);
        default: return launch_multi_ncw<T, 4>(ncw, a, dtype, ctas, smem, s);
    }
}

}  // namespace

cudaError_t launch_multi(int dtype, int L, const FusedPlanConfig& cfg, int gcap, const void* tasks, const void* items,
                         int nitems, const int* nitems_ptr, int* counter, void* partials, int ctas, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    MultiArgs a;
    a.tasks = (const MTask*)tasks;
    a.items = (const MItem*)items;
    a.nitems = nitems;
    a.nitems_ptr = nitems_ptr;
    a.counter = counter;
    a.R = cfg.R;
    a.S = cfg.S;
    a.C = cfg.copies;
    a.Gcap = gcap;
    a.partials = (unsigned char*)partials;
    const size_t smem = fused_plan_smem(dtype, L, gcap, cfg) + sizeof(StageMeta) * (size_t)cfg.S;
    return dtype == REPRO_F64 ? launch_multi_L<double>(L, cfg.ncw, a, dtype, ctas, smem, s)
                              : launch_multi_L<float>(L, cfg.ncw, a, dtype, ctas, smem, s);
}

cudaError_t launch_merge_items(int L, int dtype, const void* tasks, const void* blks, int nblks, const int* nblks_ptr,
                               const void* partials, cudaStream_t s) {
    const MTask* t = (const MTask*)tasks;
    const MergeBlk* b = (const MergeBlk*)blks;
    const unsigned char* p = (const unsigned char*)partials;
    prof_begin(PROF_MERGE, s);
    switch (L) {
        case 1: k_merge_items<1><<<nblks, 256, 0, s>>>(t, b, nblks_ptr, p, dtype); break;
        case 2: k_merge_items<2><<<nblks, 256, 0, s>>>(t, b, nblks_ptr, p, dtype); break;
        case 3: k_merge_items<3><<<nblks, 256, 0, s>>>(t, b, nblks_ptr, p, dtype); break;
        default: k_merge_items<4><<<nblks, 256, 0, s>>>(t, b, nblks_ptr, p, dtype); break;
    }
    prof_end(PROF_MERGE, s);
    count_launches(1);
    return cudaGetLastError();
}

repro_status plan_batch_host(const repro_task* tasks, int ntasks, int dtype, int L, size_t max_part_bytes,
                             HostBatch& H, int items_per_cta, const BatchClass* fixed_cfg, bool one_class) {
    if (ntasks < 0 || (ntasks > 0 && !tasks) || (dtype != REPRO_F64 && dtype != REPRO_F32) || L < 1 || L > 4)
        return REPRO_EINVAL;
    for (int t = 0; t < ntasks; ++t) {
        const repro_task& k = tasks[t];
        if (!k.state || k.n < 0 || k.num_groups < 1 || k.num_groups > INT32_MAX || (k.n > 0 && (!k.keys || !k.values)))
            return REPRO_EINVAL;
        if ((uintptr_t)k.state % 16 || (uintptr_t)k.keys % 4 || (uintptr_t)k.values % (dtype == REPRO_F64 ? 8 : 4))
            return REPRO_EINVAL;
    }
    H = HostBatch{};
    // single-pass tasks (aligned rows and a table that fits), by class
    std::vector<int> fast[kBatchClasses];
    for (int t = 0; t < ntasks; ++t) {
        const repro_task& k = tasks[t];
        if (k.n == 0) continue;
        if (fused_supported(dtype, L, k.num_groups, k.keys, k.values)) {
            int c = one_class ? kBatchClasses - 1 : 0;
            while (k.num_groups > kBatchClassBound[c]) ++c;
            fast[c].push_back(t);
            H.cls[c].gcap = std::max(H.cls[c].gcap, (int)k.num_groups);
        } else {
            H.slow.push_back(k);
            H.slow_gmax = std::max(H.slow_gmax, (long long)k.num_groups);
        }
    }
    H.tasks.resize(ntasks);
    for (int t = 0; t < ntasks; ++t)
        H.tasks[t] = MTask{tasks[t].keys, tasks[t].values, tasks[t].n, (int)tasks[t].num_groups,
                           (int)tasks[t].num_groups, (unsigned char*)tasks[t].state,
                           (unsigned char*)tasks[t].state + sizeof(repro_state_header), nullptr, 0, 0};
    long long tpi0[kBatchClasses] = {};
    long long tpi_max[kBatchClasses] = {};
    for (int c = 0; c < kBatchClasses; ++c) {
        BatchClass& B = H.cls[c];
        if (fast[c].empty()) continue;
        if (fixed_cfg && fixed_cfg[c].cfg.S) {
            if (!fused_config_fits(dtype, L, B.gcap, kMetaSmemBytes, fixed_cfg[c].cfg)) return REPRO_ERANGE;
            B.cfg = fixed_cfg[c].cfg;
        } else if (!fused_plan_config(dtype, L, B.gcap, kMetaSmemBytes, B.cfg)) {
            return REPRO_ERANGE;
        }
        const int R = B.cfg.R;
        long long total_tiles = 0;
        for (int t : fast[c]) total_tiles += (tasks[t].n + R - 1) / R;
        B.ctas = device_info().sms * B.cfg.ctas_per_sm;
        tpi_max[c] = (1ll << 23) / R;
        const long long per = (long long)std::max(1, items_per_cta) * B.ctas;
        tpi0[c] = std::max(8ll, std::min((total_tiles + per - 1) / per, tpi_max[c]));
    }
    // items grow (all classes alike) while the partial tables would exceed max_part_bytes
    auto tpi_of = [&](int c, long long f) { return std::min(tpi_max[c], tpi0[c] * f); };
    auto part_records = [&](long long f) {
        long long part = 0;
        for (int c = 0; c < kBatchClasses; ++c)
            for (int t : fast[c]) {
                const long long R = H.cls[c].cfg.R, tp = tpi_of(c, f);
                const long long nit = ((tasks[t].n + R - 1) / R + tp - 1) / tp;
                if (nit > 1) part += nit * tasks[t].num_groups;
            }
        return part;
    };
    long long f = 1;
    auto can_grow = [&]() {
        for (int c = 0; c < kBatchClasses; ++c)
            if (!fast[c].empty() && tpi_of(c, f) < tpi_max[c]) return true;
        return false;
    };
    while (can_grow() && (size_t)part_records(f) * batch_rec_bytes(L) > max_part_bytes) f *= 2;
    long long part = 0;
    for (int c = 0; c < kBatchClasses; ++c) {
        BatchClass& B = H.cls[c];
        B.item0 = (int)H.items.size();
        if (fast[c].empty()) continue;
        const long long R = B.cfg.R, tpi = tpi_of(c, f);
        for (int t : fast[c]) {
            const long long ntile = (tasks[t].n + R - 1) / R;
            const long long nit = (ntile + tpi - 1) / tpi;
            const int G = (int)tasks[t].num_groups;
            for (long long k = 0; k < nit; ++k) {
                MItem it;
                it.task = t;
                it.excl = nit == 1;
                it.row0 = k * tpi * R;
                it.row1 = std::min<long long>(tasks[t].n, (k + 1) * tpi * R);
                it.part = nit == 1 ? -1 : part + k * G;
                H.items.push_back(it);
            }
            if (nit > 1) {
                for (int g0 = 0; g0 < G; g0 += 32) H.blks.push_back(MergeBlk{t, g0, (int)nit, 0, part});
                part += nit * G;
            }
        }
        B.nitems = (int)H.items.size() - B.item0;
        B.ntasks = (int)fast[c].size();
        // largest items first: the dynamic schedule then balances the tail
        std::stable_sort(H.items.begin() + B.item0, H.items.end(),
                         [](const MItem& x, const MItem& y) { return x.row1 - x.row0 > y.row1 - y.row0; });
    }
    H.part_recs = part;
    return REPRO_OK;
}

// One launch re-initialises every task's state (grid.y = task).
__global__ void k_batch_init(const MTask* __restrict__ tasks, int task0, int dtype, int L) {
    const MTask t = tasks[task0 + blockIdx.y];
    const StateView st{t.hdr, L, t.G_hdr};
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid == 0) state_init_header(st, dtype);
    // all-zero records, cleared as one flat range (states are 16-byte aligned)
    const unsigned long long bytes = (unsigned long long)t.G_hdr * (8ull + 16ull * (unsigned long long)L);
    uint4* rec = reinterpret_cast<uint4*>(t.hdr + sizeof(repro_state_header));
    for (long long i = tid; i < (long long)(bytes / 16); i += (long long)gridDim.x * blockDim.x)
        rec[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0 && (bytes & 15))
        *reinterpret_cast<unsigned long long*>(t.hdr + sizeof(repro_state_header) + bytes - 8) = 0ull;
}

// One launch finalizes every task with an output (eq. (1) per group).
template <typename T>
__global__ void k_batch_finalize(const MTask* __restrict__ tasks, void* const* __restrict__ outs, int task0,
                                 int dtype, int L) {
    const MTask t = tasks[task0 + blockIdx.y];
    T* out = static_cast<T*>(outs[task0 + blockIdx.y]);
    if (!out) return;
    const StateView st{t.hdr, L, t.G_hdr};
    if (!cta_header_ok(st, dtype)) return;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < t.G_hdr;
         g += (long long)gridDim.x * blockDim.x)
        out[g] = state_finalize_group<T>(st, g);
}

struct BatchPlan {
    int dtype = 0, L = 0;
    BatchClass cls[kBatchClasses];      // one persistent launch per class with tasks
    int nitems = 0, nblks = 0;
    int ntasks = 0;
    long long gmax = 1;                 // largest group count of any task
    int items_per_cta = 4;              // repro_batch_tune may change it
    std::vector<repro_task> tasks;      // host copy, for re-planning
    size_t items_cap = 0, blks_cap = 0, parts_cap = 0;  // device capacities (bytes)
    void** d_outs = nullptr;            // repro_batch_set_outputs
    MTask* d_tasks = nullptr;
    MItem* d_items = nullptr;
    MergeBlk* d_blks = nullptr;
    unsigned char* d_partials = nullptr;
    int* d_counter = nullptr;
    // Tasks outside the single-pass path run through the partitioned (or
    // two-pass) path on `lanes` side streams forked from the caller's stream
    // and joined back into it, each lane with its own scratch; tasks are
    // assigned largest first to the least-loaded lane.
    std::vector<repro_task> slow;
    std::vector<int> slow_lane;
    std::vector<int> slow_part;       // 1: partitioned path with slow_choice, 0: two-pass path
    std::vector<PartChoice> slow_choice;
    std::vector<cudaStream_t> lanes;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    size_t slow_each = 0;
    unsigned char* d_slow_scratch = nullptr;
    // The aligned large-group tasks instead share one batched partition pass
    // (one hist / scan / scatter and one multi-task launch) on its own lane.
    BatchPartition bpart;
    bool has_bpart = false;
    bool bpart_overlap = true;  // on its own lane next to the persistent launch, else before it in stream order
    int bpart_tasks = 0;
    int single_tasks = 0;
    size_t dev_bytes = 0;
    unsigned char* d_bpart = nullptr;
    cudaStream_t bpart_lane = nullptr;
    cudaEvent_t bpart_join = nullptr;
};

// Largest group count routed to the batched partition pass (at most 128
// partitions per task of width up to 4096).
constexpr long long kBatchPartMaxGroups = 1 << 19;

// Side streams for the tasks beyond the single-pass table.
constexpr int kSlowLanes = 8;

// (Re)allocate the plan's item, merge-block and partial arrays for H and
// copy H's items and blocks to the device (synchronous).
repro_status upload_items(BatchPlan& P, const HostBatch& H) {
    for (int c = 0; c < kBatchClasses; ++c) P.cls[c] = H.cls[c];  // item ranges (and configurations)
    P.nitems = (int)H.items.size();
    P.nblks = (int)H.blks.size();
    if (P.nitems == 0) return REPRO_OK;
    const size_t ib = sizeof(MItem) * P.nitems;
    const size_t bb = sizeof(MergeBlk) * std::max(1, P.nblks);
    const size_t pb = std::max<size_t>(16, (size_t)H.part_recs * batch_rec_bytes(P.L));
    cudaError_t e = cudaSuccess;
    auto grow = [&](void** ptr, size_t& cap, size_t need) {
        if (e != cudaSuccess || cap >= need) return;
        cudaFree(*ptr);
        *ptr = nullptr;
        cap = 0;
        e = cudaMalloc(ptr, need);
        if (e == cudaSuccess) cap = need;
    };
    grow((void**)&P.d_items, P.items_cap, ib);
    grow((void**)&P.d_blks, P.blks_cap, bb);
    grow((void**)&P.d_partials, P.parts_cap, pb);
    if (e == cudaSuccess && !P.d_counter) e = cudaMalloc(&P.d_counter, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(P.d_items, H.items.data(), ib, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && P.nblks)
        e = cudaMemcpy(P.d_blks, H.blks.data(), sizeof(MergeBlk) * P.nblks, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? REPRO_ENOMEM : REPRO_ECUDA;
    return REPRO_OK;
}

}  // namespace rp

using namespace rp;

struct repro_batch_plan_s {
    BatchPlan p;
};

extern "C" {

repro_status repro_batch_prepare(const repro_task* tasks, int ntasks, repro_dtype dtype, int L,
                                 repro_batch_plan* out) {
    if (!out) return REPRO_EINVAL;
    *out = nullptr;
    HostBatch H;
    repro_status st = plan_batch_host(tasks, ntasks, dtype, L, kBatchPartBytes, H);
    if (st != REPRO_OK) return st;
    repro_batch_plan_s* plan = new (std::nothrow) repro_batch_plan_s;
    if (!plan) return REPRO_ENOMEM;
    BatchPlan& P = plan->p;
    P.dtype = dtype;
    P.L = L;
    for (int c = 0; c < kBatchClasses; ++c) P.cls[c] = H.cls[c];
    P.slow = H.slow;
    for (int t = 0; t < ntasks; ++t) P.single_tasks += tasks[t].n > 0 ? 1 : 0;
    P.single_tasks -= (int)H.slow.size();
    P.nitems = (int)H.items.size();
    P.nblks = (int)H.blks.size();
    P.ntasks = ntasks;
    for (int t = 0; t < ntasks; ++t) P.gmax = std::max<long long>(P.gmax, tasks[t].num_groups);
    if (ntasks > 0) {
        cudaError_t e = cudaMalloc(&P.d_tasks, sizeof(MTask) * ntasks);
        if (e == cudaSuccess) e = cudaMemcpy(P.d_tasks, H.tasks.data(), sizeof(MTask) * ntasks, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = e == cudaErrorMemoryAllocation ? REPRO_ENOMEM : REPRO_ECUDA;
    }
    P.tasks.assign(tasks, tasks + ntasks);
    if (st == REPRO_OK) st = upload_items(P, H);
    if (st == REPRO_OK && !P.slow.empty()) {
        std::vector<BatchPartInput> bin;
        std::vector<repro_task> rest;
        for (const repro_task& k : P.slow) {
            if (k.num_groups <= kBatchPartMaxGroups && (uintptr_t)k.keys % 16 == 0 && (uintptr_t)k.values % 16 == 0)
                bin.push_back(BatchPartInput{k.keys, k.values, k.n, (int)k.num_groups, (unsigned char*)k.state});
            else
                rest.push_back(k);
        }
        if (!bin.empty() && P.bpart.plan(dtype, L, bin)) {
            P.bpart_tasks = (int)bin.size();
            P.dev_bytes += P.bpart.scratch_bytes();
            cudaError_t e = cudaMalloc((void**)&P.d_bpart, P.bpart.scratch_bytes());
            if (e == cudaSuccess) e = P.bpart.upload(P.d_bpart);
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P.bpart_lane, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P.bpart_join, cudaEventDisableTiming);
            if (e == cudaSuccess && !P.fork) e = cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming);
            if (e != cudaSuccess) st = e == cudaErrorMemoryAllocation ? REPRO_ENOMEM : REPRO_ECUDA;
            P.has_bpart = true;
            P.slow = rest;
        }
    }
    if (st == REPRO_OK && !P.slow.empty()) {
        // tasks beyond the single-pass table: the partitioned path where it
        // applies, else the two-pass path
        const int nl = std::min<int>(kSlowLanes, (int)P.slow.size());
        std::stable_sort(P.slow.begin(), P.slow.end(),
                         [](const repro_task& x, const repro_task& y) { return x.n > y.n; });
        size_t need = 16;
        for (const repro_task& k : P.slow) {
            PartChoice pc{};
            const bool part = partitioned_supported(dtype, L, k.num_groups, k.n, k.keys, k.values) &&
                              partition_choose(dtype, L, k.num_groups, pc);
            P.slow_part.push_back(part ? 1 : 0);
            P.slow_choice.push_back(pc);
            need = std::max(need, part ? partitioned_scratch_bytes(pc, dtype, L, k.num_groups, k.n)
                                       : two_pass_scratch_bytes(k.num_groups));
        }
        std::vector<long long> load(nl, 0);
        for (const repro_task& k : P.slow) {
            const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            P.slow_lane.push_back(l);
            load[l] += k.n + 4096;
        }
        P.slow_each = (need + 255) & ~(size_t)255;
        if (cudaMalloc((void**)&P.d_slow_scratch, P.slow_each * nl) != cudaSuccess) st = REPRO_ENOMEM;
        cudaError_t e = cudaSuccess;
        if (st == REPRO_OK && !P.fork) e = cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming);
        for (int l = 0; l < nl && st == REPRO_OK && e == cudaSuccess; ++l) {
            cudaStream_t ls = nullptr;
            cudaEvent_t je = nullptr;
            e = cudaStreamCreateWithFlags(&ls, cudaStreamNonBlocking);
            if (e == cudaSuccess) P.lanes.push_back(ls);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&je, cudaEventDisableTiming);
            if (e == cudaSuccess) P.joins.push_back(je);
        }
        if (st == REPRO_OK && e != cudaSuccess) st = REPRO_ECUDA;
    }
    if (st != REPRO_OK) {
        repro_batch_destroy(plan);
        return st;
    }
    *out = plan;
    return REPRO_OK;
}

repro_status repro_batch_run(repro_batch_plan plan, void* stream) {
    if (!plan) return REPRO_EINVAL;
    BatchPlan& P = plan->p;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    // fork: the side lanes start with the caller's stream as it stands here,
    // and run next to the persistent launch below
    if (!P.slow.empty() || P.has_bpart) {
        if (cudaEventRecord(P.fork, s) != cudaSuccess) return REPRO_ECUDA;
        for (cudaStream_t ls : P.lanes)
            if (cudaStreamWaitEvent(ls, P.fork, 0) != cudaSuccess) return REPRO_ECUDA;
    }
    if (P.has_bpart) {
        if (P.bpart_overlap) {
            if (cudaStreamWaitEvent(P.bpart_lane, P.fork, 0) != cudaSuccess) return REPRO_ECUDA;
            if (P.bpart.launch(P.d_bpart, P.bpart_lane) != cudaSuccess) return REPRO_ECUDA;
        } else if (P.bpart.launch(P.d_bpart, s) != cudaSuccess) {
            return REPRO_ECUDA;
        }
    }
    if (!P.slow.empty()) {
        for (size_t i = 0; i < P.slow.size(); ++i) {
            const repro_task& k = P.slow[i];
            const int l = P.slow_lane[i];
            unsigned char* scratch = P.d_slow_scratch + (size_t)l * P.slow_each;
            if (P.slow_part[i])
                e = launch_groupby_partitioned(k.keys, k.values, k.n, P.dtype, P.L, k.num_groups, P.slow_choice[i],
                                               k.state, scratch, P.lanes[l]);
            else
                e = launch_groupby_two_pass(k.keys, k.values, k.n, P.dtype, P.L, k.num_groups, k.state, scratch,
                                            P.lanes[l]);
            if (e != cudaSuccess) return REPRO_ECUDA;
        }
    }
    if (P.nitems > 0) {
        for (const BatchClass& B : P.cls) {  // one persistent launch per class, in stream order
            if (B.nitems == 0) continue;
            e = launch_multi(P.dtype, P.L, B.cfg, B.gcap, P.d_tasks, P.d_items + B.item0, B.nitems, nullptr,
                             P.d_counter, P.d_partials, std::min(B.ctas, B.nitems), s);
            if (e != cudaSuccess) return REPRO_ECUDA;
        }
        if (P.nblks > 0) {
            e = launch_merge_items(P.L, P.dtype, P.d_tasks, P.d_blks, P.nblks, nullptr, P.d_partials, s);
            if (e != cudaSuccess) return REPRO_ECUDA;
        }
    }
    // join: the caller's stream continues once every lane is done
    for (size_t l = 0; l < P.lanes.size(); ++l) {
        if (cudaEventRecord(P.joins[l], P.lanes[l]) != cudaSuccess) return REPRO_ECUDA;
        if (cudaStreamWaitEvent(s, P.joins[l], 0) != cudaSuccess) return REPRO_ECUDA;
    }
    if (P.has_bpart && P.bpart_overlap) {
        if (cudaEventRecord(P.bpart_join, P.bpart_lane) != cudaSuccess) return REPRO_ECUDA;
        if (cudaStreamWaitEvent(s, P.bpart_join, 0) != cudaSuccess) return REPRO_ECUDA;
    }
    return REPRO_OK;
}

// grid.x: enough CTAs per task to cover the largest group table in a few
// passes; grid.y: tasks, at most 65535 per launch.
static dim3 batch_grid(const BatchPlan& P, int tasks_in_launch) {
    const long long bx = std::min<long long>(32, std::max<long long>(1, (P.gmax + 1023) / 1024));
    return dim3((unsigned)bx, (unsigned)tasks_in_launch, 1);
}

repro_status repro_batch_reset(repro_batch_plan plan, void* stream) {
    if (!plan) return REPRO_EINVAL;
    BatchPlan& P = plan->p;
    cudaStream_t s = (cudaStream_t)stream;
    for (int t0 = 0; t0 < P.ntasks; t0 += 65535) {
        const int nt = std::min(65535, P.ntasks - t0);
        k_batch_init<<<batch_grid(P, nt), 256, 0, s>>>(P.d_tasks, t0, P.dtype, P.L);
        count_launches(1);
        if (cudaGetLastError() != cudaSuccess) return REPRO_ECUDA;
    }
    return REPRO_OK;
}

repro_status repro_batch_set_outputs(repro_batch_plan plan, void* const* outs) {
    if (!plan || !outs) return REPRO_EINVAL;
    BatchPlan& P = plan->p;
    const size_t esz = P.dtype == REPRO_F64 ? 8 : 4;
    for (int t = 0; t < P.ntasks; ++t)
        if ((uintptr_t)outs[t] % esz) return REPRO_EINVAL;
    if (P.ntasks == 0) return REPRO_OK;
    if (!P.d_outs && cudaMalloc((void**)&P.d_outs, sizeof(void*) * P.ntasks) != cudaSuccess) return REPRO_ENOMEM;
    return cudaMemcpy(P.d_outs, outs, sizeof(void*) * P.ntasks, cudaMemcpyHostToDevice) == cudaSuccess
               ? REPRO_OK
               : REPRO_ECUDA;
}

repro_status repro_batch_finalize(repro_batch_plan plan, void* stream) {
    if (!plan) return REPRO_EINVAL;
    BatchPlan& P = plan->p;
    if (P.ntasks > 0 && !P.d_outs) return REPRO_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    prof_begin(PROF_FINALIZE, s);
    for (int t0 = 0; t0 < P.ntasks; t0 += 65535) {
        const int nt = std::min(65535, P.ntasks - t0);
        if (P.dtype == REPRO_F64)
            k_batch_finalize<double><<<batch_grid(P, nt), 256, 0, s>>>(P.d_tasks, P.d_outs, t0, P.dtype, P.L);
        else
            k_batch_finalize<float><<<batch_grid(P, nt), 256, 0, s>>>(P.d_tasks, P.d_outs, t0, P.dtype, P.L);
        count_launches(1);
        if (cudaGetLastError() != cudaSuccess) return REPRO_ECUDA;
    }
    prof_end(PROF_FINALIZE, s);
    return REPRO_OK;
}

repro_status repro_batch_tune(repro_batch_plan plan, void* stream, double* best_ms) {
    if (!plan) return REPRO_EINVAL;
    BatchPlan& P = plan->p;
    cudaStream_t s = (cudaStream_t)stream;
    if (best_ms) *best_ms = 0;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return REPRO_ECUDA;
    }
    repro_status st = REPRO_OK;
    double best = 0;
    int pick = P.items_per_cta;
    bool pick_overlap = P.bpart_overlap;
    for (int trial = 0; trial < (P.has_bpart ? 10 : 5); ++trial) {
        const int ipc = 1 << (trial % 5);
        P.bpart_overlap = trial < 5;
        HostBatch H;
        st = plan_batch_host(P.tasks.data(), P.ntasks, P.dtype, P.L, kBatchPartBytes, H, ipc, P.cls);
        if (st == REPRO_OK) st = upload_items(P, H);
        if (st != REPRO_OK) break;
        std::vector<float> t;
        for (int rep = 0; rep < 4 && st == REPRO_OK; ++rep) {  // first run untimed
            if ((st = repro_batch_reset(plan, stream)) != REPRO_OK) break;
            if (cudaEventRecord(a, s) != cudaSuccess) st = REPRO_ECUDA;
            if (st == REPRO_OK) st = repro_batch_run(plan, stream);
            if (st == REPRO_OK && cudaEventRecord(b, s) != cudaSuccess) st = REPRO_ECUDA;
            if (st == REPRO_OK && cudaEventSynchronize(b) != cudaSuccess) st = REPRO_ECUDA;
            float ms = 0;
            if (st == REPRO_OK && cudaEventElapsedTime(&ms, a, b) != cudaSuccess) st = REPRO_ECUDA;
            if (rep > 0) t.push_back(ms);
        }
        if (st != REPRO_OK) break;
        std::sort(t.begin(), t.end());
        const double med = t[t.size() / 2];
        if (best == 0 || med < best) {
            best = med;
            pick = ipc;
            pick_overlap = P.bpart_overlap;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    P.bpart_overlap = pick_overlap;
    if (st != REPRO_OK) return st;
    HostBatch H;
    st = plan_batch_host(P.tasks.data(), P.ntasks, P.dtype, P.L, kBatchPartBytes, H, pick, P.cls);
    if (st == REPRO_OK) st = upload_items(P, H);
    if (st == REPRO_OK) P.items_per_cta = pick;
    if (st == REPRO_OK) st = repro_batch_reset(plan, stream);
    if (st == REPRO_OK && cudaStreamSynchronize(s) != cudaSuccess) st = REPRO_ECUDA;
    if (best_ms) *best_ms = best;
    return st;
}

repro_status repro_batch_describe(repro_batch_plan plan, repro_batch_info* out) {
    if (!plan || !out) return REPRO_EINVAL;
    const BatchPlan& P = plan->p;
    std::memset(out, 0, sizeof(*out));
    out->tasks = P.ntasks;
    out->partition_tasks = P.bpart_tasks;
    out->lane_tasks = (int32_t)P.slow.size();
    out->single_pass_tasks = P.single_tasks;
    out->items = P.nitems;
    out->merge_blocks = P.nblks;
    out->items_per_cta = P.items_per_cta;
    out->partition_overlap = P.has_bpart && P.bpart_overlap ? 1 : 0;
    for (int c = 0; c < kBatchClasses && c < 3; ++c) out->class_tasks[c] = P.cls[c].ntasks;
    out->device_bytes = (int64_t)(P.dev_bytes + P.items_cap + P.blks_cap + P.parts_cap +
                                  sizeof(MTask) * (size_t)P.ntasks + P.slow_each * P.lanes.size());
    return REPRO_OK;
}

repro_status repro_batch_destroy(repro_batch_plan plan) {
    if (!plan) return REPRO_OK;
    BatchPlan& P = plan->p;
    cudaFree(P.d_tasks);
    cudaFree(P.d_outs);
    cudaFree(P.d_items);
    cudaFree(P.d_blks);
    cudaFree(P.d_partials);
    cudaFree(P.d_counter);
    cudaFree(P.d_slow_scratch);
    for (cudaStream_t ls : P.lanes) cudaStreamDestroy(ls);
    for (cudaEvent_t je : P.joins) cudaEventDestroy(je);
    if (P.fork) cudaEventDestroy(P.fork);
    cudaFree(P.d_bpart);
    if (P.bpart_lane) cudaStreamDestroy(P.bpart_lane);
    if (P.bpart_join) cudaEventDestroy(P.bpart_join);
    delete plan;
    return REPRO_OK;
}

repro_status repro_groupby_sum_batched(const repro_task* tasks, int ntasks, repro_dtype dtype, int L,
                                       void* stream) {
    repro_batch_plan plan = nullptr;
    repro_status st = repro_batch_prepare(tasks, ntasks, dtype, L, &plan);
    if (st != REPRO_OK) return st;
    st = repro_batch_run(plan, stream);
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess && st == REPRO_OK) st = REPRO_ECUDA;
    repro_batch_destroy(plan);
    return st;
}

}  // extern "C"
