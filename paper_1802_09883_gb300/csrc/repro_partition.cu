// repro_partition.cu -- grouped SUM for group counts beyond one shared-memory
// table: partition the rows by key range first (Algorithm 4's
// ParallelPartition on the key with fan-out F), then aggregate every
// partition as its own task with the multi-task single-pass kernel, each
// owning a disjoint slice of the caller's state (Algorithm 4's private
// tables; the slices make the merge into the shared table a plain write).
//
// Up to 1024 partitions the rows are partitioned in one pass (a measured
// choice may take one pass up to 2048; beyond 64 partitions each tile
// reserves its runs from the partitions' shared cursors, and beyond 256 the
// tiles are twice as long).  Beyond that a
// single pass writes runs of only a few rows per partition per tile, so the
// rows are partitioned twice, as the paper's multi-pass radix partitioning
// does for large fan-outs: a coarse pass by the high key bits, then, inside
// every coarse partition, a fine pass by the next bits.  A pass:
//
//   k_part_hist     per unit (a CTA's chunk of rows), rows per bucket (and
//                   bad keys); before two passes also every row's final
//                   partition, so that the fine pass needs no histogram
//   k_scan_totals / k_scan_starts / k_scan_offsets
//                   partition totals, 4-row-aligned partition starts (for the
//                   TMA copies) and every unit's write cursor per bucket
//   k_part_scatter  copy every row to its partition, tile by tile sorted in
//                   shared memory so that stores are coalesced runs, the
//                   next tile arriving by TMA meanwhile; the fine pass
//                   reserves its runs from per-partition shared cursors (row
//                   order inside a partition does not matter: the sum is
//                   exact)
//
// then k_part_plan turns the final partition sizes into tasks and work items
// on the device (no host round trip) and launch_multi / launch_merge_items
// (repro_batch.cu) aggregate them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "multi_types.h"
#include "ptx.cuh"
#include "repro_device.cuh"
#include "repro.h"
#include "repro_internal.h"

namespace rp {

namespace {

constexpr int kPartThreads = 512;
constexpr int kScatterRows = 8;          // rows per thread per scatter tile
constexpr int kWideTileBuckets = 256;    // wider passes through shared cursors: tiles of 2 kScatterRows
constexpr uint64_t kCopyWaitNs = 2000000000ull;  // a scatter tile's copy is given up after 2 s
constexpr int kMaxParts = 8192;          // final partitions
constexpr int kOneLevelParts = 64;       // beyond this a single pass reserves runs from shared cursors
constexpr int kOneLevelRuleParts = 1024;  // beyond this the rule takes two passes
constexpr int kOneLevelMaxParts = 2048;  // one pass at most this wide
constexpr long long kChunkRows = 32768;  // rows per unit of the fine pass
// Work items per CTA the aggregation aims at by default: items come from a
// shared counter, so with several per CTA the last round leaves few SMs
// idle; but every item restarts the CTA's table and windows (first touches
// and raises again), and a partition longer than an item is split into
// several (partial tables, merged afterwards).  The tuner measures 1-8.
constexpr long long kItemsPerCta = 2;
// Skewed keys (the fullest final partition above kSkewRatio times the mean,
// decided on the device from the histogram's totals) with more than
// kOneLevelParts partitions: kSkewItemsPerCta items per CTA instead, so that
// a hot partition is cut into shorter items spread over many CTAs.  With
// few partitions every partition is already cut into several items.  The
// tuner measured 8 best on Zipf keys at 2^20 and 2^24 groups, 2 at 2^16.
constexpr double kSkewRatio = 4.0;
constexpr long long kSkewItemsPerCta = 8;

// Geometry of one partition pass: a row with key k goes to bucket
// (k >> shift) & bmask and is written with key k & kmask.
struct PassGeom {
    int B;           // buckets per unit
    int shift;
    unsigned bmask;
    unsigned kmask;
    int check;       // 1: keys outside [0, G) are flagged and dropped
    int G;
    int ustride, bstride;  // counts / offsets of unit u, bucket j at u * ustride + j * bstride
};

// Rows of a unit: a CTA's fixed chunk of the input, or an entry of a chunk
// list (the fine pass over the coarse partitions).
struct PartChunk {
    long long beg, end;
    int seg;  // partition the rows belong to
    int pad;
};

// One input of a batched partition pass (a task of a batch): chunks whose
// seg is s read these columns, check keys against G and flag bad keys in
// this error word.
struct PartSeg {
    const int32_t* keys;
    const void* vals;
    int G;
    int pad;
    unsigned* errors;
};

struct Units {
    long long chunk;          // rows per CTA chunk (chunks == nullptr)
    long long n;              // rows of the input (chunks == nullptr)
    const PartChunk* chunks;  // chunk list, or nullptr
    const int* nchunks;       // its length (device)
    const PartSeg* segs;      // per chunk segment: its own input (batched pass), or nullptr
};

__device__ __forceinline__ bool unit_rows(const Units& u, int unit, long long& beg, long long& end, int& seg) {
    seg = 0;
    if (u.chunks) {
        if (unit >= *u.nchunks) return false;
        beg = u.chunks[unit].beg;
        end = u.chunks[unit].end;
        seg = u.chunks[unit].seg;
        return true;
    }
    beg = unit * u.chunk;
    end = max(beg, min(u.n, beg + u.chunk));  // units past the data hold nothing
    return true;
}

// A chunk list is walked grid-stride; a fixed chunking has one unit per CTA.
__device__ __forceinline__ int unit_step(const Units& u) { return u.chunks ? (int)gridDim.x : 1 << 30; }

__global__ void __launch_bounds__(kPartThreads) k_part_hist(const int32_t* __restrict__ keys0, Units units,
                                                            PassGeom pg, int* __restrict__ counts,
                                                            unsigned* __restrict__ errors0,
                                                            unsigned long long* __restrict__ ftot, int fshift,
                                                            int Ff, int* __restrict__ range) {
    extern __shared__ int s_hist[];  // [B] bucket counts, then [Ff] final-partition counts (ftot set)
    int* s_fin = s_hist + pg.B;
    int kmin = 0x7fffffff, kmax = (int)0x80000000;  // the key range (range set)
    for (int unit = blockIdx.x;; unit += unit_step(units)) {
        long long beg, end;
        int seg;
        if (!unit_rows(units, unit, beg, end, seg)) break;
        const int32_t* keys = units.segs ? units.segs[seg].keys : keys0;
        const int Gk = units.segs ? units.segs[seg].G : pg.G;
        unsigned* errors = units.segs ? units.segs[seg].errors : errors0;
        bool bad = false;
        for (int p = threadIdx.x; p < pg.B; p += blockDim.x) s_hist[p] = 0;
        if (ftot)
            for (int p = threadIdx.x; p < Ff; p += blockDim.x) s_fin[p] = 0;
        __syncthreads();
        // 4 keys per thread per load (beg is a multiple of 4, keys 16-byte
        // aligned), four loads in flight per thread: one load at a time
        // leaves too few bytes in flight per SM to reach HBM bandwidth
        const long long n4 = beg + ((end - beg) & ~3ll);
        const long long step = 4ll * blockDim.x;
        auto count1 = [&](int k) {
            if (range) {
                kmin = min(kmin, k);
                kmax = max(kmax, k);
            }
            if (!pg.check || (unsigned)k < (unsigned)Gk) {
                atomicAdd(&s_hist[((unsigned)k >> pg.shift) & pg.bmask], 1);
                if (ftot) atomicAdd(&s_fin[(unsigned)k >> fshift], 1);
            } else {
                bad = true;
            }
        };
        auto count4 = [&](const int4 k) {
            count1(k.x);
            count1(k.y);
            count1(k.z);
            count1(k.w);
        };
        long long i = beg + 4 * (long long)threadIdx.x;
        for (; i + 3 * step < n4; i += 4 * step) {
            int4 k[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) k[u] = *reinterpret_cast<const int4*>(keys + i + u * step);
#pragma unroll
            for (int u = 0; u < 4; ++u) count4(k[u]);
        }
        for (; i < n4; i += step) count4(*reinterpret_cast<const int4*>(keys + i));
        for (long long i = n4 + threadIdx.x; i < end; i += blockDim.x) count1(keys[i]);
        if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(errors, REPRO_ERR_KEY);
        __syncthreads();
        for (int p = threadIdx.x; p < pg.B; p += blockDim.x)
            counts[(size_t)unit * pg.ustride + (size_t)p * pg.bstride] = s_hist[p];
        if (ftot)
            for (int p = threadIdx.x; p < Ff; p += blockDim.x)
                if (s_fin[p]) atomicAdd(&ftot[p], (unsigned long long)s_fin[p]);
        __syncthreads();
        if (!units.chunks) break;
    }
    if (range) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
            kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&range[0], kmin);
            atomicMax(&range[1], kmax);
        }
    }
}

// Partitions of a scan: F = segments * B; segment s owns units
// [cbase[s], cbase[s] + nunits[s]) (one segment of `units` units when cbase is
// null); partition p = s * B + j.
struct ScanGeom {
    int F, B;
    int ustride, bstride;
    int units;
    const int* cbase;
    const int* nunits;
};

__device__ __forceinline__ void scan_segment(const ScanGeom& sg, int p, int& j, int& cb, int& nu) {
    const int s = p / sg.B;
    j = p - s * sg.B;
    cb = sg.cbase ? sg.cbase[s] : 0;
    nu = sg.cbase ? sg.nunits[s] : sg.units;
}

// One warp per partition: its row total.
__global__ void __launch_bounds__(256) k_scan_totals(const int* __restrict__ counts, ScanGeom sg,
                                                     long long* __restrict__ ptot) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < sg.F; p += nw) {
        int j, cb, nu;
        scan_segment(sg, p, j, cb, nu);
        long long t = 0;
        for (int k = lane; k < nu; k += 32) t += counts[(size_t)(cb + k) * sg.ustride + (size_t)j * sg.bstride];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) ptot[p] = t;
    }
}

// One block: 4-row-aligned partition starts (exclusive scan over partitions);
// with `cursor`, also every partition's write cursor (its start).
__global__ void __launch_bounds__(1024) k_scan_starts(const long long* __restrict__ ptot, int F,
                                                      long long* __restrict__ pstart,
                                                      long long* __restrict__ pcount,
                                                      int* __restrict__ cursor) {
    __shared__ long long s_w[33];
    const int per = (F + blockDim.x - 1) / blockDim.x;
    const int p0 = threadIdx.x * per, p1 = min(F, p0 + per);
    long long local = 0;
    for (int p = p0; p < p1; ++p) local += (ptot[p] + 3) & ~3ll;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        const long long w = lane < nw ? s_w[lane] : 0;
        long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) s_w[lane] = wi - w;
    }
    __syncthreads();
    long long run = s_w[warp] + incl - local;
    for (int p = p0; p < p1; ++p) {
        pstart[p] = run;
        pcount[p] = ptot[p];
        if (cursor) cursor[p] = (int)run;
        run += (ptot[p] + 3) & ~3ll;
    }
}

// One warp per partition: every unit's first output row in it.
__global__ void __launch_bounds__(256) k_scan_offsets(const int* __restrict__ counts, ScanGeom sg,
                                                      const long long* __restrict__ pstart,
                                                      int* __restrict__ offsets) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < sg.F; p += nw) {
        int j, cb, nu;
        scan_segment(sg, p, j, cb, nu);
        long long run = pstart[p];
        for (int k0 = 0; k0 < nu; k0 += 32) {
            const int k = k0 + lane;
            const size_t at = (size_t)(cb + k) * sg.ustride + (size_t)j * sg.bstride;
            const int v = k < nu ? counts[at] : 0;
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (k < nu) offsets[at] = (int)(run + incl - v);
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

template <typename T>
struct RowQuad;
template <>
struct RowQuad<double> {
    static __device__ __forceinline__ void load(const double* p, double v[4]) {
        const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};
template <>
struct RowQuad<float> {
    static __device__ __forceinline__ void load(const float* p, float v[4]) {
        const float4 a = reinterpret_cast<const float4*>(p)[0];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
};

// Exclusive scan of n (<= 8 * blockDim.x) ints in shared memory, in place;
// returns the total.  All threads of the block call it.
__device__ int block_exclusive_scan(int* a, int n, int* warp_tot) {
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per;
    int local = 0;
    for (int i = b0; i < min(n, b0 + per); ++i) local += a[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int w = lane < nw ? warp_tot[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) warp_tot[lane] = wi - w;  // exclusive
        if (lane == nw - 1) warp_tot[32] = wi;   // total
    }
    __syncthreads();
    int run = warp_tot[warp] + incl - local;
    for (int i = b0; i < min(n, b0 + per); ++i) {
        const int v = a[i];
        a[i] = run;
        run += v;
    }
    const int total = warp_tot[32];
    __syncthreads();
    return total;
}

// Copy every row of a unit to its bucket's cursor, one tile of
// kScatterRows * blockDim.x rows at a time: every row takes its rank in its
// bucket with one shared atomic, a block scan gives each bucket its place in
// the tile and one global slot range per tile, rows are sorted in shared
// memory, and consecutive threads then write consecutive runs (coalesced
// stores).  The next tile's rows are fetched by one TMA bulk copy into a
// staging buffer while this one is ranked, sorted and written, so reads stay
// in flight through the whole tile (unit starts are 4-row aligned, so every
// copy starts 16-byte aligned; a tile's last rows % 4 are read directly).
template <typename T, int RPT>
__global__ void __launch_bounds__(kPartThreads) k_part_scatter(const int32_t* __restrict__ keys0,
                                                               const T* __restrict__ vals0, Units units,
                                                               PassGeom pg, const int* __restrict__ offsets,
                                                               int* __restrict__ cursor,
                                                               int32_t* __restrict__ okeys, T* __restrict__ ovals,
                                                               unsigned* errors0) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    constexpr int TILE = RPT * kPartThreads;  // RPT rows per thread per tile
    T* s_vals = reinterpret_cast<T*>(s_raw);              // [TILE] rows sorted by bucket
    T* s_in_vals = s_vals + TILE;                         // [TILE] staging (TMA)
    int* s_keys = reinterpret_cast<int*>(s_in_vals + TILE);  // [TILE] keys, sorted by bucket
    int* s_in_keys = s_keys + TILE;                       // [TILE] staging (TMA)
    uint64_t* bar = reinterpret_cast<uint64_t*>(s_in_keys + TILE);
    int* s_cur = reinterpret_cast<int*>(bar + 1);         // [B] global write cursor
    int* s_cnt = s_cur + pg.B;                            // [B] rows per bucket in the tile
    int* s_gb = s_cnt + pg.B;                             // [B] global base of the tile's run
    int* s_wt = s_gb + pg.B;                              // [33] scan scratch
    const int tid = threadIdx.x;

    // the tile sequence of this CTA: its units in order, each cut into tiles
    auto seg_keys = [&](int seg) { return units.segs ? units.segs[seg].keys : keys0; };
    auto seg_vals = [&](int seg) { return units.segs ? static_cast<const T*>(units.segs[seg].vals) : vals0; };
    auto issue = [&](int seg, long long tb, long long end) {  // thread 0: the tile at tb
        const int rows_tma = (int)min((long long)TILE, end - tb) & ~3;
        mbar_arrive_expect_tx(bar, (uint32_t)rows_tma * (4 + sizeof(T)));
        if (rows_tma > 0) {
            bulk_g2s(s_in_keys, seg_keys(seg) + tb, (uint32_t)rows_tma * 4, bar);
            bulk_g2s(s_in_vals, seg_vals(seg) + tb, (uint32_t)rows_tma * sizeof(T), bar);
        }
    };
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    int unit = blockIdx.x;
    long long beg, end;
    int seg;
    bool have = unit_rows(units, unit, beg, end, seg);
    while (have && beg >= end && units.chunks) {  // the first unit with rows
        unit += unit_step(units);
        have = unit_rows(units, unit, beg, end, seg);
    }
    have = have && beg < end;
    if (have && tid == 0) issue(seg, beg, end);
    while (have) {
        const int32_t* keys = seg_keys(seg);
        const T* vals = seg_vals(seg);
        const int Gk = units.segs ? units.segs[seg].G : pg.G;
        for (int p = tid; p < pg.B; p += blockDim.x) {
            s_cur[p] = offsets ? offsets[(size_t)unit * pg.ustride + (size_t)p * pg.bstride] : 0;
            s_cnt[p] = 0;
        }
        __syncthreads();
        for (long long tb = beg; tb < end; tb += TILE) {
            const int rows = (int)min((long long)TILE, end - tb);
            const int rows_tma = rows & ~3;
            const bool ok = mbar_wait_bounded(bar, phase, kCopyWaitNs);
            phase ^= 1;
            if (__syncthreads_or(!ok)) {  // the copy never landed: flag it, wait once more, stop
                if (tid == 0) {
                    atomicOr(units.segs ? units.segs[seg].errors : errors0, REPRO_ERR_TIMEOUT);
                    mbar_wait_bounded(bar, phase ^ 1, kCopyWaitNs);
                }
                return;
            }
            int k[RPT];
            T v[RPT];
            int rank[RPT];
#pragma unroll
            for (int h = 0; h < RPT / 4; ++h) {  // quads strided by the block
                const int r0 = 4 * (tid + h * kPartThreads);
                int* kq = &k[4 * h];
                T* vq = &v[4 * h];
                kq[0] = kq[1] = kq[2] = kq[3] = -1;
                vq[0] = vq[1] = vq[2] = vq[3] = 0;
                if (r0 + 3 < rows_tma) {
                    const int4 k4 = *reinterpret_cast<const int4*>(s_in_keys + r0);
                    kq[0] = k4.x; kq[1] = k4.y; kq[2] = k4.z; kq[3] = k4.w;
                    RowQuad<T>::load(s_in_vals + r0, vq);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (r0 + j < rows) {
                            kq[j] = keys[tb + r0 + j];
                            vq[j] = vals[tb + r0 + j];
                        }
                }
            }
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                const bool okk = k[j] >= 0 && (!pg.check || k[j] < Gk);
                rank[j] = okk ? atomicAdd(&s_cnt[((unsigned)k[j] >> pg.shift) & pg.bmask], 1) : -1;
            }
            __syncthreads();  // staging read by all; counts complete
            if (tid == 0) {   // fetch the next tile (this unit's, else the next unit's first)
                fence_proxy_async_smem();
                if (tb + TILE < end) {
                    issue(seg, tb + TILE, end);
                } else if (units.chunks) {
                    long long b2, e2;
                    int s2;
                    for (int u2 = unit + unit_step(units); unit_rows(units, u2, b2, e2, s2); u2 += unit_step(units))
                        if (b2 < e2) {
                            issue(s2, b2, e2);
                            break;
                        }
                }
            }
            // reserve each bucket's run in global memory (from the unit's own
            // cursors, or from the partition's shared cursor: rows of a
            // partition in any order), then place of each bucket in the tile
            for (int p = tid; p < pg.B; p += blockDim.x) {
                if (offsets) {
                    s_gb[p] = s_cur[p];
                    s_cur[p] += s_cnt[p];
                } else {
                    s_gb[p] = s_cnt[p] ? atomicAdd(&cursor[(size_t)seg * pg.B + p], s_cnt[p]) : 0;
                }
            }
            const int nvalid = block_exclusive_scan(s_cnt, pg.B, s_wt);  // s_cnt now holds tile starts
#pragma unroll
            for (int j = 0; j < RPT; ++j)
                if (rank[j] >= 0) {
                    const int pos = s_cnt[((unsigned)k[j] >> pg.shift) & pg.bmask] + rank[j];
                    s_keys[pos] = k[j];
                    s_vals[pos] = v[j];
                }
            __syncthreads();
            for (int i = tid; i < nvalid; i += blockDim.x) {
                const int kk = s_keys[i];
                const int p = ((unsigned)kk >> pg.shift) & pg.bmask;
                const int pos = s_gb[p] + (i - s_cnt[p]);
                okeys[pos] = (int)((unsigned)kk & pg.kmask);
                ovals[pos] = s_vals[i];
            }
            __syncthreads();
            for (int p = tid; p < pg.B; p += blockDim.x) s_cnt[p] = 0;
            __syncthreads();
        }
        if (!units.chunks) break;
        // the next unit with rows (its first tile is already on its way)
        do {
            unit += unit_step(units);
            have = unit_rows(units, unit, beg, end, seg);
        } while (have && beg >= end);
    }
}

// One block: a chunk list over F partitions -- every partition cut into
// chunks of CH rows (4-row-aligned starts) -- with, when asked, each
// partition's first chunk and chunk count.  F <= 8 * blockDim.x.
__global__ void __launch_bounds__(1024) k_seg_chunks(const long long* __restrict__ pstart,
                                                     const long long* __restrict__ pcount, int F, long long CH,
                                                     PartChunk* __restrict__ chunks, int* __restrict__ cbase,
                                                     int* __restrict__ nunits, int* __restrict__ nchunks) {
    __shared__ int s_w[33];
    const int per = (F + blockDim.x - 1) / blockDim.x;
    const int p0 = threadIdx.x * per, p1 = min(F, p0 + per);
    int local = 0;
    for (int p = p0; p < p1; ++p) local += (int)((pcount[p] + CH - 1) / CH);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        const int w = lane < nw ? s_w[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) s_w[lane] = wi - w;
        if (lane == nw - 1) s_w[32] = wi;
    }
    __syncthreads();
    int cb = s_w[warp] + incl - local;
    for (int p = p0; p < p1; ++p) {
        const int nu = (int)((pcount[p] + CH - 1) / CH);
        if (cbase) {
            cbase[p] = cb;
            nunits[p] = nu;
        }
        const long long b0 = pstart[p], e0 = pstart[p] + pcount[p];
        for (int k = 0; k < nu; ++k) chunks[cb + k] = PartChunk{b0 + k * CH, min(e0, b0 + (k + 1) * CH), p, 0};
        cb += nu;
    }
    if (threadIdx.x == 0) *nchunks = s_w[32];
}

// Per group of every final partition its window: the largest K(b) over its
// finite values (the window of Algorithm 2 / the max-abs pre-pass, computed
// per partition; -1 where the group has none).  Work comes as chunks of one
// partition's rows (so a partition holding a heavy key is shared by many
// CTAs); each chunk takes its maxima in shared memory, then one global
// atomicMax per group it saw.  Used when groups have few rows, so that the
// aggregation never raises a window.
template <typename T>
__global__ void __launch_bounds__(512) k_part_window(const int32_t* __restrict__ okeys, const T* __restrict__ ovals,
                                                     const PartChunk* __restrict__ chunks,
                                                     const int* __restrict__ nchunks, int Gp, int G,
                                                     int* __restrict__ win) {
    extern __shared__ int s_win[];  // [Gp]
    for (int c = blockIdx.x; c < *nchunks; c += gridDim.x) {
        const PartChunk ch = chunks[c];
        const int Gq = min(Gp, G - ch.seg * Gp);
        for (int g = threadIdx.x; g < Gq; g += blockDim.x) s_win[g] = -1;
        __syncthreads();
        // rows 4 at a time (chunks start 4-row aligned), two groups of 4 in
        // flight per thread; the shared maximum is read before it is raised
        // (most rows of a group share its window)
        auto see = [&](int k, T v) {
            const Split sp = split_value(v);
            if (!sp.flag && sp.mant != 0 && s_win[k] < sp.kb) atomicMax(&s_win[k], sp.kb);
        };
        auto see4 = [&](const int4 k, const T* p) {  // p: four values, 16-byte aligned
            T v[4];
            RowQuad<T>::load(p, v);
            see(k.x, v[0]);
            see(k.y, v[1]);
            see(k.z, v[2]);
            see(k.w, v[3]);
        };
        const long long n4 = ch.beg + ((ch.end - ch.beg) & ~3ll);
        const long long step = 4ll * blockDim.x;
        long long r = ch.beg + 4ll * threadIdx.x;
        for (; r + step < n4; r += 2 * step) {
            const int4 ka = *reinterpret_cast<const int4*>(okeys + r);
            const int4 kb = *reinterpret_cast<const int4*>(okeys + r + step);
            T va[4], vb[4];
            RowQuad<T>::load(ovals + r, va);
            RowQuad<T>::load(ovals + r + step, vb);
            see(ka.x, va[0]);
            see(ka.y, va[1]);
            see(ka.z, va[2]);
            see(ka.w, va[3]);
            see(kb.x, vb[0]);
            see(kb.y, vb[1]);
            see(kb.z, vb[2]);
            see(kb.w, vb[3]);
        }
        if (r < n4) see4(*reinterpret_cast<const int4*>(okeys + r), ovals + r);
        for (long long t = n4 + threadIdx.x; t < ch.end; t += blockDim.x) see(okeys[t], ovals[t]);
        __syncthreads();
        int* w = win + (size_t)ch.seg * Gp;
        for (int g = threadIdx.x; g < Gq; g += blockDim.x)
            if (s_win[g] >= 0) atomicMax(&w[g], s_win[g]);
        __syncthreads();
    }
}

// Partition geometry the plan kernel reads: F final partitions of Gp groups
// each (partition p holds keys [p Gp, (p + 1) Gp)).
struct PartGeom {
    int F;
    int shift;
    int Gp;
};

// One block: partitions -> tasks, work items, merge blocks, partial offsets.
// The owner of final partition p: one input (tt null: state hdr with G
// groups, slice p) or, in a batched pass, task p / B of tt (slice p mod B).
struct PartTask {
    int G;
    int pad;
    unsigned char* hdr;
};

__device__ __forceinline__ void part_owner(int p, const PartTask* tt, int B, int G, unsigned char* hdr, int& j,
                                           int& Gt, unsigned char*& h) {
    if (tt) {
        const int t = p / B;
        j = p - t * B;
        Gt = tt[t].G;
        h = tt[t].hdr;
    } else {
        j = p;
        Gt = G;
        h = hdr;
    }
}

// Work items of a partition of cnt rows: its tiles shared out evenly over
// floor(tiles / tpi) items (at least one), so that an item holds at least
// tpi tiles -- a partition is split only when it holds two items' worth, and
// every split costs a partial table and its merge.
__device__ __forceinline__ long long part_items(long long cnt, int R, long long tpi) {
    if (cnt == 0) return 0;
    const long long tiles = (cnt + R - 1) / R;
    return max(1ll, tiles / tpi);
}

__global__ void __launch_bounds__(1024) k_part_plan(const long long* __restrict__ pstart,
                                                    const long long* __restrict__ pcount, PartGeom pg, int G, int R,
                                                    long long tpi, const int32_t* okeys, const void* ovals,
                                                    size_t vsize, unsigned char* hdr, int L,
                                                    const int* win, int win_hint, const PartTask* __restrict__ tt,
                                                    int B, MTask* __restrict__ tasks, MItem* __restrict__ items,
                                                    int* nitems, MergeBlk* __restrict__ blks, int* nblks,
                                                    long long G_hdr, long long tpi_skew) {
    __shared__ long long s_it[1024], s_pt[1024], s_bk[1024];
    const size_t rec = 8 + 16 * (size_t)L;
    const int per = (pg.F + blockDim.x - 1) / blockDim.x;
    const int p0 = threadIdx.x * per, p1 = min(pg.F, p0 + per);
    if (tpi_skew > 0) {  // skewed keys: the fullest partition above kSkewRatio x the mean
        long long mx = 0, sum = 0;
        for (int p = p0; p < p1; ++p) {
            mx = max(mx, pcount[p]);
            sum += pcount[p];
        }
        s_it[threadIdx.x] = mx;
        s_pt[threadIdx.x] = sum;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) {
                s_it[threadIdx.x] = max(s_it[threadIdx.x], s_it[threadIdx.x + o]);
                s_pt[threadIdx.x] += s_pt[threadIdx.x + o];
            }
            __syncthreads();
        }
        const bool skewed = (double)s_it[0] * pg.F > kSkewRatio * (double)s_pt[0];
        __syncthreads();
        if (skewed) tpi = tpi_skew;
    }
    long long it = 0, pt = 0, bk = 0;
    for (int p = p0; p < p1; ++p) {
        const long long cnt = pcount[p];
        int j, Gt;
        unsigned char* h;
        part_owner(p, tt, B, G, hdr, j, Gt, h);
        const int Gp = max(0, min(pg.Gp, Gt - j * pg.Gp));
        const long long nit = Gp == 0 ? 0 : part_items(cnt, R, tpi);
        it += nit;
        if (nit > 1) {
            pt += nit * Gp;
            bk += (Gp + 31) / 32;
        }
    }
    s_it[threadIdx.x] = it;
    s_pt[threadIdx.x] = pt;
    s_bk[threadIdx.x] = bk;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a = 0, b = 0, c = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            const long long x = s_it[i], y = s_pt[i], z = s_bk[i];
            s_it[i] = a;
            s_pt[i] = b;
            s_bk[i] = c;
            a += x;
            b += y;
            c += z;
        }
        *nitems = (int)a;
        *nblks = (int)c;
    }
    __syncthreads();
    it = s_it[threadIdx.x];
    pt = s_pt[threadIdx.x];
    bk = s_bk[threadIdx.x];
    for (int p = p0; p < p1; ++p) {
        const long long cnt = pcount[p];
        int j, Gt;
        unsigned char* h;
        part_owner(p, tt, B, G, hdr, j, Gt, h);
        const int Gp = max(0, min(pg.Gp, Gt - j * pg.Gp));
        MTask t;
        t.keys = okeys + pstart[p];
        t.vals = static_cast<const unsigned char*>(ovals) + (size_t)pstart[p] * vsize;
        t.n = cnt;
        t.G = Gp;
        t.G_hdr = tt ? Gt : (int)G_hdr;  // one input: its state may hold more groups than its keys reach
        t.hdr = h;
        t.recs = h + sizeof(repro_state_header) + (size_t)j * pg.Gp * rec;
        t.win = win ? win + (size_t)p * pg.Gp : nullptr;
        t.hint = win ? win_hint : 0;
        t.pad = 0;
        tasks[p] = t;
        const long long nit = Gp == 0 ? 0 : part_items(cnt, R, tpi);
        const long long tiles = (cnt + R - 1) / R;
        for (long long k = 0; k < nit; ++k) {
            MItem m;
            m.task = p;
            m.excl = nit == 1;
            m.row0 = k * tiles / nit * R;
            m.row1 = min(cnt, (k + 1) * tiles / nit * R);
            m.part = nit == 1 ? -1 : pt + k * Gp;
            items[it + k] = m;
        }
        it += nit;
        if (nit > 1) {
            for (int g0 = 0; g0 < Gp; g0 += 32) blks[bk++] = MergeBlk{p, g0, (int)nit, 0, pt};
            pt += nit * Gp;
        }
    }
}

struct PartPlan {
    int levels;          // 1 or 2 partition passes
    PassGeom p1, p2;     // first pass (coarse, or the only one); fine pass
    int F;               // final partitions (ceil(G / Gp))
    int Fs;              // final partitions the scan covers (F1 * F2 with two passes, else F)
    int F1, F2;          // coarse partitions, buckets per coarse partition
    int Gp;              // groups per final partition
    int C;               // CTAs of the partition passes
    long long chunk;     // rows per CTA chunk of the first pass
    long long max_chunks;
    FusedPlanConfig cfg;
    int ctas;            // CTAs of the multi-task kernel
    long long tpi;       // tiles per work item
    long long tpi_skew;  // tiles per work item if the keys are skewed (0: no rule)
    long long max_items, max_blks, max_part_recs;
    int windows;         // 1: compute every group's window before aggregating
    long long max_wchunks;
};

// Rows per group below which the windows are computed first: with few rows
// per group nearly every group raises its window inside the aggregation.
constexpr long long kWindowRowsPerGroup = 64;
constexpr long long kWindowChunkRows = 65536;

// Candidate partition widths 2^shift: at most kMaxParts partitions and a
// single-pass table that fits (with the 256 bytes of stage metadata).
bool shift_usable(int dtype, int L, long long G, int shift, FusedPlanConfig& cfg) {
    if (shift < 6 || shift > 12) return false;
    const long long F = (G + (1ll << shift) - 1) >> shift;
    if (F > kMaxParts) return false;
    return fused_plan_config(dtype, L, 1 << shift, kMetaSmemBytes, cfg);
}

int ceil_log2(long long x) {
    int b = 0;
    while ((1ll << b) < x) ++b;
    return b;
}

// The plan of one partitioned call, fully determined by the choice.
bool make_part_plan(const PartChoice& pc, int L, long long G, long long n, PartPlan& pp) {
    const DeviceInfo& di = device_info();
    if (pc.shift < 6 || pc.shift > 12) return false;
    const int Gp = 1 << pc.shift;
    const long long F = (G + Gp - 1) / Gp;
    if (F > kMaxParts) return false;
    pp.Gp = Gp;
    pp.F = (int)F;
    pp.C = di.sms * 2;
    pp.chunk = ((n + pp.C - 1) / pp.C + 3) & ~3ll;
    if (pp.chunk < 4) pp.chunk = 4;
    pp.levels = pc.shift1 > pc.shift ? 2 : 1;
    if (pp.levels == 1) {
        pp.F1 = pp.Fs = (int)F;
        pp.F2 = 1;
        pp.p1 = PassGeom{(int)F, pc.shift, 0xffffffffu, (unsigned)Gp - 1, 1, (int)G, 1, pp.C};
        pp.max_chunks = 0;
    } else {
        const int F2 = 1 << (pc.shift1 - pc.shift);
        const long long F1 = (G + (1ll << pc.shift1) - 1) >> pc.shift1;
        if (F1 > 1024 || F1 * F2 > 2 * (long long)kMaxParts) return false;
        pp.F1 = (int)F1;
        pp.F2 = F2;
        pp.Fs = (int)(F1 * F2);
        // coarse: keys kept whole; fine: buckets of the next bits, keys made local
        pp.p1 = PassGeom{(int)F1, pc.shift1, 0xffffffffu, 0xffffffffu, 1, (int)G, 1, pp.C};
        pp.p2 = PassGeom{F2, pc.shift, (unsigned)F2 - 1, (unsigned)Gp - 1, 0, (int)G, F2, 1};
        pp.max_chunks = (n + kChunkRows - 1) / kChunkRows + F1;
    }
    pp.cfg = pc.cfg;
    pp.ctas = di.sms * pc.cfg.ctas_per_sm;
    const long long R = pc.cfg.R;
    const long long total_tiles = (n + R - 1) / R + F;
    const long long ipc = pc.ipc > 0 ? pc.ipc : kItemsPerCta;
    auto tiles_per_item = [&](long long k) {
        return std::min(std::max(8ll, (total_tiles + k * pp.ctas - 1) / (k * pp.ctas)), (1ll << 23) / R);
    };
    pp.tpi = tiles_per_item(ipc);
    // a measured choice stands; the rule's skew split only with many partitions
    pp.tpi_skew = pc.ipc == 0 && F > kOneLevelParts ? tiles_per_item(kSkewItemsPerCta) : 0;
    const long long tpi_min = pp.tpi_skew > 0 ? std::min(pp.tpi, pp.tpi_skew) : pp.tpi;  // sizes the lists
    pp.max_items = total_tiles / tpi_min + F + 1;
    const long long max_split = std::min(F, total_tiles / tpi_min + 1);
    pp.max_blks = max_split * ((Gp + 31) / 32);
    // only partitions of at least 2 tpi tiles are split into several items
    pp.max_part_recs = (total_tiles / tpi_min + 1 + max_split) * (long long)Gp;
    pp.windows = n < kWindowRowsPerGroup * G ? 1 : 0;
    pp.max_wchunks = (n + kWindowChunkRows - 1) / kWindowChunkRows + F;
    if (pp.F > 8 * 1024) return false;  // k_seg_chunks covers 8 partitions per thread
    (void)L;
    return true;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct PartScratch {
    size_t akeys, avals;               // coarse output (two passes)
    size_t okeys, ovals;               // final partitions
    size_t counts1, offsets1, ptot1, pstart1, pcount1;
    size_t chunks, cursor;
    size_t ptot, pstart, pcount;
    size_t win, wchunks;
    size_t tasks, items, blks, parts, ints, total;
};

PartScratch part_scratch_layout(const PartPlan& pp, long long n, int dtype, int L) {
    PartScratch s{};
    const size_t vs = dtype == REPRO_F64 ? 8 : 4;
    size_t o = 0;
    auto take = [&](size_t& at, size_t bytes) {
        at = o;
        o = align256(o + bytes);
    };
    const size_t rows = (size_t)n + 4 * (size_t)pp.Fs;
    take(s.okeys, rows * 4);
    take(s.ovals, rows * vs);
    take(s.counts1, (size_t)pp.p1.B * pp.C * 4);
    take(s.offsets1, (size_t)pp.p1.B * pp.C * 4);
    if (pp.levels == 2) {
        const size_t arows = (size_t)n + 4 * (size_t)pp.F1;
        take(s.akeys, arows * 4);
        take(s.avals, arows * vs);
        take(s.ptot1, (size_t)pp.F1 * 8);
        take(s.pstart1, (size_t)pp.F1 * 8);
        take(s.pcount1, (size_t)pp.F1 * 8);
        take(s.chunks, (size_t)pp.max_chunks * sizeof(PartChunk));
    }
    take(s.cursor, (size_t)pp.Fs * 4);
    take(s.ptot, (size_t)pp.Fs * 8);
    take(s.pstart, (size_t)pp.Fs * 8);
    take(s.pcount, (size_t)pp.Fs * 8);
    take(s.win, (size_t)pp.F * pp.Gp * 4);  // exact windows, or their lower bounds
    if (pp.windows) take(s.wchunks, (size_t)pp.max_wchunks * sizeof(PartChunk));
    take(s.tasks, (size_t)pp.F * sizeof(MTask));
    take(s.items, (size_t)pp.max_items * sizeof(MItem));
    take(s.blks, (size_t)std::max(1ll, pp.max_blks) * sizeof(MergeBlk));
    take(s.parts, (size_t)pp.max_part_recs * (8 + 16 * (size_t)L));
    take(s.ints, 8 * sizeof(int));
    s.total = o;
    return s;
}

template <typename T, int RPT>
cudaError_t launch_scatter_rpt(const int32_t* keys, const void* vals, const Units& u, const PassGeom& pg, int grid,
                               const int* offsets, int* cursor, int32_t* okeys, void* ovals, unsigned* errors,
                               cudaStream_t s) {
    // sorted rows + staging rows, the mbarrier, three per-bucket arrays, scan scratch
    const size_t smem = 2 * (size_t)RPT * kPartThreads * (sizeof(T) + 4) + 8 + 3 * (size_t)pg.B * 4 + 33 * 4;
    cudaError_t e =
        cudaFuncSetAttribute(k_part_scatter<T, RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_part_scatter<T, RPT><<<grid, kPartThreads, smem, s>>>(keys, (const T*)vals, u, pg, offsets, cursor, okeys,
                                                            (T*)ovals, errors);
    return cudaGetLastError();
}

// A pass wider than kWideTileBuckets through shared cursors takes tiles
// twice as long (one CTA per SM instead of two), so that each tile's runs,
// and each global cursor atomic, cover twice the rows (measured at 2^28
// rows: 1024 partitions 2.92 -> 2.18 ms, 512: 2.18 -> 1.65 ms; at 128
// partitions the shorter tiles stay faster, 1.39 vs 1.54 ms).
template <typename T>
cudaError_t launch_scatter(const int32_t* keys, const void* vals, const Units& u, const PassGeom& pg, int grid,
                           const int* offsets, int* cursor, int32_t* okeys, void* ovals, unsigned* errors,
                           cudaStream_t s) {
    if (!offsets && pg.B > kWideTileBuckets)
        return launch_scatter_rpt<T, 2 * kScatterRows>(keys, vals, u, pg, grid, offsets, cursor, okeys, ovals,
                                                       errors, s);
    return launch_scatter_rpt<T, kScatterRows>(keys, vals, u, pg, grid, offsets, cursor, okeys, ovals, errors, s);
}

cudaError_t launch_hist(const int32_t* keys, const Units& u, const PassGeom& pg, int grid, int* counts,
                        unsigned* errors, unsigned long long* ftot, int fshift, int Ff, cudaStream_t s,
                        PartProbe* probe = nullptr) {
    const size_t smem = ((size_t)pg.B + (ftot ? (size_t)Ff : 0)) * 4;
    cudaError_t e = cudaFuncSetAttribute(k_part_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_part_hist<<<grid, kPartThreads, smem, s>>>(keys, u, pg, counts, errors, ftot, fshift, Ff,
                                                 probe ? probe->dev : nullptr);
    count_launches(1);
    return cudaGetLastError();
}

// The probe's look at the data: the key range and the F final partitions'
// row counts (totals: F x 8 bytes on the device), read back once with a
// synchronisation, then the caller's decision.
cudaError_t probe_read(PartProbe* probe, const long long* totals, int F, cudaStream_t s) {
    int r[2] = {0, 0};
    std::vector<long long> t((size_t)F);
    cudaError_t e = cudaMemcpyAsync(r, probe->dev, sizeof(r), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t.data(), totals, sizeof(long long) * (size_t)F, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    probe->abandoned = !probe->keep(r[0], r[1], t);
    return cudaSuccess;
}

cudaError_t launch_scatter_t(int dtype, const int32_t* keys, const void* vals, const Units& u, const PassGeom& pg,
                             int grid, const int* offsets, int* cursor, int32_t* okeys, void* ovals,
                             unsigned* errors, cudaStream_t s) {
    return dtype == REPRO_F64
               ? launch_scatter<double>(keys, vals, u, pg, grid, offsets, cursor, okeys, ovals, errors, s)
               : launch_scatter<float>(keys, vals, u, pg, grid, offsets, cursor, okeys, ovals, errors, s);
}

// One pass: histogram, scan, scatter.  sg describes the units' segments.
// With ftot, the histogram also counts every row's final partition
// (key >> fshift, Ff of them) into ftot (zeroed by the caller).
cudaError_t partition_pass(const int32_t* keys, const void* vals, int dtype, const Units& u, const PassGeom& pg,
                           const ScanGeom& sg, int grid, int* counts, int* offsets, long long* ptot,
                           long long* pstart, long long* pcount, int32_t* okeys, void* ovals, unsigned* errors,
                           cudaStream_t s, unsigned long long* ftot = nullptr, int fshift = 0, int Ff = 0,
                           PartProbe* probe = nullptr) {
    cudaError_t e = launch_hist(keys, u, pg, grid, counts, errors, ftot, fshift, Ff, s, probe);
    if (e != cudaSuccess) return e;
    const int sgrid = std::max(1, std::min(1024, (sg.F + 7) / 8));
    k_scan_totals<<<sgrid, 256, 0, s>>>(counts, sg, ptot);
    count_launches(1);
    if (probe) {  // the final partitions' totals: this pass's, or those the histogram counted (ftot)
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        e = ftot ? probe_read(probe, reinterpret_cast<const long long*>(ftot), Ff, s) : probe_read(probe, ptot, sg.F, s);
        if (e != cudaSuccess || probe->abandoned) return e;
    }
    k_scan_starts<<<1, 1024, 0, s>>>(ptot, sg.F, pstart, pcount, nullptr);
    k_scan_offsets<<<sgrid, 256, 0, s>>>(counts, sg, pstart, offsets);
    count_launches(3);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_scatter_t(dtype, keys, vals, u, pg, grid, offsets, nullptr, okeys, ovals, errors, s);
}

}  // namespace

bool partition_choose(int dtype, int L, long long G, PartChoice& pc) {
    // forced by the tuner (this thread) > tuned cache > rule; each only if usable
    int forced = tune_forced_shift();
    int shift = 0, levels = 0;
    pc.ipc = 0;
    pc.measured = false;
    if (forced && shift_usable(dtype, L, G, forced, pc.cfg)) {
        shift = forced;
        levels = tune_forced_levels();
        pc.measured = true;
    } else {
        int tuned = 0, tuned_levels = 0, tuned_ipc = 0;
        FusedPlanConfig tuned_cfg{};
        if (tune_lookup_shift(dtype, L, G, tuned, tuned_levels, tuned_cfg, tuned_ipc) &&
            shift_usable(dtype, L, G, tuned, pc.cfg)) {
            shift = tuned;
            levels = tuned_levels;
            if (tuned_cfg.S && fused_config_fits(dtype, L, 1 << tuned, kMetaSmemBytes, tuned_cfg)) pc.cfg = tuned_cfg;
            pc.ipc = tuned_ipc;
            pc.measured = true;
        } else {
            // rule: the widest power-of-two slice whose table keeps two CTAs
            // per SM (then one), with at most kMaxParts partitions
            for (int cps_goal = 2; cps_goal >= 1 && !shift; --cps_goal)
                for (int sh = 12; sh >= 6; --sh) {
                    FusedPlanConfig cfg;
                    if (!shift_usable(dtype, L, G, sh, cfg) || cfg.ctas_per_sm < cps_goal) continue;
                    shift = sh;
                    pc.cfg = cfg;
                    break;
                }
        }
    }
    if (!shift) return false;
    pc.shift = shift;
    // rule: one pass up to kOneLevelRuleParts partitions (measured at 2^28
    // rows, 2^20 groups: one pass into 1024 partitions 2.18 ms, two passes
    // 2.45 ms), else two with about sqrt(F) buckets per coarse partition; a
    // measured choice may take one pass up to kOneLevelMaxParts or two
    // passes beyond kOneLevelParts
    const long long F = (G + (1ll << shift) - 1) >> shift;
    if (levels == 1 && F > kOneLevelMaxParts) levels = 0;
    if (levels == 2 && F <= kOneLevelParts) levels = 0;
    if (levels == 0) levels = F > kOneLevelRuleParts ? 2 : 1;
    pc.shift1 = levels == 2 ? shift + (ceil_log2(F) + 1) / 2 : 0;
    return true;
}

bool partition_with(int dtype, int L, long long G, int shift, int levels, PartChoice& pc) {
    pc = PartChoice{};
    if (!shift_usable(dtype, L, G, shift, pc.cfg)) return false;
    const long long F = (G + (1ll << shift) - 1) >> shift;
    if ((levels == 1 && F > kOneLevelMaxParts) || (levels == 2 && F <= kOneLevelParts) || levels < 1 || levels > 2)
        return false;
    pc.shift = shift;
    pc.shift1 = levels == 2 ? shift + (ceil_log2(F) + 1) / 2 : 0;
    return true;
}

bool partitioned_supported(int dtype, int L, long long G, long long n, const void* keys, const void* vals) {
    if ((uintptr_t)keys % 16 || (uintptr_t)vals % 16) return false;
    if (n <= 0 || n > (1ll << 31) - 8ll * kMaxParts - 4096) return false;
    PartChoice pc;
    return partition_choose(dtype, L, G, pc);
}

size_t partitioned_scratch_bytes(const PartChoice& pc, int dtype, int L, long long G, long long n) {
    PartPlan pp;
    if (!make_part_plan(pc, L, G, n, pp)) return 0;
    return part_scratch_layout(pp, n, dtype, L).total;
}

cudaError_t launch_groupby_partitioned(const int32_t* keys, const void* vals, long long n, int dtype, int L,
                                       long long G, const PartChoice& pc, void* state, void* scratch,
                                       cudaStream_t s, long long G_hdr, PartProbe* probe) {
    if (G_hdr <= 0) G_hdr = G;
    PartPlan pp;
    if (!make_part_plan(pc, L, G, n, pp) || !fused_config_fits(dtype, L, pp.Gp, kMetaSmemBytes, pc.cfg))
        return cudaErrorInvalidValue;
    const PartScratch ly = part_scratch_layout(pp, n, dtype, L);
    unsigned char* b = (unsigned char*)scratch;
    int32_t* okeys = (int32_t*)(b + ly.okeys);
    void* ovals = b + ly.ovals;
    long long* pstart = (long long*)(b + ly.pstart);
    long long* pcount = (long long*)(b + ly.pcount);
    int* ints = (int*)(b + ly.ints);  // nitems, nblks, counter, nchunks
    unsigned* errors = &reinterpret_cast<repro_state_header*>(state)->errors;
    cudaError_t e;
    const Units whole{pp.chunk, n, nullptr, nullptr, nullptr};
    prof_begin(PROF_PARTITION, s);
    if (pp.levels == 1 && pp.F <= kOneLevelParts) {
        const ScanGeom sg{pp.Fs, pp.Fs, 1, pp.C, pp.C, nullptr, nullptr};
        e = partition_pass(keys, vals, dtype, whole, pp.p1, sg, pp.C, (int*)(b + ly.counts1), (int*)(b + ly.offsets1),
                           (long long*)(b + ly.ptot), pstart, pcount, okeys, ovals, errors, s, nullptr, 0, 0, probe);
    } else if (pp.levels == 1) {
        // a wide single pass: runs of a few rows per partition per tile, so
        // every tile reserves its runs from the partition's shared cursor
        // (runs of all CTAs then fill each partition front to back and its
        // lines complete in L2) rather than from per-CTA regions (about
        // F x 2 x SMs partly written runs open at once; measured at 2^28
        // rows, 1024 partitions: 5.66 -> 2.91 ms, 512: 3.35 -> 2.16 ms)
        const ScanGeom sg{pp.Fs, pp.Fs, 1, pp.C, pp.C, nullptr, nullptr};
        int* counts = (int*)(b + ly.counts1);
        long long* ptot = (long long*)(b + ly.ptot);
        int* cursor = (int*)(b + ly.cursor);
        if ((e = launch_hist(keys, whole, pp.p1, pp.C, counts, errors, nullptr, 0, 0, s, probe)) != cudaSuccess)
            return e;
        const int sgrid = std::max(1, std::min(1024, (sg.F + 7) / 8));
        k_scan_totals<<<sgrid, 256, 0, s>>>(counts, sg, ptot);
        count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (probe && ((e = probe_read(probe, ptot, sg.F, s)) != cudaSuccess || probe->abandoned)) {
            prof_end(PROF_PARTITION, s);
            return e;
        }
        k_scan_starts<<<1, 1024, 0, s>>>(ptot, sg.F, pstart, pcount, cursor);
        count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        e = launch_scatter_t(dtype, keys, vals, whole, pp.p1, pp.C, nullptr, cursor, okeys, ovals, errors, s);
    } else {
        int32_t* akeys = (int32_t*)(b + ly.akeys);
        void* avals = b + ly.avals;
        long long* pstart1 = (long long*)(b + ly.pstart1);
        long long* pcount1 = (long long*)(b + ly.pcount1);
        const ScanGeom sg1{pp.F1, pp.F1, 1, pp.C, pp.C, nullptr, nullptr};
        // the first histogram also counts the final partitions (key >> shift)
        long long* ptot = (long long*)(b + ly.ptot);
        if ((e = cudaMemsetAsync(ptot, 0, (size_t)pp.Fs * 8, s)) != cudaSuccess) return e;
        e = partition_pass(keys, vals, dtype, whole, pp.p1, sg1, pp.C, (int*)(b + ly.counts1), (int*)(b + ly.offsets1),
                           (long long*)(b + ly.ptot1), pstart1, pcount1, akeys, avals, errors, s,
                           reinterpret_cast<unsigned long long*>(ptot), pp.p2.shift, pp.Fs, probe);
        if (e != cudaSuccess || (probe && probe->abandoned)) {  // abandoned: the scans never ran
            prof_end(PROF_PARTITION, s);
            return e;
        }
        PartChunk* chunks = (PartChunk*)(b + ly.chunks);
        k_seg_chunks<<<1, 1024, 0, s>>>(pstart1, pcount1, pp.F1, kChunkRows, chunks, nullptr, nullptr, ints + 3);
        count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // so the fine pass needs no histogram of its own: the final
        // partitions' starts and write cursors, then the chunks' rows
        // scattered through the partitions' shared cursors
        int* cursor = (int*)(b + ly.cursor);
        k_scan_starts<<<1, 1024, 0, s>>>(ptot, pp.Fs, pstart, pcount, cursor);
        count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const Units fine{0, 0, chunks, ints + 3, nullptr};
        e = launch_scatter_t(dtype, akeys, avals, fine, pp.p2, pp.C, nullptr, cursor, okeys, ovals, errors, s);
        count_launches(1);
    }
    prof_end(PROF_PARTITION, s);
    if (e != cudaSuccess || (probe && probe->abandoned)) return e;
    // every group's window: exact from a window pass when groups are sparse,
    // else a lower bound the task's items raise as they end (later items of
    // a split partition then start near their groups' windows)
    int* win = (int*)(b + ly.win);
    const int win_hint = pp.windows ? 0 : 1;
    if ((e = cudaMemsetAsync(win, 0xff, (size_t)pp.F * pp.Gp * 4, s)) != cudaSuccess) return e;  // -1: none yet
    if (pp.windows) {
        PartChunk* wch = (PartChunk*)(b + ly.wchunks);
        k_seg_chunks<<<1, 1024, 0, s>>>(pstart, pcount, pp.F, kWindowChunkRows, wch, nullptr, nullptr, ints + 4);
        const int grid = device_info().sms * 4;
        const size_t smem = (size_t)pp.Gp * 4;
        if (dtype == REPRO_F64)
            k_part_window<double><<<grid, 512, smem, s>>>(okeys, (const double*)ovals, wch, ints + 4, pp.Gp, (int)G,
                                                          win);
        else
            k_part_window<float><<<grid, 512, smem, s>>>(okeys, (const float*)ovals, wch, ints + 4, pp.Gp, (int)G,
                                                         win);
        count_launches(2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    PartGeom pg{pp.F, pc.shift, pp.Gp};
    k_part_plan<<<1, 1024, 0, s>>>(pstart, pcount, pg, (int)G, pp.cfg.R, pp.tpi, okeys, ovals,
                                   dtype == REPRO_F64 ? 8 : 4, (unsigned char*)state, L, win, win_hint, nullptr, 0,
                                   (MTask*)(b + ly.tasks),
                                   (MItem*)(b + ly.items), ints, (MergeBlk*)(b + ly.blks), ints + 1, G_hdr,
                                   pp.tpi_skew);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_multi(dtype, L, pp.cfg, pp.Gp, b + ly.tasks, b + ly.items, (int)pp.max_items, ints, ints + 2,
                     b + ly.parts, pp.ctas, s);
    if (e != cudaSuccess) return e;
    if (pp.max_blks > 0)
        e = launch_merge_items(L, dtype, b + ly.tasks, b + ly.blks, (int)pp.max_blks, ints + 1, b + ly.parts, s);
    return e;
}

// ------------------------------------------------------------------
// Batched partition pass: many inputs (a batch's large-group tasks), each
// with its own columns, group count and state, partitioned by one hist /
// scan / scatter over a chunk list of all of them, aggregated by one
// multi-task launch.  Partition width and single-pass configuration are
// common; B = the largest task's partition count, and final partition p
// belongs to task p / B, slice p mod B.

namespace {

constexpr long long kBatchBuckets = 128;  // partitions per task of a batched pass

struct BatchLayout {
    size_t chunks, segs, ptask, cbase, nunits, ints, tables;  // host-built tables: bytes [0, tables)
    size_t okeys, ovals, counts, offsets, ptot, pstart, pcount;
    size_t tasks, items, blks, parts, total;
};

}  // namespace

struct BatchPartition::Impl {
    int dtype = 0, L = 0, T = 0, B = 0, F = 0, Gp = 0, ctas = 0;
    PartChoice pc{};
    long long rows_out = 0, tpi = 0, max_items = 0, max_blks = 0, max_part_recs = 0;
    std::vector<PartChunk> chunks;
    std::vector<PartSeg> segs;
    std::vector<PartTask> ptask;
    std::vector<int> cbase, nunits;
    BatchLayout ly{};
};

BatchPartition::BatchPartition() : impl(new Impl) {}
BatchPartition::~BatchPartition() { delete impl; }

bool BatchPartition::plan(int dtype, int L, const std::vector<BatchPartInput>& in) {
    Impl& P = *impl;
    P = Impl{};
    if (in.empty()) return false;
    long long Gmax = 1, total_rows = 0;
    for (const BatchPartInput& t : in) {
        if ((uintptr_t)t.keys % 16 || (uintptr_t)t.vals % 16 || t.n <= 0 || t.G < 1) return false;
        Gmax = std::max<long long>(Gmax, t.G);
        total_rows += t.n;
    }
    if (total_rows > (1ll << 31) - 8ll * kMaxParts - 4096) return false;
    if (!partition_choose(dtype, L, Gmax, P.pc)) return false;
    // one pass: a chunk's rows spread over at most kBatchBuckets buckets of
    // its own task (tiles of 4096 rows still write runs of 32+ rows); widen
    // the partitions if the largest task needs it
    const int need = ceil_log2((Gmax + kBatchBuckets - 1) / kBatchBuckets);
    if (need > P.pc.shift) {
        if (!shift_usable(dtype, L, Gmax, need, P.pc.cfg)) return false;
        P.pc.shift = need;
    }
    P.pc.shift1 = 0;
    P.dtype = dtype;
    P.L = L;
    P.T = (int)in.size();
    P.Gp = 1 << P.pc.shift;
    P.B = (int)((Gmax + P.Gp - 1) / P.Gp);
    if (P.B > kBatchBuckets || (long long)P.T * P.B > (1ll << 24)) return false;
    P.F = P.T * P.B;
    for (int t = 0; t < P.T; ++t) {
        const BatchPartInput& x = in[t];
        P.cbase.push_back((int)P.chunks.size());
        for (long long b = 0; b < x.n; b += kChunkRows)
            P.chunks.push_back(PartChunk{b, std::min(x.n, b + kChunkRows), t, 0});
        P.nunits.push_back((int)P.chunks.size() - P.cbase.back());
        P.segs.push_back(PartSeg{x.keys, x.vals, x.G, 0, &reinterpret_cast<repro_state_header*>(x.state)->errors});
        P.ptask.push_back(PartTask{x.G, 0, x.state});
    }
    const DeviceInfo& di = device_info();
    P.ctas = di.sms * P.pc.cfg.ctas_per_sm;
    const long long R = P.pc.cfg.R;
    long long total_tiles = P.F;
    for (const BatchPartInput& x : in) total_tiles += (x.n + R - 1) / R;
    P.tpi = std::max(8ll, (total_tiles + kItemsPerCta * P.ctas - 1) / (kItemsPerCta * P.ctas));
    P.tpi = std::min(P.tpi, (1ll << 23) / R);
    P.max_items = total_tiles / P.tpi + P.F + 1;
    const long long max_split = std::min<long long>(P.F, total_tiles / P.tpi + 1);
    P.max_blks = max_split * ((P.Gp + 31) / 32);
    P.max_part_recs = (total_tiles / P.tpi + 1 + max_split) * (long long)P.Gp;
    P.rows_out = total_rows + 4ll * P.F;
    const size_t vs = dtype == REPRO_F64 ? 8 : 4;
    const size_t nch = P.chunks.size();
    BatchLayout& ly = P.ly;
    size_t o = 0;
    auto take = [&](size_t& at, size_t bytes) {
        at = o;
        o = align256(o + bytes);
    };
    // the host-built tables first (one contiguous image, see pack_tables)
    take(ly.chunks, nch * sizeof(PartChunk));
    take(ly.segs, (size_t)P.T * sizeof(PartSeg));
    take(ly.ptask, (size_t)P.T * sizeof(PartTask));
    take(ly.cbase, (size_t)P.T * 4);
    take(ly.nunits, (size_t)P.T * 4);
    take(ly.ints, 8 * sizeof(int));
    ly.tables = o;
    take(ly.okeys, (size_t)P.rows_out * 4);
    take(ly.ovals, (size_t)P.rows_out * vs);
    take(ly.counts, nch * (size_t)P.B * 4);
    take(ly.offsets, nch * (size_t)P.B * 4);
    take(ly.ptot, (size_t)P.F * 8);
    take(ly.pstart, (size_t)P.F * 8);
    take(ly.pcount, (size_t)P.F * 8);
    take(ly.tasks, (size_t)P.F * sizeof(MTask));
    take(ly.items, (size_t)P.max_items * sizeof(MItem));
    take(ly.blks, (size_t)std::max(1ll, P.max_blks) * sizeof(MergeBlk));
    take(ly.parts, (size_t)P.max_part_recs * (8 + 16 * (size_t)L));
    ly.total = o;
    return true;
}

size_t BatchPartition::scratch_bytes() const { return impl->ly.total; }

size_t BatchPartition::table_bytes() const { return impl->ly.tables; }

void BatchPartition::pack_tables(void* host) const {
    const Impl& P = *impl;
    unsigned char* b = (unsigned char*)host;
    std::memset(b, 0, P.ly.tables);
    std::memcpy(b + P.ly.chunks, P.chunks.data(), P.chunks.size() * sizeof(PartChunk));
    std::memcpy(b + P.ly.segs, P.segs.data(), P.segs.size() * sizeof(PartSeg));
    std::memcpy(b + P.ly.ptask, P.ptask.data(), P.ptask.size() * sizeof(PartTask));
    std::memcpy(b + P.ly.cbase, P.cbase.data(), P.cbase.size() * 4);
    std::memcpy(b + P.ly.nunits, P.nunits.data(), P.nunits.size() * 4);
    const int nch = (int)P.chunks.size();
    std::memcpy(b + P.ly.ints + 4 * sizeof(int), &nch, sizeof(int));
}

cudaError_t BatchPartition::upload(void* scratch) const {
    std::vector<unsigned char> img(impl->ly.tables);
    pack_tables(img.data());
    return cudaMemcpy(scratch, img.data(), img.size(), cudaMemcpyHostToDevice);
}

cudaError_t BatchPartition::upload_async(void* scratch, void* pinned, cudaStream_t s) const {
    pack_tables(pinned);
    return cudaMemcpyAsync(scratch, pinned, impl->ly.tables, cudaMemcpyHostToDevice, s);
}

cudaError_t BatchPartition::launch(void* scratch, cudaStream_t s) const {
    const Impl& P = *impl;
    unsigned char* b = (unsigned char*)scratch;
    int* ints = (int*)(b + P.ly.ints);  // nitems, nblks, counter, -, nchunks
    const Units u{0, 0, (const PartChunk*)(b + P.ly.chunks), ints + 4, (const PartSeg*)(b + P.ly.segs)};
    const PassGeom pg{P.B, P.pc.shift, 0xffffffffu, (unsigned)P.Gp - 1, 1, 0, P.B, 1};
    const ScanGeom sg{P.F, P.B, P.B, 1, 0, (const int*)(b + P.ly.cbase), (const int*)(b + P.ly.nunits)};
    int32_t* okeys = (int32_t*)(b + P.ly.okeys);
    void* ovals = b + P.ly.ovals;
    long long* pstart = (long long*)(b + P.ly.pstart);
    long long* pcount = (long long*)(b + P.ly.pcount);
    prof_begin(PROF_PARTITION, s);
    cudaError_t e = partition_pass(nullptr, nullptr, P.dtype, u, pg, sg, device_info().sms * 2, (int*)(b + P.ly.counts),
                                   (int*)(b + P.ly.offsets), (long long*)(b + P.ly.ptot), pstart, pcount, okeys, ovals,
                                   nullptr, s);
    prof_end(PROF_PARTITION, s);
    if (e != cudaSuccess) return e;
    const PartGeom geo{P.F, P.pc.shift, P.Gp};
    k_part_plan<<<1, 1024, 0, s>>>(pstart, pcount, geo, 0, P.pc.cfg.R, P.tpi, okeys, ovals,
                                   P.dtype == REPRO_F64 ? 8 : 4, nullptr, P.L, nullptr, 0,
                                   (const PartTask*)(b + P.ly.ptask), P.B, (MTask*)(b + P.ly.tasks),
                                   (MItem*)(b + P.ly.items), ints, (MergeBlk*)(b + P.ly.blks), ints + 1, 0, 0);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_multi(P.dtype, P.L, P.pc.cfg, P.Gp, b + P.ly.tasks, b + P.ly.items, (int)P.max_items, ints, ints + 2,
                     b + P.ly.parts, P.ctas, s);
    if (e != cudaSuccess) return e;
    if (P.max_blks > 0)
        e = launch_merge_items(P.L, P.dtype, b + P.ly.tasks, b + P.ly.blks, (int)P.max_blks, ints + 1, b + P.ly.parts,
                               s);
    return e;
}

// ------------------------------------------------------------------
}  // namespace rp
