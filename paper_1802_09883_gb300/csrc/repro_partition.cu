// repro_partition.cu -- grouped SUM for group counts beyond one shared-memory
// table: partition the rows by key range first (Algorithm 4, line 1:
// ParallelPartition on the key with fan-out F), then aggregate every
// partition as its own task with the multi-task single-pass kernel, each
// owning a disjoint slice of the caller's state (Algorithm 4's private
// tables; the slices make the merge into the shared table a plain write).
//
//   k_part_hist     per CTA chunk, rows per partition (and bad keys)
//   k_part_scan     partition starts (4-row aligned for the TMA copies) and
//                   each CTA's write cursor in every partition
//   k_part_scatter  copy every row to its partition with its key made local
//                   (row order inside a partition does not matter: the sum
//                   is exact)
//   k_part_plan     turn partition sizes into tasks and work items on the
//                   device (no host round trip)
// then launch_multi / launch_merge_items (repro_batch.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "multi_types.h"
#include "repro.h"
#include "repro_internal.h"

namespace rp {

namespace {

constexpr int kPartThreads = 512;
constexpr int kScatterRows = 8;  // rows per thread per scatter tile
constexpr int kMaxParts = 4096;

struct PartGeom {
    int F;            // partitions
    int shift;        // partition = key >> shift
    int Gp;           // groups per partition (2^shift)
    int C;            // CTAs of the partition passes
    long long chunk;  // rows per CTA chunk (multiple of 4)
};

__global__ void __launch_bounds__(kPartThreads) k_part_hist(const int32_t* __restrict__ keys, long long n, int G,
                                                            PartGeom pg, int* __restrict__ counts,
                                                            unsigned* __restrict__ errors) {
    extern __shared__ int s_hist[];
    for (int p = threadIdx.x; p < pg.F; p += blockDim.x) s_hist[p] = 0;
    __syncthreads();
    const long long beg = blockIdx.x * pg.chunk;
    const long long end = max(beg, min(n, beg + pg.chunk));  // CTAs past the data count nothing
    bool bad = false;
    // 4 keys per thread per step (beg is a multiple of 4 and keys 16-byte aligned)
    const long long n4 = beg + ((end - beg) & ~3ll);
    for (long long i = beg + 4 * (long long)threadIdx.x; i < n4; i += 4ll * blockDim.x) {
        const int4 k = *reinterpret_cast<const int4*>(keys + i);
        const int ks[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if ((unsigned)ks[q] < (unsigned)G) atomicAdd(&s_hist[ks[q] >> pg.shift], 1);
            else bad = true;
        }
    }
    for (long long i = n4 + threadIdx.x; i < end; i += blockDim.x) {
        const int k = keys[i];
        if ((unsigned)k < (unsigned)G) atomicAdd(&s_hist[k >> pg.shift], 1);
        else bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(errors, REPRO_ERR_KEY);
    __syncthreads();
    for (int p = threadIdx.x; p < pg.F; p += blockDim.x) counts[(size_t)p * pg.C + blockIdx.x] = s_hist[p];
}

// One block: per partition its total and 4-aligned start; per (partition, CTA)
// the CTA's first output row.
__global__ void __launch_bounds__(1024) k_part_scan(const int* __restrict__ counts, PartGeom pg,
                                                    int* __restrict__ offsets, long long* __restrict__ pstart,
                                                    long long* __restrict__ pcount) {
    __shared__ long long s_tot[1024];
    const int per = (pg.F + blockDim.x - 1) / blockDim.x;  // partitions per thread (consecutive)
    const int p0 = threadIdx.x * per;
    long long mine = 0;
    for (int p = p0; p < min(pg.F, p0 + per); ++p) {
        long long t = 0;
        for (int c = 0; c < pg.C; ++c) t += counts[(size_t)p * pg.C + c];
        pcount[p] = t;
        mine += (t + 3) & ~3ll;
    }
    s_tot[threadIdx.x] = mine;
    __syncthreads();
    // exclusive scan over the per-thread totals (1024 entries, simple and rare)
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            const long long v = s_tot[i];
            s_tot[i] = run;
            run += v;
        }
    }
    __syncthreads();
    long long run = s_tot[threadIdx.x];
    for (int p = p0; p < min(pg.F, p0 + per); ++p) {
        pstart[p] = run;
        long long cur = run;
        for (int c = 0; c < pg.C; ++c) {
            offsets[(size_t)p * pg.C + c] = (int)cur;
            cur += counts[(size_t)p * pg.C + c];
        }
        run += (pcount[p] + 3) & ~3ll;
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

// Copy every row to its partition, one tile of kScatterRows * blockDim.x rows at a
// time: every row takes its rank in its partition with one shared atomic, a
// block scan gives each partition its place in the tile and one global slot
// range per tile, rows are sorted in shared memory, and consecutive threads
// then write consecutive runs (coalesced stores).
template <typename T>
__global__ void __launch_bounds__(kPartThreads) k_part_scatter(const int32_t* __restrict__ keys,
                                                               const T* __restrict__ vals, long long n, int G,
                                                               PartGeom pg, const int* __restrict__ offsets,
                                                               int32_t* __restrict__ okeys, T* __restrict__ ovals) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    constexpr int RPT = kScatterRows;  // rows per thread per tile
    const int TILE = RPT * kPartThreads;
    T* s_vals = reinterpret_cast<T*>(s_raw);                              // [TILE]
    int* s_keys = reinterpret_cast<int*>(s_vals + TILE);                  // [TILE] global keys, sorted
    int* s_cur = s_keys + TILE;                                           // [F] global write cursor
    int* s_cnt = s_cur + pg.F;                                            // [F] rows per partition in the tile
    int* s_gb = s_cnt + pg.F;                                             // [F] global base of the tile's run
    int* s_wt = s_gb + pg.F;                                              // [33] scan scratch
    for (int p = threadIdx.x; p < pg.F; p += blockDim.x) {
        s_cur[p] = offsets[(size_t)p * pg.C + blockIdx.x];
        s_cnt[p] = 0;
    }
    __syncthreads();
    const long long beg = blockIdx.x * pg.chunk;
    const long long end = max(beg, min(n, beg + pg.chunk));
    const int mask = pg.Gp - 1;
    for (long long tb = beg; tb < end; tb += TILE) {
        int k[RPT];
        T v[RPT];
        int rank[RPT];
#pragma unroll
        for (int h = 0; h < RPT / 4; ++h) {  // quads strided by the block: coalesced 16-byte loads
            const long long r0 = tb + 4ll * (threadIdx.x + h * kPartThreads);
            int* kq = &k[4 * h];
            T* vq = &v[4 * h];
            kq[0] = kq[1] = kq[2] = kq[3] = -1;
            vq[0] = vq[1] = vq[2] = vq[3] = 0;
            if (r0 + 3 < end) {
                const int4 k4 = *reinterpret_cast<const int4*>(keys + r0);
                kq[0] = k4.x; kq[1] = k4.y; kq[2] = k4.z; kq[3] = k4.w;
                RowQuad<T>::load(vals + r0, vq);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (r0 + j < end) {
                        kq[j] = keys[r0 + j];
                        vq[j] = vals[r0 + j];
                    }
            }
        }
#pragma unroll
        for (int j = 0; j < RPT; ++j)
            rank[j] = (unsigned)k[j] < (unsigned)G ? atomicAdd(&s_cnt[k[j] >> pg.shift], 1) : -1;
        __syncthreads();
        // reserve each partition's run in global memory, then place of each partition in the tile
        for (int p = threadIdx.x; p < pg.F; p += blockDim.x) {
            s_gb[p] = s_cur[p];
            s_cur[p] += s_cnt[p];
        }
        const int nvalid = block_exclusive_scan(s_cnt, pg.F, s_wt);  // s_cnt now holds tile starts
#pragma unroll
        for (int j = 0; j < RPT; ++j)
            if (rank[j] >= 0) {
                const int pos = s_cnt[k[j] >> pg.shift] + rank[j];
                s_keys[pos] = k[j];
                s_vals[pos] = v[j];
            }
        __syncthreads();
        for (int i = threadIdx.x; i < nvalid; i += blockDim.x) {
            const int kk = s_keys[i];
            const int p = kk >> pg.shift;
            const int pos = s_gb[p] + (i - s_cnt[p]);
            okeys[pos] = kk & mask;
            ovals[pos] = s_vals[i];
        }
        __syncthreads();
        for (int p = threadIdx.x; p < pg.F; p += blockDim.x) s_cnt[p] = 0;
        __syncthreads();
    }
}

// One block: partitions -> tasks, work items, merge blocks, partial offsets.
__global__ void __launch_bounds__(1024) k_part_plan(const long long* __restrict__ pstart,
                                                    const long long* __restrict__ pcount, PartGeom pg, int G, int R,
                                                    long long tpi, const int32_t* okeys, const void* ovals,
                                                    size_t vsize, unsigned char* hdr, int L, MTask* __restrict__ tasks,
                                                    MItem* __restrict__ items, int* nitems, MergeBlk* __restrict__ blks,
                                                    int* nblks) {
    __shared__ long long s_it[1024], s_pt[1024], s_bk[1024];
    const size_t rec = 8 + 16 * (size_t)L;
    const int per = (pg.F + blockDim.x - 1) / blockDim.x;
    const int p0 = threadIdx.x * per, p1 = min(pg.F, p0 + per);
    long long it = 0, pt = 0, bk = 0;
    for (int p = p0; p < p1; ++p) {
        const long long cnt = pcount[p];
        const int Gp = min(pg.Gp, G - p * pg.Gp);
        const long long nit = cnt == 0 ? 0 : (((cnt + R - 1) / R) + tpi - 1) / tpi;
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
        const int Gp = min(pg.Gp, G - p * pg.Gp);
        MTask t;
        t.keys = okeys + pstart[p];
        t.vals = static_cast<const unsigned char*>(ovals) + (size_t)pstart[p] * vsize;
        t.n = cnt;
        t.G = Gp;
        t.G_hdr = G;
        t.hdr = hdr;
        t.recs = hdr + sizeof(repro_state_header) + (size_t)p * pg.Gp * rec;
        tasks[p] = t;
        const long long nit = cnt == 0 ? 0 : (((cnt + R - 1) / R) + tpi - 1) / tpi;
        for (long long k = 0; k < nit; ++k) {
            MItem m;
            m.task = p;
            m.excl = nit == 1;
            m.row0 = k * tpi * R;
            m.row1 = min(cnt, (k + 1) * tpi * R);
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
    PartGeom pg;
    FusedPlanConfig cfg;
    int ctas;          // CTAs of the multi-task kernel
    long long tpi;     // tiles per work item
    long long max_items, max_blks, max_part_recs;
};

// Candidate partition widths 2^shift: at most kMaxParts partitions and a
// single-pass table that fits (with the 256 bytes of stage metadata).
bool shift_usable(int dtype, int L, long long G, int shift, FusedPlanConfig& cfg) {
    if (shift < 6 || shift > 12) return false;
    const long long F = (G + (1ll << shift) - 1) >> shift;
    if (F > kMaxParts) return false;
    return fused_plan_config(dtype, L, 1 << shift, 256, cfg);
}

// The plan of one partitioned call, fully determined by the choice.
bool make_part_plan(const PartChoice& pc, int L, long long G, long long n, PartPlan& pp) {
    const DeviceInfo& di = device_info();
    const int Gp = 1 << pc.shift;
    const long long F = (G + Gp - 1) / Gp;
    if (F > kMaxParts || pc.shift < 6 || pc.shift > 12) return false;
    pp.pg.F = (int)F;
    pp.pg.shift = pc.shift;
    pp.pg.Gp = Gp;
    pp.cfg = pc.cfg;
    pp.ctas = di.sms * pc.cfg.ctas_per_sm;
    const long long R = pc.cfg.R;
    const long long total_tiles = (n + R - 1) / R + F;
    pp.tpi = std::max(8ll, (total_tiles + 2ll * pp.ctas - 1) / (2ll * pp.ctas));
    pp.tpi = std::min(pp.tpi, (1ll << 23) / R);
    pp.max_items = total_tiles / pp.tpi + F + 1;
    const long long max_split = std::min(F, total_tiles / pp.tpi + 1);
    pp.max_blks = max_split * ((Gp + 31) / 32);
    // only partitions with more than tpi tiles are split into several items
    pp.max_part_recs = (total_tiles / pp.tpi + 1 + max_split) * (long long)Gp;
    pp.pg.C = di.sms * 2;
    pp.pg.chunk = ((n + pp.pg.C - 1) / pp.pg.C + 3) & ~3ll;
    if (pp.pg.chunk < 4) pp.pg.chunk = 4;
    (void)L;
    return true;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct PartScratch {
    size_t okeys, ovals, counts, offsets, pstart, pcount, tasks, items, blks, parts, ints, total;
};

PartScratch part_scratch_layout(const PartPlan& pp, long long n, int dtype, int L) {
    PartScratch s;
    const size_t vs = dtype == REPRO_F64 ? 8 : 4;
    const size_t rows = (size_t)n + 4 * (size_t)pp.pg.F;
    size_t o = 0;
    s.okeys = o; o = align256(o + rows * 4);
    s.ovals = o; o = align256(o + rows * vs);
    s.counts = o; o = align256(o + (size_t)pp.pg.F * pp.pg.C * 4);
    s.offsets = o; o = align256(o + (size_t)pp.pg.F * pp.pg.C * 4);
    s.pstart = o; o = align256(o + (size_t)pp.pg.F * 8);
    s.pcount = o; o = align256(o + (size_t)pp.pg.F * 8);
    s.tasks = o; o = align256(o + (size_t)pp.pg.F * sizeof(MTask));
    s.items = o; o = align256(o + (size_t)pp.max_items * sizeof(MItem));
    s.blks = o; o = align256(o + (size_t)std::max(1ll, pp.max_blks) * sizeof(MergeBlk));
    s.parts = o; o = align256(o + (size_t)pp.max_part_recs * (8 + 16 * (size_t)L));
    s.ints = o; o = align256(o + 4 * sizeof(int));
    s.total = o;
    return s;
}

}  // namespace

bool partition_choose(int dtype, int L, long long G, PartChoice& pc) {
    // forced by the tuner (this thread) > tuned cache > rule; each only if usable
    int forced = tune_forced_shift();
    if (forced && shift_usable(dtype, L, G, forced, pc.cfg)) {
        pc.shift = forced;
        return true;
    }
    int tuned = 0;
    if (tune_lookup_shift(dtype, L, G, tuned) && shift_usable(dtype, L, G, tuned, pc.cfg)) {
        pc.shift = tuned;
        return true;
    }
    // rule: the widest power-of-two slice whose table keeps two CTAs per SM
    // (then one), with at most kMaxParts partitions
    for (int cps_goal = 2; cps_goal >= 1; --cps_goal)
        for (int shift = 12; shift >= 6; --shift) {
            FusedPlanConfig cfg;
            if (!shift_usable(dtype, L, G, shift, cfg)) continue;
            if (cfg.ctas_per_sm < cps_goal) continue;
            pc.shift = shift;
            pc.cfg = cfg;
            return true;
        }
    return false;
}

bool partitioned_supported(int dtype, int L, long long G, long long n, const void* keys, const void* vals) {
    if ((uintptr_t)keys % 16 || (uintptr_t)vals % 16) return false;
    if (n <= 0 || n > (1ll << 31) - 4ll * kMaxParts) return false;
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
                                       cudaStream_t s) {
    PartPlan pp;
    if (!make_part_plan(pc, L, G, n, pp) || !fused_config_fits(dtype, L, pp.pg.Gp, 256, pc.cfg))
        return cudaErrorInvalidValue;
    const PartScratch ly = part_scratch_layout(pp, n, dtype, L);
    unsigned char* b = (unsigned char*)scratch;
    int32_t* okeys = (int32_t*)(b + ly.okeys);
    void* ovals = b + ly.ovals;
    int* counts = (int*)(b + ly.counts);
    int* offsets = (int*)(b + ly.offsets);
    long long* pstart = (long long*)(b + ly.pstart);
    long long* pcount = (long long*)(b + ly.pcount);
    int* ints = (int*)(b + ly.ints);  // nitems, nblks, counter
    unsigned* errors = &reinterpret_cast<repro_state_header*>(state)->errors;
    const size_t hsmem = (size_t)pp.pg.F * 4;
    cudaError_t e;
    prof_begin(PROF_PARTITION, s);
    k_part_hist<<<pp.pg.C, kPartThreads, hsmem, s>>>(keys, n, (int)G, pp.pg, counts, errors);
    k_part_scan<<<1, 1024, 0, s>>>(counts, pp.pg, offsets, pstart, pcount);
    const size_t vsz = dtype == REPRO_F64 ? 8 : 4;
    const size_t ssmem = (size_t)kScatterRows * kPartThreads * (vsz + 4) + 3 * (size_t)pp.pg.F * 4 + 33 * 4;
    if (dtype == REPRO_F64) {
        if ((e = cudaFuncSetAttribute(k_part_scatter<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)ssmem)) != cudaSuccess)
            return e;
        k_part_scatter<double><<<pp.pg.C, kPartThreads, ssmem, s>>>(keys, (const double*)vals, n, (int)G, pp.pg,
                                                                     offsets, okeys, (double*)ovals);
    } else {
        if ((e = cudaFuncSetAttribute(k_part_scatter<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)ssmem)) != cudaSuccess)
            return e;
        k_part_scatter<float><<<pp.pg.C, kPartThreads, ssmem, s>>>(keys, (const float*)vals, n, (int)G, pp.pg,
                                                                    offsets, okeys, (float*)ovals);
    }
    prof_end(PROF_PARTITION, s);
    k_part_plan<<<1, 1024, 0, s>>>(pstart, pcount, pp.pg, (int)G, pp.cfg.R, pp.tpi, okeys, ovals,
                                   dtype == REPRO_F64 ? 8 : 4, (unsigned char*)state, L, (MTask*)(b + ly.tasks),
                                   (MItem*)(b + ly.items), ints, (MergeBlk*)(b + ly.blks), ints + 1);
    count_launches(4);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_multi(dtype, L, pp.cfg, pp.pg.Gp, b + ly.tasks, b + ly.items, (int)pp.max_items, ints, ints + 2,
                     b + ly.parts, pp.ctas, s);
    if (e != cudaSuccess) return e;
    if (pp.max_blks > 0)
        e = launch_merge_items(L, dtype, b + ly.tasks, b + ly.blks, (int)pp.max_blks, ints + 1, b + ly.parts, s);
    return e;
}

}  // namespace rp
