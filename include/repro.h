/*
 * repro.h -- C ABI of the reproducible grouped SUM library (librepro.so).
 *
 * The library computes SQL's SUM ... GROUP BY over floating-point values so
 * that the bits of every group's result are the same for any order of the
 * rows, any split of the input into calls, and any GPU schedule.  It
 * implements the repro<T,L> aggregate of Mueller, Arteaga, Hoefler, Alonso,
 * "Reproducible Floating-Point Aggregation in RDBMSs" (arXiv 1802.09883):
 * each value is cut into L digits on a grid fixed by the group's largest
 * |value| (Sec. III-C, Algorithm 2), digits are summed exactly, and the
 * result is the per-level sum rounded to T and folded from the lowest level
 * (eq. (1)).  Reproducibility comes from exact integer bins, not from a
 * fixed order, so atomics and any launch configuration give the same bits.
 *
 * Conventions for every entry point:
 *  - Arrays are DEVICE pointers owned by the caller; the library never frees
 *    them.  `stream` is a cudaStream_t (NULL = the legacy default stream).
 *  - Calls are stream-ordered and asynchronous: they enqueue kernels on
 *    `stream` and return.  Argument errors are returned synchronously, before
 *    anything is enqueued.  Errors found in the data (a key outside
 *    [0, num_groups)) are recorded in the state's header and reported by
 *    repro_state_check().
 *  - Scratch memory is taken stream-ordered (cudaMallocFromPoolAsync) from a
 *    memory pool the library creates per device and returned to it on the
 *    same stream; the pool keeps freed bytes cached for the next call
 *    (repro_release_cached_memory hands them back).  REPRO_ENOMEM if scratch
 *    cannot be had.
 *  - L (levels) is 1..4; num_groups is 1 .. 2^31 - 1; keys are dense int32
 *    group ids in [0, num_groups) (the paper's IdentityHashing, Sec. VI-A).
 */
#ifndef REPRO_H
#define REPRO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    REPRO_OK = 0,
    REPRO_EINVAL = 1,   /* bad argument (NULL pointer, L, num_groups, n, dtype) */
    REPRO_EKEY = 2,     /* a key outside [0, num_groups) was seen (row skipped) */
    REPRO_ERANGE = 3,   /* reserved: size beyond a documented maximum */
    REPRO_ENOMEM = 4,   /* scratch memory could not be allocated */
    REPRO_ECUDA = 5,    /* a CUDA call failed (launch, copy, allocation) */
    REPRO_ETIMEOUT = 6, /* a bounded device-side wait gave up */
    REPRO_ELAYOUT = 7   /* the state header does not match dtype / L / num_groups */
} repro_status;

typedef enum {
    REPRO_F64 = 0, /* double: W = 40 bits per level, grid unit 2^(-1074 + 40 k) */
    REPRO_F32 = 1  /* float:  W = 18 bits per level, grid unit 2^(-149 + 18 k)  */
} repro_dtype;

/* Per-group flags (state layout below). */
#define REPRO_FLAG_NAN 1u     /* a NaN was summed: result is NaN */
#define REPRO_FLAG_POS_INF 2u /* +Inf summed (with -Inf too: NaN) */
#define REPRO_FLAG_NEG_INF 4u /* -Inf summed */
#define REPRO_FLAG_RANGE 8u   /* a finite value >= 2^1005 (double) / 2^120 (float)
                                 was summed: its window would overflow the
                                 running sum of Algorithm 2; result is NaN */

/* Header error bits (repro_state_header.errors). */
#define REPRO_ERR_KEY 1u
#define REPRO_ERR_TIMEOUT 2u
#define REPRO_ERR_LAYOUT 4u

#define REPRO_STATE_MAGIC 0x4f525052u /* "RPRO" */

/*
 * State layout (device memory, canonical: equal sums give equal bytes).
 *
 *   repro_state_header                         64 bytes
 *   group g at 64 + g * (8 + 16 L):
 *     int32_t  K;        grid index of level 0 (level j has unit
 *                        u(K - j) = 2^(g_min + (K - j) W)); the smallest K
 *                        with max |value| < 2^(W-1) u(K) (Algorithm 2's
 *                        raise condition)
 *     uint32_t flags;    REPRO_FLAG_*
 *     { int64_t lo; int64_t hi; } bin[L];
 *                        the exact integer T_j = hi * 2^64 + lo of level j
 *                        (both halves signed), the sum of the digits of the
 *                        group's values at that level; level 0 is the top.
 * An empty group has K = 0, flags = 0 and zero bins.  T_j * u(K - j) is the
 * level's exact value, i.e. (S - 1.5 ufp(S)) + 0.25 ufp(S) C of the paper's
 * <S, C> pair.
 */
typedef struct {
    uint32_t magic;      /* REPRO_STATE_MAGIC */
    uint32_t dtype;      /* repro_dtype */
    uint32_t L;
    uint32_t errors;     /* REPRO_ERR_* bits, OR-ed by kernels */
    int64_t num_groups;
    uint8_t reserved[40];
} repro_state_header;

/* Bytes of a state for num_groups groups: 64 + num_groups * (8 + 16 L).
   Returns 0 for invalid arguments. */
size_t repro_state_bytes(repro_dtype dtype, int L, int64_t num_groups);

/* Write an empty state (header + all groups empty) into `state`, which must
   hold repro_state_bytes() bytes and be 16-byte aligned. */
repro_status repro_state_init(void* state, repro_dtype dtype, int L, int64_t num_groups,
                              void* stream);

/*
 * Grouped reproducible SUM: for each row i, add values[i] to group keys[i]
 * of `state` (accumulating: the state may already hold earlier calls' rows,
 * which is how the paper's resumable summation state is used, Sec. III-C).
 *
 * keys:   int32[n] device array, group ids in [0, num_groups).  Rows with a
 *         key outside that range are skipped and set REPRO_ERR_KEY.
 * values: double[n] (REPRO_F64) or float[n] (REPRO_F32) device array.
 *         NaN / +-Inf / out-of-range values set the group's flags and add
 *         nothing to its bins.
 * n:      rows; 0 is allowed (no-op).  keys and values must be 4- and
 *         8/4-byte aligned.
 * state:  in-out, initialised by repro_state_init with the same dtype / L /
 *         num_groups.
 * Steps (paper sections): per-group window from max |value| (Algorithm 2,
 * check extractor validity); L-digit extraction against the window
 * (Algorithm 2, transform; constant extractor so ties round to even);
 * exact accumulation (the carry-bit counts of Algorithm 2 become wide
 * integer bins); per-call partial states merged into `state` with
 * operator+=(repro) (Sec. V-B, Algorithm 4).  Group counts beyond one
 * shared-memory table are partitioned first (Algorithm 4's
 * ParallelPartition, one or two passes); when the keys are skewed (the
 * fullest partition above four times the mean, seen on the device) and
 * there are more than 64 partitions, partitions are cut into shorter work
 * items (8 per CTA instead of 2) unless a tuned choice says otherwise.
 */
repro_status repro_groupby_sum(const int32_t* keys, const void* values, int64_t n,
                               repro_dtype dtype, int L, int64_t num_groups, void* state,
                               void* stream);

/*
 * repro_groupby_sum with the partitioning depth chosen from the data.  The
 * paper picks the number of partitioning levels by the number of groups:
 * enough levels that the last one aggregates in cache, no more, and it
 * proposes choosing them adaptively, from the groups actually met, instead
 * of offline (Sec. V-C, "Tuning Buffer Size and Partitioning Depth").  Here
 * num_groups only bounds the keys.  When it exceeds one shared-memory table,
 * the partitioned path planned for num_groups starts, and its first
 * histogram pass (which reads every key anyway) also takes the keys' range;
 * the stream is synchronised once (range and partition row counts read
 * back), and if the groups the keys reach,
 * max(key) + 1, call for another plan -- no partitioning while one table
 * holds them (a single pass over records [0, max(key)]), else one or two
 * partition passes sized for that many groups; when the keys are skewed
 * (the fullest partition above four times the mean) and no tuned choice
 * applies, one pass into partitions small enough for lane-private table
 * copies where at most 2048 partitions cover the groups, else one wide pass
 * instead of two where that covers them -- the call stops there and runs
 * that plan instead; otherwise it goes on.  In both plans skewed keys
 * (the fullest partition above four times the mean, seen on the device)
 * cut their partitions into shorter work items when there are more than 64
 * partitions and no tuned choice, as in repro_groupby_sum.  Same
 * arguments and the same result bits as repro_groupby_sum.  *depth_out (may
 * be NULL) receives the partition passes taken: 0, 1 or 2, or -1 when the
 * call went the plain way without looking at the keys (keys or values not
 * 16-byte aligned, a stream under capture, or the two-pass path).  Keys
 * outside [0, num_groups) keep the plan for num_groups, which flags them.
 * Unlike repro_groupby_sum this call synchronises `stream` once when it
 * reads the range.
 */
repro_status repro_groupby_sum_adaptive(const int32_t* keys, const void* values, int64_t n, repro_dtype dtype, int L,
                                        int64_t num_groups, void* state, int* depth_out, void* stream);

/*
 * repro_groupby_sum on columns in page-locked HOST memory (cudaHostAlloc /
 * pinned tensors; anything else is REPRO_EINVAL): the rows are staged in
 * chunks of 2^24 through two device buffers from the library's pool, copied
 * on a library-owned stream, each chunk aggregated on `stream` behind its
 * copy while the next one is in flight (chunks merge exactly, so the state
 * is that of one call on the whole input).  Asynchronous: the host columns
 * must stay unchanged until `stream` has passed this call.  Not for stream
 * capture (the copy stream is shared by all callers on a device).
 */
repro_status repro_groupby_sum_host(const int32_t* keys, const void* values, int64_t n, repro_dtype dtype, int L,
                                    int64_t num_groups, void* state, void* stream);

/*
 * Several SUM aggregates over one grouping given as two low-cardinality
 * uint8 key columns (SQL: SELECT SUM(c0), SUM(c1), ... GROUP BY k1, k2, the
 * shape of the paper's TPC-H Q1 aggregation, Sec. VI-E): the group of row i
 * is key1[i] * card2 + key2[i] (rows whose composite key is not below
 * num_groups are skipped and flag REPRO_ERR_KEY in every state), and column
 * c is added into states[c] exactly as repro_groupby_sum would.
 * cols and states are HOST arrays of ncols DEVICE pointers.  Scratch: 4
 * bytes per row for the composite keys.
 */
repro_status repro_groupby_sum_cols(const uint8_t* key1, const uint8_t* key2, int card2,
                                    const void* const* cols, int ncols, int64_t n, repro_dtype dtype,
                                    int L, int64_t num_groups, void* const* states, void* stream);

/*
 * Reproducible SUM without GROUP BY (one group): values[0 .. n) are added
 * into `state`, a state made with num_groups = 1 (its header is checked on
 * the device; a mismatch sets REPRO_ERR_LAYOUT).  Same bits as
 * repro_groupby_sum with an all-zero key column, without reading one: the
 * single-pass kernel runs keyless when values are 16-byte aligned, else the
 * grouped path runs on a zero key column in scratch.  Across ranks the
 * states merge like any other (the paper's MPI_Reduce remark, Sec. III).
 */
repro_status repro_sum(const void* values, int64_t n, repro_dtype dtype, int L, void* state, void* stream);

/*
 * The paper's unbuffered data type as a library routine (Sec. IV): the same
 * SUM as repro_sum (same state bits), but every thread adds its rows one by
 * one into its own repro_accum (include/repro_accum.cuh), and the CTAs merge
 * their accumulators.  A comparison point for the cost of the naive type
 * next to the buffered shared-memory tables.  state: num_groups = 1.
 */
repro_status repro_sum_unbuffered(const void* values, int64_t n, repro_dtype dtype, int L, void* state,
                                  void* stream);

/*
 * DECIMAL baseline: SUM of int64 values (a fixed-point column as scaled
 * integers, e.g. cents) per group into out[num_groups] (zeroed first),
 * exact and order-independent by integer arithmetic (wraps around on
 * int64 overflow).  Keys outside [0, num_groups) are skipped.  A comparison
 * point: fixed-point types are the reproducible alternative the paper sets
 * the floating-point method against (Sec. II, VI).
 */
repro_status groupby_sum_decimal64(const int32_t* keys, const int64_t* values, int64_t n, int64_t num_groups,
                                   int64_t* out, void* stream);

/*
 * repro_groupby_sum without any allocation.  The paper has no counterpart:
 * this is a deployment variant of repro_groupby_sum for callers that cannot
 * allocate device memory while they aggregate -- a host whose buffer
 * manager has reserved the GPU's memory up front, a process whose allocator
 * belongs to another runtime, or a request path that must not wait on, or
 * fail in, an allocation.  Same arguments, same result bits as
 * repro_groupby_sum.
 *
 * It runs the single-pass shared-memory path only, with its per-CTA partial
 * tables in a fixed 16 MiB device array inside the library (held by every
 * GPU that loads the library until the process exits), using fewer CTAs
 * when needed so that they fit.  Limits: keys and values 16-byte aligned,
 * and a group table that fits the single-pass path (num_groups up to a few
 * thousand, depending on L and dtype) with num_groups * (8 + 16 L) <= 16 MiB;
 * otherwise REPRO_ERANGE and nothing is enqueued.  Each call that is not
 * under stream capture looks the array's address up (cudaGetSymbolAddress,
 * with the device current), so a context created after cudaDeviceReset is
 * served correctly; a call under capture reuses the address of the last
 * uncaptured call on that device, so make one such call on each device
 * before any capture (else REPRO_ECUDA).  Every call uses the same array:
 * calls that overlap on the GPU race (serialise them on one stream).
 * Nothing needs clearing between calls.
 */
repro_status repro_groupby_sum_noalloc(const int32_t* keys, const void* values, int64_t n,
                                       repro_dtype dtype, int L, int64_t num_groups, void* state,
                                       void* stream);

/*
 * Batched grouped SUM: many independent aggregations (each with its own
 * keys, values, group count and state) in a few persistent launches.  Same
 * result bits per task as repro_groupby_sum on that task alone.
 *
 * repro_batch_prepare builds a plan on the host (it allocates device memory
 * with cudaMalloc and copies the task list and the work items to it; not
 * capturable).  repro_batch_run enqueues the plan's kernels on `stream`
 * without host copies or allocations, so it may be captured in a CUDA graph
 * and replayed; every run adds the tasks' rows into their states again.
 * repro_batch_destroy frees the plan (it synchronises the device).
 * repro_groupby_sum_batched = prepare + run + stream synchronise + destroy.
 *
 * Tasks whose rows are 16-byte aligned and whose group table fits the
 * single-pass path share persistent launches, one per table class (up to 64
 * groups, up to 1024, larger), each configured for its own largest table:
 * the plan cuts them into work items of whole tiles (the item size is tuned
 * to the batch: about four items per CTA, at most 2^23 rows), largest first;
 * an item that covers a whole task merges straight into its state.  Tasks with more groups
 * than one shared-memory table holds (and 16-byte aligned rows, up to 2^19
 * groups) share one batched partition pass -- one partitioning of all of
 * them and one multi-task launch over their partitions -- on a side stream
 * forked from `stream` and joined back; any other task (larger group
 * counts, unaligned rows) runs its own partitioned or two-pass chain on
 * eight more side streams.
 * All tasks use the same dtype and L; states must not overlap.
 */
typedef struct {
    const int32_t* keys;   /* device, int32[n] */
    const void* values;    /* device, double[n] or float[n] */
    int64_t n;             /* rows, >= 0 */
    int64_t num_groups;    /* 1 .. 2^31 - 1 */
    void* state;           /* device state (repro_state_init with the batch's dtype and L) */
} repro_task;

typedef struct repro_batch_plan_s* repro_batch_plan;

repro_status repro_batch_prepare(const repro_task* tasks, int ntasks, repro_dtype dtype, int L,
                                 repro_batch_plan* plan);
repro_status repro_batch_run(repro_batch_plan plan, void* stream);
repro_status repro_batch_destroy(repro_batch_plan plan);
/* How a prepared plan runs its tasks (a diagnostic; nothing is launched). */
typedef struct {
    int32_t tasks;             /* tasks of the plan (including empty ones) */
    int32_t single_pass_tasks; /* in the persistent launches */
    int32_t partition_tasks;   /* in the batched partition pass */
    int32_t lane_tasks;        /* each on its own side-stream chain */
    int32_t items;             /* work items of the persistent launches */
    int32_t merge_blocks;
    int32_t items_per_cta;     /* item sizing target (repro_batch_tune may change it) */
    int32_t partition_overlap; /* 1: the partition pass runs beside the persistent launches, 0: before them */
    int64_t device_bytes;      /* device memory the plan holds */
    int32_t class_tasks[3];    /* single-pass tasks per table class (G <= 64, <= 1024, larger), one
                                  persistent launch per class with tasks, each sized for its own largest table */
    int32_t reserved;
} repro_batch_info;

repro_status repro_batch_describe(repro_batch_plan plan, repro_batch_info* out);

/* Re-initialise every task's state (one launch; capturable). */
repro_status repro_batch_reset(repro_batch_plan plan, void* stream);

/* Give the plan one output per task (HOST array of ntasks DEVICE pointers to
   num_groups elements of the dtype, or NULL to skip a task); copied to the
   device synchronously, like repro_batch_prepare. */
repro_status repro_batch_set_outputs(repro_batch_plan plan, void* const* outs);

/* Finalize every task with an output into it (one launch; capturable).
   REPRO_EINVAL before repro_batch_set_outputs. */
repro_status repro_batch_finalize(repro_batch_plan plan, void* stream);

repro_status repro_groupby_sum_batched(const repro_task* tasks, int ntasks, repro_dtype dtype, int L,
                                       void* stream);

/* dst += src, group by group (operator+=(repro), Sec. V-B; eq. (2)/(3) for
   equal windows): both are aligned to the larger window, levels that fall
   below it are dropped, bins are added exactly and flags OR-ed.  Exact, so
   any merge order or tree gives the same bytes.  dst and src may not
   overlap. */
repro_status repro_merge(void* dst, const void* src, repro_dtype dtype, int L,
                         int64_t num_groups, void* stream);

/*
 * dst += src over two arrays of num_records bare group records (the record
 * layout above, no header), in place: the same per-record merge as
 * repro_merge (operator+=(repro), Sec. V-B; eq. (2)/(3) for equal windows,
 * the larger window and dropped low levels otherwise).  For blocks of
 * records that ranks exchange (a reduce-scatter of states by group ranges):
 * no state has to be built around a block to merge it.  Both arrays 8-byte
 * aligned, device memory, not overlapping; src is only read.  The dtype is
 * not needed (records are integers).  REPRO_EINVAL for bad arguments.
 */
repro_status repro_merge_records(void* dst, const void* src, int L, int64_t num_records, void* stream);

/* out[g] = the group's reproducible sum (eq. (1)): V_j = T_j * u(K - j)
   rounded to nearest even in T (gradual underflow, overflow to +-Inf), then
   Q = (((V_{L-1} + V_{L-2}) + ...) + V_0) in T arithmetic.  A group with
   NaN or RANGE flags, or both infinities, gives the quiet NaN
   0x7ff8000000000000 / 0x7fc00000; +Inf or -Inf alone gives that infinity;
   an empty group gives +0.0.  out is double[num_groups] or float[num_groups]. */
repro_status repro_finalize(const void* state, repro_dtype dtype, int L, int64_t num_groups,
                            void* out, void* stream);

/* Synchronise `stream` and report the state's error bits: REPRO_EKEY,
   REPRO_ETIMEOUT or REPRO_ELAYOUT (first one set, in that order), else
   REPRO_OK.  If errors_out is not NULL it receives the raw bits.  The bits
   stay set until repro_state_init. */
repro_status repro_state_check(const void* state, uint32_t* errors_out, void* stream);

/* Conventional, NON-reproducible grouped SUM: out[g] = sum of values[i]
   with keys[i] == g, added with built-in floating-point adds in whatever
   order the GPU runs them (the "built-in" baseline the paper compares
   against, Sec. VI-C and VI-D).  out (double[num_groups]) is overwritten.
   Rows with a key outside [0, num_groups) are skipped.  Same input handling
   as the reproducible kernels (16-byte vector loads when keys and values
   are 16-byte aligned, persistent grid); the table strategy is picked by
   group count: one shared-memory copy per lane for small tables, one shared
   table with equal keys of a warp combined first up to the shared-memory
   limit, global atomics (again combined per warp) beyond. */
repro_status groupby_sum_fp64(const int32_t* keys, const double* values, int64_t n,
                              int64_t num_groups, double* out, void* stream);

/* Float variant of the conventional baseline (float accumulators). */
repro_status groupby_sum_fp32(const int32_t* keys, const float* values, int64_t n,
                              int64_t num_groups, float* out, void* stream);

/* The conventional baseline with an explicit table strategy, so that a
   benchmark can time them all and keep the fastest: mode 0 shared table
   (one copy per lane when the copies fit), 1 shared table with equal keys
   combined per warp (__match_any_sync), 2 one shared table per warp (plain
   adds after the combining), 3 global atomics, 4 global atomics after the
   combining.  values: double or float per dtype; out: num_groups of that
   type, overwritten.  REPRO_ERANGE if the mode's tables do not fit in shared
   memory for num_groups, REPRO_EINVAL for a bad mode or argument. */
repro_status groupby_sum_fp_mode(const int32_t* keys, const void* values, int64_t n, repro_dtype dtype,
                                 int64_t num_groups, int mode, void* out, void* stream);

/*
 * SQL aggregates from reproducible sums.  The paper observes that with a
 * reproducible SUM every SQL aggregate becomes reproducible: COUNT needs no
 * floating point, AVG, VARIANCE and STDDEV are functions of SUM(x) and
 * SUM(x^2) (Sec. I).  A stats state holds a repro state of x, one of x*x
 * (each product rounded to nearest in the dtype) and an exact uint64 row
 * count per group; repro_stats_state_bytes gives its size (16-byte aligned
 * device memory, caller-owned).  repro_groupby_stats accumulates rows like
 * repro_groupby_sum (keys outside [0, num_groups) are skipped and flag
 * REPRO_ERR_KEY in the first part's header, read by repro_state_check);
 * scratch: none beyond the single pass's partial tables when the group
 * table fits on chip (the x*x pass squares each staged value in place),
 * else one value column.  repro_stats_merge adds one state into another
 * (states of the same shape, not overlapping).
 *
 * repro_stats_finalize writes, per group g (any pointer may be NULL; value
 * arrays are of the dtype, count int64):
 *   count = rows (the presence column: count > 0),
 *   sum = SUM(x) as repro_finalize, mean = sum / count,
 *   D = SUMSQ - (sum * sum) / count, clamped at 0 (each operation rounded to
 *   nearest in the dtype, in this order),
 *   var_samp = D / (count - 1), var_pop = D / count, stddev_* = sqrt(var_*).
 * Empty groups give NaN for mean and the variances, one row NaN for var_samp
 * (SQL's NULL).  The count is converted to the dtype exactly below 2^53
 * (2^24 for float), rounded above.
 */
typedef struct {
    int64_t* count;
    void* sum;
    void* mean;
    void* var_samp;
    void* var_pop;
    void* stddev_samp;
    void* stddev_pop;
} repro_stats_out;

size_t repro_stats_state_bytes(repro_dtype dtype, int L, int64_t num_groups);
repro_status repro_stats_init(void* state, repro_dtype dtype, int L, int64_t num_groups, void* stream);
repro_status repro_groupby_stats(const int32_t* keys, const void* values, int64_t n, repro_dtype dtype, int L,
                                 int64_t num_groups, void* state, void* stream);
repro_status repro_stats_merge(void* dst, const void* src, repro_dtype dtype, int L, int64_t num_groups,
                               void* stream);
repro_status repro_stats_finalize(const void* state, repro_dtype dtype, int L, int64_t num_groups,
                                  const repro_stats_out* out, void* stream);

/*
 * Request server: continuous batching of aggregation queries.
 *
 * The paper aggregates one relation per query (Sec. II problem statement,
 * Sec. V Algorithm 4); a server answers many such queries that arrive over
 * time, without changing any query's result: every bin add is exact, so a
 * query's state, and so its result, is the same whatever it shares the
 * device with (Sec. III reproducibility requirement).
 *
 * A scheduler thread admits submitted queries in arrival order while their
 * device memory (state plus scratch, estimated at submit) fits the budget and
 * a slot is free.  It then runs iterations: each iteration takes the next
 * chunk_rows rows of every admitted query; chunks whose group table fits the
 * single-pass kernel go into one multi-task persistent launch (one per table
 * class when the iteration holds 2^26 rows or more); the chunks of
 * queries that need partitioning go into one batched partition pass on a
 * second stream (aligned columns, up to 2^19 groups) or, otherwise, through
 * the partitioned path on one of three more streams.  Partial states stay on
 * the device between iterations.  After its last chunk a query is finalized
 * into its output and its state freed; a host callback stamps the completion
 * time.  At most max_inflight iterations are queued ahead of the device.
 */
typedef struct repro_server_s* repro_server;

typedef struct {
    int64_t memory_budget; /* bytes for admitted queries' states + scratch; 0: a quarter of free memory */
    int64_t chunk_rows;    /* rows per query per iteration, rounded up to a multiple of 4096; 0: 2^24 */
    int32_t max_active;    /* admitted queries at a time; 0: 256 */
    int32_t max_inflight;  /* iterations queued on the device; 0: 3 */
} repro_server_config;

typedef struct {
    int32_t done;       /* 1 once out holds the result */
    int32_t status;     /* repro_status of the query: data errors as repro_state_check reports them */
    uint32_t errors;    /* the state's error word (REPRO_ERR_*) */
    uint32_t reserved;
    int64_t arrival_ns; /* repro_server_now_ns() clock: arrival, admission, result in out */
    int64_t admit_ns;
    int64_t done_ns;
} repro_request_info;

typedef struct {
    int64_t submitted, completed;
    int64_t iterations;     /* scheduler iterations issued */
    int64_t batch_launches; /* multi-task launches */
    int64_t large_calls;    /* partitioned-path chunk calls */
    /* Device memory, bytes: in use now and the peak -- the admitted queries'
       charges (state + one chunk's partitioned-path scratch each) plus the
       server's own buffers (iteration plans and partial tables, held until
       destroy; partition-pass scratch while its iteration is in flight).
       Admission keeps this within memory_budget, except that a query is
       always admitted when no other one is, so the peak can exceed the
       budget by at most memory_server_peak. */
    int64_t memory_in_use, memory_peak, memory_budget;
    int32_t active, waiting; /* admitted and not finished; arrived and not admitted */
    int64_t memory_server_peak; /* peak of the server's own buffers alone */
} repro_server_stats;

/* Monotonic clock of the server's timestamps, in nanoseconds. */
int64_t repro_server_now_ns(void);

/* Create a server on the current device (cfg may be NULL for defaults). */
repro_status repro_server_create(const repro_server_config* cfg, repro_server* out);

/*
 * Submit one query: SUM of values grouped by keys (as repro_groupby_sum) into
 * a fresh state, finalized into out (num_groups elements of the dtype).
 * keys and values: DEVICE memory of the server's device, unchanged until the
 * query is done.  out: device memory or page-locked host memory.
 * ready_event (cudaEvent_t, may be NULL): the server's streams wait on it
 * before reading the inputs.  arrival_ns: the query is not admitted before
 * this time of repro_server_now_ns() (0: now); it is the start of the query's
 * latency.  *id receives the query's handle.
 * REPRO_EINVAL for bad arguments or pointers that are not device-accessible,
 * REPRO_ERANGE if the query alone needs more than the memory budget.
 */
repro_status repro_server_submit(repro_server srv, const int32_t* keys, const void* values, int64_t n,
                                 repro_dtype dtype, int L, int64_t num_groups, void* out, void* ready_event,
                                 int64_t arrival_ns, uint64_t* id);

/* Non-blocking state of a query (info->done = 0 while it runs).  REPRO_EINVAL
   for an unknown or released id. */
repro_status repro_server_poll(repro_server srv, uint64_t id, repro_request_info* info);

/* Wait up to timeout_s seconds for a query: REPRO_ETIMEOUT if it is not done. */
repro_status repro_server_wait(repro_server srv, uint64_t id, double timeout_s, repro_request_info* info);

/* Forget a finished query (REPRO_EINVAL if unknown or still running). */
repro_status repro_server_release(repro_server srv, uint64_t id);

repro_status repro_server_stats_get(repro_server srv, repro_server_stats* st);

/* Finish every submitted query (honouring arrival times), then free the
   server.  Results of unreleased queries are no longer readable. */
repro_status repro_server_destroy(repro_server srv);

/*
 * Autotuning.  The paper picks its partitioning fan-out and buffer sizes per
 * machine offline and notes that the best values depend on the group count
 * (Sec. V-C, Sec. VI).  repro_tune_groupby times every configuration that
 * fits on the caller's inputs -- for the single-pass path its stages, rows
 * per tile, consumer warps, CTAs per SM and table copies; for the
 * partitioned path its partition width (fan-out), the number of partition
 * passes, the aggregation kernel's configuration and its work items per CTA
 * -- and records the fastest
 * for (dtype, L, num_groups rounded up to a power of two); later calls in that
 * bucket use it.  It allocates its own state and scratch, runs each
 * candidate a few times on `stream` and synchronises; the inputs are only
 * read.  No choice changes any result (every candidate computes the same
 * exact bins).  A batch plan or a call that has already chosen keeps its
 * choice.  REPRO_EINVAL for bad arguments or n == 0.
 */
typedef struct {
    int32_t path;            /* 0 single pass, 1 partitioned, 2 two pass (nothing to tune) */
    int32_t candidates;      /* configurations timed */
    int32_t stages, tile_rows, consumer_warps, ctas_per_sm, table_copies; /* single-pass choice */
    int32_t partition_shift; /* partitioned choice: log2 of the groups per partition */
    double best_ms;          /* median time of one call with the choice */
    double default_ms;       /* the same with the built-in rule's choice */
    int32_t partition_levels; /* partitioned choice: partition passes over the rows (1 or 2) */
    int32_t partition_items_per_cta; /* partitioned choice: work items per CTA (0: the built-in default) */
} repro_tune_result;

repro_status repro_tune_groupby(const int32_t* keys, const void* values, int64_t n, repro_dtype dtype, int L,
                                int64_t num_groups, void* stream, repro_tune_result* out);

/* Write / read the recorded choices as text (one choice per line; load
   merges into what is recorded).  REPRO_EINVAL if the file cannot be
   opened or a line is malformed (nothing is loaded then). */
repro_status repro_tune_save(const char* path);
repro_status repro_tune_load(const char* path);

/* Forget every recorded choice (the built-in rule applies again). */
void repro_tune_clear(void);

/* Time the plan with work items of several sizes (about 1, 2, 4, 8 and 16
   items per CTA) and, when it has a batched partition pass, with that pass
   beside the persistent launches and before them; keep the fastest; *best_ms (may be NULL) receives its
   median time per run.  Runs the plan several times on `stream` and
   synchronises; afterwards every task's state is re-initialised (as
   repro_batch_reset). */
repro_status repro_batch_tune(repro_batch_plan plan, void* stream, double* best_ms);

/* Human-readable text for a status code (static storage). */
const char* repro_strerror(repro_status status);

/* Version of the state layout and the library (major * 100 + minor). */
int repro_version(void);

/* Synchronise the current device and return the scratch bytes cached in the
   library's memory pool to the driver. */
repro_status repro_release_cached_memory(void);

/* Profiling aid (not part of the computation).  While enabled, the library
   records a pair of CUDA events on the caller's stream around every launch
   of its row-pass kernels, keyed by kernel name ("window", "accum",
   "fused", "partition", "merge", "finalize", "fp64", "fp32").
   repro_profile_read() waits for the recorded events of that name, returns
   their summed duration in milliseconds and their count, and forgets them.
   Unknown names give REPRO_EINVAL. */
void repro_profile_enable(int on);
repro_status repro_profile_read(const char* kernel, double* total_ms, int64_t* launches);

/* Number of kernel launches the library has made since it was loaded. */
int64_t repro_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* REPRO_H */
