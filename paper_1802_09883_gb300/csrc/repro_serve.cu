// repro_serve.cu -- request server: continuous batching of reproducible
// grouped-SUM queries over a device-memory budget (repro_server_* in
// include/repro.h).
//
// One scheduler thread owns the device work.  Per iteration it
//   1. moves queries whose arrival time has come into the FIFO wait queue and
//      admits from its head while the budget and the slots allow (state from
//      the library pool, initialised in stream order);
//   2. takes the next chunk of every admitted query: chunks of single-pass
//      queries (table fits shared memory) become the tasks of one multi-task
//      persistent launch per (dtype, L) on the batch stream; the chunks of
//      queries that need partitioning join one batched partition pass on a
//      second stream (aligned columns, up to 2^19 groups) or, otherwise, run
//      the partitioned path on one of three more streams (fixed per query,
//      the least loaded at admission);
//   3. finalizes queries that received their last chunk, copies each state's
//      error word to a pinned slot, frees the state in stream order and
//      enqueues a host callback that stamps the completion time and returns
//      the query's memory and slot to the scheduler.
// Reproducibility does not depend on any of these choices: the bins are
// exact integers, so a query's state is the same whichever chunks shared its
// launches (the order-independence of Sec. III / Algorithm 2 with exact
// bins, and the state merge of Algorithm 4).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include "batch_plan.h"
#include "multi_types.h"
#include "repro.h"
#include "repro_internal.h"

namespace rp {
namespace {

using Clock = std::chrono::steady_clock;

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

repro_status status_of(uint32_t err) {
    if (err & REPRO_ERR_KEY) return REPRO_EKEY;
    if (err & REPRO_ERR_TIMEOUT) return REPRO_ETIMEOUT;
    if (err & REPRO_ERR_LAYOUT) return REPRO_ELAYOUT;
    return REPRO_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Partial tables of one iteration's batch stay below this where the work
// allows (the planner makes items longer otherwise).
constexpr size_t kServePartBytes = 256ull << 20;
constexpr long long kServeClassRows = 1ll << 26;  // iterations with fewer rows: one persistent launch

// Stream 0 runs the batched single-pass launches; stream 1 the batched
// partition pass of the queries whose tables need partitioning (aligned
// columns, at most kPartLaneGroups groups); streams 2 .. kLanes-1 run the
// remaining large queries, each query on one of them.
constexpr int kLanes = 5;
constexpr long long kPartLaneGroups = 1 << 19;

struct Req {
    uint64_t id = 0;
    const int32_t* keys = nullptr;
    const void* vals = nullptr;
    long long n = 0;
    int dtype = 0, L = 0;
    long long G = 0;
    void* out = nullptr;
    cudaEvent_t ready = nullptr;
    int64_t arrival_ns = 0, admit_ns = 0, done_ns = 0;
    bool done = false;
    repro_status status = REPRO_OK;
    uint32_t errors = 0;
    long long pos = 0;   // rows issued so far
    int lane = 0;        // 0: batch stream, 1: batched partition pass, else a partitioned-path stream
    bool large = false;  // needs the partitioned path
    bool part_lane = false;  // its chunks join the batched partition pass
    void* state = nullptr;
    size_t need = 0;     // bytes charged to the budget while admitted
    int slot = -1;       // pinned error-word slot
};

// Device + pinned host buffers of one batch launch, reused across iterations.
struct Arena {
    unsigned char* host = nullptr;
    size_t host_cap = 0;
    unsigned char* dev = nullptr;
    size_t dev_cap = 0;
};

struct Iter {
    std::vector<Arena*> arenas;
    cudaEvent_t ev[kLanes] = {};
    long long pass_bytes = 0;  // partition-pass scratch of this iteration, charged until it retires
};

struct Server;

struct Completion {
    Server* srv;
    std::vector<Req*> reqs;
};

void CUDART_CB on_complete(void* p);

struct Server {
    repro_server_config cfg{};
    int device = 0;
    cudaMemPool_t pool = nullptr;
    cudaStream_t stream[kLanes] = {};
    uint32_t* err_words = nullptr;  // pinned, one per slot

    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::multimap<int64_t, Req*> pending;  // by arrival time
    std::deque<Req*> waitq;
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    std::vector<int> free_slots;
    long long in_use = 0, peak = 0;
    // the server's own device buffers: iteration arenas (held until destroy)
    // and the partition-pass scratch of iterations in flight
    long long own = 0, own_peak = 0;
    int admitted = 0;  // admitted and not yet completed
    uint64_t next_id = 1;
    bool stop = false;
    repro_status fatal = REPRO_OK;
    repro_server_stats st{};

    // scheduler-thread state
    std::vector<Req*> active;  // admitted queries with rows left to issue
    std::deque<Iter> inflight;
    std::vector<Arena*> free_arenas, all_arenas;
    std::vector<cudaEvent_t> free_events;
    std::thread thr;

    cudaEvent_t take_event() {
        if (!free_events.empty()) {
            cudaEvent_t e = free_events.back();
            free_events.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        return e;
    }

    // Charge (bytes > 0) or release the server's own device memory; the
    // footprint's peak counts it with the admitted queries' charges.
    void charge_own(long long bytes) {
        std::lock_guard<std::mutex> lk(mu);
        own += bytes;
        own_peak = std::max(own_peak, own);
        peak = std::max(peak, in_use + own);
    }

    Arena* take_arena() {
        if (!free_arenas.empty()) {
            Arena* a = free_arenas.back();
            free_arenas.pop_back();
            return a;
        }
        Arena* a = new Arena;
        all_arenas.push_back(a);
        return a;
    }

    void retire_oldest() {
        Iter& it = inflight.front();
        for (cudaEvent_t e : it.ev)
            if (e) {
                cudaEventSynchronize(e);
                free_events.push_back(e);
            }
        for (Arena* a : it.arenas) free_arenas.push_back(a);
        if (it.pass_bytes) charge_own(-it.pass_bytes);
        inflight.pop_front();
    }

    // Fail every query that is not yet on the device (after a launch error).
    void fail_all(repro_status why) {
        std::lock_guard<std::mutex> lk(mu);
        fatal = why;
        const int64_t t = now_ns();
        auto fail = [&](Req* r) {
            r->status = why;
            r->done = true;
            r->done_ns = t;
        };
        for (auto& kv : pending) fail(kv.second);
        pending.clear();
        for (Req* r : waitq) fail(r);
        waitq.clear();
        for (Req* r : active) fail(r);
        active.clear();
        cv_done.notify_all();
    }

    cudaError_t launch_batch(int dtype, int L, const std::vector<repro_task>& tasks, Iter& it) {
        // a light iteration runs as one persistent launch (latency), a heavy
        // one by table class (throughput)
        long long rows = 0;
        for (const repro_task& k : tasks) rows += k.n;
        HostBatch H;
        if (plan_batch_host(tasks.data(), (int)tasks.size(), dtype, L, kServePartBytes, H, 4, nullptr,
                            rows < kServeClassRows) != REPRO_OK)
            return cudaErrorInvalidValue;
        if (!H.slow.empty()) return cudaErrorInvalidValue;  // admission routes these to the other lane
        if (H.items.empty()) return cudaSuccess;
        const size_t tb = align256(sizeof(MTask) * H.tasks.size());
        const size_t ib = align256(sizeof(MItem) * H.items.size());
        const size_t bb = align256(sizeof(MergeBlk) * std::max<size_t>(1, H.blks.size()));
        const size_t host_need = tb + ib + bb;
        const size_t dev_need = host_need + 256 + std::max<size_t>(16, (size_t)H.part_recs * batch_rec_bytes(L));
        Arena* a = take_arena();
        it.arenas.push_back(a);
        cudaError_t e = cudaSuccess;
        if (a->host_cap < host_need) {
            if (a->host) cudaFreeHost(a->host);
            a->host = nullptr;
            a->host_cap = std::max(host_need, (size_t)256 << 10);
            e = cudaHostAlloc((void**)&a->host, a->host_cap, cudaHostAllocDefault);
            if (e != cudaSuccess) {
                a->host_cap = 0;
                return e;
            }
        }
        if (a->dev_cap < dev_need) {
            if (a->dev) cudaFreeAsync(a->dev, stream[0]);
            a->dev = nullptr;
            const long long old_cap = (long long)a->dev_cap;
            a->dev_cap = std::max(dev_need, a->dev_cap * 2);
            charge_own((long long)a->dev_cap - old_cap);
            e = cudaMallocFromPoolAsync((void**)&a->dev, a->dev_cap, pool, stream[0]);
            if (e != cudaSuccess) {
                charge_own(-(long long)a->dev_cap);
                a->dev_cap = 0;
                return e;
            }
        }
        std::memcpy(a->host, H.tasks.data(), sizeof(MTask) * H.tasks.size());
        std::memcpy(a->host + tb, H.items.data(), sizeof(MItem) * H.items.size());
        if (!H.blks.empty()) std::memcpy(a->host + tb + ib, H.blks.data(), sizeof(MergeBlk) * H.blks.size());
        e = cudaMemcpyAsync(a->dev, a->host, host_need, cudaMemcpyHostToDevice, stream[0]);
        if (e != cudaSuccess) return e;
        int* counter = (int*)(a->dev + host_need);
        unsigned char* partials = a->dev + host_need + 256;
        for (const BatchClass& B : H.cls) {  // one persistent launch per table class, in stream order
            if (B.nitems == 0) continue;
            e = launch_multi(dtype, L, B.cfg, B.gcap, a->dev, a->dev + tb + sizeof(MItem) * (size_t)B.item0, B.nitems,
                             nullptr, counter, partials, std::min(B.ctas, B.nitems), stream[0]);
            if (e != cudaSuccess) return e;
        }
        if (!H.blks.empty())
            e = launch_merge_items(L, dtype, a->dev, a->dev + tb + ib, (int)H.blks.size(), nullptr, partials,
                                   stream[0]);
        return e;
    }

    // The batched partition pass over this iteration's chunks of the
    // partition-lane queries: tables from a pinned arena, scratch from the
    // pool in stream order, all on stream 1.  If the chunks do not qualify
    // as one pass (they always should), each runs the dispatcher instead.
    cudaError_t launch_part(int dtype, int L, const std::vector<BatchPartInput>& in, Iter& it) {
        BatchPartition bp;
        cudaStream_t s = stream[1];
        if (!bp.plan(dtype, L, in)) {
            for (const BatchPartInput& x : in)
                if (groupby_dispatch(x.keys, x.vals, x.n, dtype, L, x.G, x.state, s) != REPRO_OK)
                    return cudaErrorUnknown;
            return cudaSuccess;
        }
        Arena* a = take_arena();
        it.arenas.push_back(a);
        cudaError_t e = cudaSuccess;
        if (a->host_cap < bp.table_bytes()) {
            if (a->host) cudaFreeHost(a->host);
            a->host = nullptr;
            a->host_cap = std::max(bp.table_bytes(), (size_t)256 << 10);
            e = cudaHostAlloc((void**)&a->host, a->host_cap, cudaHostAllocDefault);
            if (e != cudaSuccess) {
                a->host_cap = 0;
                return e;
            }
        }
        void* scratch = nullptr;
        it.pass_bytes += (long long)bp.scratch_bytes();
        charge_own((long long)bp.scratch_bytes());
        e = cudaMallocFromPoolAsync(&scratch, bp.scratch_bytes(), pool, s);
        if (e == cudaSuccess) e = bp.upload_async(scratch, a->host, s);
        if (e == cudaSuccess) e = bp.launch(scratch, s);
        if (scratch) cudaFreeAsync(scratch, s);
        return e;
    }

    // One iteration over the admitted queries; false after a launch error.
    bool issue(std::vector<Req*>& admitted_now) {
        cudaError_t e = cudaSuccess;
        for (Req* r : admitted_now) {
            if (r->part_lane) {
                r->lane = 1;
            } else if (r->large) {  // the partitioned lane with the fewest rows left to issue
                long long left[kLanes] = {};
                for (Req* q : active) left[q->lane] += q->n - q->pos;
                r->lane = 2;
                for (int l = 3; l < kLanes; ++l)
                    if (left[l] < left[r->lane]) r->lane = l;
            }
            cudaStream_t s = stream[r->lane];
            if (r->ready) e = cudaStreamWaitEvent(s, r->ready, 0);
            const size_t sb = repro_state_bytes((repro_dtype)r->dtype, r->L, r->G);
            if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&r->state, sb, pool, s);
            if (e == cudaSuccess) e = launch_init_state(r->state, r->dtype, r->L, r->G, s);
            if (e != cudaSuccess) return false;
            active.push_back(r);
        }
        admitted_now.clear();
        if (active.empty()) return true;
        while ((int)inflight.size() >= cfg.max_inflight) retire_oldest();
        inflight.emplace_back();
        Iter& it = inflight.back();
        std::map<std::pair<int, int>, std::vector<repro_task>> batches;
        std::map<std::pair<int, int>, std::vector<BatchPartInput>> parts;
        std::vector<Req*> fin[kLanes], keep;
        long long large_calls = 0;
        for (Req* r : active) {
            const long long rows = std::min<long long>(cfg.chunk_rows, r->n - r->pos);
            if (rows > 0) {
                const int32_t* k = r->keys + r->pos;
                const void* v = (const char*)r->vals + (size_t)r->pos * (r->dtype == REPRO_F64 ? 8 : 4);
                if (r->lane == 0) {
                    batches[{r->dtype, r->L}].push_back(repro_task{k, v, rows, r->G, r->state});
                } else if (r->lane == 1) {
                    parts[{r->dtype, r->L}].push_back(
                        BatchPartInput{k, v, rows, (int)r->G, (unsigned char*)r->state});
                } else {
                    const int st_ = groupby_dispatch(k, v, rows, r->dtype, r->L, r->G, r->state, stream[r->lane]);
                    if (st_ != REPRO_OK) {
                        for (Req* q : keep) active.push_back(q);
                        return false;
                    }
                    ++large_calls;
                }
                r->pos += rows;
            }
            (r->pos >= r->n ? fin[r->lane] : keep).push_back(r);
        }
        active.swap(keep);
        // on an error, queries not yet handed to a completion callback go back
        // to the active list, which fail_all() then reports
        auto give_back = [&](int from) {
            for (int l = from; l < kLanes; ++l)
                for (Req* r : fin[l]) active.push_back(r);
            return false;
        };
        long long launches = 0;
        for (auto& b : batches) {
            if (launch_batch(b.first.first, b.first.second, b.second, it) != cudaSuccess) return give_back(0);
            ++launches;
        }
        for (auto& b : parts) {
            if (launch_part(b.first.first, b.first.second, b.second, it) != cudaSuccess) return give_back(0);
            ++large_calls;
        }
        for (int l = 0; l < kLanes; ++l) {
            if (fin[l].empty()) continue;
            for (Req* r : fin[l]) {
                e = launch_finalize(r->state, r->dtype, r->L, r->G, r->out, stream[l]);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(&err_words[r->slot], &((const repro_state_header*)r->state)->errors,
                                        sizeof(uint32_t), cudaMemcpyDeviceToHost, stream[l]);
                if (e == cudaSuccess) e = cudaFreeAsync(r->state, stream[l]);
                if (e != cudaSuccess) return give_back(l);
                r->state = nullptr;
            }
            Completion* c = new (std::nothrow) Completion{this, fin[l]};
            if (!c || cudaLaunchHostFunc(stream[l], on_complete, c) != cudaSuccess) {
                delete c;
                return give_back(l);
            }
            fin[l].clear();
        }
        for (int l = 0; l < kLanes; ++l) {
            it.ev[l] = take_event();
            if (!it.ev[l] || cudaEventRecord(it.ev[l], stream[l]) != cudaSuccess) return false;
        }
        std::lock_guard<std::mutex> lk(mu);
        st.iterations += 1;
        st.batch_launches += launches;
        st.large_calls += large_calls;
        return true;
    }

    void run() {
        cudaSetDevice(device);
        std::vector<Req*> admitted_now;
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(mu);
                for (;;) {
                    if (fatal != REPRO_OK) break;
                    const int64_t t = now_ns();
                    while (!pending.empty() && pending.begin()->first <= t) {
                        waitq.push_back(pending.begin()->second);
                        pending.erase(pending.begin());
                    }
                    // the server's own buffers count against the budget; a query
                    // is always admitted when no other one is (progress)
                    while (!waitq.empty() && admitted < cfg.max_active && !free_slots.empty() &&
                           (admitted == 0 ||
                            in_use + own + (long long)waitq.front()->need <= cfg.memory_budget)) {
                        Req* r = waitq.front();
                        waitq.pop_front();
                        r->slot = free_slots.back();
                        free_slots.pop_back();
                        r->admit_ns = now_ns();
                        in_use += (long long)r->need;
                        peak = std::max(peak, in_use + own);
                        ++admitted;
                        admitted_now.push_back(r);
                    }
                    if (!active.empty() || !admitted_now.empty()) break;
                    if (stop && pending.empty() && waitq.empty()) break;
                    if (!pending.empty())
                        cv_sched.wait_until(lk, Clock::time_point(std::chrono::nanoseconds(pending.begin()->first)));
                    else
                        cv_sched.wait(lk);
                }
                if (fatal != REPRO_OK) break;
                if (active.empty() && admitted_now.empty()) break;  // stopping, nothing left to issue
            }
            if (!issue(admitted_now)) {
                for (Req* r : admitted_now) active.push_back(r);
                admitted_now.clear();
                fail_all(REPRO_ECUDA);
                break;
            }
        }
        for (cudaStream_t st_ : stream) cudaStreamSynchronize(st_);
        while (!inflight.empty()) retire_oldest();
    }
};

void CUDART_CB on_complete(void* p) {
    Completion* c = (Completion*)p;
    Server* S = c->srv;
    const int64_t t = now_ns();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (Req* r : c->reqs) {
            r->errors = S->err_words[r->slot];
            r->status = status_of(r->errors);
            S->free_slots.push_back(r->slot);
            r->slot = -1;
            S->in_use -= (long long)r->need;
            --S->admitted;
            r->done_ns = t;
            r->done = true;
            S->st.completed += 1;
        }
    }
    S->cv_done.notify_all();
    S->cv_sched.notify_all();
    delete c;
}

bool device_accessible(const void* p, int device, bool host_ok) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return a.device == device;
    return host_ok && a.type == cudaMemoryTypeHost;
}

void fill_info(const Req& r, repro_request_info* info) {
    if (!info) return;
    std::memset(info, 0, sizeof(*info));
    info->done = r.done ? 1 : 0;
    info->status = r.status;
    info->errors = r.errors;
    info->arrival_ns = r.arrival_ns;
    info->admit_ns = r.admit_ns;
    info->done_ns = r.done_ns;
}

}  // namespace
}  // namespace rp

using namespace rp;

struct repro_server_s {
    Server s;
};

extern "C" {

int64_t repro_server_now_ns(void) { return now_ns(); }

repro_status repro_server_create(const repro_server_config* cfg, repro_server* out) {
    if (!out) return REPRO_EINVAL;
    *out = nullptr;
    repro_server_config c{};
    if (cfg) c = *cfg;
    if (c.memory_budget < 0 || c.chunk_rows < 0 || c.max_active < 0 || c.max_inflight < 0) return REPRO_EINVAL;
    if (c.chunk_rows == 0) c.chunk_rows = 1ll << 24;
    c.chunk_rows = (c.chunk_rows + 4095) / 4096 * 4096;
    if (c.max_active == 0) c.max_active = 256;
    if (c.max_inflight == 0) c.max_inflight = 3;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return REPRO_ECUDA;
    if (c.memory_budget == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return REPRO_ECUDA;
        c.memory_budget = (int64_t)(free_b / 4);
    }
    repro_server_s* h = new (std::nothrow) repro_server_s;
    if (!h) return REPRO_ENOMEM;
    Server& S = h->s;
    S.cfg = c;
    S.device = dev;
    cudaError_t e = cudaSuccess;
    S.pool = library_pool(e);
    for (int l = 0; l < kLanes && S.pool && e == cudaSuccess; ++l)
        e = cudaStreamCreateWithFlags(&S.stream[l], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&S.err_words, sizeof(uint32_t) * c.max_active, cudaHostAllocDefault);
    if (!S.pool || e != cudaSuccess) {
        for (cudaStream_t st_ : S.stream)
            if (st_) cudaStreamDestroy(st_);
        if (S.err_words) cudaFreeHost(S.err_words);
        delete h;
        return e == cudaErrorMemoryAllocation ? REPRO_ENOMEM : REPRO_ECUDA;
    }
    for (int i = c.max_active - 1; i >= 0; --i) S.free_slots.push_back(i);
    S.st.memory_budget = c.memory_budget;
    try {
        S.thr = std::thread([&S] { S.run(); });
    } catch (...) {
        for (cudaStream_t st_ : S.stream) cudaStreamDestroy(st_);
        cudaFreeHost(S.err_words);
        delete h;
        return REPRO_ENOMEM;
    }
    *out = h;
    return REPRO_OK;
}

repro_status repro_server_submit(repro_server srv, const int32_t* keys, const void* values, int64_t n,
                                 repro_dtype dtype, int L, int64_t num_groups, void* out, void* ready_event,
                                 int64_t arrival_ns, uint64_t* id) {
    if (!srv || !id || n < 0 || (dtype != REPRO_F64 && dtype != REPRO_F32) || L < 1 || L > 4 || num_groups < 1 ||
        num_groups > INT32_MAX || !out)
        return REPRO_EINVAL;
    Server& S = srv->s;
    const size_t esz = dtype == REPRO_F64 ? 8 : 4;
    if ((uintptr_t)out % esz || !device_accessible(out, S.device, true)) return REPRO_EINVAL;
    if (n > 0) {
        if (!keys || !values || (uintptr_t)keys % 4 || (uintptr_t)values % esz) return REPRO_EINVAL;
        if (!device_accessible(keys, S.device, false) || !device_accessible(values, S.device, false))
            return REPRO_EINVAL;
    }
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return REPRO_ECUDA;
    if (cur != S.device) cudaSetDevice(S.device);
    std::unique_ptr<Req> r(new (std::nothrow) Req);
    if (!r) return REPRO_ENOMEM;
    r->keys = keys;
    r->vals = values;
    r->n = n;
    r->dtype = dtype;
    r->L = L;
    r->G = num_groups;
    r->out = out;
    r->ready = (cudaEvent_t)ready_event;
    r->arrival_ns = arrival_ns > 0 ? arrival_ns : now_ns();
    r->large = !(n == 0 || fused_supported(dtype, L, num_groups, keys, values));
    r->part_lane = r->large && num_groups <= kPartLaneGroups && (uintptr_t)keys % 16 == 0 &&
                   (uintptr_t)values % 16 == 0;
    r->need = repro_state_bytes(dtype, L, num_groups);
    if (r->large) {
        const long long rows = std::min<long long>(n, S.cfg.chunk_rows);
        PartChoice pc;
        r->need += partitioned_supported(dtype, L, num_groups, rows, keys, values) &&
                           partition_choose(dtype, L, num_groups, pc)
                       ? partitioned_scratch_bytes(pc, dtype, L, num_groups, rows)
                       : two_pass_scratch_bytes(num_groups);
    }
    if (cur != S.device) cudaSetDevice(cur);
    if ((long long)r->need > S.cfg.memory_budget) return REPRO_ERANGE;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        if (S.stop) return REPRO_EINVAL;
        if (S.fatal != REPRO_OK) return S.fatal;
        r->id = S.next_id++;
        *id = r->id;
        S.pending.emplace(r->arrival_ns, r.get());
        S.reqs.emplace(r->id, std::move(r));
        S.st.submitted += 1;
    }
    S.cv_sched.notify_all();
    return REPRO_OK;
}

repro_status repro_server_poll(repro_server srv, uint64_t id, repro_request_info* info) {
    if (!srv) return REPRO_EINVAL;
    Server& S = srv->s;
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.reqs.find(id);
    if (it == S.reqs.end()) return REPRO_EINVAL;
    fill_info(*it->second, info);
    return REPRO_OK;
}

repro_status repro_server_wait(repro_server srv, uint64_t id, double timeout_s, repro_request_info* info) {
    if (!srv || !(timeout_s >= 0)) return REPRO_EINVAL;
    Server& S = srv->s;
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.reqs.find(id);
    if (it == S.reqs.end()) return REPRO_EINVAL;
    Req* r = it->second.get();
    const auto deadline = Clock::now() + std::chrono::nanoseconds((long long)(std::min(timeout_s, 1e9) * 1e9));
    if (!S.cv_done.wait_until(lk, deadline, [r] { return r->done; })) {
        fill_info(*r, info);
        return REPRO_ETIMEOUT;
    }
    fill_info(*r, info);
    return REPRO_OK;
}

repro_status repro_server_release(repro_server srv, uint64_t id) {
    if (!srv) return REPRO_EINVAL;
    Server& S = srv->s;
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.reqs.find(id);
    if (it == S.reqs.end() || !it->second->done) return REPRO_EINVAL;
    S.reqs.erase(it);
    return REPRO_OK;
}

repro_status repro_server_stats_get(repro_server srv, repro_server_stats* out) {
    if (!srv || !out) return REPRO_EINVAL;
    Server& S = srv->s;
    std::lock_guard<std::mutex> lk(S.mu);
    *out = S.st;
    out->memory_in_use = S.in_use + S.own;
    out->memory_peak = S.peak;
    out->memory_server_peak = S.own_peak;
    out->active = S.admitted;
    out->waiting = (int32_t)S.waitq.size();
    return REPRO_OK;
}

repro_status repro_server_destroy(repro_server srv) {
    if (!srv) return REPRO_OK;
    Server& S = srv->s;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.stop = true;
    }
    S.cv_sched.notify_all();
    if (S.thr.joinable()) S.thr.join();
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(S.device);
    for (cudaEvent_t e : S.free_events) cudaEventDestroy(e);
    for (Arena* a : S.all_arenas) {
        if (a->dev) cudaFreeAsync(a->dev, S.stream[0]);
        if (a->host) cudaFreeHost(a->host);
        delete a;
    }
    cudaStreamSynchronize(S.stream[0]);
    for (cudaStream_t st_ : S.stream) cudaStreamDestroy(st_);
    cudaFreeHost(S.err_words);
    cudaSetDevice(cur);
    const repro_status st = S.fatal;
    delete srv;
    return st;
}

}  // extern "C"
