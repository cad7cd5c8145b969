// batch_plan.h -- host-side planning of a multi-task single-pass launch,
// shared by repro_batch_prepare (repro_batch.cu) and the request server
// (repro_serve.cu).  Not installed.
#pragma once

#include <vector>

#include "multi_types.h"
#include "repro.h"
#include "repro_internal.h"

namespace rp {

// Bytes of one partial-table record: int32 K, uint32 flags, L 128-bit bins.
constexpr size_t batch_rec_bytes(int L) { return 8 + 16 * (size_t)L; }

// The single-pass tasks are launched in classes by group count, one
// persistent launch per class, each with the configuration of its own
// largest table: small tables keep several CTAs per SM (and lane-private
// copies for the smallest) instead of all tasks running at the occupancy
// of the batch's largest table.
constexpr int kBatchClasses = 3;
constexpr long long kBatchClassBound[kBatchClasses] = {64, 1024, 1ll << 31};  // largest G of each class

struct BatchClass {
    FusedPlanConfig cfg{};  // cfg.S == 0: the class holds no task
    int gcap = 1;           // largest group table among its tasks
    int ctas = 0;           // CTAs of its persistent launch
    int item0 = 0, nitems = 0;  // its items in HostBatch::items (largest first)
    int ntasks = 0;
};

struct HostBatch {
    BatchClass cls[kBatchClasses];
    std::vector<MTask> tasks;      // one per input task (index = task number)
    std::vector<MItem> items;      // class by class
    std::vector<MergeBlk> blks;    // partial-merge blocks of the tasks cut into several items
    long long part_recs = 0;       // partial-table records the items write
    std::vector<repro_task> slow;  // tasks outside the single-pass path (two-pass path)
    long long slow_gmax = 0;
};

// Cut tasks into items: about items_per_cta items per CTA, each at least 8
// tiles and at most 2^23 rows (no 64-bit table bin can overflow within an
// item); items grow further while the partial tables would exceed
// max_part_bytes.  Validates the tasks (REPRO_EINVAL) and the table size
// (REPRO_ERANGE).
// With fixed_cfg (one per class) each class's configuration is that one (it
// must fit) instead of a fresh choice, so a re-plan keeps an existing plan's
// kernels.
// With one_class, every single-pass task goes to the last class (one
// persistent launch: fewer launches for a small batch).
repro_status plan_batch_host(const repro_task* tasks, int ntasks, int dtype, int L, size_t max_part_bytes,
                             HostBatch& H, int items_per_cta = 4, const BatchClass* fixed_cfg = nullptr,
                             bool one_class = false);

}  // namespace rp
