// multi_types.h -- work descriptors shared by the multi-task single-pass
// kernel (repro_batch.cu) and the device-side planners that build them
// (repro_batch.cu on the host, repro_partition.cu on the device).
#pragma once

#include <cstdint>

namespace rp {

struct MTask {
    const int32_t* keys;
    const void* vals;
    long long n;
    int G;                // groups of this task: records recs[0 .. G)
    int G_hdr;            // num_groups its state header must show
    unsigned char* hdr;   // the state's header (checks, error word)
    unsigned char* recs;  // the task's first group record
    const int* win;       // per group its window (K of its largest |value|, -1: none), or null
    int hint;             // 1: win is only a lower bound, raised by every item of the task at its end
    int pad;
};

struct MItem {
    int task;
    int excl;             // 1: the item covers the whole task -> merge into its state
    long long row0, row1; // rows [row0, row1) of the task; row0 is a multiple of R
    long long part;       // first record of this item's partial table (excl == 0)
};

struct MergeBlk {
    int task;
    int g0;               // first group of this block (32 groups per block)
    int nparts;           // partial tables of the task
    int pad;
    long long part;       // first record of the task's first partial table
};

// What the consumers of a stage need, written by the producer with the tile
// (so the per-tile work reads no descriptor from global memory).
struct StageMeta {
    int item;             // -1: no more work
    int rows;             // rows of this tile
    int rows_tma;         // rows delivered by TMA (a multiple of 4), the rest read from global
    int last;             // last tile of the item
    long long row0;       // first row of the tile within the task
    int G;                // groups of the item's task
    int first;            // first tile of the item
    const int32_t* keys;  // the task's key and value columns at row0
    const void* vals;
    const int* win;       // the task's preset windows, or null
    int hint;             // win is a lower bound that other CTAs raise meanwhile
    int pad;
};

// Shared memory the multi-task kernel reserves for its stage records (S <= 8).
constexpr size_t kMetaSmemBytes = sizeof(StageMeta) * 8;

struct MultiArgs {
    const MTask* tasks;
    const MItem* items;
    int nitems;
    const int* nitems_ptr;  // when set, the item count is read from device memory
    int* counter;
    int R, S, C, Gcap;
    unsigned char* partials;
};

}  // namespace rp
