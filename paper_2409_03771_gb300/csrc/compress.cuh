// Path compression by pointer jumping (in place), with device-side
// convergence detection and active-list compaction.
#pragma once

#include "common.cuh"

namespace msc {

constexpr int kMaxJumpSteps = 64;

// Per pointer array; zeroed at the start of every compression.
struct JumpCtl {
    uint32_t cnt[kMaxJumpSteps];    // vertices changed in each step
    uint32_t built[kMaxJumpSteps];  // step wrote its changed vertices to a list
};

struct CompressTune {
    bool fill_lists = true;  // build the active list whenever the previous sweep's count is at
                             // most 1.5x its capacity (an overflow leaves a full sweep next)
    int build_shift = 3;     // fill_lists off: build it once <= n >> build_shift changed
    bool trusted = false;  // pointers from the stencil kernels: skip range / cycle tests
    uint32_t* roots = nullptr;  // roots[i] += #self-pointers of array i (first sweep)
};

// Sweeps launched for n vertices: ceil(log5 n) + 2 (enough for any forest
// at a fivefold advance per sweep; more are needed only by a cycle).
int compress_steps(int64_t n);

// Workspace pieces for `count` arrays of n entries.
void size_compress_scratch(Sizer& s, int64_t n, int count);
struct CompressScratch {
    JumpCtl* ctl;     // [count]
    int32_t* lists;   // [count][2][list_cap]
    int64_t list_cap;
};
CompressScratch carve_compress_scratch(Carver& c, int64_t n, int count);

// Compress `count` (1 or 2) arrays of n entries in place.  Negative entries
// are inactive.  Errors go to status (MSC_ERR_ARG, MSC_ERR_NOT_CONVERGED).
int run_compress(int32_t* const* ptrs, int count, int32_t n, const CompressScratch& sc,
                 int32_t* status, cudaStream_t s, const CompressTune& tune = CompressTune());

}  // namespace msc
