// Connected components: feature mask on a grid, explicit mesh (CSR).
#pragma once

#include "common.cuh"

namespace msc {

// label[v] = smallest id of v's component among mask != 0 voxels under
// `conn` (6 or 14) connectivity, -1 where mask is 0.
int run_cc_mask(const uint8_t* mask, msc_grid g, int conn, int32_t* label, int32_t* status,
                cudaStream_t s);

// label[v] = smallest id of v's component of the symmetric CSR graph.
// `frequent` is one device int32 of scratch.
int run_cc_mesh(const int32_t* row, const int32_t* col, int32_t n, int32_t* label, int32_t* status,
                cudaStream_t s, int32_t* frequent);

}  // namespace msc
