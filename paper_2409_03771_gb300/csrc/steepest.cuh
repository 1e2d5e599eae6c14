// Steepest-ascent / steepest-descent pointer kernels (grid stencil, CSR).
#pragma once

#include "common.cuh"

namespace msc {

// asc[v] / desc[v] = neighbour of smallest / largest order (or v).  When
// `extrema` is non-null, extrema[0] += #minima and extrema[1] += #maxima.
int run_steepest_grid(const int32_t* order, msc_grid g, int32_t* asc, int32_t* desc,
                      uint32_t* extrema, int32_t* status, cudaStream_t s, bool allow_tma = true);

int run_steepest_csr(const int32_t* order, const int32_t* row, const int32_t* col, int32_t n,
                     int32_t* asc, int32_t* desc, int32_t* status, cudaStream_t s);

}  // namespace msc
