// Steepest-ascent / steepest-descent pointer kernels (grid stencil, CSR).
#pragma once

#include "common.cuh"

namespace msc {

// asc[v] / desc[v] = neighbour of smallest / largest order (or v).  When
// `extrema` is non-null, extrema[0] += #minima and extrema[1] += #maxima.
int run_steepest_grid(const int32_t* order, msc_grid g, int32_t* asc, int32_t* desc,
                      uint32_t* extrema, int32_t* status, cudaStream_t s, bool allow_tma = true);

// One instance of a packed batch (host-built table, one entry per grid).
struct BatchInst {
    int32_t nx, ny, nz;
    int32_t off;  // packed id of the instance's first vertex
    int32_t vec;  // asc / desc rows of this instance take 16-byte stores
    int32_t pad[3];
};

// Batched grid stencil: tile shapes 0..steepest_batch_shapes()-1;
// tile0[i] = first tile of instance i under that shape (count + 1
// entries, tile0[count] = ntiles).  asc / desc get packed ids, ext[2i] /
// ext[2i+1] += the minima / maxima of instance i.  `packed`: every
// instance has at most 2^27 vertices.
int steepest_batch_shapes();
int64_t steepest_batch_tiles(int shape, msc_grid g);
const char* steepest_batch_shape_name(int shape);
int run_steepest_batch(const int32_t* order, const BatchInst* inst, const int32_t* tile0, int count,
                       int64_t ntiles, int shape, bool packed, int32_t* asc, int32_t* desc, uint32_t* ext,
                       cudaStream_t s);

int run_steepest_csr(const int32_t* order, const int32_t* row, const int32_t* col, int32_t n,
                     int32_t* asc, int32_t* desc, int32_t* status, cudaStream_t s);

}  // namespace msc
