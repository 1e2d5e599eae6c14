// Adjacency of labelled regions on a regular grid.
#pragma once

#include "common.cuh"
#include "sort.cuh"

namespace msc {

// False when 7 * n does not fit the int32 key count.
bool adjacency_size_ok(int64_t n);

// Workspace of run_adjacency_grid; `saddle`: with the crossing vertices.
void size_adjacency_scratch(Sizer& s, int64_t n, bool saddle);

// Distinct label pairs across the edges of the grid (conn 6 or 14):
// out_a / out_b receive the first min(out_cap, K) pairs in lexicographic
// order, *num_pairs (device) = K.  Labels must be < bound.  With `order`
// (not null), saddle[r] also receives pair r's crossing vertex: the end of
// its highest (sense +1) or lowest (sense -1) crossing edge in the order.
// The same over an explicit mesh: row[n+1], col[nnz] (symmetric CSR, nnz =
// row[n]); each edge is taken from its smaller end.
void size_adjacency_csr_scratch(Sizer& s, int64_t nnz, bool saddle);
int run_adjacency_csr(const int32_t* label, const int32_t* row, const int32_t* col, int32_t n, int64_t nnz,
                      int32_t bound, int32_t* out_a, int32_t* out_b, int64_t out_cap, int64_t* num_pairs, void* ws,
                      size_t ws_bytes, int32_t* status, cudaStream_t s, const int32_t* order = nullptr,
                      int sense = 1, int32_t* saddle = nullptr);

int run_adjacency_grid(const int32_t* label, msc_grid g, int conn, int32_t bound, int32_t* out_a,
                       int32_t* out_b, int64_t out_cap, int64_t* num_pairs, void* ws, size_t ws_bytes,
                       int32_t* status, cudaStream_t s, const int32_t* order = nullptr, int sense = 1,
                       int32_t* saddle = nullptr);

}  // namespace msc
