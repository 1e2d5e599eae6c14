// Dense Morse-Smale cell ids from (ascending, descending) label pairs.
#pragma once

#include "common.cuh"
#include "sort.cuh"

namespace msc {

struct MsScratch {
    unsigned long long* table_keys;  // [cap_max]
    uint32_t* table_vals;            // [cap_max]
    int64_t cap_max;
    unsigned long long* ukeys[2];    // [n] unique pair keys (ping-pong)
    int32_t* uvals[2];               // [n] their table slots
    uint32_t* ctl;                   // [0] nmin [1] nmax [2] cap [3] K; words 9..19 private
    uint32_t* chunk;                 // [2][chunks of 4096 minimum ids]: pair counts, their scan
    SortScratch sort;
};

// b of the pair keys (asc << b) | desc: ceil(log2 n).
int ms_pair_shift(int64_t n);

void size_ms_scratch(Sizer& s, int64_t n);
MsScratch carve_ms_scratch(Carver& c, int64_t n);

// ms[v] = rank of (asc[v], desc[v]) among the distinct pairs, num_cells = K.
// When `counts_known` is false the labels are validated (in range, every
// label labels itself) and the extrema counted first; otherwise ctl[0..1]
// must already hold the number of minima and maxima.
// `sorted_keys` (optional) receives the device array of the K distinct
// pair keys (asc << ms_pair_shift(n)) | desc in ascending order (K = ctl[3]).
int run_ms_id(const int32_t* asc, const int32_t* desc, int32_t n, int32_t* ms, int32_t* num_cells,
              const MsScratch& sc, bool counts_known, int32_t* status, cudaStream_t s,
              const unsigned long long** sorted_keys = nullptr);

}  // namespace msc
