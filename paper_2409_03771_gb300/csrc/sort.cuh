// Onesweep LSD radix sort: float32 -> vertex order, and 64-bit keys with an
// int32 payload (used to sort unique Morse-Smale pairs).
#pragma once

#include "common.cuh"

namespace msc {

struct SortScratch {
    uint32_t* hist;                   // [8][256] digit histograms
    uint32_t* tile_counters;          // [8] dynamic tile ids, one per pass
    unsigned long long* lookback;     // [max_tiles][256] decoupled look-back words
    int64_t max_tiles;
    uint32_t* sub_fill;               // order inversion: slots taken per sub-bucket of 2^15 ids
};

constexpr int kSortTile = 4096;       // keys per onesweep tile

// Bytes of scratch (hist + counters + look-back) for up to n keys.
void size_sort_scratch(Sizer& s, int64_t n);
SortScratch carve_sort_scratch(Carver& c, int64_t n);

// order[v] = rank of (f[v], v).  Uses two (key, id) ping-pong buffers of n
// entries each.  Records MSC_ERR_NAN in status when f holds a NaN.
int run_order(const float* f, int64_t n, int32_t* order, uint32_t* key_a, int32_t* id_a,
              uint32_t* key_b, int32_t* id_b, const SortScratch& sc, int32_t* status,
              cudaStream_t s);

// Packed segments sorted independently (batched instances).  Segment i
// holds keys [off[i], off[i+1]) and tiles [tile0[i], tile0[i+1]) of
// kSortTile keys; tile_seg[t] is the segment of tile t.  Device arrays,
// built once on the host; total < 2^31.
struct SegTable {
    const int32_t* off;       // [count + 1]
    const int32_t* tile0;     // [count + 1]
    const int32_t* tile_seg;  // [tiles]
    int32_t count;
    int64_t total;
    int64_t tiles;
};

void size_seg_sort_scratch(Sizer& s, int count, int64_t tiles);
SortScratch carve_seg_sort_scratch(Carver& c, int count, int64_t tiles);

// order[v] = rank of (f[v], v) within v's segment, for every segment at
// once (4 segmented onesweep passes).  Ping-pong buffers of `total` entries.
int run_order_seg(const float* f, const SegTable& t, int32_t* order, uint32_t* key_a, int32_t* id_a,
                  uint32_t* key_b, int32_t* id_b, const SortScratch& sc, int32_t* status,
                  cudaStream_t s);

// Stable sort of (keys, vals) by the low `key_bits` bits of keys.  The
// count is read on the device from *d_count (<= max_count).  Returns, via
// *result_in_alt, whether the sorted data ended in the alt buffers.  With
// vals and vals_alt both null the keys are sorted alone.
int run_sort_u64(unsigned long long* keys, int32_t* vals, unsigned long long* keys_alt,
                 int32_t* vals_alt, const int32_t* d_count, int64_t max_count, int key_bits,
                 const SortScratch& sc, int32_t* status, cudaStream_t s, bool* result_in_alt,
                 const char* hist_label = "msid.sort_hist", const char* pass_label = "msid.sort_pass");

}  // namespace msc
