// Onesweep LSD radix sort: float32 -> vertex order, and 64-bit keys with an
// int32 payload (used to sort unique Morse-Smale pairs).
#pragma once

#include "common.cuh"

namespace msc {

struct SortScratch {
    uint32_t* ord_cnt;                // vertex order: [256][kOrderMaxSuper] super-tile counts, [4][256]
                                      // pass totals, [kOrderMaxBuckets][kOrderFillStride] bucket fills
    uint32_t* hist;                   // [8][256] digit histograms
    uint32_t* tile_counters;          // [8] dynamic tile ids, one per pass
    unsigned long long* lookback;     // [max_tiles][256] decoupled look-back words
    int64_t max_tiles;
    uint32_t* sub_fill;               // order inversion: slots taken per sub-bucket of 2^15 ids
};

constexpr int kSortTile = 4096;       // keys per onesweep tile
constexpr int kOrderMaxSuper = 8192;  // super-tiles (runs of consecutive tiles) of a vertex-order pass
constexpr int kOrderMaxBuckets = 256; // id buckets the last order pass files pairs into
constexpr int kOrderFillStride = 32;  // words between bucket fill counters (one 128-byte line each)
constexpr size_t kOrderCntWords = (size_t)256 * kOrderMaxSuper + 4 * 256 + kOrderMaxBuckets * kOrderFillStride;

// Width of the id buckets of the order's last pass: 2^19 ids at least, at
// most kOrderMaxBuckets buckets.
int order_bucket_shift(int64_t n);

// Inverse permutation of the (id, position) pairs filed by id bucket
// (bucket b holds the ids [b << shift, (b + 1) << shift)): order[id] =
// position, through sub-buckets of 2^15 ids (ids2 / pos2: n-entry scratch).
int order_invert(int shift, const int32_t* ids, const uint32_t* pos, int32_t* ids2, uint32_t* pos2,
                 uint32_t* sub_fill, int64_t n, int32_t* order, int32_t* status, cudaStream_t s);

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
