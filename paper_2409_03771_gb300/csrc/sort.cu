// Onesweep LSD radix sorts: the vertex order of many packed instances at
// once (Simulation of Simplicity, section "Preprocessing": sort by value,
// ties by global id, per instance) and 64-bit keys with an int32 payload
// (unique Morse-Smale pairs, region-adjacency keys); plus the inversion of
// the vertex order that order.cu shares.
//
// Keys of a float field: float32 bits mapped to an order-preserving uint32
// (-0.0 first folded onto +0.0 so that the two tie, as IEEE '<' says).
// 8-bit digit passes, least significant first; every pass is stable, and
// the first pass reads the vertices in id order, so equal keys stay in id
// order: the final position of v is its rank under (f[v], v).
//
// One pass = one kernel.  A block takes tiles of 4096 keys from a global
// atomic counter (so every predecessor tile is owned by a running block),
// ranks its keys per digit stably within each warp (ballot peers +
// per-warp counters), publishes its per-digit counts to a decoupled
// look-back array, sums its predecessors' counts and scatters through
// shared memory.  The last pass of an order files (vertex id, position)
// pairs into buckets of consecutive ids; the order field is their inverse
// permutation, written through shared memory: the buckets are split into
// sub-buckets of 2^15 ids, each scattered into one CTA's shared memory and
// written out as whole lines (k_pair_split, k_pair_scatter_local).
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "radix.cuh"
#include "sort.cuh"
#include "tma.cuh"

namespace msc {
#ifdef MSC_DEBUG_BOUNDS
__device__ uint32_t g_sort_dbg[16];
#endif
namespace {

constexpr int kThreads = 256;
constexpr int kItems = kSortTile / kThreads;  // 16
constexpr int kWarps = kThreads / kWarp;      // 8
constexpr int kBins = 256;
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr uint32_t kSpinLimit = 1u << 22;
// The last pass of the vertex order files (id, position) pairs into
// buckets of 2^shift consecutive ids; bucket b holds exactly the ids
// [b << shift, (b + 1) << shift) and so occupies pair slots of the same
// range.  At most kMaxBuckets buckets (see bucket_shift).
constexpr int kMaxBuckets = kOrderMaxBuckets;
constexpr int kFillStride = kOrderFillStride;  // one 128-byte line per bucket counter: the
                                 // tiles' reservations spread over L2 slices
constexpr int kCounterWords = 8 + kMaxBuckets * kFillStride;  // tile counters, bucket fills

// Digit histograms for `npass` passes over n keys (keys read from `keys`,
// or made from the float field `f`).  Each thread counts runs of equal
// digits over 16 consecutive keys (neighbouring grid values share their
// high digits, so the skewed digits cost one update per run) into a
// warp-private shared histogram; blocks then add theirs to the global one.
template <typename KeyT, bool FROM_F>
__global__ void __launch_bounds__(256) k_hist(const KeyT* __restrict__ keys,
                                              const float* __restrict__ f, int64_t n_host,
                                              const int32_t* __restrict__ d_n, int npass,
                                              uint32_t* __restrict__ hist, int32_t* status) {
    extern __shared__ uint32_t sh[];  // [kWarps][npass][256]
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < kWarps * npass * kBins; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    uint32_t* wsh = sh + warp * npass * kBins;
    const int64_t n = d_n ? min((int64_t)*d_n, n_host) : n_host;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * kHistRun;
    bool saw_nan = false;
    for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + tid) * kHistRun; i0 < n; i0 += stride) {
        KeyT k[kHistRun];
        const int cnt = (int)min((int64_t)kHistRun, n - i0);
        if constexpr (FROM_F) {
            load_float_keys16(f, i0, cnt, k, saw_nan);
        } else {
#pragma unroll
            for (int j = 0; j < kHistRun; ++j) k[j] = j < cnt ? keys[i0 + j] : KeyT(0);
        }
        count_runs(k, cnt, npass, wsh);
    }
    if (saw_nan) record_error(status, MSC_ERR_NAN);
    __syncthreads();
    for (int i = tid; i < npass * kBins; i += blockDim.x) {
        uint32_t c = 0;
        for (int w = 0; w < kWarps; ++w) c += sh[w * npass * kBins + i];
        if (c) atomicAdd(&hist[i], c);
    }
}

// Per-segment histograms of the float keys for the 4 passes of a
// segmented sort: hist[seg][pass][256].  Block b takes a contiguous run of
// tiles (one tile = 256 threads x 16 keys, inside one segment) and adds
// its warp-private shared counts to the segment's global histogram each
// time the segment changes and at the end.
constexpr int kSegPasses = 4;

__global__ void __launch_bounds__(256) k_hist_seg(const float* __restrict__ f,
                                                  const int32_t* __restrict__ tile_seg,
                                                  const int32_t* __restrict__ seg_off,
                                                  const int32_t* __restrict__ seg_tile0, int64_t tiles,
                                                  uint32_t* __restrict__ hist, int32_t* status) {
    extern __shared__ uint32_t sh[];  // [kWarps][4][256]
    constexpr int kSeg = kSegPasses * kBins;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < kWarps * kSeg; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    uint32_t* wsh = sh + warp * kSeg;
    const int64_t t0 = tiles * blockIdx.x / gridDim.x, t1 = tiles * (blockIdx.x + 1) / gridDim.x;
    bool saw_nan = false;
    auto flush = [&](int seg) {
        __syncthreads();
        for (int i = tid; i < kSeg; i += blockDim.x) {
            uint32_t c = 0;
            for (int w = 0; w < kWarps; ++w) {
                c += sh[w * kSeg + i];
                sh[w * kSeg + i] = 0;
            }
            if (c) atomicAdd(&hist[(int64_t)seg * kSeg + i], c);
        }
        __syncthreads();
    };
    int cur = t0 < t1 ? tile_seg[t0] : 0;
    for (int64_t t = t0; t < t1; ++t) {
        const int seg = tile_seg[t];  // uniform over the block
        if (seg != cur) {
            flush(cur);
            cur = seg;
        }
        const int64_t off = seg_off[seg], n = seg_off[seg + 1] - off;
        const int64_t i0 = (t - seg_tile0[seg]) * kSortTile + (int64_t)tid * kHistRun;
        if (i0 < n) {
            uint32_t k[kHistRun];
            const int cnt = (int)min((int64_t)kHistRun, n - i0);
            load_float_keys16(f + off, i0, cnt, k, saw_nan);
            count_runs(k, cnt, kSegPasses, wsh);
        }
    }
    if (t0 < t1) flush(cur);
    if (saw_nan) record_error(status, MSC_ERR_NAN);
}

// hist[seg][pass][.] -> exclusive bin starts, one block per (seg, pass).
__global__ void __launch_bounds__(256) k_seg_bstart(uint32_t* hist) {
    __shared__ uint32_t s_w[kWarps];
    uint32_t* h = hist + (int64_t)blockIdx.x * kBins;
    const uint32_t c = h[threadIdx.x];
    h[threadIdx.x] = block_scan_256(c, s_w) - c;
}

template <typename KeyT>
struct PassArgs {
    const KeyT* keys_in;
    const float* f_in;
    const int32_t* vals_in;
    KeyT* keys_out;
    int32_t* vals_out;
    int64_t n;
    const int32_t* d_n;
    const uint32_t* hist;  // this pass's 256 counts
    uint32_t* pair_pos;    // BUCKET pass: position of the id in vals_out[slot]
    uint32_t* bucket_fill; // BUCKET pass: slots taken per bucket (stride kFillStride)
    int bucket_shift;      // BUCKET pass: log2 of the ids per bucket
    int shift;
    unsigned long long* lookback;
    uint32_t* tile_counter;
    uint32_t epoch;
    int32_t* status;
    // segmented sort (packed instances): segment of each tile, key offset
    // of each segment, first tile of each segment; `hist` then holds the
    // per-segment exclusive bin starts with a stride of seg_stride words
    const int32_t* tile_seg;
    const int32_t* seg_off;
    const int32_t* seg_tile0;
    int64_t seg_tiles;
    int seg_stride;
};

template <typename KeyT, bool STAGE>
constexpr size_t pass_smem_bytes() {
    return (size_t)(kWarps * kBins + 4 * kBins + 32 + 2 * kMaxBuckets) * 4 +
           (STAGE ? (size_t)kSortTile * (sizeof(KeyT) + 4) : 0);
}

// One onesweep digit pass.  FROM_F: keys come from the float field and
// the payload is the vertex id.  BUCKET (last pass of the vertex order):
// instead of the sorted (key, payload) arrays, file every (payload,
// position) pair into the bucket of its payload's top bits (a tile
// reserves its share of each bucket with one atomic per bucket).
//
// SEG: the keys are packed segments sorted independently (batched
// instances).  Tiles never straddle two segments, the look-back stops at
// the segment's first tile, bin starts come per segment, and positions are
// segment-local (keys land at seg_off + position; order gets the position).
template <typename KeyT, bool FROM_F, bool BUCKET, bool SEG = false>
__global__ void __launch_bounds__(kThreads, 3) k_onesweep(const PassArgs<KeyT> a) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t* s_whist = reinterpret_cast<uint32_t*>(smem);  // [kWarps][256]
    uint32_t* s_total = s_whist + kWarps * kBins;          // [256]
    uint32_t* s_excl = s_total + kBins;                    // [256] tile-local bin starts
    uint32_t* s_gbase = s_excl + kBins;                    // [256] global base of the bin
    uint32_t* s_bstart = s_gbase + kBins;                  // [256] global bin starts
    uint32_t* s_misc = s_bstart + kBins;                   // [0] tile id, [1..8] scan
    uint32_t* s_bucket = s_misc + 32;                      // [2][kMaxBuckets] counts, bases
    KeyT* s_keys = reinterpret_cast<KeyT*>(s_bucket + 2 * kMaxBuckets);
    int32_t* s_vals = reinterpret_cast<int32_t*>(s_keys + kSortTile);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n_all = a.d_n ? min((int64_t)*a.d_n, a.n) : a.n;  // a device count never exceeds the buffers
    const int64_t ntiles = SEG ? a.seg_tiles : (n_all + kSortTile - 1) / kSortTile;
    if constexpr (!SEG) {
        const uint32_t c = a.hist[tid];
        s_bstart[tid] = block_scan_256(c, s_misc + 1) - c;
    }
    for (;;) {
        if (tid == 0) s_misc[0] = atomicAdd(a.tile_counter, 1u);
        for (int i = tid; i < kWarps * kBins; i += kThreads) s_whist[i] = 0;
        __syncthreads();
        const int64_t tile = s_misc[0];
        if (tile >= ntiles) break;
        // this tile's segment: key offset, key count, tile index within it
        int64_t seg_base = 0, n = n_all, ltile = tile;
        if constexpr (SEG) {
            const int seg = a.tile_seg[tile];
            seg_base = a.seg_off[seg];
            n = a.seg_off[seg + 1] - seg_base;
            ltile = tile - a.seg_tile0[seg];
            s_bstart[tid] = a.hist[(int64_t)seg * a.seg_stride + tid];  // read by this thread only
        }
        // tile-local 32-bit indices from here on: the tile's keys are
        // [tbase, tbase + cnt) of the packed arrays
        const int64_t tbase = seg_base + ltile * kSortTile;
        const int cnt = (int)min((int64_t)kSortTile, n - ltile * kSortTile);
        const int wbase = warp * (kItems * 32) + lane;

        KeyT key[kItems];
        int32_t val[kItems];
        uint32_t rk[kItems];  // (digit << 16) | rank among the warp's equal digits
        {
            const KeyT* kin = FROM_F ? nullptr : a.keys_in + tbase;
            const int32_t* vin = FROM_F || !a.vals_in ? nullptr : a.vals_in + tbase;  // keys only: no payload
            const float* fin = FROM_F ? a.f_in + tbase : nullptr;
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                const int li = wbase + k * 32;
                if (li < cnt) {
                    if constexpr (FROM_F) {
                        key[k] = (KeyT)float_key(fin[li]);
                        val[k] = (int32_t)tbase + li;
                    } else {
                        key[k] = kin[li];
                        val[k] = vin ? vin[li] : 0;
                    }
                } else {
                    key[k] = 0;
                    val[k] = -1;
                }
            }
        }
        uint32_t* wh = s_whist + warp * kBins;
        const uint32_t lt = lanemask_lt();
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            // stable rank among the warp's equal digits: earlier iterations
            // (warp counter) + lower lanes of this iteration (ballot peers)
            const bool valid = wbase + k * 32 < cnt;
            const uint32_t d = (uint32_t)(key[k] >> a.shift) & 255u;
            const uint32_t peers = digit_peers(d, valid);
            const uint32_t lower = __popc(peers & lt);
            const uint32_t before = wh[d];
            if (valid && lower == 0) wh[d] = before + __popc(peers);
            rk[k] = ((valid ? d : 256u) << 16) | (before + lower);
            __syncwarp();
        }
        __syncthreads();
#ifdef MSC_DEBUG_BOUNDS
        {   // each warp's histogram must hold exactly its valid items
            uint32_t sum = 0;
            for (int i = lane; i < kBins; i += 32) sum += wh[i];
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            const int64_t wv = min(kItems * 32, max(0, cnt - warp * kItems * 32));
            if (lane == 0 && sum != (uint32_t)wv && atomicCAS(&g_sort_dbg[14], 0u, 1u) == 0u) {
                g_sort_dbg[15] = (uint32_t)((tile & 0xffffu) << 16 | (warp << 12) | (sum & 0xfffu));
            }
        }
        __syncthreads();
#endif
        // per-digit tile totals; warp counts become warp-exclusive prefixes
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = s_whist[w * kBins + tid];
            s_whist[w * kBins + tid] = run;
            run += c;
        }
        s_total[tid] = run;
        {
            unsigned long long* lb = a.lookback + (size_t)tile * kBins + tid;
            const unsigned long long ep = (unsigned long long)a.epoch << 32;
            st_volatile_u64(lb, (ltile == 0 ? kFlagInc : kFlagAgg) | ep | run);
            uint32_t excl = 0;
            if (ltile > 0) {  // the segment's first tile publishes inclusive: the walk ends there
                int64_t j = tile - 1;
                uint32_t spins = 0;
                while (j >= 0) {
                    const unsigned long long w = ld_volatile_u64(a.lookback + (size_t)j * kBins + tid);
                    const uint32_t wep = (uint32_t)(w >> 32) & 0x3fffffffu;
                    const unsigned long long flag = w & (3ull << 62);
                    if (wep != a.epoch || flag == 0) {
                        if (++spins > kSpinLimit) {
                            record_error(a.status, MSC_ERR_INTERNAL);
                            break;
                        }
                        __nanosleep(32);
                        continue;
                    }
                    excl += (uint32_t)w;
                    if (flag == kFlagInc) break;
                    --j;
                }
                st_volatile_u64(lb, kFlagInc | ep | (unsigned long long)(excl + run));
            }
            s_gbase[tid] = s_bstart[tid] + excl;
        }
        s_excl[tid] = block_scan_256(run, s_misc + 1) - run;
        __syncthreads();  // s_excl is read across threads below
        {
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                const uint32_t d = rk[k] >> 16;
                if (d < 256u) {
                    const uint32_t lpos = s_excl[d] + s_whist[warp * kBins + d] + (rk[k] & 0xffffu);
#ifdef MSC_DEBUG_BOUNDS
                    if (lpos >= (uint32_t)kSortTile && atomicCAS(&g_sort_dbg[0], 0u, 1u) == 0u) {
                        g_sort_dbg[1] = (uint32_t)tile; g_sort_dbg[2] = warp; g_sort_dbg[3] = lane;
                        g_sort_dbg[4] = k; g_sort_dbg[5] = d; g_sort_dbg[6] = s_excl[d];
                        g_sort_dbg[7] = s_whist[warp * kBins + d]; g_sort_dbg[8] = rk[k] & 0xffffu;
                        g_sort_dbg[9] = a.shift; g_sort_dbg[10] = s_total[d]; g_sort_dbg[11] = blockIdx.x;
                        g_sort_dbg[12] = (uint32_t)ntiles; g_sort_dbg[13] = gridDim.x;
                    }
#endif
                    MSC_GUARD(lpos < (uint32_t)kSortTile, a.status, -103) {
                        s_keys[lpos] = key[k];
                        s_vals[lpos] = val[k];
                    }
                }
            }
            __syncthreads();
            if constexpr (BUCKET) {
                // (id, position) pairs regrouped by bucket in shared memory, then
                // each bucket's run written with consecutive lanes on consecutive slots
                static_assert(kMaxBuckets == kThreads, "one bucket per thread");
                uint32_t* s_bstart2 = s_bucket;              // counts, then tile-local bucket starts
                uint32_t* s_bbase = s_bucket + kMaxBuckets;  // first global slot of the tile's run
                s_bstart2[tid] = 0;
                __syncthreads();
                uint32_t pid[kItems], ppos[kItems], prank[kItems / 2];  // two 16-bit ranks per word
#pragma unroll
                for (int k = 0; k < kItems; ++k) {
                    const int i = tid + k * kThreads;
                    if (k % 2 == 0) prank[k / 2] = 0;
                    if (i < cnt) {
                        pid[k] = (uint32_t)s_vals[i];
                        const uint32_t d = (uint32_t)(s_keys[i] >> a.shift) & 255u;
                        ppos[k] = s_gbase[d] + (uint32_t)i - s_excl[d];
                        prank[k / 2] |= atomicAdd(&s_bstart2[pid[k] >> a.bucket_shift], 1u) << (16 * (k % 2));
                    }
                }
                __syncthreads();
                {
                    const uint32_t c = s_bstart2[tid];
                    const uint32_t start = block_scan_256(c, s_misc + 1) - c;
                    s_bbase[tid] = c ? ((uint32_t)tid << a.bucket_shift) +
                                           atomicAdd(&a.bucket_fill[tid * kFillStride], c)
                                     : 0u;
                    s_bstart2[tid] = start;
                }
                __syncthreads();
#pragma unroll
                for (int k = 0; k < kItems; ++k) {
                    const int i = tid + k * kThreads;
                    if (i < cnt) {
                        const uint32_t j = s_bstart2[pid[k] >> a.bucket_shift] + ((prank[k / 2] >> (16 * (k % 2))) & 0xffffu);
                        s_keys[j] = (KeyT)ppos[k];
                        s_vals[j] = (int32_t)pid[k];
                    }
                }
                __syncthreads();
                for (int i = tid; i < cnt; i += kThreads) {
                    const uint32_t id = (uint32_t)s_vals[i];
                    const uint32_t b = id >> a.bucket_shift;
                    const uint32_t slot = s_bbase[b] + ((uint32_t)i - s_bstart2[b]);
                    const uint32_t pos = (uint32_t)s_keys[i];
                    MSC_GUARD(slot < (uint64_t)a.n && pos < (uint64_t)n, a.status, -102) {
                        a.vals_out[slot] = (int32_t)id;
                        a.pair_pos[slot] = pos;
                    }
                }
            } else {
                KeyT* kout = a.keys_out + seg_base;
                int32_t* vout = a.vals_out ? a.vals_out + seg_base : nullptr;
                for (int i = tid; i < cnt; i += kThreads) {
                    const KeyT kk = s_keys[i];
                    const uint32_t d = (uint32_t)(kk >> a.shift) & 255u;
                    const uint32_t pos = s_gbase[d] + (uint32_t)i - s_excl[d];
                    MSC_GUARD(pos < (uint64_t)n, a.status, -102) {
                        kout[pos] = kk;
                        if (vout) vout[pos] = s_vals[i];
                    }
                }
            }
        }
        __syncthreads();
    }
}

// Width of the id buckets the last pass files pairs into: 2^19 ids at
// least (so that each bucket splits into 16 sub-buckets of 2^15), and at
// most kMaxBuckets buckets.
int bucket_shift(int64_t n) {
    return std::max(19, ceil_log2(ceil_div(std::max<int64_t>(n, 1), kMaxBuckets)));
}

// Two-level order inversion.  (1) k_pair_split: every
// chunk of 4096 filed pairs (a chunk lies inside one bucket of 2^shift ids)
// re-files its pairs into sub-buckets of 2^15 ids; sub-bucket j holds
// exactly the ids j * 2^15 + [0, 2^15) and so fills those pair slots.  A
// chunk reserves its share of each sub-bucket with one atomic per
// sub-bucket and regroups its pairs in shared memory, so that each run is
// written with consecutive lanes.  (2) k_pair_scatter_local: one CTA per
// sub-bucket stores its 2^15 positions into a 128 KiB shared-memory slice
// of the order array and writes the slice out as whole lines.
constexpr int kSubLog2 = 15;
constexpr int kSubIds = 1 << kSubLog2;
constexpr int kSplitThreads = 512;
constexpr int kSplitChunk = 4096;
constexpr int kSplitPer = kSplitChunk / kSplitThreads;  // 8
constexpr int kMaxSub = 1 << 8;  // sub-buckets per bucket (shift <= 23)

// The chunk's pairs arrive by 1D TMA bulk copy into one half of a shared
// double buffer while the previous chunk is filed (plain loads for a ragged
// last chunk or unaligned arrays); they are counted per sub-bucket,
// regrouped in place and written out as runs.
constexpr size_t kSplitSmem = (size_t)2 * 2 * kSplitChunk * 4 + (2 * kMaxSub + 32) * 4 + 2 * 8;

__global__ void __launch_bounds__(kSplitThreads, 2) k_pair_split(const int32_t* __restrict__ ids_in,
                                                                 const uint32_t* __restrict__ pos_in, int64_t n,
                                                                 int shift, int use_tma, uint32_t* sub_fill,
                                                                 int32_t* __restrict__ ids_out,
                                                                 uint32_t* __restrict__ pos_out, int32_t* status) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t* buf = reinterpret_cast<uint32_t*>(smem);     // [2][ids kSplitChunk | positions kSplitChunk]
    uint32_t* s_cnt = buf + 2 * 2 * kSplitChunk;            // [kMaxSub] counts, then chunk-local starts
    uint32_t* s_base = s_cnt + kMaxSub;                     // [kMaxSub] first slot of the run in each sub-bucket
    uint32_t* s_w = s_base + kMaxSub;                       // [32]
    uint64_t* mbar = reinterpret_cast<uint64_t*>(s_w + 32); // [2]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nsub = 1 << (shift - kSubLog2);
    const int64_t nchunks = (n + kSplitChunk - 1) / kSplitChunk;
    if ((int64_t)blockIdx.x >= nchunks) return;  // block-uniform
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto by_tma = [&](int64_t c) { return use_tma && (c + 1) * kSplitChunk <= n; };
    auto issue = [&](int64_t c, int slot) {  // one thread
        if (c >= nchunks || !by_tma(c)) return;
        uint32_t* dst = buf + slot * 2 * kSplitChunk;
        mbar_expect_tx(&mbar[slot], 2 * kSplitChunk * 4);
        bulk_load(dst, ids_in + c * kSplitChunk, kSplitChunk * 4, &mbar[slot]);
        bulk_load(dst + kSplitChunk, pos_in + c * kSplitChunk, kSplitChunk * 4, &mbar[slot]);
    };
    if (tid == 0) issue(blockIdx.x, 0);
    int it = 0;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x, ++it) {
        const int slot = it & 1;
        uint32_t* bi = buf + slot * 2 * kSplitChunk;
        uint32_t* bp = bi + kSplitChunk;
        if (tid == 0) issue(c + gridDim.x, slot ^ 1);
        const int64_t c0 = c * kSplitChunk;
        const int cnt = (int)min((int64_t)kSplitChunk, n - c0);
        const int64_t s0 = (c0 >> shift) << shift;  // first id of the chunk's bucket
        for (int i = tid; i < nsub; i += kSplitThreads) s_cnt[i] = 0;
        if (by_tma(c)) {
            const bool ok = mbar_wait(&mbar[slot], (uint32_t)(it >> 1) & 1u, kSpinLimit);
            if (__syncthreads_or(!ok)) {  // a copy never landed: report, let the prefetch finish, stop
                if (tid == 0) {
                    record_error(status, MSC_ERR_INTERNAL);
                    if (c + gridDim.x < nchunks && by_tma(c + gridDim.x))
                        mbar_wait(&mbar[slot ^ 1], (uint32_t)((it + 1) >> 1) & 1u, kSpinLimit);
                }
                return;
            }
        } else {
            for (int i = tid; i < cnt; i += kSplitThreads) {
                bi[i] = (uint32_t)ids_in[c0 + i];
                bp[i] = pos_in[c0 + i];
            }
            __syncthreads();
        }
        int32_t id[kSplitPer];
        uint32_t ps[kSplitPer], rank[kSplitPer];
#pragma unroll
        for (int k = 0; k < kSplitPer; ++k) {
            const int i = tid + k * kSplitThreads;
            id[k] = -1;
            if (i < cnt) {
                id[k] = (int32_t)bi[i];
                ps[k] = bp[i];
                const int64_t off = (int64_t)id[k] - s0;
                MSC_GUARD(off >= 0 && off < (int64_t(1) << shift), status, -106)
                rank[k] = atomicAdd(&s_cnt[off >> kSubLog2], 1u);
            }
        }
        __syncthreads();
        // chunk-local exclusive starts over the nsub (<= 256) sub-buckets, and
        // the chunk's reservation in each of them
        const uint32_t cc = tid < nsub ? s_cnt[tid] : 0u;
        uint32_t incl = cc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += s_w[w];
        if (tid < nsub) {
            s_base[tid] = cc ? atomicAdd(&sub_fill[(s0 >> kSubLog2) + tid], cc) : 0u;
            s_cnt[tid] = before + incl - cc;
        }
        __syncthreads();
        // regroup in place: every pair of the chunk was read before the barriers above
#pragma unroll
        for (int k = 0; k < kSplitPer; ++k)
            if (id[k] >= 0) {
                const uint32_t j = s_cnt[(uint32_t)(id[k] - s0) >> kSubLog2] + rank[k];
                MSC_GUARD(j < (uint32_t)kSplitChunk, status, -109) {
                    bi[j] = (uint32_t)id[k];
                    bp[j] = ps[k];
                }
            }
        __syncthreads();
        for (int i = tid; i < cnt; i += kSplitThreads) {
            const int32_t v = (int32_t)bi[i];
            const int sub = (int)((uint32_t)(v - s0) >> kSubLog2);
            const uint32_t slot_ = s_base[sub] + (uint32_t)i - s_cnt[sub];
            const int64_t dst = s0 + ((int64_t)sub << kSubLog2) + slot_;
            MSC_GUARD(slot_ < (uint32_t)kSubIds && dst < n, status, -107) {
                ids_out[dst] = v;
                pos_out[dst] = bp[i];
            }
        }
        // this buffer is refilled by a bulk copy (async proxy) two chunks on
        fence_proxy_async_smem();
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_pair_scatter_local(const int32_t* __restrict__ ids,
                                                             const uint32_t* __restrict__ pos, int64_t n,
                                                             int32_t* __restrict__ order, int32_t* status) {
    extern __shared__ __align__(16) int32_t slice[];  // kSubIds
    const int64_t nsub = (n + kSubIds - 1) >> kSubLog2;
    for (int64_t sb = blockIdx.x; sb < nsub; sb += gridDim.x) {
        const int64_t s0 = sb << kSubLog2, s1 = min(n, s0 + kSubIds);
        const int cnt = (int)(s1 - s0);
        for (int i = threadIdx.x; i < cnt; i += 1024) {
            const int32_t id = __ldcs(ids + s0 + i);
            const uint32_t p = __ldcs(pos + s0 + i);
            const int64_t off = (int64_t)id - s0;
            MSC_GUARD(off >= 0 && off < cnt, status, -108)
            slice[off] = (int32_t)p;
        }
        __syncthreads();
        // 16-byte stores when the caller's array allows them (s0 is a multiple
        // of 2^15, so the base pointer decides), else one word at a time
        const int full = ((uintptr_t)order & 15) == 0 ? cnt >> 2 : 0;
        for (int i = threadIdx.x; i < full; i += 1024)
            reinterpret_cast<int4*>(order + s0)[i] = reinterpret_cast<const int4*>(slice)[i];
        for (int i = full * 4 + threadIdx.x; i < cnt; i += 1024) order[s0 + i] = slice[i];
        __syncthreads();
    }
}

int launch_pair_split_scatter(int shift, const int32_t* ids, const uint32_t* pos, int32_t* ids2, uint32_t* pos2,
                              uint32_t* sub_fill, int64_t n, int32_t* order, int32_t* status, cudaStream_t s) {
    const int sms = current_device().sms;
    MSC_TRY(cudaMemsetAsync(sub_fill, 0, (size_t)(ceil_div(n, kSubIds) + 1) * sizeof(uint32_t), s));
    static int configured_dev = -1;
    if (configured_dev != current_device().id) {
        MSC_TRY(cudaFuncSetAttribute(k_pair_scatter_local, cudaFuncAttributeMaxDynamicSharedMemorySize, kSubIds * 4));
        MSC_TRY(cudaFuncSetAttribute(k_pair_split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSplitSmem));
        configured_dev = current_device().id;
    }
    {
        const int64_t chunks = ceil_div(n, kSplitChunk);
        const int use_tma = ((uintptr_t)ids & 15) == 0 && ((uintptr_t)pos & 15) == 0;
        TraceScope ts_("order.split", s);
        k_pair_split<<<(unsigned)std::min<int64_t>(chunks, (int64_t)sms * 2), kSplitThreads, kSplitSmem, s>>>(
            ids, pos, n, shift, use_tma, sub_fill, ids2, pos2, status);
    }
    MSC_LAUNCHED();
    const int64_t nsub = ceil_div(n, kSubIds);
    {
        TraceScope ts_("order.scatter", s);
        k_pair_scatter_local<<<(unsigned)std::min<int64_t>(nsub, (int64_t)sms), 1024, kSubIds * 4, s>>>(
            ids2, pos2, n, order, status);
    }
    MSC_LAUNCHED();
    return MSC_OK;
}

template <typename KeyT, bool FROM_F, bool BUCKET, bool SEG = false>
int launch_pass(const PassArgs<KeyT>& a, int64_t max_n, cudaStream_t s, const char* label) {
    constexpr size_t smem = pass_smem_bytes<KeyT, true>();
    auto kern = k_onesweep<KeyT, FROM_F, BUCKET, SEG>;
    static int configured_dev = -1;  // the attribute is set once per device
    if (configured_dev != current_device().id) {
        MSC_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured_dev = current_device().id;
    }
    int occ = 0;
    MSC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem));
    const int64_t ntiles = SEG ? a.seg_tiles : ceil_div(max_n, kSortTile);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)current_device().sms * std::max(occ, 1)));
    {
        TraceScope ts_(label, s);
        kern<<<(unsigned)grid, kThreads, smem, s>>>(a);
    }
    MSC_LAUNCHED();
    return MSC_OK;
}

}  // namespace

int order_bucket_shift(int64_t n) { return bucket_shift(n); }

int order_invert(int shift, const int32_t* ids, const uint32_t* pos, int32_t* ids2, uint32_t* pos2,
                 uint32_t* sub_fill, int64_t n, int32_t* order, int32_t* status, cudaStream_t s) {
    return launch_pair_split_scatter(shift, ids, pos, ids2, pos2, sub_fill, n, order, status, s);
}

void size_sort_scratch(Sizer& s, int64_t n) {
    s.take<uint32_t>(kOrderCntWords);
    s.take<uint32_t>(8 * kBins + kCounterWords);
    s.take<uint32_t>(ceil_div(std::max<int64_t>(n, 1), kSubIds) + 1);
    s.take<unsigned long long>((size_t)std::max<int64_t>(1, ceil_div(n, kSortTile)) * kBins);
}

SortScratch carve_sort_scratch(Carver& c, int64_t n) {
    SortScratch sc;
    sc.ord_cnt = c.take<uint32_t>(kOrderCntWords);
    sc.hist = c.take<uint32_t>(8 * kBins + kCounterWords);
    sc.tile_counters = sc.hist + 8 * kBins;
    sc.sub_fill = c.take<uint32_t>(ceil_div(std::max<int64_t>(n, 1), kSubIds) + 1);
    sc.max_tiles = std::max<int64_t>(1, ceil_div(n, kSortTile));
    sc.lookback = c.take<unsigned long long>((size_t)sc.max_tiles * kBins);
    return sc;
}

// Clears the look-back words of the tiles that *d_n keys occupy (a sort
// whose count is known only on the device touches no other tile).
__global__ void k_clear_lookback(unsigned long long* lookback, const int32_t* __restrict__ d_n,
                                 int64_t max_n) {
    const int64_t words = ((min((int64_t)*d_n, max_n) + kSortTile - 1) / kSortTile) * kBins;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (int64_t)gridDim.x * blockDim.x)
        lookback[i] = 0ull;
}

static size_t hist_smem(int npass) { return (size_t)kWarps * npass * kBins * sizeof(uint32_t); }

// Allow both histogram kernels the shared memory of 8 passes (64 KiB).
static int configure_hist() {
    static int configured_dev = -1;
    if (configured_dev != current_device().id) {
        const int bytes = (int)hist_smem(8);
        MSC_TRY(cudaFuncSetAttribute(k_hist<uint32_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        MSC_TRY(cudaFuncSetAttribute(k_hist<unsigned long long, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        configured_dev = current_device().id;
    }
    return MSC_OK;
}

static int hist_grid(int64_t n) {
    const int64_t want = ceil_div(std::max<int64_t>(n, 1), 256 * kHistRun);
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)current_device().sms * 8));
}

void size_seg_sort_scratch(Sizer& s, int count, int64_t tiles) {
    s.take<uint32_t>((size_t)count * kSegPasses * kBins + kCounterWords);
    s.take<uint32_t>(ceil_div(std::max<int64_t>(tiles, 1) * kSortTile, kSubIds) + 1);
    s.take<unsigned long long>((size_t)std::max<int64_t>(1, tiles) * kBins);
}

SortScratch carve_seg_sort_scratch(Carver& c, int count, int64_t tiles) {
    SortScratch sc;
    sc.ord_cnt = nullptr;
    const size_t hist_words = (size_t)count * kSegPasses * kBins;
    sc.hist = c.take<uint32_t>(hist_words + kCounterWords);
    sc.tile_counters = sc.hist + hist_words;
    sc.sub_fill = c.take<uint32_t>(ceil_div(std::max<int64_t>(tiles, 1) * kSortTile, kSubIds) + 1);
    sc.max_tiles = std::max<int64_t>(1, tiles);
    sc.lookback = c.take<unsigned long long>((size_t)sc.max_tiles * kBins);
    return sc;
}

int run_order_seg(const float* f, const SegTable& t, int32_t* order, uint32_t* key_a, int32_t* id_a,
                  uint32_t* key_b, int32_t* id_b, const SortScratch& sc, int32_t* status,
                  cudaStream_t s) {
    if (t.tiles <= 0) return MSC_OK;
    const size_t hist_words = (size_t)t.count * kSegPasses * kBins;
    MSC_TRY(cudaMemsetAsync(sc.hist, 0, (hist_words + kCounterWords) * sizeof(uint32_t), s));
    MSC_TRY(cudaMemsetAsync(sc.lookback, 0, (size_t)t.tiles * kBins * sizeof(unsigned long long), s));
    int r = configure_hist();
    if (r) return r;
    {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(t.tiles, (int64_t)current_device().sms * 4));
        TraceScope ts_("order.hist", s);
        k_hist_seg<<<grid, 256, hist_smem(kSegPasses), s>>>(f, t.tile_seg, t.off, t.tile0, t.tiles, sc.hist, status);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("order.bstart", s);
        k_seg_bstart<<<(unsigned)(t.count * kSegPasses), 256, 0, s>>>(sc.hist);
    }
    MSC_LAUNCHED();
    PassArgs<uint32_t> a{};
    a.n = t.total;
    a.status = status;
    a.lookback = sc.lookback;
    a.tile_seg = t.tile_seg;
    a.seg_off = t.off;
    a.seg_tile0 = t.tile0;
    a.seg_tiles = t.tiles;
    a.seg_stride = kSegPasses * kBins;
    a.f_in = f;
    a.keys_out = key_a;
    a.vals_out = id_a;
    a.hist = sc.hist;
    a.shift = 0;
    a.tile_counter = sc.tile_counters + 0;
    a.epoch = 1;
    if ((r = launch_pass<uint32_t, true, false, true>(a, t.total, s, "order.pass_first"))) return r;
    uint32_t* kin = key_a;
    int32_t* iin = id_a;
    uint32_t* kout = key_b;
    int32_t* iout = id_b;
    for (int p = 1; p <= 2; ++p) {
        a.f_in = nullptr;
        a.keys_in = kin;
        a.vals_in = iin;
        a.keys_out = kout;
        a.vals_out = iout;
        a.hist = sc.hist + p * kBins;
        a.shift = 8 * p;
        a.tile_counter = sc.tile_counters + p;
        a.epoch = (uint32_t)(p + 1);
        if ((r = launch_pass<uint32_t, false, false, true>(a, t.total, s, "order.pass"))) return r;
        std::swap(kin, kout);
        std::swap(iin, iout);
    }
    a.keys_in = kin;
    a.vals_in = iin;
    a.keys_out = nullptr;
    a.vals_out = iout;
    a.pair_pos = kout;
    a.bucket_fill = sc.tile_counters + 8;
    a.bucket_shift = bucket_shift(t.total);
    a.hist = sc.hist + 3 * kBins;
    a.shift = 24;
    a.tile_counter = sc.tile_counters + 3;
    a.epoch = 4;
    if ((r = launch_pass<uint32_t, false, true, true>(a, t.total, s, "order.pass_last"))) return r;
    return launch_pair_split_scatter(a.bucket_shift, iout, kout, iin, kin, sc.sub_fill, t.total, order, status, s);
}

int run_sort_u64(unsigned long long* keys, int32_t* vals, unsigned long long* keys_alt,
                 int32_t* vals_alt, const int32_t* d_count, int64_t max_count, int key_bits,
                 const SortScratch& sc, int32_t* status, cudaStream_t s, bool* result_in_alt,
                 const char* hist_label, const char* pass_label) {
    *result_in_alt = false;
    if (max_count <= 0 || key_bits <= 0) return MSC_OK;
    const int npass = std::min(8, (key_bits + 7) / 8);
    MSC_TRY(cudaMemsetAsync(sc.hist, 0, (8 * kBins + kCounterWords) * sizeof(uint32_t), s));
    {
        TraceScope ts_("sort.clear_lookback", s);
        k_clear_lookback<<<(unsigned)std::min<int64_t>(ceil_div(ceil_div(max_count, kSortTile) * kBins, 256),
                                                       (int64_t)current_device().sms * 8),
                           256, 0, s>>>(sc.lookback, d_count, max_count);
    }
    MSC_LAUNCHED();
    int r = configure_hist();
    if (r) return r;
    {
        TraceScope ts_(hist_label, s);
        k_hist<unsigned long long, false><<<hist_grid(max_count), 256, hist_smem(npass), s>>>(keys, nullptr, max_count, d_count, npass, sc.hist, status);
    }
    MSC_LAUNCHED();
    PassArgs<unsigned long long> a{};
    a.n = max_count;
    a.d_n = d_count;
    a.status = status;
    a.lookback = sc.lookback;
    unsigned long long* kin = keys;
    int32_t* vin = vals;
    unsigned long long* kout = keys_alt;
    int32_t* vout = vals_alt;
    for (int p = 0; p < npass; ++p) {
        a.keys_in = kin;
        a.vals_in = vin;
        a.keys_out = kout;
        a.vals_out = vout;
        a.hist = sc.hist + p * kBins;
        a.shift = 8 * p;
        a.tile_counter = sc.tile_counters + p;
        a.epoch = (uint32_t)(p + 1);
        if ((r = launch_pass<unsigned long long, false, false>(a, max_count, s, pass_label))) return r;
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    *result_in_alt = (npass & 1) != 0;
    return MSC_OK;
}

}  // namespace msc

#ifdef MSC_DEBUG_BOUNDS
extern "C" MSC_API int msc_debug_sort(uint32_t* out16) {
    return cudaMemcpyFromSymbol(out16, msc::g_sort_dbg, sizeof(uint32_t) * 16) == cudaSuccess ? 0 : -3;
}
#endif
