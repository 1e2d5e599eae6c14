// Dense Morse-Smale cell ids.  A cell is the set of vertices sharing one
// (minimum, maximum) pair (section "Ascending and Descending
// Segmentation"); its id is the pair's rank among the distinct pairs in
// lexicographic order, minimum first.
//
// 1. A linear-probing hash table de-duplicates the pair keys
//    (asc << b) | desc, b = ceil(log2 n).  Its capacity is a power of two
//    >= 2 * #minima * #maxima, or >= n when that is more than n (there are
//    at most n distinct pairs), chosen on the device, so smooth fields (few
//    extrema) use a table that lives in L2.  Probing never wraps: the table
//    has kPad slots past its capacity.  Within a warp, a run of consecutive
//    vertices with the same key (neighbours usually share a cell) probes
//    once.  Each vertex keeps its slot in `ms` for now.
// 2. Ranks, by one of two routes chosen on the device:
//    (a) tables too big for the cache place a pair at the slot
//        base(asc) = asc * cap / n plus a small spread and the probe
//        distance; the insert records the largest distance M of a pair from
//        its base.  A pair whose base lies in the chunk of slots
//        [jC, (j+1)C) then sits in [jC, (j+1)C + M), and the pairs before
//        chunk j in key order are the occupied slots below jC plus the
//        pairs in [jC, jC + M) whose base is below jC.  One block per chunk
//        loads that window, groups its pairs by base (counting sort over the
//        C bases), ranks each pair inside its base's group by counting the
//        group's smaller keys (groups of at most kGroupMax), and writes
//        rank = (pairs before the chunk) + position into the table.  No
//        global sort.
//    (b) otherwise -- small tables with random home slots, a group or a
//        chunk too big for (a), a caller that needs the sorted keys --
//        the occupied slots are compacted, radix-sorted by key and ranked.
// 3. ms[v] = table_vals[ms[v]].
#include <cuda_runtime.h>

#include <algorithm>

#include "msid.cuh"
#include "radix.cuh"

namespace msc {
namespace {

constexpr int kThreads = 256;
constexpr unsigned long long kEmpty = ~0ull;
constexpr uint32_t kSpread = 64;  // random spread of a pair around its home slot
constexpr uint32_t kCacheResidentSlots = 1u << 20;  // 8 MiB of keys: plain random hashing
constexpr uint32_t kPad = 4096;   // slots past the capacity: probing never wraps
constexpr int kChunkLog2 = 12;    // route (a): chunks of 4096 slots (bases)
constexpr int kChunk = 1 << kChunkLog2;
constexpr uint32_t kMaxWindow = 2048;                 // route (a): largest M it accepts
constexpr int kRankThreads = 512;
constexpr int kWinPer = (kChunk + kMaxWindow) / kRankThreads;  // window slots per thread (12)
constexpr int kGroupMax = 128;        // route (a): pairs of one base ranked by counting

// control words (ctl[0..3] are shared with the callers: nmin, nmax, cap, K)
constexpr int kCtlRoute = 16;   // 0: route (a); nonzero: route (b)
constexpr int kCtlM = 17;       // largest slot - asc * cap / n of a pair
constexpr int kCtlCompact = 18; // route (b): compacted pairs
constexpr int kCtlShift = 19;   // b of the pair keys

__device__ __forceinline__ unsigned long long mix64(unsigned long long k) {
    // 64-bit finaliser of MurmurHash3
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// Validate labels and count extrema (labels that label themselves).
__global__ void k_ms_prepare(const int32_t* __restrict__ asc, const int32_t* __restrict__ desc,
                             int32_t n, uint32_t* ctl, int32_t* status) {
    uint32_t nmin = 0, nmax = 0;
    bool bad = false;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = asc[v], d = desc[v];
        if ((uint32_t)a >= (uint32_t)n || (uint32_t)d >= (uint32_t)n) {
            bad = true;
            continue;
        }
        if (asc[a] != a || desc[d] != d) bad = true;
        nmin += a == v;
        nmax += d == v;
    }
    if (bad) record_error(status, MSC_ERR_ARG);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nmin += __shfl_xor_sync(0xffffffffu, nmin, o);
        nmax += __shfl_xor_sync(0xffffffffu, nmax, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (nmin) atomicAdd(&ctl[0], nmin);
        if (nmax) atomicAdd(&ctl[1], nmax);
    }
}

__global__ void k_ms_setcap(uint32_t* ctl, int64_t n, int64_t cap_max, int sh, int force_sort) {
    const unsigned long long pairs = (unsigned long long)ctl[0] * ctl[1];
    const unsigned long long bound = pairs < (unsigned long long)n ? pairs : (unsigned long long)n;
    // twice the bound on the distinct pairs while that stays within n, else
    // the bound itself (there are at most n pairs; white noise fills a
    // table of n slots to about a third)
    const unsigned long long want = 2 * bound <= (unsigned long long)n ? 2 * bound : bound;
    unsigned long long cap = 64;
    while (cap < want) cap <<= 1;
    if ((long long)cap > cap_max) cap = (unsigned long long)cap_max;
    ctl[2] = (uint32_t)cap;  // cap_max <= 2^31
    ctl[3] = 0;
    // home-slot multiplier: asc * cap / n as (asc * F) >> 32, F = cap * 2^32 / n
    const unsigned long long f = (cap << 32) / (unsigned long long)n;
    ctl[9] = (uint32_t)f;
    ctl[10] = (uint32_t)(f >> 32);
    ctl[kCtlRoute] = (cap <= kCacheResidentSlots || force_sort) ? 1u : 0u;
    ctl[kCtlM] = 0;
    ctl[kCtlCompact] = 0;
    ctl[kCtlShift] = (uint32_t)sh;
}

__global__ void k_ms_clear(unsigned long long* keys, const uint32_t* ctl) {
    const int64_t slots = (int64_t)ctl[2] + kPad;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < slots;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = kEmpty;
}

// asc * cap / n by a fixed-point multiply (f = cap * 2^32 / n), no division.
__device__ __forceinline__ uint32_t slot_base(uint32_t asc, unsigned long long f) {
    return (uint32_t)((unsigned long long)asc * (f >> 32) + (((unsigned long long)asc * (uint32_t)f) >> 32));
}

// Home slot of a pair.  In a table too big for the cache: proportional to
// its minimum's id plus a small random spread.  The minimum of a vertex
// lies near the vertex, so the vertices of a warp, and the warps in flight,
// probe a narrow band of the table (L2 hits instead of random DRAM
// sectors), and a pair's slot is at most M past asc * cap / n.
__device__ __forceinline__ uint32_t home_slot(uint32_t asc, unsigned long long key, uint32_t cap,
                                              unsigned long long f) {
    if (cap <= kCacheResidentSlots) return (uint32_t)mix64(key) & (cap - 1);  // fits in cache: spread
    return slot_base(asc, f) + (uint32_t)(mix64(key) & (kSpread - 1));
}

// Linear probing over the cap + kPad slots; `fresh` when this call stored
// the key.  Probe i looks at slot home + i; after kNearProbes slots it goes
// on from a second, random home, so that the many pairs of one minimum (all
// with one home window) cannot build one long cluster.  Every insert of a
// key follows the same sequence, so equal keys meet.  Leaving the home
// window or running off the end (the probe then continues at slot 0) sets
// `broke`: a pair is no longer within M of its base.  The probe resumes at
// step i0 (slot h0), after the steps a caller made itself.
constexpr uint32_t kNearProbes = 1024;
static_assert(kPad % 4 == 0, "the table's slot count is a multiple of four");

__device__ __forceinline__ uint32_t probe_insert(unsigned long long* keys, uint32_t cap, unsigned long long key,
                                                 uint32_t i0, uint32_t h0, bool& fresh, bool& broke,
                                                 int32_t* status) {
    const uint32_t lim = cap + kPad;
    uint32_t h = h0;
    // One round trip reads the aligned group of four slots (one 32-byte
    // sector) holding slot h and takes the first of slots h, h+1, ... in it
    // that holds the key or is empty.  The steps stop exactly at kNearProbes
    // and at the end of the table (lim, a multiple of four), so every insert
    // of a key visits the same slots in the same order.
    uint32_t i = i0;
    while (i < lim + kNearProbes) {
        if (i == kNearProbes) {
            h = (uint32_t)mix64(key ^ 0x9e3779b97f4a7c15ull) & (cap - 1);
            broke = true;
        }
        const uint32_t g0 = h & ~3u, start = h - g0;
        const uint32_t end = i < kNearProbes ? min(4u, start + (kNearProbes - i)) : 4u;
        const ulonglong2 lo = *reinterpret_cast<const ulonglong2*>(keys + g0);
        const ulonglong2 hi = *reinterpret_cast<const ulonglong2*>(keys + g0 + 2);
        const unsigned long long sl[4] = {lo.x, lo.y, hi.x, hi.y};
        uint32_t q = 4;
        unsigned long long v = 0;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            if ((uint32_t)j >= start && (uint32_t)j < end && (sl[j] == key || sl[j] == kEmpty)) {
                q = (uint32_t)j;
                v = sl[j];
            }
        }
        if (q == 4) {  // none in the group: on to the next one
            i += end - start;
            h = g0 + end;
        } else {
            const uint32_t slot = g0 + q;
            if (v == key) return slot;
            const unsigned long long old = atomicCAS(&keys[slot], kEmpty, key);
            if (old == kEmpty) {
                fresh = true;
                return slot;
            }
            if (old == key) return slot;
            i += q - start + 1;  // another key took the slot first
            h = slot + 1;
        }
        if (h == lim) {
            h = 0;
            broke = true;
        }
    }
    record_error(status, MSC_ERR_INTERNAL);  // table full: impossible at load <= 1/2
    return 0;
}

// Each thread takes kInsJ vertices per step (lane-consecutive within each
// of them), so that the first probe load, and the claiming CAS, of all of
// them are in flight together; the rare longer probe then goes on alone.
#ifndef MSC_MS_INSERT_J
#define MSC_MS_INSERT_J 4
#endif
constexpr int kInsJ = MSC_MS_INSERT_J;

__global__ void __launch_bounds__(kThreads) k_ms_insert(const int32_t* __restrict__ asc,
                                                        const int32_t* __restrict__ desc, int32_t n,
                                                        unsigned long long* keys, uint32_t* ctl, int32_t* ms,
                                                        int32_t* status) {
    const uint32_t cap = ctl[2];
    const uint32_t lim = cap + kPad;
    const int sh = (int)ctl[kCtlShift];
    const bool ordered = ctl[kCtlRoute] == 0u;
    const unsigned long long f = (unsigned long long)ctl[9] | ((unsigned long long)ctl[10] << 32);
    const int lane = threadIdx.x & 31;
    constexpr int64_t kStep = (int64_t)kThreads * kInsJ;
    uint32_t added = 0, far = 0;
    bool broke = false;
    for (int64_t c0 = (int64_t)blockIdx.x * kStep; c0 < n; c0 += (int64_t)gridDim.x * kStep) {
        unsigned long long key[kInsJ], w[kInsJ], old[kInsJ];
        uint32_t a[kInsJ], h[kInsJ], slot[kInsJ];
        uint32_t probing = 0, heads_mask[kInsJ];
#pragma unroll
        for (int j = 0; j < kInsJ; ++j) {
            const int64_t v = c0 + (int64_t)j * kThreads + threadIdx.x;
            const bool valid = v < n;
            key[j] = kEmpty - 1 - lane;  // distinct per idle lane
            a[j] = 0;
            if (valid) {
                a[j] = (uint32_t)asc[v];
                key[j] = ((unsigned long long)a[j] << sh) | (uint32_t)desc[v];
            }
            // neighbouring vertices usually share their cell: only the first
            // lane of each run of equal keys probes, the others take its slot
            const unsigned long long prev = __shfl_up_sync(0xffffffffu, key[j], 1);
            const bool head = lane == 0 || key[j] != prev;
            heads_mask[j] = __ballot_sync(0xffffffffu, head);
            if (valid && head) probing |= 1u << j;
        }
#pragma unroll
        for (int j = 0; j < kInsJ; ++j) {
            slot[j] = 0;
            if (probing >> j & 1u) {
                h[j] = home_slot(a[j], key[j], cap, f);
                w[j] = keys[h[j]];
            }
        }
#pragma unroll
        for (int j = 0; j < kInsJ; ++j)
            if ((probing >> j & 1u) && w[j] == kEmpty) old[j] = atomicCAS(&keys[h[j]], kEmpty, key[j]);
#pragma unroll
        for (int j = 0; j < kInsJ; ++j) {
            if (!(probing >> j & 1u)) continue;
            bool fresh = false;
            if (w[j] == key[j] || (w[j] == kEmpty && old[j] == key[j])) {
                slot[j] = h[j];
            } else if (w[j] == kEmpty && old[j] == kEmpty) {
                slot[j] = h[j];
                fresh = true;
            } else {  // the home slot holds another key: go on probing
                uint32_t h1 = h[j] + 1;
                if (h1 == lim) {
                    h1 = 0;
                    broke = true;
                }
                slot[j] = probe_insert(keys, cap, key[j], 1, h1, fresh, broke, status);
            }
            added += fresh;
            // how far past its base a pair landed (route (a))
            if (ordered && fresh && !broke) far = max(far, slot[j] - slot_base(a[j], f));
        }
#pragma unroll
        for (int j = 0; j < kInsJ; ++j) {
            const int my_head = 31 - __clz(heads_mask[j] & (0xffffffffu >> (31 - lane)));
            const uint32_t mine = __shfl_sync(0xffffffffu, slot[j], my_head);
            const int64_t v = c0 + (int64_t)j * kThreads + threadIdx.x;
            if (v < n) ms[v] = (int32_t)mine;
        }
    }
    added = __reduce_add_sync(0xffffffffu, added);
    far = __reduce_max_sync(0xffffffffu, far);
    if (__any_sync(0xffffffffu, broke) && lane == 0) atomicOr(&ctl[kCtlRoute], 16u);
    if (lane == 0) {
        if (added) atomicAdd(&ctl[3], added);
        if (far) atomicMax(&ctl[kCtlM], far);
    }
}

// Route (a), step 1: occupied slots per chunk of slots.
__global__ void __launch_bounds__(kThreads) k_ms_occ(const unsigned long long* __restrict__ keys,
                                                     uint32_t* __restrict__ occ, int64_t nchunks,
                                                     const uint32_t* ctl) {
    __shared__ uint32_t s_w[kThreads / 32];
    if (ctl[kCtlRoute] != 0u) return;
    const int64_t lim = (int64_t)ctl[2] + kPad;
    const int tid = threadIdx.x;
    for (int64_t j = blockIdx.x; j < nchunks; j += gridDim.x) {
        uint32_t c = 0;
        const int64_t s0 = j << kChunkLog2;
        if (s0 >= lim) {  // past the table in use
            if (tid == 0) occ[j] = 0;
            continue;
        }
#pragma unroll
        for (int q = 0; q < kChunk / kThreads / 2; ++q) {  // two slots per 16-byte load
            const int64_t h = s0 + 2 * ((int64_t)q * kThreads + tid);
            if (h + 1 < lim) {
                const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(keys + h);
                c += (v.x != kEmpty) + (v.y != kEmpty);
            } else if (h < lim) {
                c += keys[h] != kEmpty;
            }
        }
        c = __reduce_add_sync(0xffffffffu, c);
        if ((tid & 31) == 0) s_w[tid >> 5] = c;
        __syncthreads();
        if (tid == 0) {
            uint32_t t = 0;
            for (int w = 0; w < kThreads / 32; ++w) t += s_w[w];
            occ[j] = t;
        }
        __syncthreads();
    }
}

// Route (a), step 2: exclusive scan of the chunk counts (one block).
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) k_ms_chunk_scan(const uint32_t* __restrict__ cnt,
                                                                 uint32_t* __restrict__ base, int64_t nchunks,
                                                                 const uint32_t* ctl) {
    __shared__ uint32_t s_w[kScanThreads / 32];
    if (ctl[kCtlRoute] != 0u) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t per = (nchunks + kScanThreads - 1) / kScanThreads;
    const int64_t i0 = (int64_t)tid * per, i1 = min(nchunks, i0 + per);
    uint32_t sum = 0;
    for (int64_t i = i0; i < i1; ++i) sum += cnt[i];
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t q = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += q;
        }
        s_w[lane] = t;
    }
    __syncthreads();
    uint32_t run = incl - sum + (warp ? s_w[warp - 1] : 0u);
    for (int64_t i = i0; i < i1; ++i) {
        base[i] = run;
        run += cnt[i];
    }
}

// Route (a), step 3: one block per chunk of slots at a time.  The window's
// keys are loaded into registers at once (kWinPer per thread).
constexpr size_t kRankSmem = (size_t)(kChunk + kMaxWindow) * 12 + kChunk * 4 + 32 * 4;

__global__ void __launch_bounds__(kRankThreads, 2) k_ms_chunk_rank(const unsigned long long* __restrict__ keys,
                                                                   uint32_t* __restrict__ vals,
                                                                   const uint32_t* __restrict__ occ_before,
                                                                   int64_t nchunks, uint32_t* ctl) {
    constexpr int kWin = kChunk + kMaxWindow;
    extern __shared__ __align__(16) uint8_t smem[];
    unsigned long long* s_key = reinterpret_cast<unsigned long long*>(smem);  // [kWin]
    uint32_t* s_slot = reinterpret_cast<uint32_t*>(s_key + kWin);            // [kWin]
    uint32_t* s_hist = s_slot + kWin;                                        // [kChunk]
    uint32_t* s_misc = s_hist + kChunk;  // [32]: [1] pairs with base below the chunk [2..17] scan
    if (ctl[kCtlRoute] != 0u) return;
    const uint32_t M = ctl[kCtlM];
    if (M > kMaxWindow) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ctl[kCtlRoute], 1u);
        return;
    }
    const int64_t lim = (int64_t)ctl[2] + kPad;
    const int sh = (int)ctl[kCtlShift];
    const unsigned long long f = (unsigned long long)ctl[9] | ((unsigned long long)ctl[10] << 32);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // the window of chunk j, all loads in flight at once (the next chunk's
    // window is loaded while the current one is sorted and written)
    unsigned long long k[kWinPer];
    // slots of a window: the chunk plus M (rows of kRankThreads)
    const int nq = (int)((kChunk + M + kRankThreads - 1) / kRankThreads);
    auto load_window = [&](int64_t j) {
        const int64_t s0 = j << kChunkLog2;
        const int64_t s1 = min(lim, s0 + kChunk + (int64_t)M);
#pragma unroll
        for (int q = 0; q < kWinPer; ++q) {
            const int64_t h = s0 + (int64_t)q * kRankThreads + tid;
            k[q] = (q < nq && h < s1) ? keys[h] : kEmpty;
        }
    };
    if ((int64_t)blockIdx.x < nchunks) load_window(blockIdx.x);
    for (int64_t j = blockIdx.x; j < nchunks; j += gridDim.x) {
        const int64_t s0 = j << kChunkLog2;
        if (s0 >= lim) break;  // past the table in use (block-uniform)
        for (int i = tid; i < kChunk; i += kRankThreads) s_hist[i] = 0;
        if (tid < 2) s_misc[tid] = 0;
        // each key's offset of its base from s0 (or -1: empty, or a base
        // outside the chunk)
        int32_t off[kWinPer];
        __syncthreads();
        uint32_t below = 0;
#pragma unroll
        for (int q = 0; q < kWinPer; ++q) {
            off[q] = -1;
            if (q >= nq || k[q] == kEmpty) continue;
            const int64_t b = (int64_t)slot_base((uint32_t)(k[q] >> sh), f) - s0;
            if (b < 0) {
                ++below;
            } else if (b < kChunk) {
                off[q] = (int32_t)b;
                atomicAdd(&s_hist[b], 1u);
            }
        }
        below = __reduce_add_sync(0xffffffffu, below);
        if (lane == 0 && below) atomicAdd(&s_misc[1], below);
        __syncthreads();
        {   // exclusive starts of the bases (8 consecutive per thread)
            constexpr int kPer = kChunk / kRankThreads;
            uint32_t x[kPer], sum = 0;
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                x[i] = s_hist[tid * kPer + i];
                sum += x[i];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane == 31) s_misc[2 + warp] = incl;
            __syncthreads();
            uint32_t run = incl - sum;
            for (int w = 0; w < warp; ++w) run += s_misc[2 + w];
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                s_hist[tid * kPer + i] = run;
                run += x[i];
            }
        }
        __syncthreads();
        // gather the pairs grouped by base (cursors advance the starts)
#pragma unroll
        for (int q = 0; q < kWinPer; ++q) {
            if (q >= nq || off[q] < 0) continue;
            const uint32_t p = atomicAdd(&s_hist[off[q]], 1u);
            s_key[p] = k[q];
            s_slot[p] = (uint32_t)(s0 + (int64_t)q * kRankThreads + tid);
        }
        if (j + gridDim.x < nchunks) load_window(j + gridDim.x);
        __syncthreads();
        // each pair's position: the start of its base's group plus the pairs
        // of the group with a smaller key (s_hist[i] is now the end of group
        // i); pairs of one thread are spread over the whole chunk
        const uint32_t count = s_hist[kChunk - 1];
        const uint32_t first = occ_before[j] + s_misc[1];
        bool big = false;
        for (uint32_t p = tid; p < count; p += kRankThreads) {
            const unsigned long long kk = s_key[p];
            const uint32_t b = slot_base((uint32_t)(kk >> sh), f) - (uint32_t)s0;
            const uint32_t beg = b ? s_hist[b - 1] : 0u, end = s_hist[b];
            if (end - beg > (uint32_t)kGroupMax) {
                big = true;
                continue;
            }
            uint32_t r = 0;
            for (uint32_t q = beg; q < end; ++q) r += s_key[q] < kk;
            vals[s_slot[p]] = first + beg + r;
        }
        if (big) atomicOr(&ctl[kCtlRoute], 4u);
        __syncthreads();
    }
}

// Route (b): compact occupied slots into (key, slot) pairs: each thread
// scans 8 consecutive slots with 16-byte loads; one atomic append per
// block chunk.
constexpr int kCompactPer = 8;

__global__ void __launch_bounds__(kThreads) k_ms_compact(const unsigned long long* __restrict__ keys,
                                                         uint32_t* ctl, unsigned long long* ukeys,
                                                         int32_t* uvals, int32_t* status) {
    __shared__ uint32_t s_warp[kThreads / 32];
    __shared__ uint32_t s_base;
    if (ctl[kCtlRoute] == 0u) return;
    const int64_t slots = (int64_t)ctl[2] + kPad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int64_t kChunkSlots = (int64_t)kThreads * kCompactPer;
    const int64_t nchunks = (slots + kChunkSlots - 1) / kChunkSlots;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int64_t i0 = c * kChunkSlots + (int64_t)tid * kCompactPer;
        unsigned long long k[kCompactPer];
        if (i0 + kCompactPer <= slots) {  // cap and kPad are multiples of 8: whole groups
#pragma unroll
            for (int q = 0; q < kCompactPer / 2; ++q) {
                const ulonglong2 v = reinterpret_cast<const ulonglong2*>(keys + i0)[q];
                k[2 * q] = v.x;
                k[2 * q + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kCompactPer; ++j) k[j] = i0 + j < slots ? keys[i0 + j] : kEmpty;
        }
        uint32_t cnt = 0;
#pragma unroll
        for (int j = 0; j < kCompactPer; ++j) cnt += k[j] != kEmpty;
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (tid == 0) {
            uint32_t run = 0;
            for (int w = 0; w < kThreads / 32; ++w) {
                const uint32_t t = s_warp[w];
                s_warp[w] = run;
                run += t;
            }
            s_base = run ? atomicAdd(&ctl[kCtlCompact], run) : 0u;
        }
        __syncthreads();
        uint32_t pos = s_base + s_warp[warp] + incl - cnt;
#pragma unroll
        for (int j = 0; j < kCompactPer; ++j) {
            if (k[j] != kEmpty) {
                MSC_GUARD(pos < (uint32_t)slots, status, -131) {
                    ukeys[pos] = k[j];
                    uvals[pos] = (int32_t)(i0 + j);
                }
                ++pos;
            }
        }
        __syncthreads();
    }
}

// Route (b): table_vals[slot] = rank of the slot's key.
__global__ void k_ms_rank(const int32_t* __restrict__ slots, const uint32_t* ctl, uint32_t* vals,
                          int32_t* status) {
    if (ctl[kCtlRoute] == 0u) return;
    const int64_t K = ctl[kCtlCompact];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K;
         i += (int64_t)gridDim.x * blockDim.x)
        MSC_GUARD((uint32_t)slots[i] < ctl[2] + kPad, status, -132)
        vals[slots[i]] = (uint32_t)i;
}

// ms[v] = vals[ms[v]]: 8 vertices per thread, lane-consecutive, so the
// gathers of a warp fall on neighbouring slots.
constexpr int kLookupPer = 8;

__global__ void __launch_bounds__(kThreads) k_ms_lookup(int32_t* ms, int32_t n, const uint32_t* __restrict__ vals,
                                                        const uint32_t* ctl, int32_t* num_cells) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *num_cells = (int32_t)ctl[3];
    constexpr int64_t kChunk = (int64_t)kThreads * kLookupPer;
    for (int64_t c = blockIdx.x; c * kChunk < n; c += gridDim.x) {
        uint32_t s[kLookupPer];
#pragma unroll
        for (int j = 0; j < kLookupPer; ++j) {
            const int64_t v = c * kChunk + (int64_t)j * kThreads + threadIdx.x;
            s[j] = v < n ? (uint32_t)ms[v] : 0u;
        }
#pragma unroll
        for (int j = 0; j < kLookupPer; ++j) {
            const int64_t v = c * kChunk + (int64_t)j * kThreads + threadIdx.x;
            if (v < n) s[j] = vals[s[j]];
        }
#pragma unroll
        for (int j = 0; j < kLookupPer; ++j) {
            const int64_t v = c * kChunk + (int64_t)j * kThreads + threadIdx.x;
            if (v < n) ms[v] = (int32_t)s[j];
        }
    }
}

int grid_for(int64_t work, int per_sm = 8) {
    const int64_t want = ceil_div(std::max<int64_t>(work, 1), kThreads);
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)current_device().sms * per_sm));
}

int64_t cap_max_for(int64_t n) {
    int64_t cap = 64;
    while (cap < 2 * n) cap <<= 1;
    return std::min<int64_t>(cap, int64_t(1) << 31);
}

// chunks of slots of route (a): the whole table (capacity + pad)
int64_t chunks_for(int64_t cap_max) { return ceil_div(cap_max + kPad, kChunk); }

}  // namespace

int ms_pair_shift(int64_t n) { return ceil_log2(std::max<int64_t>(n, 1)); }

void size_ms_scratch(Sizer& s, int64_t n) {
    const int64_t cap = cap_max_for(n) + kPad;
    s.take<unsigned long long>(cap);
    s.take<uint32_t>(cap);
    for (int i = 0; i < 2; ++i) {
        s.take<unsigned long long>(std::max<int64_t>(n, 1) + kPad);
        s.take<int32_t>(std::max<int64_t>(n, 1) + kPad);
    }
    s.take<uint32_t>(64);
    s.take<uint32_t>(2 * chunks_for(cap_max_for(n)));
    size_sort_scratch(s, n + kPad);
}

MsScratch carve_ms_scratch(Carver& c, int64_t n) {
    MsScratch sc;
    sc.cap_max = cap_max_for(n);
    sc.table_keys = c.take<unsigned long long>(sc.cap_max + kPad);
    sc.table_vals = c.take<uint32_t>(sc.cap_max + kPad);
    for (int i = 0; i < 2; ++i) {
        sc.ukeys[i] = c.take<unsigned long long>(std::max<int64_t>(n, 1) + kPad);
        sc.uvals[i] = c.take<int32_t>(std::max<int64_t>(n, 1) + kPad);
    }
    sc.ctl = c.take<uint32_t>(64);
    sc.chunk = c.take<uint32_t>(2 * chunks_for(sc.cap_max));
    sc.sort = carve_sort_scratch(c, n + kPad);
    return sc;
}

int run_ms_id(const int32_t* asc, const int32_t* desc, int32_t n, int32_t* ms, int32_t* num_cells,
              const MsScratch& sc, bool counts_known, int32_t* status, cudaStream_t s,
              const unsigned long long** sorted_keys) {
    if (n <= 0) {
        MSC_TRY(cudaMemsetAsync(num_cells, 0, sizeof(int32_t), s));
        return MSC_OK;
    }
    const int sh = ms_pair_shift(n);
    if (!counts_known) MSC_TRY(cudaMemsetAsync(sc.ctl, 0, 4 * sizeof(uint32_t), s));
    if (!counts_known) {
        TraceScope ts_("msid.prepare", s);
        k_ms_prepare<<<grid_for(n), kThreads, 0, s>>>(asc, desc, n, sc.ctl, status);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("msid.setcap", s);
        k_ms_setcap<<<1, 1, 0, s>>>(sc.ctl, n, sc.cap_max, sh, sorted_keys ? 1 : 0);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("msid.clear", s);
        k_ms_clear<<<grid_for(sc.cap_max + kPad, 4), kThreads, 0, s>>>(sc.table_keys, sc.ctl);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("msid.insert", s);
        k_ms_insert<<<grid_for(ceil_div(n, kInsJ)), kThreads, 0, s>>>(asc, desc, n, sc.table_keys, sc.ctl, ms, status);
    }
    MSC_LAUNCHED();
    // route (a); each kernel returns at once on route (b).  The chunks cover
    // the largest table; those past the one in use are empty.
    const int64_t nchunks = chunks_for(sc.cap_max);
    uint32_t* occ = sc.chunk;
    uint32_t* occ_before = sc.chunk + nchunks;
    {
        TraceScope ts_("msid.occ", s);
        k_ms_occ<<<grid_for(nchunks * kThreads, 8), kThreads, 0, s>>>(sc.table_keys, occ, nchunks, sc.ctl);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("msid.chunk_scan", s);
        k_ms_chunk_scan<<<1, kScanThreads, 0, s>>>(occ, occ_before, nchunks, sc.ctl);
    }
    MSC_LAUNCHED();
    {
        static int configured_dev = -1;
        if (configured_dev != current_device().id) {
            MSC_TRY(cudaFuncSetAttribute(k_ms_chunk_rank, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRankSmem));
            configured_dev = current_device().id;
        }
        TraceScope ts_("msid.chunk_rank", s);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nchunks, (int64_t)current_device().sms * 2));
        k_ms_chunk_rank<<<grid, kRankThreads, kRankSmem, s>>>(sc.table_keys, sc.table_vals, occ_before, nchunks,
                                                               sc.ctl);
    }
    MSC_LAUNCHED();
    // route (b), run when the flag asks for it (every kernel returns at once otherwise)
    {
        TraceScope ts_("msid.compact", s);
        k_ms_compact<<<grid_for((sc.cap_max + kPad) / kCompactPer, 4), kThreads, 0, s>>>(
            sc.table_keys, sc.ctl, sc.ukeys[0], sc.uvals[0], status);
    }
    MSC_LAUNCHED();
    bool in_alt = false;
    int r = run_sort_u64(sc.ukeys[0], sc.uvals[0], sc.ukeys[1], sc.uvals[1],
                         reinterpret_cast<const int32_t*>(sc.ctl + kCtlCompact), n + kPad, 2 * sh, sc.sort, status,
                         s, &in_alt);
    if (r) return r;
    if (sorted_keys) *sorted_keys = in_alt ? sc.ukeys[1] : sc.ukeys[0];
    {
        TraceScope ts_("msid.rank", s);
        k_ms_rank<<<grid_for(n), kThreads, 0, s>>>(in_alt ? sc.uvals[1] : sc.uvals[0], sc.ctl, sc.table_vals, status);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("msid.lookup", s);
        k_ms_lookup<<<grid_for(n / kLookupPer + 1), kThreads, 0, s>>>(ms, n, sc.table_vals, sc.ctl, num_cells);
    }
    MSC_LAUNCHED();
    return MSC_OK;
}

}  // namespace msc
