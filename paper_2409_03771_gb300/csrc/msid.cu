// Dense Morse-Smale cell ids.  A cell is the set of vertices sharing one
// (minimum, maximum) pair (section "Ascending and Descending
// Segmentation"); its id is the pair's rank among the distinct pairs in
// lexicographic order, minimum first.
//
// 1. A linear-probing hash table de-duplicates the pair keys
//    asc * n + desc.  Its capacity is a power of two >= 2 * #minima *
//    #maxima, or >= n when that is more than n (there are at most n
//    distinct pairs), chosen on the device, so smooth fields (few extrema)
//    use a table that lives in L2.  Within a warp, a run of
//    consecutive vertices with the same key (neighbours usually share a
//    cell) probes once.
//    Each vertex keeps its slot in `ms` for now.
// 2. The occupied slots are compacted and radix-sorted by key.
// 3. table_vals[slot] = rank; ms[v] = table_vals[ms[v]].
#include <cuda_runtime.h>

#include <algorithm>

#include "msid.cuh"

namespace msc {
namespace {

constexpr int kThreads = 256;
constexpr unsigned long long kEmpty = ~0ull;
constexpr uint32_t kSpread = 64;  // random spread of a pair around its home slot
constexpr uint32_t kCacheResidentSlots = 1u << 20;  // 8 MiB of keys: plain random hashing

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

__global__ void k_ms_setcap(uint32_t* ctl, int64_t n, int64_t cap_max) {
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
}

__global__ void k_ms_clear(unsigned long long* keys, const uint32_t* ctl) {
    const int64_t cap = ctl[2];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = kEmpty;
}

// Home slot of a pair in a table too big for the cache: proportional to
// its minimum's id plus a small random spread.  The minimum of a vertex lies near the vertex, so the
// vertices of a warp, and the warps in flight, probe a narrow band of the
// table (L2 hits instead of random DRAM sectors), and the slots of sorted
// pairs are nearly increasing, which keeps the rank writes and the final
// lookups almost sequential too.
__device__ __forceinline__ uint32_t home_slot(uint32_t asc, unsigned long long key, uint32_t cap,
                                              unsigned long long f) {
    if (cap <= kCacheResidentSlots) return (uint32_t)mix64(key) & (cap - 1);  // fits in cache: spread
    // asc * cap / n by a fixed-point multiply (f = cap * 2^32 / n), no division
    const uint32_t base = (uint32_t)((unsigned long long)asc * (f >> 32) + (((unsigned long long)asc * (uint32_t)f) >> 32));
    return (base + (uint32_t)(mix64(key) & (kSpread - 1))) & (cap - 1);
}

__device__ __forceinline__ uint32_t probe_insert(unsigned long long* keys, uint32_t cap,
                                                 unsigned long long key, uint32_t home, int32_t* status) {
    uint32_t h = home;
    for (uint32_t i = 0; i < cap; ++i) {
        const unsigned long long k = keys[h];
        if (k == key) return h;
        if (k == kEmpty) {
            const unsigned long long old = atomicCAS(&keys[h], kEmpty, key);
            if (old == kEmpty || old == key) return h;
        }
        h = (h + 1) & (cap - 1);
    }
    record_error(status, MSC_ERR_INTERNAL);  // table full: impossible at load <= 1/2
    return 0;
}

__global__ void __launch_bounds__(kThreads) k_ms_insert(const int32_t* __restrict__ asc,
                                                        const int32_t* __restrict__ desc, int32_t n,
                                                        unsigned long long* keys, const uint32_t* ctl,
                                                        int32_t* ms, int32_t* status) {
    const uint32_t cap = ctl[2];
    const unsigned long long f = (unsigned long long)ctl[9] | ((unsigned long long)ctl[10] << 32);
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v - lane < n; v += stride) {
        const bool valid = v < n;
        unsigned long long key = kEmpty - 1 - lane;  // distinct per idle lane
        if (valid) key = (unsigned long long)(uint32_t)asc[v] * (unsigned long long)n + (uint32_t)desc[v];
        // neighbouring vertices usually share their cell: only the first lane
        // of each run of equal keys probes, the others take its slot
        const unsigned long long prev = __shfl_up_sync(0xffffffffu, key, 1);
        const bool head = lane == 0 || key != prev;
        const uint32_t heads = __ballot_sync(0xffffffffu, head);
        const int my_head = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
        uint32_t slot = 0;
        if (valid && head) slot = probe_insert(keys, cap, key, home_slot((uint32_t)asc[v], key, cap, f), status);
        slot = __shfl_sync(0xffffffffu, slot, my_head);
        if (valid) ms[v] = (int32_t)slot;
    }
}

// Compact occupied slots into (key, slot) pairs: each thread scans 8
// consecutive slots with 16-byte loads; one atomic append per block chunk.
constexpr int kCompactPer = 8;

__global__ void __launch_bounds__(kThreads) k_ms_compact(const unsigned long long* __restrict__ keys,
                                                         uint32_t* ctl, unsigned long long* ukeys,
                                                         int32_t* uvals, int32_t* status) {
    __shared__ uint32_t s_warp[kThreads / 32];
    __shared__ uint32_t s_base;
    const int64_t cap = ctl[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int64_t kChunkSlots = (int64_t)kThreads * kCompactPer;
    const int64_t nchunks = (cap + kChunkSlots - 1) / kChunkSlots;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int64_t i0 = c * kChunkSlots + (int64_t)tid * kCompactPer;
        unsigned long long k[kCompactPer];
        if (i0 + kCompactPer <= cap) {  // cap is a power of two >= 64: whole groups
#pragma unroll
            for (int q = 0; q < kCompactPer / 2; ++q) {
                const ulonglong2 v = reinterpret_cast<const ulonglong2*>(keys + i0)[q];
                k[2 * q] = v.x;
                k[2 * q + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kCompactPer; ++j) k[j] = i0 + j < cap ? keys[i0 + j] : kEmpty;
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
            s_base = run ? atomicAdd(&ctl[3], run) : 0u;
        }
        __syncthreads();
        uint32_t pos = s_base + s_warp[warp] + incl - cnt;
#pragma unroll
        for (int j = 0; j < kCompactPer; ++j) {
            if (k[j] != kEmpty) {
                MSC_GUARD(pos < (uint32_t)cap, status, -131) {
                    ukeys[pos] = k[j];
                    uvals[pos] = (int32_t)(i0 + j);
                }
                ++pos;
            }
        }
        __syncthreads();
    }
}

__global__ void k_ms_rank(const int32_t* __restrict__ slots, const uint32_t* ctl, uint32_t* vals,
                          int32_t* status) {
    const int64_t K = ctl[3];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K;
         i += (int64_t)gridDim.x * blockDim.x)
        MSC_GUARD((uint32_t)slots[i] < ctl[2], status, -132)
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

}  // namespace

void size_ms_scratch(Sizer& s, int64_t n) {
    const int64_t cap = cap_max_for(n);
    s.take<unsigned long long>(cap);
    s.take<uint32_t>(cap);
    for (int i = 0; i < 2; ++i) {
        s.take<unsigned long long>(std::max<int64_t>(n, 1));
        s.take<int32_t>(std::max<int64_t>(n, 1));
    }
    s.take<uint32_t>(64);
    size_sort_scratch(s, n);
}

MsScratch carve_ms_scratch(Carver& c, int64_t n) {
    MsScratch sc;
    sc.cap_max = cap_max_for(n);
    sc.table_keys = c.take<unsigned long long>(sc.cap_max);
    sc.table_vals = c.take<uint32_t>(sc.cap_max);
    for (int i = 0; i < 2; ++i) {
        sc.ukeys[i] = c.take<unsigned long long>(std::max<int64_t>(n, 1));
        sc.uvals[i] = c.take<int32_t>(std::max<int64_t>(n, 1));
    }
    sc.ctl = c.take<uint32_t>(64);
    sc.sort = carve_sort_scratch(c, n);
    return sc;
}

int run_ms_id(const int32_t* asc, const int32_t* desc, int32_t n, int32_t* ms, int32_t* num_cells,
              const MsScratch& sc, bool counts_known, int32_t* status, cudaStream_t s,
              const unsigned long long** sorted_keys) {
    if (n <= 0) {
        MSC_TRY(cudaMemsetAsync(num_cells, 0, sizeof(int32_t), s));
        return MSC_OK;
    }
    if (!counts_known) {
        MSC_TRY(cudaMemsetAsync(sc.ctl, 0, 4 * sizeof(uint32_t), s));
        {
            TraceScope ts_("msid.prepare", s);
            k_ms_prepare<<<grid_for(n), kThreads, 0, s>>>(asc, desc, n, sc.ctl, status);
        }
        MSC_LAUNCHED();
    }
    {
        TraceScope ts_("msid.setcap", s);
        k_ms_setcap<<<1, 1, 0, s>>>(sc.ctl, n, sc.cap_max);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("msid.clear", s);
        k_ms_clear<<<grid_for(sc.cap_max, 4), kThreads, 0, s>>>(sc.table_keys, sc.ctl);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("msid.insert", s);
        k_ms_insert<<<grid_for(n), kThreads, 0, s>>>(asc, desc, n, sc.table_keys, sc.ctl, ms, status);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("msid.compact", s);
        k_ms_compact<<<grid_for(sc.cap_max / kCompactPer, 4), kThreads, 0, s>>>(sc.table_keys, sc.ctl, sc.ukeys[0], sc.uvals[0], status);
    }
    MSC_LAUNCHED();
    const int key_bits = ceil_log2((int64_t)n * (int64_t)n);
    bool in_alt = false;
    int r = run_sort_u64(sc.ukeys[0], sc.uvals[0], sc.ukeys[1], sc.uvals[1],
                         reinterpret_cast<const int32_t*>(sc.ctl + 3), n, key_bits, sc.sort, status, s,
                         &in_alt);
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
