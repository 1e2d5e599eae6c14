// Dense Morse-Smale cell ids.  A cell is the set of vertices sharing one
// (minimum, maximum) pair (section "Ascending and Descending
// Segmentation"); its id is the pair's rank among the distinct pairs in
// lexicographic order, minimum first.
//
// 1. A linear-probing hash table de-duplicates the pair keys
//    asc * n + desc.  Its capacity is a power of two >= 2 * min(n,
//    #minima * #maxima), chosen on the device, so smooth fields (few
//    extrema) use a table that lives in L2.  Lanes of a warp holding the
//    same key (neighbouring vertices usually share a cell) probe once.
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
    unsigned long long cap = 64;
    while (cap < 2 * bound) cap <<= 1;
    if ((long long)cap > cap_max) cap = (unsigned long long)cap_max;
    ctl[2] = (uint32_t)cap;  // cap_max <= 2^31
    ctl[3] = 0;
}

__global__ void k_ms_clear(unsigned long long* keys, const uint32_t* ctl) {
    const int64_t cap = ctl[2];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = kEmpty;
}

__device__ __forceinline__ uint32_t probe_insert(unsigned long long* keys, uint32_t cap,
                                                 unsigned long long key, int32_t* status) {
    uint32_t h = (uint32_t)mix64(key) & (cap - 1);
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
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v - lane < n; v += stride) {
        const bool valid = v < n;
        unsigned long long key = kEmpty - 1 - lane;  // distinct per idle lane
        if (valid) key = (unsigned long long)(uint32_t)asc[v] * (unsigned long long)n + (uint32_t)desc[v];
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(peers) - 1;
        uint32_t slot = 0;
        if (valid && lane == leader) slot = probe_insert(keys, cap, key, status);
        slot = __shfl_sync(0xffffffffu, slot, leader);
        if (valid) ms[v] = (int32_t)slot;
    }
}

// Compact occupied slots: (key, slot) pairs, block-aggregated appends.
__global__ void __launch_bounds__(kThreads) k_ms_compact(const unsigned long long* __restrict__ keys,
                                                         uint32_t* ctl, unsigned long long* ukeys,
                                                         int32_t* uvals, int32_t* status) {
    __shared__ uint32_t s_warp[kThreads / 32];
    __shared__ uint32_t s_base;
    const int64_t cap = ctl[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t nchunks = (cap + kThreads - 1) / kThreads;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int64_t i = c * kThreads + tid;
        const unsigned long long k = i < cap ? keys[i] : kEmpty;
        const bool keep = k != kEmpty;
        const uint32_t m = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_warp[warp] = __popc(m);
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
        if (keep) {
            const uint32_t pos = s_base + s_warp[warp] + __popc(m & lanemask_lt());
            MSC_GUARD(pos < (uint32_t)cap, status, -131) {
                ukeys[pos] = k;
                uvals[pos] = (int32_t)i;
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

__global__ void k_ms_lookup(int32_t* ms, int32_t n, const uint32_t* __restrict__ vals,
                            const uint32_t* ctl, int32_t* num_cells) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) *num_cells = (int32_t)ctl[3];
    const int64_t nq = n / 4;
    int4* m4 = reinterpret_cast<int4*>(ms);
    if (((uintptr_t)ms & 15) == 0) {
        for (int64_t q = t; q < nq; q += stride) {
            int4 s = m4[q];
            s.x = (int32_t)vals[(uint32_t)s.x];
            s.y = (int32_t)vals[(uint32_t)s.y];
            s.z = (int32_t)vals[(uint32_t)s.z];
            s.w = (int32_t)vals[(uint32_t)s.w];
            m4[q] = s;
        }
        for (int64_t v = nq * 4 + t; v < n; v += stride) ms[v] = (int32_t)vals[(uint32_t)ms[v]];
    } else {
        for (int64_t v = t; v < n; v += stride) ms[v] = (int32_t)vals[(uint32_t)ms[v]];
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
              const MsScratch& sc, bool counts_known, int32_t* status, cudaStream_t s) {
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
        k_ms_compact<<<grid_for(sc.cap_max, 4), kThreads, 0, s>>>(sc.table_keys, sc.ctl, sc.ukeys[0], sc.uvals[0], status);
    }
    MSC_LAUNCHED();
    const int key_bits = ceil_log2((int64_t)n * (int64_t)n);
    bool in_alt = false;
    int r = run_sort_u64(sc.ukeys[0], sc.uvals[0], sc.ukeys[1], sc.uvals[1],
                         reinterpret_cast<const int32_t*>(sc.ctl + 3), n, key_bits, sc.sort, status, s,
                         &in_alt);
    if (r) return r;
    {
        TraceScope ts_("msid.rank", s);
        k_ms_rank<<<grid_for(n), kThreads, 0, s>>>(in_alt ? sc.uvals[1] : sc.uvals[0], sc.ctl, sc.table_vals, status);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("msid.lookup", s);
        k_ms_lookup<<<grid_for(n / 4 + 1), kThreads, 0, s>>>(ms, n, sc.table_vals, sc.ctl, num_cells);
    }
    MSC_LAUNCHED();
    return MSC_OK;
}

}  // namespace msc
