// Adjacency of labelled regions on a regular grid: the distinct pairs
// (a, b), a < b, of non-negative labels that meet across an edge of the
// implicit triangulation (14-neighbour link) or of the face grid (6).
// Applied to the minimum / maximum labels or the cell ids of a
// segmentation, the pairs are the connectivity preview of the Morse-Smale
// complex that the paper's related work builds from the segmentations, and
// the edges of an extremum graph (Conclusion).
//
// 1. k_adj_emit: one CTA per 32 x 8 x 4 tile stages the tile's labels and
//    its +1 halo in shared memory, follows every positive link offset of
//    every vertex (each edge once), and de-duplicates the pair keys
//    (lo << shift) | hi in a shared hash set: a region boundary crosses a
//    tile in many edges but few pairs.  The distinct keys of the tile are
//    appended to a global buffer with one atomic per tile; a key that finds
//    no free slot within a few probes is appended on its own.
// 2. The appended keys are radix-sorted (keys only).
// 3. k_adj_heads / k_adj_scan / k_adj_write keep the first key of every run
//    of equal keys and split it into (a, b).
#include <cuda_runtime.h>

#include <algorithm>

#include "adjacency.cuh"

namespace msc {
namespace {

constexpr int kThreads = 256;
constexpr int kTX = 32, kTY = 8, kTZ = 4;  // warp w owns row y = w of each z plane
constexpr int kHX = kTX + 1, kHY = kTY + 1, kHZ = kTZ + 1;  // with the +1 halo
constexpr int kSetSlots = 4096;  // shared hash set: 32 KiB of keys
constexpr int kProbes = 32;
constexpr unsigned long long kNoKey = ~0ull;
constexpr int kChunk = 4096;  // sorted keys per block in the unique pass
constexpr int kPer = kChunk / kThreads;

// positive link offsets: the three face directions, then the four
// diagonals of the Freudenthal split (x, y, z)
__constant__ int8_t c_off[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};

__device__ __forceinline__ unsigned long long mix64(unsigned long long k) {
    // 64-bit finaliser of MurmurHash3
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

struct EmitArgs {
    const int32_t* label;
    int32_t nx, ny, nz;
    int half;     // positive offsets followed: 3 (conn 6) or 7 (conn 14)
    int32_t bound;
    int shift;
    unsigned long long* out;
    int32_t* count;
    int64_t cap;  // entries of `out`
    int32_t* status;
};

__device__ __forceinline__ void append_global(const EmitArgs& a, unsigned long long key) {
    const uint32_t pos = atomicAdd(reinterpret_cast<uint32_t*>(a.count), 1u);
    if ((int64_t)pos < a.cap)
        a.out[pos] = key;
    else
        record_error(a.status, MSC_ERR_INTERNAL);  // more keys than edges: impossible
}

__global__ void __launch_bounds__(kThreads) k_adj_emit(const EmitArgs a) {
    __shared__ unsigned long long s_set[kSetSlots];
    __shared__ uint16_t s_used[kSetSlots];
    __shared__ int32_t s_lab[kHZ][kHY][kHX];
    __shared__ uint32_t s_nused, s_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < kSetSlots; i += kThreads) s_set[i] = kNoKey;
    if (tid == 0) s_nused = 0;
    const int64_t tx = (a.nx + kTX - 1) / kTX, ty = (a.ny + kTY - 1) / kTY, tz = (a.nz + kTZ - 1) / kTZ;
    const int64_t ntiles = tx * ty * tz;
    const int64_t plane = (int64_t)a.nx * a.ny;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t bx = t % tx, by = (t / tx) % ty, bz = t / (tx * ty);
        const int x0 = (int)(bx * kTX), y0 = (int)(by * kTY), z0 = (int)(bz * kTZ);
        // stage labels (tile + halo; -1 outside the grid); a label at or
        // above the bound is an argument error and counts as unlabelled
        for (int i = tid; i < kHX * kHY * kHZ; i += kThreads) {
            const int hx = i % kHX, hy = (i / kHX) % kHY, hz = i / (kHX * kHY);
            const int x = x0 + hx, y = y0 + hy, z = z0 + hz;
            int32_t l = -1;
            if (x < a.nx && y < a.ny && z < a.nz) {
                l = __ldg(a.label + x + (int64_t)a.nx * y + plane * z);
                if (l >= a.bound) {
                    record_error(a.status, MSC_ERR_ARG);
                    l = -1;
                }
            }
            s_lab[hz][hy][hx] = l;
        }
        __syncthreads();
        for (int z = 0; z < kTZ; ++z) {
            // halo vertices (x = 32, y = 8 or z = 4 in the tile) are only
            // ever edge ends: s_lab holds -1 past the grid
            const int32_t l = s_lab[z][warp][lane];
            for (int k = 0; k < a.half; ++k) {
                const int32_t m = s_lab[z + c_off[k][2]][warp + c_off[k][1]][lane + c_off[k][0]];
                unsigned long long key = kNoKey;
                if (l >= 0 && m >= 0 && l != m) {
                    const uint32_t lo = (uint32_t)min(l, m), hi = (uint32_t)max(l, m);
                    key = ((unsigned long long)lo << a.shift) | hi;
                }
                // a boundary usually crosses neighbouring lanes with the same pair
                const unsigned long long prev = __shfl_up_sync(0xffffffffu, key, 1);
                if (key == kNoKey || (lane > 0 && prev == key)) continue;
                uint32_t h = (uint32_t)mix64(key) & (kSetSlots - 1);
                bool placed = false;
                for (int p = 0; p < kProbes; ++p) {
                    const unsigned long long cur = s_set[h];
                    if (cur == key) {
                        placed = true;
                        break;
                    }
                    if (cur == kNoKey) {
                        const unsigned long long old = atomicCAS(&s_set[h], kNoKey, key);
                        if (old == kNoKey) {
                            s_used[atomicAdd(&s_nused, 1u)] = (uint16_t)h;
                            placed = true;
                            break;
                        }
                        if (old == key) {
                            placed = true;
                            break;
                        }
                    }
                    h = (h + 1) & (kSetSlots - 1);
                }
                if (!placed) append_global(a, key);
            }
        }
        __syncthreads();
        const uint32_t nu = s_nused;
        if (tid == 0 && nu) s_base = atomicAdd(reinterpret_cast<uint32_t*>(a.count), nu);
        __syncthreads();
        for (uint32_t i = tid; i < nu; i += kThreads) {
            const uint32_t slot = s_used[i];
            const uint32_t pos = s_base + i;
            if ((int64_t)pos < a.cap)
                a.out[pos] = s_set[slot];
            else
                record_error(a.status, MSC_ERR_INTERNAL);
            s_set[slot] = kNoKey;  // cleared for the next tile
        }
        __syncthreads();
        if (tid == 0) s_nused = 0;
        // the next tile's staging loop writes s_lab only after this barrier
        // and s_nused is read after the staging barrier
    }
}

__device__ __forceinline__ int64_t clamp_count(const int32_t* d_count, int64_t cap) {
    return min((int64_t)max(*d_count, 0), cap);
}

// Heads (first key of each run of equal keys) per chunk of kChunk keys.
__global__ void __launch_bounds__(kThreads) k_adj_heads(const unsigned long long* __restrict__ keys,
                                                        const int32_t* d_count, int64_t cap,
                                                        uint32_t* chunk_heads) {
    __shared__ uint32_t s_w[kThreads / 32];
    const int64_t m = clamp_count(d_count, cap);
    const int64_t nchunks = (m + kChunk - 1) / kChunk;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        uint32_t cnt = 0;
        for (int j = 0; j < kPer; ++j) {
            const int64_t i = c * kChunk + (int64_t)j * kThreads + threadIdx.x;
            if (i < m) cnt += i == 0 || keys[i] != keys[i - 1];
        }
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < kThreads / 32; ++w) t += s_w[w];
            chunk_heads[c] = t;
        }
        __syncthreads();
    }
}

// Exclusive scan of the chunk counts in place (one block); the total is the
// number of distinct pairs.
__global__ void __launch_bounds__(1024) k_adj_scan(uint32_t* chunk_heads, const int32_t* d_count, int64_t cap,
                                                   int64_t* num_pairs) {
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_carry;
    const int64_t m = clamp_count(d_count, cap);
    const int64_t nchunks = (m + kChunk - 1) / kChunk;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nchunks; base += 1024) {
        const int64_t i = base + tid;
        const uint32_t v = i < nchunks ? chunk_heads[i] : 0u;
        uint32_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = s_w[lane];
            uint32_t wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            s_w[lane] = wi - w;
        }
        __syncthreads();
        const uint32_t carry = s_carry;
        if (i < nchunks) chunk_heads[i] = carry + s_w[warp] + incl - v;
        __syncthreads();
        if (tid == 1023) s_carry = carry + s_w[warp] + incl;
        __syncthreads();
    }
    if (tid == 0) *num_pairs = (int64_t)s_carry;
}

// Writes the heads of each chunk at their ranks: a = key >> shift,
// b = key & (2^shift - 1); ranks at or beyond `out_cap` are dropped.
__global__ void __launch_bounds__(kThreads) k_adj_write(const unsigned long long* __restrict__ keys,
                                                        const int32_t* d_count, int64_t cap,
                                                        const uint32_t* __restrict__ chunk_base, int shift,
                                                        int32_t* out_a, int32_t* out_b, int64_t out_cap) {
    __shared__ uint32_t s_w[kThreads / 32];
    const int64_t m = clamp_count(d_count, cap);
    const int64_t nchunks = (m + kChunk - 1) / kChunk;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long mask = (1ull << shift) - 1;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        // thread tid takes the kPer consecutive keys [c*kChunk + tid*kPer, ...)
        const int64_t i0 = c * kChunk + (int64_t)tid * kPer;
        uint32_t heads = 0;  // bit j: key i0 + j starts a run
        for (int j = 0; j < kPer; ++j) {
            const int64_t i = i0 + j;
            if (i < m && (i == 0 || keys[i] != keys[i - 1])) heads |= 1u << j;
        }
        const uint32_t cnt = __popc(heads);
        uint32_t incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += s_w[w];
        int64_t r = (int64_t)chunk_base[c] + before + incl - cnt;
        for (int j = 0; j < kPer; ++j) {
            if (heads >> j & 1u) {
                if (r < out_cap) {
                    const unsigned long long k = keys[i0 + j];
                    out_a[r] = (int32_t)(k >> shift);
                    out_b[r] = (int32_t)(k & mask);
                }
                ++r;
            }
        }
        __syncthreads();
    }
}

int64_t emit_capacity(int64_t n) { return 7 * std::max<int64_t>(n, 1); }

int blocks_for(int64_t work, int per_sm) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(std::max<int64_t>(work, 1), (int64_t)current_device().sms * per_sm));
}

}  // namespace

bool adjacency_size_ok(int64_t n) { return n >= 0 && emit_capacity(n) <= (int64_t)INT32_MAX; }

void size_adjacency_scratch(Sizer& s, int64_t n) {
    const int64_t cap = emit_capacity(n);
    s.take<int32_t>(64);
    s.take<unsigned long long>(cap);
    s.take<unsigned long long>(cap);
    s.take<uint32_t>(ceil_div(cap, kChunk) + 1);
    size_sort_scratch(s, cap);
}

int run_adjacency_grid(const int32_t* label, msc_grid g, int conn, int32_t bound, int32_t* out_a,
                       int32_t* out_b, int64_t out_cap, int64_t* num_pairs, void* ws, size_t ws_bytes,
                       int32_t* status, cudaStream_t s) {
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    const int64_t cap = emit_capacity(n);
    Carver c(ws, ws_bytes);
    int32_t* ctl = c.take<int32_t>(64);
    unsigned long long* k0 = c.take<unsigned long long>(cap);
    unsigned long long* k1 = c.take<unsigned long long>(cap);
    uint32_t* chunk = c.take<uint32_t>(ceil_div(cap, kChunk) + 1);
    SortScratch sc = carve_sort_scratch(c, cap);
    if (!c.ok()) return MSC_ERR_WS;
    MSC_TRY(cudaMemsetAsync(ctl, 0, 64 * sizeof(int32_t), s));
    const int shift = ceil_log2(bound);
    EmitArgs ea{label, g.nx, g.ny, g.nz, conn == 6 ? 3 : 7, bound, shift, k0, ctl, cap, status};
    const int64_t tiles = ceil_div(g.nx, kTX) * ceil_div(g.ny, kTY) * ceil_div(g.nz, kTZ);
    {
        TraceScope ts_("adjacency.emit", s);
        k_adj_emit<<<blocks_for(tiles, 4), kThreads, 0, s>>>(ea);
    }
    MSC_LAUNCHED();
    bool in_alt = false;
    int r = run_sort_u64(k0, nullptr, k1, nullptr, ctl, cap, 2 * shift, sc, status, s, &in_alt,
                         "adjacency.sort_hist", "adjacency.sort_pass");
    if (r) return r;
    const unsigned long long* sorted = in_alt ? k1 : k0;
    const int grid = blocks_for(ceil_div(cap, kChunk), 8);
    {
        TraceScope ts_("adjacency.heads", s);
        k_adj_heads<<<grid, kThreads, 0, s>>>(sorted, ctl, cap, chunk);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("adjacency.scan", s);
        k_adj_scan<<<1, 1024, 0, s>>>(chunk, ctl, cap, num_pairs);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("adjacency.write", s);
        k_adj_write<<<grid, kThreads, 0, s>>>(sorted, ctl, cap, chunk, shift, out_a, out_b, out_cap);
    }
    MSC_LAUNCHED();
    return MSC_OK;
}

}  // namespace msc
