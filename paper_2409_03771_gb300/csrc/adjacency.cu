// Adjacency of labelled regions on a regular grid: the distinct pairs
// (a, b), a < b, of non-negative labels that meet across an edge of the
// implicit triangulation (14-neighbour link) or of the face grid (6).
// Applied to the minimum / maximum labels or the cell ids of a
// segmentation, the pairs are the connectivity preview of the Morse-Smale
// complex that the paper's related work builds from the segmentations, and
// the edges of an extremum graph (Conclusion).
//
// 1. k_adj_emit: warps march rows of 32 vertices through z with two planes
//    of labels in registers, follow every positive link offset of every
//    vertex (each edge once), and de-duplicate the pair keys
//    (lo << shift) | hi in a hash set per CTA in shared memory: a region
//    boundary crosses a tile in many edges but few pairs.  The set's keys
//    are appended to a global buffer with one atomic per flush; a key that
//    finds no free slot within a few probes is appended on its own.
// 2. The appended keys are radix-sorted (keys only).
// 3. k_adj_heads / k_adj_scan / k_adj_write keep the first key of every run
//    of equal keys and split it into (a, b).
#include <cuda_runtime.h>

#include <algorithm>

#include "adjacency.cuh"

namespace msc {
namespace {

constexpr int kThreads = 256;
constexpr int kTX = 32, kTY = 8;  // a tile: 32 x 8 rows, warp w owns row y0 + w
constexpr int kZR = 32;           // planes a tile marches through
constexpr int kAhead = 2;         // planes loaded ahead of their use
constexpr int kCheckDense = 2;    // planes between checks of the set's fill where boundaries are dense
constexpr int kCheckSparse = 8;   // ... and where the set stayed nearly empty
constexpr int kSetBits = 12;
constexpr int kSetSlots = 1 << kSetBits;  // shared hash set: 32 KiB of keys
constexpr int kProbes = 16;
constexpr unsigned long long kNoKey = ~0ull;
constexpr int kChunk = 4096;  // sorted keys per block in the unique pass
constexpr int kPer = kChunk / kThreads;

// Positive link offsets k = 0..6: the three face directions (1,0,0),
// (0,1,0), (0,0,1), then the four diagonals of the Freudenthal split
// (1,1,0), (1,0,1), (0,1,1), (1,1,1); conn 6 follows the first three.

struct EmitArgs {
    const int32_t* label;
    int32_t nx, ny, nz;
    int32_t bound;
    int shift;
    unsigned long long* out;
    int32_t* count;
    int64_t cap;  // entries of `out`
    int32_t* status;
    // saddles (extremum graph): the vertex order, +1 for maximum labels or
    // -1 for minimum labels, and the crossing vertex of each emitted key
    const int32_t* order;
    int sense;
    int32_t* out_w;
};

// A crossing vertex w at order level l as a value whose maximum is the
// saddle: (l << 32 | w) for maxima (highest crossing), its complement for
// minima (lowest crossing).  0 is below every value.
__device__ __forceinline__ unsigned long long crossing_val(int sense, int32_t level, int32_t w) {
    const unsigned long long p = (unsigned long long)(uint32_t)level << 32 | (uint32_t)w;
    return sense > 0 ? p : ~p;
}

__device__ __forceinline__ int32_t crossing_vertex(int sense, unsigned long long val) {
    return (int32_t)(uint32_t)(sense > 0 ? val : ~val);
}

__device__ __forceinline__ void append_global(const EmitArgs& a, unsigned long long key, unsigned long long val) {
    const uint32_t pos = atomicAdd(reinterpret_cast<uint32_t*>(a.count), 1u);
    if ((int64_t)pos < a.cap) {
        a.out[pos] = key;
        if (a.out_w) a.out_w[pos] = crossing_vertex(a.sense, val);
    } else {
        record_error(a.status, MSC_ERR_INTERNAL);  // more keys than edges: impossible
    }
}

// Key of the pair of labels c and m (both non-negative): (lo << shift) | hi.
__device__ __forceinline__ unsigned long long pair_key_of(int shift, int32_t c, int32_t m) {
    const uint32_t lo = (uint32_t)min(c, m), hi = (uint32_t)max(c, m);
    return ((unsigned long long)lo << shift) | hi;
}

// Key of the pair of labels c and m, or kNoKey when m < 0.
__device__ __forceinline__ unsigned long long pair_key(const EmitArgs& a, int32_t c, int32_t m) {
    if (m < 0) return kNoKey;
    return pair_key_of(a.shift, c, m);
}

// Home slot of a key in the shared set: a multiplicative hash of both
// halves (the set is rebuilt per tile, so a cheap hash suffices).
__device__ __forceinline__ uint32_t set_home(unsigned long long key) {
    const uint32_t h = (uint32_t)key * 0x9E3779B1u ^ (uint32_t)(key >> 32) * 0x85EBCA77u;
    return h >> (32 - kSetBits);
}

// Inserts `key` (kNoKey = nothing) into the tile's shared set; with
// SADDLE, also raises the key's value to `val`.  Called by the whole warp;
// records new slots in s_used with one shared atomic per warp.
template <bool SADDLE>
__device__ __forceinline__ void set_insert(const EmitArgs& a, unsigned long long key, unsigned long long val,
                                           unsigned long long* s_set, unsigned long long* s_val, uint16_t* s_used,
                                           uint32_t* s_nused, int lane) {
    if constexpr (SADDLE) {
        // the first lane of a run of equal keys carries the run's maximum
        // (lanes further on with the same key only add to the same maximum)
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long k2 = __shfl_down_sync(0xffffffffu, key, o);
            const unsigned long long v2 = __shfl_down_sync(0xffffffffu, val, o);
            if (lane + o < 32 && k2 == key && v2 > val) val = v2;
        }
    }
    // a boundary usually crosses neighbouring lanes with the same pair
    const unsigned long long prev = __shfl_up_sync(0xffffffffu, key, 1);
    int new_slot = -1;
    if (key != kNoKey && !(lane > 0 && prev == key)) {
        uint32_t h = set_home(key);
        int slot = -1;
        for (int p = 0; p < kProbes; ++p) {
            const unsigned long long cur = s_set[h];
            if (cur == key) {
                slot = (int)h;
                break;
            }
            if (cur == kNoKey) {
                const unsigned long long old = atomicCAS(&s_set[h], kNoKey, key);
                if (old == kNoKey) new_slot = (int)h;
                if (old == kNoKey || old == key) {
                    slot = (int)h;
                    break;
                }
            }
            h = (h + 1) & (kSetSlots - 1);
        }
        if (slot < 0)
            append_global(a, key, val);
        else if constexpr (SADDLE)
            atomicMax(&s_val[slot], val);
    }
    const uint32_t fresh = __ballot_sync(0xffffffffu, new_slot >= 0);
    if (fresh) {
        const int leader = __ffs(fresh) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(s_nused, (uint32_t)__popc(fresh));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (new_slot >= 0) s_used[base + __popc(fresh & lanemask_lt())] = (uint16_t)new_slot;
    }
}

// Labels of plane z of rows y and y + 1 of a tile (lanes hold x0 + lane)
// and the labels at x0 + 32 of both rows (every lane the same); -1 outside
// the grid.
struct Plane {
    int32_t c, u;  // (x, y, z), (x, y + 1, z)
    int32_t e, f;  // (x0 + 32, y, z), (x0 + 32, y + 1, z)
};

// Plane z of the two rows; -1 past the grid.  Only the row's own label (c)
// is checked against the bound: every vertex is the own label of exactly
// one (warp, lane, plane), so each label is checked once; an unchecked
// label past the bound can only make a key of a call that reports
// MSC_ERR_ARG.
__device__ __forceinline__ Plane load_plane(const EmitArgs& a, int x, int y, int xe, int z) {
    Plane p;
    const bool in_z = z < a.nz;
    const int32_t* r = a.label + (int64_t)a.nx * y + (int64_t)a.nx * a.ny * z;
    p.c = in_z && y < a.ny && x < a.nx ? __ldg(r + x) : -1;
    p.u = in_z && y + 1 < a.ny && x < a.nx ? __ldg(r + a.nx + x) : -1;
    p.e = in_z && y < a.ny && xe < a.nx ? __ldg(r + xe) : -1;
    p.f = in_z && y + 1 < a.ny && xe < a.nx ? __ldg(r + a.nx + xe) : -1;
    return p;
}

__device__ __forceinline__ int32_t checked(const EmitArgs& a, int32_t l) {
    if (l >= a.bound) {
        record_error(a.status, MSC_ERR_ARG);
        return -1;
    }
    return l;
}

// Called by the whole CTA: when `force` or the set holds a quarter of its
// slots, appends the set's keys (and crossing vertices) to the global
// buffer (one atomic) and empties the set.  Returns the planes to the next
// check (the same in every thread): few when the set is filling, more when
// it stayed nearly empty.
template <bool SADDLE>
__device__ __forceinline__ int flush_set(const EmitArgs& a, unsigned long long* s_set, unsigned long long* s_val,
                                         const uint16_t* s_used, uint32_t* s_nused, uint32_t* s_base, bool force) {
    const int tid = threadIdx.x;
    const bool go = __syncthreads_or(force || (tid == 0 && *s_nused >= kSetSlots / 4));
    const uint32_t nu = *s_nused;  // every insert is behind the barrier above
    const int next = nu < kSetSlots / 16 ? kCheckSparse : kCheckDense;
    if (!go) {
        __syncthreads();  // nobody may insert before every thread has read s_nused
        return next;
    }
    __syncthreads();
    if (tid == 0) {
        *s_base = nu ? atomicAdd(reinterpret_cast<uint32_t*>(a.count), nu) : 0u;
        *s_nused = 0;
    }
    __syncthreads();
    for (uint32_t i = tid; i < nu; i += kThreads) {
        const uint32_t slot = s_used[i];
        const uint32_t pos = *s_base + i;
        if ((int64_t)pos < a.cap) {
            a.out[pos] = s_set[slot];
            if constexpr (SADDLE) a.out_w[pos] = crossing_vertex(a.sense, s_val[slot]);
        } else {
            record_error(a.status, MSC_ERR_INTERNAL);
        }
        s_set[slot] = kNoKey;  // cleared for the keys that follow
        if constexpr (SADDLE) s_val[slot] = 0;
    }
    __syncthreads();
    return next;
}

// HALF: positive offsets followed, 3 (conn 6) or 7 (conn 14).  A CTA takes
// tiles of 32 x 8 rows by kZR planes; each warp marches its row through the
// planes with the labels of planes z and z + 1 in registers (neighbours in
// x from a lane shuffle, in y from the row above, which L2 serves to both
// warps that read it), so every label comes from DRAM about once and the
// only barriers are the set's fill checks.
// Offset k of the link as a vertex-id difference.
__device__ __forceinline__ int32_t offset_id(const EmitArgs& a, int k) {
    const int dx = k == 0 || k == 3 || k == 4 || k == 6, dy = k == 1 || k == 3 || k == 5 || k == 6;
    const int dz = k == 2 || k == 4 || k == 5 || k == 6;
    return dx + a.nx * (dy + a.ny * dz);
}

// Shared memory of k_adj_emit: the set's keys, (SADDLE) their values, the
// list of used slots.
template <bool SADDLE>
constexpr size_t emit_smem_bytes() {
    return (size_t)kSetSlots * (sizeof(unsigned long long) * (SADDLE ? 2 : 1) + sizeof(uint16_t));
}

template <int HALF, bool SADDLE>
__global__ void __launch_bounds__(kThreads) k_adj_emit(const EmitArgs a) {
    extern __shared__ __align__(16) unsigned long long emit_smem[];
    unsigned long long* s_set = emit_smem;
    unsigned long long* s_val = emit_smem + kSetSlots;  // SADDLE only
    uint16_t* s_used = reinterpret_cast<uint16_t*>(emit_smem + kSetSlots * (SADDLE ? 2 : 1));
    __shared__ uint32_t s_nused, s_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < kSetSlots; i += kThreads) {
        s_set[i] = kNoKey;
        if constexpr (SADDLE) s_val[i] = 0;
    }
    if (tid == 0) s_nused = 0;
    __syncthreads();
    // tile counts fit 32 bits: n < 2^31 vertices and every tile holds one
    const uint32_t tx = (a.nx + kTX - 1) / kTX, ty = (a.ny + kTY - 1) / kTY, tz = (a.nz + kZR - 1) / kZR;
    const uint32_t ntiles = tx * ty * tz;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint32_t txy = tx * ty, bz = t / txy, rem = t - bz * txy, by = rem / tx, bx = rem - by * tx;
        const int x0 = (int)bx * kTX, x = x0 + lane, xe = x0 + kTX, y = (int)by * kTY + warp;
        const int zs = (int)bz * kZR, ze = min(zs + kZR, a.nz);
        Plane cur = load_plane(a, x, y, xe, zs);
        Plane q[kAhead];  // planes z + 1 .. z + kAhead, loads in flight
#pragma unroll
        for (int i = 0; i < kAhead; ++i) q[i] = load_plane(a, x, y, xe, zs + 1 + i);
        cur.c = checked(a, cur.c);
        // (x + 1) neighbours of the current plane: the next lane's label,
        // or the label at x0 + 32 for the last lane
        int32_t xn = __shfl_down_sync(0xffffffffu, cur.c, 1), dn = __shfl_down_sync(0xffffffffu, cur.u, 1);
        if (lane == 31) {
            xn = cur.e;
            dn = cur.f;
        }
        int until = kCheckDense;  // planes to the next check of the set (uniform across the CTA)
#pragma unroll 1
        for (int z = zs; z < ze; ++z) {
            const Plane nx1 = {checked(a, q[0].c), q[0].u, q[0].e, q[0].f};
#pragma unroll
            for (int i = 0; i + 1 < kAhead; ++i) q[i] = q[i + 1];
            q[kAhead - 1] = load_plane(a, x, y, xe, z + 1 + kAhead);  // used kAhead planes from now
            int32_t xn1 = __shfl_down_sync(0xffffffffu, nx1.c, 1), dn1 = __shfl_down_sync(0xffffffffu, nx1.u, 1);
            if (lane == 31) {
                xn1 = nx1.e;
                dn1 = nx1.f;
            }
            const int32_t c0 = cur.c;
            // neighbours in the order of the offsets k = 0..6
            const int32_t nb[7] = {xn, cur.u, nx1.c, dn, xn1, nx1.u, dn1};
            uint32_t diff = 0;  // nonzero iff some neighbour's label differs from c0
#pragma unroll
            for (int k = 0; k < HALF; ++k) diff |= (uint32_t)(nb[k] ^ c0);
            // usually no lane of the row sits at a region boundary
            if (__any_sync(0xffffffffu, diff != 0 && c0 >= 0)) {
                // the distinct labels across this vertex's boundary edges:
                // one for a boundary between two regions, two where three
                // meet; offsets with a third or later one go to `extra`
                int32_t m0 = -1, m1 = -1;
                uint32_t extra = 0;
                // SADDLE: the best crossing towards m0 and m1 and per offset
                unsigned long long v0 = 0, v1 = 0, vk[7] = {0, 0, 0, 0, 0, 0, 0};
                if (c0 >= 0) {
                    const int32_t v = x + a.nx * (y + a.ny * z);
                    const int32_t ov = SADDLE ? __ldg(a.order + v) : 0;
#pragma unroll
                    for (int k = 0; k < HALF; ++k) {
                        const int32_t m = nb[k];
                        if (m >= 0 && m != c0) {
                            if constexpr (SADDLE) {
                                // the crossing vertex of edge (v, u): the lower end
                                // for maxima, the higher for minima
                                const int32_t u = v + offset_id(a, k), ou = __ldg(a.order + u);
                                const bool u_is = a.sense > 0 ? ou < ov : ou > ov;
                                vk[k] = crossing_val(a.sense, u_is ? ou : ov, u_is ? u : v);
                                if (m == m0) v0 = max(v0, vk[k]);
                                if (m == m1) v1 = max(v1, vk[k]);
                            }
                            if (m != m0 && m != m1) {
                                if (m0 < 0) {
                                    m0 = m;
                                    v0 = vk[k];
                                } else if (m1 < 0) {
                                    m1 = m;
                                    v1 = vk[k];
                                } else {
                                    extra |= 1u << k;
                                }
                            }
                        }
                    }
                }
                // rounds: m0, m1 when some lane has one, then one round per
                // offset in the warp's union of `extra`
                uint32_t wextra = __reduce_or_sync(0xffffffffu, extra);
                const bool two = __any_sync(0xffffffffu, m1 >= 0);
                for (int round = 0;; ++round) {
                    int32_t m;
                    unsigned long long val = 0;
                    if (round == 0) {
                        m = m0;
                        val = v0;
                    } else if (round == 1 && two) {
                        m = m1;
                        val = v1;
                    } else {
                        if (!wextra) break;
                        const int k = __ffs(wextra) - 1;
                        wextra &= wextra - 1;
                        m = extra >> k & 1u ? (k == 0 ? nb[0] : k == 1 ? nb[1] : k == 2 ? nb[2] : k == 3 ? nb[3]
                                               : k == 4 ? nb[4] : k == 5 ? nb[5] : nb[6])
                                            : -1;
                        if constexpr (SADDLE)
                            val = k == 0 ? vk[0] : k == 1 ? vk[1] : k == 2 ? vk[2] : k == 3 ? vk[3]
                                : k == 4 ? vk[4] : k == 5 ? vk[5] : vk[6];
                    }
                    set_insert<SADDLE>(a, pair_key(a, c0, m), val, s_set, s_val, s_used, &s_nused, lane);
                }
            }
            cur = nx1;
            xn = xn1;
            dn = dn1;
            // hand the set's keys to the global buffer when it is a quarter
            // full, checked often enough that the keys added before the next
            // check still find room (a full set only costs de-duplication:
            // keys that find no slot go out on their own), and at the
            // tile's end
            const bool last = z + 1 == ze;
            if (--until == 0 || last) until = flush_set<SADDLE>(a, s_set, s_val, s_used, &s_nused, &s_base, last);
        }
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
// b = key & (2^shift - 1); ranks at or beyond `out_cap` are dropped.  The
// chunk goes in kPer rounds of one key per thread (coalesced); a round's
// ranks come from a block-wide count of the heads before each thread.
// SADDLE: every key (head or not) also raises the value of its run's rank
// in `best` to its crossing vertex's value (a warp first combines the
// lanes of one run).
template <bool SADDLE>
__global__ void __launch_bounds__(kThreads) k_adj_write(const unsigned long long* __restrict__ keys,
                                                        const int32_t* d_count, int64_t cap,
                                                        const uint32_t* __restrict__ chunk_base, int shift,
                                                        int32_t* out_a, int32_t* out_b, int64_t out_cap,
                                                        const int32_t* __restrict__ cross, const int32_t* __restrict__ order,
                                                        int sense, unsigned long long* best) {
    __shared__ uint32_t s_w[kThreads / 32];
    const int64_t m = clamp_count(d_count, cap);
    const int64_t nchunks = (m + kChunk - 1) / kChunk;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long mask = (1ull << shift) - 1;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        int64_t run = chunk_base[c];
        for (int j = 0; j < kPer; ++j) {
            const int64_t i = c * kChunk + (int64_t)j * kThreads + tid;
            unsigned long long k = 0;
            bool head = false;
            if (i < m) {
                k = keys[i];
                head = i == 0 || k != keys[i - 1];
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, head);
            if (lane == 0) s_w[warp] = __popc(bal);
            __syncthreads();
            uint32_t before = __popc(bal & lanemask_lt()), total = 0;
            for (int w = 0; w < kThreads / 32; ++w) {
                const uint32_t c_w = s_w[w];
                before += w < warp ? c_w : 0u;
                total += c_w;
            }
            const int64_t r = run + before;
            if (head && r < out_cap) {
                out_a[r] = (int32_t)(k >> shift);
                out_b[r] = (int32_t)(k & mask);
            }
            if constexpr (SADDLE) {
                // rank of this key's run: the heads up to and including it, less one
                const int64_t rr = r + (head ? 0 : -1);
                unsigned long long val = 0;
                if (i < m) {
                    const int32_t w = cross[i];
                    val = crossing_val(sense, __ldg(order + w), w);
                }
                int64_t rk = i < m ? rr : -1 - lane;  // lanes past the end never match
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned long long v2 = __shfl_down_sync(0xffffffffu, val, o);
                    const int64_t r2 = __shfl_down_sync(0xffffffffu, rk, o);
                    if (lane + o < 32 && r2 == rk && v2 > val) val = v2;
                }
                const int64_t rprev = __shfl_up_sync(0xffffffffu, rk, 1);
                if (i < m && (lane == 0 || rprev != rk)) atomicMax(&best[rk], val);
            }
            run += total;
            __syncthreads();  // s_w is rewritten by the next round
        }
    }
}

// best[0 .. K) = 0 (K distinct pairs, read on the device).
__global__ void k_adj_zero(unsigned long long* best, const int64_t* num_pairs) {
    const int64_t k = *num_pairs;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
        best[i] = 0ull;
}

// saddle[r] = the crossing vertex held in best[r], r < min(K, out_cap).
__global__ void k_adj_saddle(const unsigned long long* __restrict__ best, const int64_t* num_pairs, int sense,
                             int32_t* saddle, int64_t out_cap) {
    const int64_t k = min(*num_pairs, out_cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
        saddle[i] = crossing_vertex(sense, best[i]);
}

int64_t emit_capacity(int64_t n) { return 7 * std::max<int64_t>(n, 1); }

int blocks_for(int64_t work, int per_sm) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(std::max<int64_t>(work, 1), (int64_t)current_device().sms * per_sm));
}

}  // namespace

bool adjacency_size_ok(int64_t n) { return n >= 0 && emit_capacity(n) <= (int64_t)INT32_MAX; }

namespace {

// Workspace of one adjacency call: `cap` emitted keys (and crossing
// vertices), the unique pass's chunk counts, the sort's scratch.
struct PairScratch {
    int32_t* ctl;
    unsigned long long* k0;
    unsigned long long* k1;
    int32_t* w0;
    int32_t* w1;
    uint32_t* chunk;
    SortScratch sort;
    int64_t cap;
};

// The same sequence of pieces, sized (Sizer) and carved (Carver).
void size_pair_scratch(Sizer& c, int64_t cap, bool saddle) {
    c.take<int32_t>(64);
    c.take<unsigned long long>(cap);
    c.take<unsigned long long>(cap);
    if (saddle) {
        c.take<int32_t>(cap);
        c.take<int32_t>(cap);
    }
    c.take<uint32_t>(ceil_div(cap, kChunk) + 1);
    size_sort_scratch(c, cap);
}

PairScratch take_pair_scratch(Carver& c, int64_t cap, bool saddle) {
    PairScratch p;
    p.cap = cap;
    p.ctl = c.take<int32_t>(64);
    p.k0 = c.take<unsigned long long>(cap);
    p.k1 = c.take<unsigned long long>(cap);
    p.w0 = saddle ? c.take<int32_t>(cap) : nullptr;
    p.w1 = saddle ? c.take<int32_t>(cap) : nullptr;
    p.chunk = c.take<uint32_t>(ceil_div(cap, kChunk) + 1);
    p.sort = carve_sort_scratch(c, cap);
    return p;
}

// Sort the emitted keys (with their crossing vertices), keep the first of
// each run, and (saddles) reduce each run to its best crossing.
int finish_pairs(const PairScratch& p, int shift, int32_t* out_a, int32_t* out_b, int64_t out_cap,
                 int64_t* num_pairs, const int32_t* order, int sense, int32_t* saddle, int32_t* status,
                 cudaStream_t s) {
    const bool with_saddle = order != nullptr;
    const int64_t cap = p.cap;
    bool in_alt = false;
    int r = run_sort_u64(p.k0, p.w0, p.k1, p.w1, p.ctl, cap, 2 * shift, p.sort, status, s, &in_alt,
                         "adjacency.sort_hist", "adjacency.sort_pass");
    if (r) return r;
    const unsigned long long* sorted = in_alt ? p.k1 : p.k0;
    const int32_t* cross = in_alt ? p.w1 : p.w0;
    unsigned long long* best = in_alt ? p.k0 : p.k1;  // the other key buffer is free now
    const int grid = blocks_for(ceil_div(cap, kChunk), 8);
    {
        TraceScope ts_("adjacency.heads", s);
        k_adj_heads<<<grid, kThreads, 0, s>>>(sorted, p.ctl, cap, p.chunk);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("adjacency.scan", s);
        k_adj_scan<<<1, 1024, 0, s>>>(p.chunk, p.ctl, cap, num_pairs);
    }
    MSC_LAUNCHED();
    if (with_saddle) {
        {
            TraceScope ts_("adjacency.zero", s);
            k_adj_zero<<<blocks_for(ceil_div(cap, kThreads), 8), kThreads, 0, s>>>(best, num_pairs);
        }
        MSC_LAUNCHED();
        {
            TraceScope ts_("adjacency.write", s);
            k_adj_write<true><<<grid, kThreads, 0, s>>>(sorted, p.ctl, cap, p.chunk, shift, out_a, out_b, out_cap,
                                                        cross, order, sense, best);
        }
        MSC_LAUNCHED();
        {
            TraceScope ts_("adjacency.saddle", s);
            k_adj_saddle<<<blocks_for(ceil_div(cap, kThreads), 8), kThreads, 0, s>>>(best, num_pairs, sense,
                                                                                     saddle, out_cap);
        }
        MSC_LAUNCHED();
    } else {
        {
            TraceScope ts_("adjacency.write", s);
            k_adj_write<false><<<grid, kThreads, 0, s>>>(sorted, p.ctl, cap, p.chunk, shift, out_a, out_b, out_cap,
                                                         nullptr, nullptr, 0, nullptr);
        }
        MSC_LAUNCHED();
    }
    return MSC_OK;
}

// Explicit mesh: one lane per vertex, the warp stepping through the rows of
// its 32 vertices together (one entry per lane per step), each edge taken
// from its smaller end.  A lane skips a key equal to the one it emitted
// last (plain adjacency); the warp's keys of a step go out with one atomic.
template <bool SADDLE>
__global__ void __launch_bounds__(kThreads) k_adj_emit_csr(const int32_t* __restrict__ label,
                                                           const int32_t* __restrict__ row,
                                                           const int32_t* __restrict__ col, int32_t n, int64_t nnz,
                                                           int32_t bound, int shift, const int32_t* __restrict__ order,
                                                           int sense, unsigned long long* out, int32_t* out_w,
                                                           int32_t* count, int64_t cap, int32_t* status) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t v = base + threadIdx.x;  // warp-uniform loop: every lane runs every step
        int32_t l = -1, e0 = 0, e1 = 0, ov = 0;
        if (v < n) {
            l = __ldg(label + v);
            if (l >= bound) {
                record_error(status, MSC_ERR_ARG);
                l = -1;
            }
            e0 = __ldg(row + v);
            e1 = __ldg(row + v + 1);
            if (e0 < 0 || e1 < e0 || (int64_t)e1 > nnz) {
                record_error(status, MSC_ERR_ARG);
                e1 = e0;
            }
            if (SADDLE && l >= 0) ov = __ldg(order + v);
        }
        const int32_t deg = l >= 0 ? e1 - e0 : 0;
        int32_t steps = deg;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) steps = max(steps, __shfl_xor_sync(0xffffffffu, steps, o));
        unsigned long long last = kNoKey;
        for (int32_t k = 0; k < steps; ++k) {
            unsigned long long key = kNoKey;
            int32_t w = 0;
            if (k < deg) {
                const int32_t u = __ldg(col + e0 + k);
                if ((uint32_t)u >= (uint32_t)n) {
                    record_error(status, MSC_ERR_ARG);
                } else if (u > v) {
                    const int32_t m = __ldg(label + u);
                    if (m >= 0 && m < bound && m != l) {
                        key = pair_key_of(shift, l, m);
                        if constexpr (SADDLE) {
                            const int32_t ou = __ldg(order + u);
                            const bool u_is = sense > 0 ? ou < ov : ou > ov;
                            w = u_is ? u : (int32_t)v;
                        } else {
                            if (key == last) key = kNoKey;  // the same pair as this lane's previous edge
                            else last = key;
                        }
                    }
                }
            }
            const uint32_t emit = __ballot_sync(0xffffffffu, key != kNoKey);
            if (!emit) continue;
            const int leader = __ffs(emit) - 1;
            uint32_t pos0 = 0;
            if (lane == leader) pos0 = atomicAdd(reinterpret_cast<uint32_t*>(count), (uint32_t)__popc(emit));
            pos0 = __shfl_sync(0xffffffffu, pos0, leader);
            if (key != kNoKey) {
                const uint32_t pos = pos0 + __popc(emit & lanemask_lt());
                if ((int64_t)pos < cap) {
                    out[pos] = key;
                    if constexpr (SADDLE) out_w[pos] = w;
                } else {
                    record_error(status, MSC_ERR_INTERNAL);  // more keys than entries: impossible
                }
            }
        }
    }
}

}  // namespace

void size_adjacency_scratch(Sizer& s, int64_t n, bool saddle) { size_pair_scratch(s, emit_capacity(n), saddle); }

void size_adjacency_csr_scratch(Sizer& s, int64_t nnz, bool saddle) {
    size_pair_scratch(s, std::max<int64_t>(nnz, 1), saddle);
}

template <bool SADDLE>
static int launch_emit(const EmitArgs& ea, int conn, int64_t tiles, cudaStream_t s) {
    auto kern = conn == 6 ? k_adj_emit<3, SADDLE> : k_adj_emit<7, SADDLE>;
    constexpr size_t smem = emit_smem_bytes<SADDLE>();
    MSC_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // persistent: as many CTAs as fit on the GPU at once
    int occ = 0;
    MSC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem));
    {
        TraceScope ts_("adjacency.emit", s);
        kern<<<blocks_for(tiles, std::max(occ, 1)), kThreads, smem, s>>>(ea);
    }
    MSC_LAUNCHED();
    return MSC_OK;
}

int run_adjacency_grid(const int32_t* label, msc_grid g, int conn, int32_t bound, int32_t* out_a,
                       int32_t* out_b, int64_t out_cap, int64_t* num_pairs, void* ws, size_t ws_bytes,
                       int32_t* status, cudaStream_t s, const int32_t* order, int sense, int32_t* saddle) {
    const bool with_saddle = order != nullptr;
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    Carver c(ws, ws_bytes);
    PairScratch p = take_pair_scratch(c, emit_capacity(n), with_saddle);
    if (!c.ok()) return MSC_ERR_WS;
    MSC_TRY(cudaMemsetAsync(p.ctl, 0, 64 * sizeof(int32_t), s));
    const int shift = ceil_log2(bound);
    const EmitArgs ea{label, g.nx, g.ny, g.nz, bound, shift, p.k0, p.ctl, p.cap, status, order, sense, p.w0};
    const int64_t tiles = ceil_div(g.nx, kTX) * ceil_div(g.ny, kTY) * ceil_div(g.nz, kZR);
    int r = with_saddle ? launch_emit<true>(ea, conn, tiles, s) : launch_emit<false>(ea, conn, tiles, s);
    if (r) return r;
    return finish_pairs(p, shift, out_a, out_b, out_cap, num_pairs, order, sense, saddle, status, s);
}

int run_adjacency_csr(const int32_t* label, const int32_t* row, const int32_t* col, int32_t n, int64_t nnz,
                      int32_t bound, int32_t* out_a, int32_t* out_b, int64_t out_cap, int64_t* num_pairs, void* ws,
                      size_t ws_bytes, int32_t* status, cudaStream_t s, const int32_t* order, int sense,
                      int32_t* saddle) {
    const bool with_saddle = order != nullptr;
    Carver c(ws, ws_bytes);
    PairScratch p = take_pair_scratch(c, std::max<int64_t>(nnz, 1), with_saddle);
    if (!c.ok()) return MSC_ERR_WS;
    MSC_TRY(cudaMemsetAsync(p.ctl, 0, 64 * sizeof(int32_t), s));
    const int shift = ceil_log2(bound);
    if (n > 0) {
        TraceScope ts_("adjacency.emit_csr", s);
        const int grid = blocks_for(ceil_div(n, kThreads), 8);
        if (with_saddle)
            k_adj_emit_csr<true><<<grid, kThreads, 0, s>>>(label, row, col, n, nnz, bound, shift, order, sense, p.k0,
                                                           p.w0, p.ctl, p.cap, status);
        else
            k_adj_emit_csr<false><<<grid, kThreads, 0, s>>>(label, row, col, n, nnz, bound, shift, nullptr, 1, p.k0,
                                                            nullptr, p.ctl, p.cap, status);
    }
    MSC_LAUNCHED();
    return finish_pairs(p, shift, out_a, out_b, out_cap, num_pairs, order, sense, saddle, status, s);
}

}  // namespace msc
