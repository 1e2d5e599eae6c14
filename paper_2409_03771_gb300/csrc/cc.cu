// Connected components with smallest-id labels: feature mask on a grid
// (6- or 14-connectivity) and explicit mesh adjacency (CSR).
//
// The paper (Alg. 3) points every feature vertex at its largest feature
// neighbour, compresses, hooks segment roots across segment borders
// ("d[d[v]] <- d[u]") and compresses again, first per rank and then across
// ranks.  Here the same local-then-global structure is applied to GPU
// tiles, mirrored to the smallest id, with the hooking made exact by a
// union-find on roots (hook the larger root under the smaller with
// atomicMin; retry if another thread moved it first):
//   1. k_cc_local: a 64x8x8 tile of the mask as 64 row bitmasks in shared
//      memory, x-runs labelled by bit arithmetic, runs of neighbouring rows
//      united once per overlap segment, each feature voxel written with
//      the global id of its tile-local root (the smallest id of its
//      tile-local component), -1 elsewhere;
//   2. k_cc_merge: for every edge that leaves a tile through its +x, +y or
//      +z side, union the two roots in global memory (path halving);
//   3. k_cc_flatten: pointer jumping to the final root.
// The final root of a component is its smallest vertex id because every
// hook points a root at a smaller one.
//
// Mesh: union-find over the CSR edges with subgraph sampling (see the mesh
// kernels below).
#include <cuda_runtime.h>

#include <algorithm>

#include "cc.cuh"

namespace msc {
namespace {

#ifndef MSC_CC_LOCAL_MIN_BLOCKS
#define MSC_CC_LOCAL_MIN_BLOCKS 6
#endif
constexpr int CX = 64, CY = 8, CZ = 8;
constexpr int CT = CX * CY * CZ;  // 4096
constexpr int kThreads = 256;
constexpr uint32_t kUnionLimit = 1u << 20;

struct CcGrid {
    int32_t nx, ny, nz;
    int32_t tx, ty;
    int64_t ntiles;
    int conn;
    int vec;  // nx % 8 == 0, mask 8-byte and label 16-byte aligned: rows move as 8-byte / 16-byte words
};

__device__ __forceinline__ void cc_tile_coords(const CcGrid& g, int64_t t, int& x0, int& y0, int& z0) {
    const int64_t txy = (int64_t)g.tx * g.ty;
    const int64_t tz = t / txy;
    const int64_t r = t - tz * txy;
    const int64_t ty = r / g.tx;
    x0 = (int)((r - ty * g.tx) * CX);
    y0 = (int)(ty * CY);
    z0 = (int)(tz * CZ);
}

// positive half of the neighbourhood: 3 face offsets, then 4 diagonals
__constant__ int8_t c_pos[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0},
                                   {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};

// Root of x in a shared-memory forest whose entries point at smaller
// local indices, halving the path on the way (atomicMin: never undoes a
// hook made by another thread).
__device__ __forceinline__ int find_s(int* L, int x) {
    int p = L[x];
    while (p != x) {
        const int gp = L[p];
        if (gp != p) atomicMin(&L[x], gp);
        x = gp;
        p = L[x];
    }
    return x;
}

__device__ __forceinline__ void union_s(int* L, int a, int b) {
    for (int it = 0; it < CT * 4; ++it) {
        a = find_s(L, a);
        b = find_s(L, b);
        if (a == b) return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(&L[b], a);
        if (old == b) return;
        b = old;
    }
}

// Root of x in global memory, halving the path on the way.  The halving
// write is an atomicMin: labels only ever decrease (every entry points at a
// smaller or equal id of the same component), so a halving write can never
// undo a hook or overwrite a final root written by another thread.
__device__ __forceinline__ int32_t find_g(int32_t* L, int32_t x) {
    for (uint32_t it = 0; it < kUnionLimit; ++it) {
        const int32_t p = ld_volatile_s32(L + x);
        if (p == x) return x;
        const int32_t gp = ld_volatile_s32(L + p);
        if (gp != p) atomicMin(L + x, gp);
        x = gp;
    }
    return x;
}

__device__ __forceinline__ void union_g(int32_t* L, int32_t a, int32_t b, int32_t* status) {
    for (uint32_t it = 0; it < kUnionLimit; ++it) {
        a = find_g(L, a);
        b = find_g(L, b);
        if (a == b) return;
        if (a > b) {
            const int32_t t = a;
            a = b;
            b = t;
        }
        const int32_t old = atomicMin(L + b, a);
        if (old == b) return;
        b = old;
    }
    record_error(status, MSC_ERR_INTERNAL);
}

// Tile-local labelling, run based.  Rows are x-lines of 64 voxels (one
// 64-bit mask each, from two ballots).  A masked voxel starts at the first
// voxel of its x-run; runs of neighbouring rows are united once per
// overlap segment (a maximal x-range where both rows' voxels, shifted by
// the offset's dx, are masked); then every voxel takes its root.
constexpr int kRows = CY * CZ;  // 64 rows of CX = 64 voxels

__device__ __forceinline__ uint64_t run_start_mask_below(uint64_t m, int x) {
    return ~m & ((x ? (~0ull >> (64 - x)) : 0ull));
}

__global__ void __launch_bounds__(kThreads, MSC_CC_LOCAL_MIN_BLOCKS) k_cc_local(const uint8_t* __restrict__ mask, const CcGrid g,
                                                       int32_t* __restrict__ label) {
    __shared__ int s_l[CT];
    __shared__ uint64_t s_row[kRows];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int64_t t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        int x0, y0, z0;
        cc_tile_coords(g, t, x0, y0, z0);
        // the 64 row bitmasks
        if (g.vec) {
            // 8 lanes per row, 8 mask bytes per lane: byte j nonzero -> bit j
            const int sub = lane & 7;
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
                const int r = warp * 4 + (lane >> 3) + 32 * pass;
                const int ly = r & (CY - 1), lz = r / CY;
                const int gy = y0 + ly, gz = z0 + lz, gx = x0 + 8 * sub;
                uint32_t bits = 0;
                if (gy < g.ny && gz < g.nz && gx < g.nx) {
                    const uint2 w = *reinterpret_cast<const uint2*>(
                        mask + (gx + (int64_t)g.nx * (gy + (int64_t)g.ny * gz)));
                    // high bit of each byte set iff the byte is nonzero; then
                    // the four high bits gathered into bits 28..31
                    const uint32_t lo = (w.x | ((w.x & 0x7f7f7f7fu) + 0x7f7f7f7fu)) & 0x80808080u;
                    const uint32_t hi = (w.y | ((w.y & 0x7f7f7f7fu) + 0x7f7f7f7fu)) & 0x80808080u;
                    bits = ((lo * 0x00204081u) >> 28) | (((hi * 0x00204081u) >> 28) << 4);
                }
                reinterpret_cast<uint8_t*>(s_row)[8 * r + sub] = (uint8_t)bits;
            }
            __syncthreads();
            for (int r = warp; r < kRows; r += kThreads / 32) {
                const uint64_t m = s_row[r];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int x = lane + 32 * h;
                    int lab = -1;
                    if (m >> x & 1ull) {
                        const uint64_t z = run_start_mask_below(m, x);
                        lab = (z ? 64 - __clzll((long long)z) : 0) + CX * r;
                    }
                    s_l[x + CX * r] = lab;
                }
            }
        } else {
        // rows: warp w takes rows w, w + 8, ..., 8 rows per warp
        for (int r = warp; r < kRows; r += kThreads / 32) {
            const int ly = r & (CY - 1), lz = r / CY;
            const int gy = y0 + ly, gz = z0 + lz;
            bool a = false, b = false;
            if (gy < g.ny && gz < g.nz) {
                const int64_t rb = (int64_t)g.nx * (gy + (int64_t)g.ny * gz);
                if (x0 + lane < g.nx) a = mask[rb + x0 + lane] != 0;
                if (x0 + 32 + lane < g.nx) b = mask[rb + x0 + 32 + lane] != 0;
            }
            const uint64_t m = (uint64_t)__ballot_sync(0xffffffffu, a) | ((uint64_t)__ballot_sync(0xffffffffu, b) << 32);
            if (lane == 0) s_row[r] = m;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int x = lane + 32 * h;
                int lab = -1;
                if (m >> x & 1ull) {
                    const uint64_t z = run_start_mask_below(m, x);
                    const int start = z ? 64 - __clzll((long long)z) : 0;
                    lab = start + CX * r;
                }
                s_l[x + CX * r] = lab;
            }
        }
        }
        __syncthreads();
        // unite runs of neighbouring rows, once per overlap segment
        const int npairs = g.conn == 6 ? 2 * 56 : 2 * 56 + 2 * 56 + 2 * 49;
        for (int q = tid; q < npairs; q += kThreads) {
            int r, r2, dx;
            int k = q;
            if (k < 112) {  // (0,1,0) / (1,1,0): y + 1 ; (0,0,1) / (1,0,1): z + 1
                const bool ystep = k < 56;
                const int i = ystep ? k : k - 56;
                const int ly = ystep ? i % 7 : i % 8, lz = ystep ? i / 7 : i / 8;
                r = ly + CY * lz;
                r2 = ystep ? r + 1 : r + CY;
                dx = 0;
            } else if (k < 224) {
                k -= 112;
                const bool ystep = k < 56;
                const int i = ystep ? k : k - 56;
                const int ly = ystep ? i % 7 : i % 8, lz = ystep ? i / 7 : i / 8;
                r = ly + CY * lz;
                r2 = ystep ? r + 1 : r + CY;
                dx = 1;
            } else {  // (0,1,1) / (1,1,1): y + 1 and z + 1
                k -= 224;
                const int i = k % 49;
                const int ly = i % 7, lz = i / 7;
                r = ly + CY * lz;
                r2 = r + 1 + CY;
                dx = k < 49 ? 0 : 1;
            }
            const uint64_t o = s_row[r] & (s_row[r2] >> dx);
            uint64_t seg = o & ~(o << 1);
            while (seg) {
                const int x = __ffsll((long long)seg) - 1;
                seg &= seg - 1;
                union_s(s_l, s_l[x + CX * r], s_l[x + dx + CX * r2]);
            }
        }
        __syncthreads();
        // every run start takes its root (four threads per row, a quarter
        // of the row each); a voxel's entry names its run start
        {
            const int r = tid >> 2, q = tid & 3;
            const uint64_t m = s_row[r];
            uint64_t st = m & ~(m << 1) & (0xffffull << (16 * q));
            while (st) {
                const int xs = __ffsll((long long)st) - 1;
                st &= st - 1;
                s_l[xs + CX * r] = find_s(s_l, xs + CX * r);
            }
        }
        __syncthreads();
        // every voxel takes its run start's root: 16 threads per row, four
        // consecutive voxels each, stored as one 16-byte word where the row
        // allows
        const int64_t tbase = x0 + (int64_t)g.nx * (y0 + (int64_t)g.ny * z0);
        const int64_t nxy = (int64_t)g.nx * g.ny;
        const int x = 4 * (tid & 15);
#pragma unroll
        for (int pass = 0; pass < kRows / 16; ++pass) {
            const int r = (tid >> 4) + 16 * pass;
            const int ly = r & (CY - 1), lz = r / CY;
            if (y0 + ly >= g.ny || z0 + lz >= g.nz || x0 + x >= g.nx) continue;
            int32_t out[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = x + j + CX * r;
                out[j] = -1;
                const int ls = s_l[i];
                if (ls >= 0) {
                    const int rt = s_l[ls];
                    const int rx = rt & (CX - 1), ry = (rt / CX) & (CY - 1), rz = rt / (CX * CY);
                    out[j] = (int32_t)(tbase + rx + (int64_t)g.nx * ry + nxy * rz);
                }
            }
            int32_t* dst = label + tbase + x + (int64_t)g.nx * ly + nxy * lz;
            if (g.vec) {
                *reinterpret_cast<int4*>(dst) = make_int4(out[0], out[1], out[2], out[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (x0 + x + j < g.nx) dst[j] = out[j];
            }
        }
        __syncthreads();
    }
}

// Voxels of a tile's +z face, then +y face (without z face), then +x face
// (without the other two): 512 + 448 + 49 = 1009 per full tile.
constexpr int kShell = CX * CY + CX * (CZ - 1) + (CY - 1) * (CZ - 1);

// The crossing edges of one tile mostly join the same few pairs of
// tile-local components.  Each tile's distinct pairs (a, b) are collected in
// a shared-memory hash set (after a warp-level skip of repeated pairs in
// consecutive lanes), then united in parallel, one thread per pair; a pair
// that finds the set full is united at once.
constexpr int kPairSlots = 256;

__global__ void __launch_bounds__(kThreads) k_cc_merge(const CcGrid g, int32_t* label, int32_t* status) {
    __shared__ unsigned long long s_pair[kPairSlots];
    const int npos = g.conn == 6 ? 3 : 7;
    const int lane = threadIdx.x & 31;
    for (int64_t t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        int x0, y0, z0;
        cc_tile_coords(g, t, x0, y0, z0);
        for (int i = threadIdx.x; i < kPairSlots; i += kThreads) s_pair[i] = ~0ull;
        __syncthreads();
        // the trip count is warp-uniform: kShell rounded up to whole warps
        for (int s0 = threadIdx.x - lane; s0 < kShell; s0 += kThreads) {
            const int s = s0 + lane;
            int lx = 0, ly = 0, lz = 0;
            if (s < CX * CY) {
                lx = s % CX;
                ly = s / CX;
                lz = CZ - 1;
            } else if (s < CX * CY + CX * (CZ - 1)) {
                const int r = s - CX * CY;
                lx = r % CX;
                lz = r / CX;
                ly = CY - 1;
            } else {
                const int r = s - CX * CY - CX * (CZ - 1);
                ly = r % (CY - 1);
                lz = r / (CY - 1);
                lx = CX - 1;
            }
            const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
            const bool in = s < kShell && gx < g.nx && gy < g.ny && gz < g.nz;
            const int64_t v = gx + (int64_t)g.nx * (gy + (int64_t)g.ny * gz);
            const int32_t a = in ? label[v] : -1;
            for (int o = 0; o < npos; ++o) {
                const int dx = c_pos[o][0], dy = c_pos[o][1], dz = c_pos[o][2];
                const int ux = gx + dx, uy = gy + dy, uz = gz + dz;
                const bool cross = in && a >= 0 && !(lx + dx < CX && ly + dy < CY && lz + dz < CZ) && ux < g.nx &&
                                   uy < g.ny && uz < g.nz;
                const int32_t b = cross ? label[ux + (int64_t)g.nx * (uy + (int64_t)g.ny * uz)] : -1;
                const bool want = cross && b >= 0 && b != a;
                const int32_t pa = __shfl_up_sync(0xffffffffu, want ? a : -1, 1);
                const int32_t pb = __shfl_up_sync(0xffffffffu, want ? b : -1, 1);
                if (want && (lane == 0 || pa != a || pb != b)) {
                    const unsigned long long key = ((unsigned long long)(uint32_t)a << 32) | (uint32_t)b;
                    uint32_t h = (uint32_t)((key * 0x9e3779b97f4a7c15ull) >> 56) & (kPairSlots - 1);
                    bool placed = false;
                    for (int probe = 0; probe < 16 && !placed; ++probe, h = (h + 1) & (kPairSlots - 1)) {
                        const unsigned long long old = atomicCAS(&s_pair[h], ~0ull, key);
                        placed = old == ~0ull || old == key;
                    }
                    if (!placed) union_g(label, a, b, status);  // set full: unite now
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kPairSlots; i += kThreads) {
            const unsigned long long key = s_pair[i];
            if (key != ~0ull) union_g(label, (int32_t)(key >> 32), (int32_t)(uint32_t)key, status);
        }
        __syncthreads();
    }
}

// Pointer jumping to the roots.  A thread takes 8 labels, lane-consecutive
// (label c*2048 + j*256 + tid), and follows their chains hop by hop
// together until the warp's chains have all ended: 8 independent gathers
// in flight, and the 32 lanes of each gather read neighbouring labels,
// whose roots are mostly shared (the union-find before it halved the
// paths, so chains are short).  Once every hook is done the root reached is
// the component minimum, so a plain store of it cannot lose anything.
constexpr int kFlatPer = 8;
constexpr int kFlatHops = (int)kUnionLimit;  // bound only: a forest's chains end far sooner
constexpr int kFlatThreads = 256;

__global__ void __launch_bounds__(kFlatThreads) k_flatten(int32_t* label, int64_t n) {
    constexpr int64_t kChunk = (int64_t)kFlatThreads * kFlatPer;
    for (int64_t c = blockIdx.x; c * kChunk < n; c += gridDim.x) {
        int32_t l[kFlatPer], r[kFlatPer];
        uint32_t open = 0;
#pragma unroll
        for (int j = 0; j < kFlatPer; ++j) {
            const int64_t v = c * kChunk + (int64_t)j * kFlatThreads + threadIdx.x;
            l[j] = v < n ? label[v] : -1;
            r[j] = l[j];
            open |= (l[j] >= 0 ? 1u : 0u) << j;
        }
        // cached loads: a label read stale is still an ancestor of the
        // vertex (labels only decrease), so following it stays correct
#pragma unroll 1
        for (int h = 0; h < kFlatHops; ++h) {
            if (!__any_sync(0xffffffffu, open)) break;  // the warp's chains all ended
            int32_t w[kFlatPer];
#pragma unroll
            for (int j = 0; j < kFlatPer; ++j) w[j] = (open >> j & 1u) ? label[r[j]] : 0;
#pragma unroll
            for (int j = 0; j < kFlatPer; ++j)
                if (open >> j & 1u) {
                    if (w[j] == r[j]) open &= ~(1u << j);
                    else r[j] = w[j];
                }
        }
#pragma unroll
        for (int j = 0; j < kFlatPer; ++j) {
            const int64_t v = c * kChunk + (int64_t)j * kFlatThreads + threadIdx.x;
            if (v < n && r[j] != l[j]) label[v] = r[j];
        }
    }
}

// ----------------------------------------------------------------------------
// mesh

// Mesh kernels (subgraph sampling, after the Afforest scheme):
//   1. label[v] = v; unite every vertex with its first and second neighbour
//      (one lane per vertex and round);
//   2. flatten; sample 1024 vertices and take the most frequent label --
//      on a well-connected mesh, nearly every vertex is already in that
//      component;
//   3. every vertex outside it unites all its remaining edges (8 lanes per
//      row); an edge to a vertex of the frequent component is found from
//      this side, since the adjacency is symmetric;
//   4. flatten.
// Every union hooks the larger root under the smaller, so the final root of
// a component is its smallest vertex id, whatever the order of unions.
constexpr int kRowLanes = 8;
constexpr int kSamples = 1024;

__global__ void k_mesh_init(int32_t* label, int32_t n) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        label[v] = (int32_t)v;
}

// Unite every vertex with its k-th neighbour (k = 0 or 1).
__global__ void k_mesh_link_k(const int32_t* __restrict__ row, const int32_t* __restrict__ col, int32_t n,
                              int k, int32_t* label, int32_t* status) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = row[v] + k;
        if (e >= row[v + 1]) continue;
        const int32_t u = col[e];
        if ((uint32_t)u >= (uint32_t)n) {
            record_error(status, MSC_ERR_ARG);
            continue;
        }
        union_g(label, (int32_t)v, u, status);
    }
}

// The most frequent label among kSamples vertices spread over the ids
// (one block; labels sorted in shared memory, longest run wins, ties to
// the smaller label).
__global__ void __launch_bounds__(kSamples) k_mesh_sample(const int32_t* label, int32_t n, int32_t* frequent) {
    __shared__ int32_t s[kSamples];
    const int t = threadIdx.x;
    const uint64_t mixed = (uint64_t)(t + 1) * 0x9e3779b97f4a7c15ull;
    s[t] = label[(int64_t)((mixed >> 11) % (uint64_t)n)];
    __syncthreads();
    for (int k = 2; k <= kSamples; k <<= 1)  // bitonic sort
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int p = t ^ j;
            if (p > t) {
                const bool up = (t & k) == 0;
                const int32_t a = s[t], b = s[p];
                if ((a > b) == up) {
                    s[t] = b;
                    s[p] = a;
                }
            }
            __syncthreads();
        }
    if (t == 0) {
        int32_t best = s[0], best_len = 0, cur = s[0], len = 0;
        for (int i = 0; i < kSamples; ++i) {
            if (s[i] == cur) ++len;
            else {
                cur = s[i];
                len = 1;
            }
            if (len > best_len) {
                best_len = len;
                best = cur;
            }
        }
        *frequent = best;
    }
}

// Vertices outside the frequent component unite their remaining edges.
__global__ void __launch_bounds__(256) k_mesh_hook(const int32_t* __restrict__ row,
                                                   const int32_t* __restrict__ col, int32_t n,
                                                   const int32_t* __restrict__ frequent, int32_t* label,
                                                   int32_t* status) {
    const int lane = threadIdx.x & 31, sub = lane & (kRowLanes - 1);
    const int32_t big = *frequent;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) / 32;
    constexpr int kPerWarp = 32 / kRowLanes;
    for (int64_t wbase = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32) * kPerWarp; wbase < n;
         wbase += warps * kPerWarp) {
        const int64_t v = wbase + lane / kRowLanes;
        if (v >= n || label[v] == big) continue;
        const int32_t e1 = row[v + 1];
        for (int32_t e = row[v] + 2 + sub; e < e1; e += kRowLanes) {
            const int32_t u = col[e];
            if ((uint32_t)u >= (uint32_t)n) {
                record_error(status, MSC_ERR_ARG);
                continue;
            }
            union_g(label, (int32_t)v, u, status);
        }
    }
}

int cc_grid_for(int64_t work, int per_sm = 8) {
    const int64_t want = ceil_div(std::max<int64_t>(work, 1), 256);
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)current_device().sms * per_sm));
}

}  // namespace

int run_cc_mask(const uint8_t* mask, msc_grid gd, int conn, int32_t* label, int32_t* status,
                cudaStream_t s) {
    CcGrid g;
    g.nx = gd.nx;
    g.ny = gd.ny;
    g.nz = gd.nz;
    g.tx = (int)ceil_div(gd.nx, CX);
    g.ty = (int)ceil_div(gd.ny, CY);
    g.ntiles = (int64_t)g.tx * g.ty * ceil_div(gd.nz, CZ);
    g.conn = conn;
    g.vec = gd.nx % 8 == 0 && ((uintptr_t)mask & 7) == 0 && ((uintptr_t)label & 15) == 0;
    const int64_t n = (int64_t)gd.nx * gd.ny * gd.nz;
    const int sms = current_device().sms;
    int occ = 1;
    MSC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cc_local, kThreads, 0));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(g.ntiles, (int64_t)sms * std::max(occ, 1)));
    {
        TraceScope ts_("cc.local", s);
        k_cc_local<<<grid, kThreads, 0, s>>>(mask, g, label);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("cc.merge", s);
        k_cc_merge<<<grid, kThreads, 0, s>>>(g, label, status);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("cc.flatten", s);
        k_flatten<<<cc_grid_for(ceil_div(n, kFlatPer)), kFlatThreads, 0, s>>>(label, n);
    }
    MSC_LAUNCHED();
    return MSC_OK;
}

int run_cc_mesh(const int32_t* row, const int32_t* col, int32_t n, int32_t* label, int32_t* status,
                cudaStream_t s, int32_t* frequent) {
    if (n <= 0) return MSC_OK;
    const int grid = cc_grid_for(n);
    const int fgrid = cc_grid_for(ceil_div(n, kFlatPer));
    {
        TraceScope ts_("mesh.init", s);
        k_mesh_init<<<grid, 256, 0, s>>>(label, n);
    }
    MSC_LAUNCHED();
    for (int k = 0; k < 2; ++k) {
        TraceScope ts_("mesh.link", s);
        k_mesh_link_k<<<grid, 256, 0, s>>>(row, col, n, k, label, status);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("mesh.flatten", s);
        k_flatten<<<fgrid, kFlatThreads, 0, s>>>(label, n);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("mesh.sample", s);
        k_mesh_sample<<<1, kSamples, 0, s>>>(label, n, frequent);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("mesh.hook", s);
        k_mesh_hook<<<grid, 256, 0, s>>>(row, col, n, frequent, label, status);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("mesh.flatten", s);
        k_flatten<<<fgrid, kFlatThreads, 0, s>>>(label, n);
    }
    MSC_LAUNCHED();
    return MSC_OK;
}

}  // namespace msc
