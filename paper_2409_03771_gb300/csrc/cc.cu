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
//   1. k_cc_local: a 64x8x8 tile of the mask in shared memory, union-find
//      over its internal edges in shared memory, each feature voxel
//      written with the global id of its tile-local root (the smallest id
//      of its tile-local component), -1 elsewhere;
//   2. k_cc_merge: for every edge that leaves a tile through its +x, +y or
//      +z side, union the two roots in global memory (path halving);
//   3. k_cc_flatten: pointer jumping to the final root.
// The final root of a component is its smallest vertex id because every
// hook points a root at a smaller one.
//
// Mesh: label[v] <- min(v, smallest neighbour), union over every edge
// (u < v) in global memory, flatten.
#include <cuda_runtime.h>

#include <algorithm>

#include "cc.cuh"

namespace msc {
namespace {

constexpr int CX = 64, CY = 8, CZ = 8;
constexpr int CT = CX * CY * CZ;  // 4096
constexpr int kThreads = 256;
constexpr int kPer = CT / kThreads;  // 16
constexpr uint32_t kUnionLimit = 1u << 20;

struct CcGrid {
    int32_t nx, ny, nz;
    int32_t tx, ty;
    int64_t ntiles;
    int conn;
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

__global__ void __launch_bounds__(kThreads) k_cc_local(const uint8_t* __restrict__ mask, const CcGrid g,
                                                       int32_t* __restrict__ label) {
    __shared__ int s_l[CT];
    __shared__ uint8_t s_m[CT];
    const int tid = threadIdx.x;
    const int npos = g.conn == 6 ? 3 : 7;
    for (int64_t t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        int x0, y0, z0;
        cc_tile_coords(g, t, x0, y0, z0);
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int i = tid + k * kThreads;
            const int lx = i & (CX - 1), ly = (i / CX) & (CY - 1), lz = i / (CX * CY);
            const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
            uint8_t m = 0;
            if (gx < g.nx && gy < g.ny && gz < g.nz)
                m = mask[gx + (int64_t)g.nx * (gy + (int64_t)g.ny * gz)] != 0;
            s_m[i] = m;
            s_l[i] = m ? i : -1;
        }
        __syncthreads();
#pragma unroll 1
        for (int k = 0; k < kPer; ++k) {
            const int i = tid + k * kThreads;
            if (!s_m[i]) continue;
            const int lx = i & (CX - 1), ly = (i / CX) & (CY - 1), lz = i / (CX * CY);
            for (int o = 0; o < npos; ++o) {
                const int jx = lx + c_pos[o][0], jy = ly + c_pos[o][1], jz = lz + c_pos[o][2];
                if (jx >= CX || jy >= CY || jz >= CZ) continue;
                const int j = jx + CX * (jy + CY * jz);
                if (s_m[j]) union_s(s_l, i, j);
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int i = tid + k * kThreads;
            if (s_m[i]) s_l[i] = find_s(s_l, i);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int i = tid + k * kThreads;
            const int lx = i & (CX - 1), ly = (i / CX) & (CY - 1), lz = i / (CX * CY);
            const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
            if (gx < g.nx && gy < g.ny && gz < g.nz) {
                int32_t out = -1;
                const int r = s_l[i];
                if (r >= 0) {
                    const int rx = r & (CX - 1), ry = (r / CX) & (CY - 1), rz = r / (CX * CY);
                    out = (int32_t)((x0 + rx) + (int64_t)g.nx * ((y0 + ry) + (int64_t)g.ny * (z0 + rz)));
                }
                label[gx + (int64_t)g.nx * (gy + (int64_t)g.ny * gz)] = out;
            }
        }
        __syncthreads();
    }
}

// Voxels of a tile's +z face, then +y face (without z face), then +x face
// (without the other two): 512 + 448 + 49 = 1009 per full tile.
constexpr int kShell = CX * CY + CX * (CZ - 1) + (CY - 1) * (CZ - 1);

__global__ void __launch_bounds__(kThreads) k_cc_merge(const CcGrid g, int32_t* label, int32_t* status) {
    const int npos = g.conn == 6 ? 3 : 7;
    for (int64_t t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        int x0, y0, z0;
        cc_tile_coords(g, t, x0, y0, z0);
        for (int s = threadIdx.x; s < kShell; s += kThreads) {
            int lx, ly, lz;
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
            if (gx >= g.nx || gy >= g.ny || gz >= g.nz) continue;
            const int64_t v = gx + (int64_t)g.nx * (gy + (int64_t)g.ny * gz);
            int32_t a = -2;  // loaded lazily
            for (int o = 0; o < npos; ++o) {
                const int dx = c_pos[o][0], dy = c_pos[o][1], dz = c_pos[o][2];
                if (lx + dx < CX && ly + dy < CY && lz + dz < CZ) continue;  // inside the tile
                const int ux = gx + dx, uy = gy + dy, uz = gz + dz;
                if (ux >= g.nx || uy >= g.ny || uz >= g.nz) continue;
                if (a == -2) a = label[v];
                if (a < 0) break;
                const int32_t b = label[ux + (int64_t)g.nx * (uy + (int64_t)g.ny * uz)];
                if (b >= 0 && b != a) union_g(label, a, b, status);
            }
        }
    }
}

// Pointer jumping to the roots.  A thread takes 8 labels, lane-consecutive
// (label c*2048 + j*256 + tid), and follows their chains hop by hop
// together: 8 independent gathers in flight, and the 32 lanes of each
// gather read neighbouring labels, whose roots are mostly shared.  The few
// chains still open after kFlatHops hops finish one by one.  Once every
// hook is done the root reached is the component minimum, so a plain store
// of it cannot lose anything.
constexpr int kFlatPer = 8;
constexpr int kFlatHops = 4;
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
#pragma unroll
        for (int h = 0; h < kFlatHops; ++h) {
            int32_t w[kFlatPer];
#pragma unroll
            for (int j = 0; j < kFlatPer; ++j) w[j] = (open >> j & 1u) ? ld_volatile_s32(label + r[j]) : 0;
#pragma unroll
            for (int j = 0; j < kFlatPer; ++j)
                if (open >> j & 1u) {
                    if (w[j] == r[j]) open &= ~(1u << j);
                    else r[j] = w[j];
                }
        }
#pragma unroll
        for (int j = 0; j < kFlatPer; ++j)
            if (open >> j & 1u) r[j] = find_g(label, r[j]);
#pragma unroll
        for (int j = 0; j < kFlatPer; ++j) {
            const int64_t v = c * kChunk + (int64_t)j * kFlatThreads + threadIdx.x;
            if (v < n && r[j] != l[j]) label[v] = r[j];
        }
    }
}

// ----------------------------------------------------------------------------
// mesh

// Mesh kernels: 8 lanes per vertex, each lane taking every 8th entry of
// the row, so a row's column indices are read as contiguous 32-byte runs.
constexpr int kRowLanes = 8;

__global__ void __launch_bounds__(256) k_mesh_init(const int32_t* __restrict__ row,
                                                   const int32_t* __restrict__ col, int32_t n,
                                                   int32_t* label, int32_t* status) {
    const int sub = threadIdx.x & (kRowLanes - 1);
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) / 32;
    constexpr int kPerWarp = 32 / kRowLanes;
    for (int64_t wbase = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32) * kPerWarp; wbase < n;
         wbase += warps * kPerWarp) {
        const int64_t v = wbase + (threadIdx.x & 31) / kRowLanes;
        int32_t m = INT32_MAX;
        if (v < n) {
            m = (int32_t)v;
            const int32_t e1 = row[v + 1];
            for (int32_t e = row[v] + sub; e < e1; e += kRowLanes) {
                const int32_t u = col[e];
                if ((uint32_t)u >= (uint32_t)n) {
                    record_error(status, MSC_ERR_ARG);
                    continue;
                }
                m = u < m ? u : m;
            }
        }
#pragma unroll
        for (int o = kRowLanes / 2; o > 0; o >>= 1) {
            const int32_t t = __shfl_xor_sync(0xffffffffu, m, o);
            m = t < m ? t : m;
        }
        if (v < n && sub == 0) label[v] = m;
    }
}

// Union every edge (v, u) with u < v, after label[] holds, for every v, the
// smallest of v and its neighbours.  The root of v is found once per row.
__global__ void __launch_bounds__(256) k_mesh_hook(const int32_t* __restrict__ row,
                                                   const int32_t* __restrict__ col, int32_t n,
                                                   int32_t* label, int32_t* status) {
    const int lane = threadIdx.x & 31, sub = lane & (kRowLanes - 1);
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) / 32;
    constexpr int kPerWarp = 32 / kRowLanes;
    for (int64_t wbase = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32) * kPerWarp; wbase < n;
         wbase += warps * kPerWarp) {
        const int64_t v = wbase + lane / kRowLanes;
        int32_t rv = 0;
        if (v < n && sub == 0) rv = find_g(label, (int32_t)v);
        rv = __shfl_sync(0xffffffffu, rv, lane & ~(kRowLanes - 1));
        if (v >= n) continue;
        const int32_t e1 = row[v + 1];
        for (int32_t e = row[v] + sub; e < e1; e += kRowLanes) {
            const int32_t u = col[e];
            if ((uint32_t)u >= (uint32_t)v) continue;  // each edge once (u < v); bad u skipped
            if (ld_volatile_s32(label + u) == rv) continue;  // already hooked to v's root
            union_g(label, rv, u, status);
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
                cudaStream_t s) {
    if (n <= 0) return MSC_OK;
    const int grid = cc_grid_for(n);
    {
        TraceScope ts_("mesh.init", s);
        k_mesh_init<<<grid, 256, 0, s>>>(row, col, n, label, status);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("mesh.hook", s);
        k_mesh_hook<<<grid, 256, 0, s>>>(row, col, n, label, status);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("mesh.flatten", s);
        k_flatten<<<cc_grid_for(ceil_div(n, kFlatPer)), kFlatThreads, 0, s>>>(label, n);
    }
    MSC_LAUNCHED();
    return MSC_OK;
}

}  // namespace msc
