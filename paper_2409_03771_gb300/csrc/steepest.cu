// Steepest-ascent / steepest-descent pointers on the implicit Freudenthal
// triangulation of a regular grid (Alg. 1 initialisation, and its mirror
// for the ascending manifold), plus the explicit-adjacency (CSR) variant.
//
// Grid kernel: persistent CTAs walk 32x8x8 vertex tiles.  Each tile's
// order values plus a halo (4 cells in x to keep the TMA x coordinate
// 16-byte aligned, 1 cell in y and z) land in shared memory through one 3D
// TMA box (40x10x10 int32), three boxes in flight against the compute of the
// previous tiles.  Cells outside the grid get -1, which loses every signed
// max and (as 0xffffffff) every unsigned min, so border vertices see only
// their in-grid neighbours.  A thread handles four consecutive x vertices
// in two z planes, reading each neighbour row once as an int4 plus edge
// scalars, and keeps argmax / argmin as packed (order * 16 + code) keys.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "steepest.cuh"
#include "tma.cuh"

namespace msc {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr int kStages = 3;  // TMA boxes in flight per CTA (3 x 16 000 B of shared memory)

// A tile of TX x TY x TZ vertices and its shared-memory box (4 halo cells
// in x, keeping 16-byte alignment, 1 in y and z).  A thread takes four
// consecutive x vertices in REPS (= 2) consecutive z planes.
template <int TX_, int TY_, int TZ_>
struct Shape {
    static constexpr int TX = TX_, TY = TY_, TZ = TZ_;
    static constexpr int BX = TX + 8, BY = TY + 2, BZ = TZ + 2;
    static constexpr int PLANE = BX * BY;
    static constexpr int BOX = PLANE * BZ;
    static constexpr int XQ = TX / 4;            // threads along x
    static constexpr int LAYER = XQ * TY;        // threads per z plane
    static constexpr int ZL = kThreads / LAYER;  // z planes per pass
    static constexpr int REPS = TZ / ZL;
    static_assert(TX % 4 == 0 && kThreads % LAYER == 0 && TZ % ZL == 0, "tile shape");
};
using Tile = Shape<32, 8, 8>;  // single-grid kernels (TMA box 40 x 10 x 10)
constexpr int TX = Tile::TX, TY = Tile::TY, TZ = Tile::TZ;
constexpr int BX = Tile::BX, BY = Tile::BY, BZ = Tile::BZ;
constexpr int PLANE = Tile::PLANE;  // 400
constexpr int BOX = Tile::BOX;      // 4000

// Neighbour codes 0..13 (matching the row reads below), 14 = the vertex.
__constant__ int8_t c_off[15][3] = {
    {0, 0, -1}, {-1, 0, -1}, {0, -1, -1}, {-1, -1, -1}, {0, -1, 0},
    {-1, -1, 0}, {-1, 0, 0}, {1, 0, 0},   {0, 1, 0},    {1, 1, 0},
    {0, 0, 1},  {1, 0, 1},  {0, 1, 1},    {1, 1, 1},    {0, 0, 0}};

struct GridInfo {
    int32_t nx, ny, nz;
    int32_t tx, ty;  // tiles along x and y
    int64_t ntiles;
    int vec_store;  // asc/desc rows can take int4 stores
    int32_t off;    // id of the grid's first vertex (packed batches; else 0)
};

// Packed candidate: order * 16 + neighbour code.  Out-of-grid cells hold
// -1: negative as signed (loses every max), huge as unsigned (loses every
// min).  PK = int32 when order * 16 + 15 fits (n <= 2^27), else int64.
template <typename PK>
__device__ __forceinline__ PK pack(int val, int code) {
    return (PK)val * 16 + code;
}

// argmax / argmin codes over the 15 packed candidates c[0..14] (two-input
// min / max: measured faster here than the three-input DPX forms).
__device__ __forceinline__ void best_codes(const int32_t (&c)[15], int& hi, int& lo) {
    int mx = c[0];
    unsigned mn = (unsigned)c[0];
#pragma unroll
    for (int k = 1; k < 15; ++k) {
        mx = max(mx, c[k]);
        mn = min(mn, (unsigned)c[k]);
    }
    hi = mx & 15;
    lo = (int)(mn & 15u);
}

__device__ __forceinline__ void best_codes(const long long (&c)[15], int& hi, int& lo) {
    long long mx = c[0];
    unsigned long long mn = (unsigned long long)c[0];
#pragma unroll
    for (int k = 1; k < 15; ++k) {
        mx = c[k] > mx ? c[k] : mx;
        mn = (unsigned long long)c[k] < mn ? (unsigned long long)c[k] : mn;
    }
    hi = (int)(mx & 15);
    lo = (int)(mn & 15);
}

__device__ __forceinline__ void load_row(const int* r, int (&o)[6]) {
    // o[j] = value at x offset j-1 relative to the thread's first vertex
    const int4 q = *reinterpret_cast<const int4*>(r);
    o[0] = r[-1];
    o[1] = q.x;
    o[2] = q.y;
    o[3] = q.z;
    o[4] = q.w;
    o[5] = r[4];
}

// COUNT: add the tile's minima / maxima to nmin / nmax.
template <typename PK, typename S = Tile, bool COUNT = true>
__device__ __forceinline__ void tile_compute(const int* buf, const GridInfo& g, int x0, int y0,
                                             int z0, const int32_t* s_off, int32_t* __restrict__ asc,
                                             int32_t* __restrict__ desc, uint32_t& nmin,
                                             uint32_t& nmax) {
    static_assert(S::REPS == 2, "a thread takes two consecutive z planes");
    const int tid = threadIdx.x;
    const int xq = tid % S::XQ, ly = (tid / S::XQ) % S::TY, lzq = tid / S::LAYER;
    const int gx0 = x0 + 4 * xq, gy = y0 + ly;
    if (gx0 >= g.nx || gy >= g.ny) return;
    // Rows around the thread's 4 vertices in plane z: A (z-1, y), B (z-1, y-1),
    // C (z, y-1), D (z, y), E (z, y+1), F (z+1, y), G (z+1, y+1).  For plane
    // z+1, A = D, B = C, D = F and E = G of plane z: only C, F, G are read.
    const int lz0 = 2 * lzq;
    const int* b = buf + (lz0 + 1) * S::PLANE + (ly + 1) * S::BX + 4 * xq + 4;
    int A[6], B[6], C[6], D[6], E[6], F[6], G[6];
    load_row(b - S::PLANE, A);
    load_row(b - S::PLANE - S::BX, B);
    load_row(b - S::BX, C);
    load_row(b, D);
    load_row(b + S::BX, E);
    load_row(b + S::PLANE, F);
    load_row(b + S::PLANE + S::BX, G);
#pragma unroll
    for (int rep = 0; rep < 2; ++rep) {
        const int gz = z0 + lz0 + rep;
        if (gz >= g.nz) break;
        if (rep == 1) {
#pragma unroll
            for (int t = 0; t < 6; ++t) {
                A[t] = D[t];
                B[t] = C[t];
                D[t] = F[t];
                E[t] = G[t];
            }
            b += S::PLANE;
            load_row(b - S::BX, C);
            load_row(b + S::PLANE, F);
            load_row(b + S::PLANE + S::BX, G);
        }
        int hi_code[4], lo_code[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int j = i + 1;  // index of x offset 0
            using P = typename std::conditional<sizeof(PK) == 4, int32_t, long long>::type;
            const P c[15] = {pack<P>(D[j], 14),     pack<P>(A[j], 0),     pack<P>(A[j - 1], 1),
                             pack<P>(B[j], 2),      pack<P>(B[j - 1], 3), pack<P>(C[j], 4),
                             pack<P>(C[j - 1], 5),  pack<P>(D[j - 1], 6), pack<P>(D[j + 1], 7),
                             pack<P>(E[j], 8),      pack<P>(E[j + 1], 9), pack<P>(F[j], 10),
                             pack<P>(F[j + 1], 11), pack<P>(G[j], 12),    pack<P>(G[j + 1], 13)};
            best_codes(c, hi_code[i], lo_code[i]);
        }
        const int32_t v0 = g.off + gx0 + g.nx * (gy + g.ny * gz);  // total < 2^31
        int out_hi[4], out_lo[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            out_hi[i] = v0 + i + s_off[hi_code[i]];
            out_lo[i] = v0 + i + s_off[lo_code[i]];
            if (COUNT) {
                nmax += hi_code[i] == 14 && gx0 + i < g.nx;
                nmin += lo_code[i] == 14 && gx0 + i < g.nx;
            }
        }
#ifdef MSC_DEBUG_BOUNDS
        if (v0 < 0) return;
#endif
        if (g.vec_store && gx0 + 3 < g.nx) {
            *reinterpret_cast<int4*>(desc + v0) = make_int4(out_hi[0], out_hi[1], out_hi[2], out_hi[3]);
            *reinterpret_cast<int4*>(asc + v0) = make_int4(out_lo[0], out_lo[1], out_lo[2], out_lo[3]);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (gx0 + i < g.nx) {
                    desc[v0 + i] = out_hi[i];
                    asc[v0 + i] = out_lo[i];
                }
        }
    }
}

template <typename S = Tile>
__device__ __forceinline__ void tile_coords(const GridInfo& g, int64_t tile, int& x0, int& y0,
                                            int& z0) {
    const int64_t txy = (int64_t)g.tx * g.ty;
    const int64_t tz = tile / txy;
    const int64_t r = tile - tz * txy;
    const int64_t ty = r / g.tx;
    x0 = (int)((r - ty * g.tx) * S::TX);
    y0 = (int)(ty * S::TY);
    z0 = (int)(tz * S::TZ);
}

__device__ __forceinline__ bool box_crosses_border(const GridInfo& g, int x0, int y0, int z0) {
    return x0 < 4 || y0 < 1 || z0 < 1 || x0 + TX + 4 > g.nx || y0 + TY + 1 > g.ny ||
           z0 + TZ + 1 > g.nz;
}

__device__ __forceinline__ void mark_outside(int* buf, const GridInfo& g, int x0, int y0, int z0) {
    for (int i = threadIdx.x; i < BOX; i += kThreads) {
        const int lz = i / PLANE, r = i - lz * PLANE, ly = r / BX, lx = r - ly * BX;
        const int gx = x0 - 4 + lx, gy = y0 - 1 + ly, gz = z0 - 1 + lz;
        if (gx < 0 || gy < 0 || gz < 0 || gx >= g.nx || gy >= g.ny || gz >= g.nz) buf[i] = -1;
    }
}

__device__ __forceinline__ void flush_counts(uint32_t nmin, uint32_t nmax, uint32_t* extrema) {
    if (!extrema) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nmin += __shfl_xor_sync(0xffffffffu, nmin, o);
        nmax += __shfl_xor_sync(0xffffffffu, nmax, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (nmin) atomicAdd(&extrema[0], nmin);
        if (nmax) atomicAdd(&extrema[1], nmax);
    }
}

template <typename PK, bool COUNT>
__global__ void __launch_bounds__(kThreads, 4) k_steepest_tma(const __grid_constant__ CUtensorMap map,
                                                          const GridInfo g, int32_t* asc,
                                                          int32_t* desc, uint32_t* extrema,
                                                          int32_t* status) {
    __shared__ alignas(128) int buf[kStages][BOX];
    __shared__ alignas(8) uint64_t bar[kStages];
    __shared__ int32_t s_off[15];
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) mbar_init(&bar[q], 1);
        fence_mbar_init();
    }
    if (tid < 15)
        s_off[tid] = c_off[tid][0] + g.nx * (c_off[tid][1] + g.ny * c_off[tid][2]);
    __syncthreads();
    auto issue = [&](int64_t t, int b) {
        int x0, y0, z0;
        tile_coords(g, t, x0, y0, z0);
        mbar_expect_tx(&bar[b], BOX * 4);
        tma_load_3d(buf[b], &map, x0 - 4, y0 - 1, z0 - 1, &bar[b]);
    };
    int64_t tile = blockIdx.x;
    if (tid == 0)
        for (int q = 0; q < kStages; ++q)
            if (tile + q * (int64_t)gridDim.x < g.ntiles) issue(tile + q * (int64_t)gridDim.x, q);
    uint32_t phase[kStages] = {};
    uint32_t nmin = 0, nmax = 0;
    for (int it = 0; tile < g.ntiles; ++it, tile += gridDim.x) {
        const int b = it % kStages;
        const bool ok = mbar_wait(&bar[b], phase[b], kWaitLimit);
        if (ok) {
            int x0, y0, z0;
            tile_coords(g, tile, x0, y0, z0);
            if (box_crosses_border(g, x0, y0, z0)) {  // block-uniform
                mark_outside(buf[b], g, x0, y0, z0);
                __syncthreads();
            }
            tile_compute<PK, Tile, COUNT>(buf[b], g, x0, y0, z0, s_off, asc, desc, nmin, nmax);
        }
        // one barrier per tile: the buffer is free again, and a failed wait
        // (never expected) is seen by every thread
        if (__syncthreads_or(!ok)) {
            if (tid == 0) record_error(status, MSC_ERR_INTERNAL);
            for (int q = 0; q < kStages; ++q) mbar_wait(&bar[q], phase[q], kWaitLimit);
            return;
        }
        phase[b] ^= 1u;
        if (tid == 0 && tile + kStages * (int64_t)gridDim.x < g.ntiles) {
            fence_proxy_async_smem();
            issue(tile + kStages * (int64_t)gridDim.x, b);
        }
    }
    if (COUNT) flush_counts(nmin, nmax, extrema);
}

// Same stencil with plain coalesced loads (grids whose rows TMA cannot
// address: nx not a multiple of 4, or an unaligned base pointer).
template <typename PK, bool COUNT>
__global__ void __launch_bounds__(kThreads) k_steepest_ld(const int32_t* __restrict__ order,
                                                         const GridInfo g, int32_t* asc,
                                                         int32_t* desc, uint32_t* extrema) {
    __shared__ alignas(16) int buf[BOX];
    __shared__ int32_t s_off[15];
    const int tid = threadIdx.x;
    if (tid < 15)
        s_off[tid] = c_off[tid][0] + g.nx * (c_off[tid][1] + g.ny * c_off[tid][2]);
    uint32_t nmin = 0, nmax = 0;
    for (int64_t tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
        int x0, y0, z0;
        tile_coords(g, tile, x0, y0, z0);
        for (int i = tid; i < BOX; i += kThreads) {
            const int lz = i / PLANE, r = i - lz * PLANE, ly = r / BX, lx = r - ly * BX;
            const int gx = x0 - 4 + lx, gy = y0 - 1 + ly, gz = z0 - 1 + lz;
            int val = -1;
            if (gx >= 0 && gy >= 0 && gz >= 0 && gx < g.nx && gy < g.ny && gz < g.nz)
                val = order[gx + (int64_t)g.nx * (gy + (int64_t)g.ny * gz)];
            buf[i] = val;
        }
        __syncthreads();
        tile_compute<PK, Tile, COUNT>(buf, g, x0, y0, z0, s_off, asc, desc, nmin, nmax);
        __syncthreads();
    }
    if (COUNT) flush_counts(nmin, nmax, extrema);
}

// ----------------------------------------------------------------------------
// Batched grids packed one after another.  Persistent CTAs walk the tiles
// of all instances (instance i owns tiles [tile0[i], tile0[i+1])); the
// block's instance comes from a binary search over tile0 (in shared memory
// when the table fits), the box is staged with plain coalesced loads (an
// instance's rows need not be 16-byte aligned, so no TMA), and pointers
// are packed ids (instance offset + local id).  ext[2i], ext[2i+1] count
// the instance's minima and maxima.

constexpr int kSmemTileTable = 2048;  // instances whose tile table goes to shared memory

template <typename S>
__device__ __forceinline__ void load_box(const int32_t* __restrict__ order, const GridInfo& g, int x0,
                                         int y0, int z0, int* buf) {
    for (int i = threadIdx.x; i < S::BOX; i += kThreads) {
        const int lz = i / S::PLANE, r = i - lz * S::PLANE, ly = r / S::BX, lx = r - ly * S::BX;
        const int gx = x0 - 4 + lx, gy = y0 - 1 + ly, gz = z0 - 1 + lz;
        int val = -1;
        if (gx >= 0 && gy >= 0 && gz >= 0 && gx < g.nx && gy < g.ny && gz < g.nz)
            val = order[(int64_t)g.off + gx + (int64_t)g.nx * (gy + (int64_t)g.ny * gz)];
        buf[i] = val;
    }
}

template <typename PK, typename S>
__global__ void __launch_bounds__(kThreads) k_steepest_batch(const int32_t* __restrict__ order,
                                                            const BatchInst* __restrict__ inst,
                                                            const int32_t* __restrict__ tile0, int count,
                                                            int32_t* asc, int32_t* desc, uint32_t* ext) {
    __shared__ alignas(16) int buf[S::BOX];
    __shared__ int32_t s_off[15];
    __shared__ int32_t s_tile0[kSmemTileTable + 1];
    __shared__ int s_inst;
    const int tid = threadIdx.x;
    const bool smem_table = count <= kSmemTileTable;
    if (smem_table)
        for (int i = tid; i <= count; i += kThreads) s_tile0[i] = tile0[i];
    __syncthreads();
    const int32_t* t0 = smem_table ? s_tile0 : tile0;
    const int64_t ntiles = t0[count];
    int cur = -1;
    GridInfo g{};
    uint32_t nmin = 0, nmax = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (tid == 0) {  // largest i with t0[i] <= tile (empty instances own no tile)
            int lo = 0, hi = count - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (t0[mid] <= tile) lo = mid; else hi = mid - 1;
            }
            s_inst = lo;
        }
        __syncthreads();
        const int i = s_inst;
        if (i != cur) {  // block-uniform
            if (cur >= 0) flush_counts(nmin, nmax, ext + 2 * cur);
            nmin = nmax = 0;
            cur = i;
            const BatchInst b = inst[i];
            g.nx = b.nx;
            g.ny = b.ny;
            g.nz = b.nz;
            g.off = b.off;
            g.tx = (b.nx + S::TX - 1) / S::TX;
            g.ty = (b.ny + S::TY - 1) / S::TY;
            g.vec_store = b.vec;
            if (tid < 15) s_off[tid] = c_off[tid][0] + g.nx * (c_off[tid][1] + g.ny * c_off[tid][2]);
        }
        int x0, y0, z0;
        tile_coords<S>(g, tile - t0[i], x0, y0, z0);
        load_box<S>(order, g, x0, y0, z0, buf);
        __syncthreads();
        tile_compute<PK, S>(buf, g, x0, y0, z0, s_off, asc, desc, nmin, nmax);
        __syncthreads();
    }
    if (cur >= 0) flush_counts(nmin, nmax, ext + 2 * cur);
}

// ----------------------------------------------------------------------------
// CSR variant: 8 lanes per vertex, each lane scans every 8th neighbour.

constexpr int kCsrLanes = 8;

__global__ void __launch_bounds__(256) k_steepest_csr(const int32_t* __restrict__ order,
                                                      const int32_t* __restrict__ row,
                                                      const int32_t* __restrict__ col, int32_t n,
                                                      int32_t* asc, int32_t* desc,
                                                      int32_t* status) {
    const int sub = threadIdx.x & (kCsrLanes - 1);
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) / 32;
    constexpr int kPerWarp = 32 / kCsrLanes;
    // warp-uniform loop: the warp's 4 vertices are wbase .. wbase+3
    for (int64_t wbase = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32) * kPerWarp;
         wbase < n; wbase += warps * kPerWarp) {
        const int64_t v = wbase + (threadIdx.x & 31) / kCsrLanes;
        const bool live = v < n;
        int hi_v = -1, hi_u = -1, lo_v = INT32_MAX, lo_u = -1;
        if (live) {
            const int ov = order[v];
            hi_v = ov;
            hi_u = (int)v;
            lo_v = ov;
            lo_u = (int)v;
            const int e0 = row[v], e1 = row[v + 1];
            for (int e = e0 + sub; e < e1; e += kCsrLanes) {
                const int u = col[e];
                if ((unsigned)u >= (unsigned)n) {
                    record_error(status, MSC_ERR_ARG);
                    continue;
                }
                const int ou = order[u];
                if (ou > hi_v) {
                    hi_v = ou;
                    hi_u = u;
                }
                if (ou < lo_v) {
                    lo_v = ou;
                    lo_u = u;
                }
            }
        }
#pragma unroll
        for (int o = kCsrLanes / 2; o > 0; o >>= 1) {
            const int hv = __shfl_xor_sync(0xffffffffu, hi_v, o);
            const int hu = __shfl_xor_sync(0xffffffffu, hi_u, o);
            const int lv = __shfl_xor_sync(0xffffffffu, lo_v, o);
            const int lu = __shfl_xor_sync(0xffffffffu, lo_u, o);
            if (hv > hi_v) {
                hi_v = hv;
                hi_u = hu;
            }
            if (lv < lo_v) {
                lo_v = lv;
                lo_u = lu;
            }
        }
        if (live && sub == 0) {
            desc[v] = hi_u;
            asc[v] = lo_u;
        }
    }
}

}  // namespace

int run_steepest_grid(const int32_t* order, msc_grid gd, int32_t* asc, int32_t* desc,
                      uint32_t* extrema, int32_t* status, cudaStream_t s, bool allow_tma) {
    GridInfo g;
    g.off = 0;
    g.nx = gd.nx;
    g.ny = gd.ny;
    g.nz = gd.nz;
    g.tx = (int)ceil_div(gd.nx, TX);
    g.ty = (int)ceil_div(gd.ny, TY);
    const int64_t tz = ceil_div(gd.nz, TZ);
    g.ntiles = (int64_t)g.tx * g.ty * tz;
    g.vec_store = (gd.nx % 4 == 0) && ((uintptr_t)asc % 16 == 0) && ((uintptr_t)desc % 16 == 0);
    const int64_t n = (int64_t)gd.nx * gd.ny * gd.nz;
    const bool packed = n <= (int64_t(1) << 27);
    const int sms = current_device().sms;
    CUtensorMap map;
    const bool tma = allow_tma && make_tensor_map_3d(&map, order, 4, gd.nx, gd.ny, gd.nz, BX, BY, BZ);
    int occ = 1;
    if (tma) {
        auto kern = extrema ? (packed ? k_steepest_tma<int32_t, true> : k_steepest_tma<int64_t, true>)
                            : (packed ? k_steepest_tma<int32_t, false> : k_steepest_tma<int64_t, false>);
        MSC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, 0));
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(g.ntiles, (int64_t)sms * std::max(occ, 1)));
        {
            TraceScope ts_("steepest.grid", s);
            kern<<<(unsigned)grid, kThreads, 0, s>>>(map, g, asc, desc, extrema, status);
        }
    } else {
        auto kern = extrema ? (packed ? k_steepest_ld<int32_t, true> : k_steepest_ld<int64_t, true>)
                            : (packed ? k_steepest_ld<int32_t, false> : k_steepest_ld<int64_t, false>);
        MSC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, 0));
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(g.ntiles, (int64_t)sms * std::max(occ, 1)));
        {
            TraceScope ts_("steepest.grid", s);
            kern<<<(unsigned)grid, kThreads, 0, s>>>(order, g, asc, desc, extrema);
        }
    }
    MSC_LAUNCHED();
    return MSC_OK;
}

namespace {

template <typename S>
int64_t tiles_of(msc_grid g) {
    return ceil_div(g.nx, S::TX) * ceil_div(g.ny, S::TY) * ceil_div(g.nz, S::TZ);
}

template <typename S>
int launch_batch(const int32_t* order, const BatchInst* inst, const int32_t* tile0, int count,
                 int64_t ntiles, bool packed, int32_t* asc, int32_t* desc, uint32_t* ext, cudaStream_t s) {
    auto kern = packed ? k_steepest_batch<int32_t, S> : k_steepest_batch<int64_t, S>;
    int occ = 1;
    MSC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, 0));
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)current_device().sms * std::max(occ, 1)));
    {
        TraceScope ts_("steepest.batch", s);
        kern<<<(unsigned)grid, kThreads, 0, s>>>(order, inst, tile0, count, asc, desc, ext);
    }
    MSC_LAUNCHED();
    return MSC_OK;
}

}  // namespace

int steepest_batch_shapes() { return 4; }

int64_t steepest_batch_tiles(int shape, msc_grid g) {
    switch (shape) {
        case 1: return tiles_of<Shape<16, 8, 16>>(g);
        case 2: return tiles_of<Shape<64, 4, 8>>(g);
        case 3: return tiles_of<Shape<16, 16, 8>>(g);
        default: return tiles_of<Tile>(g);
    }
}

const char* steepest_batch_shape_name(int shape) {
    switch (shape) {
        case 1: return "16x8x16";
        case 2: return "64x4x8";
        case 3: return "16x16x8";
        default: return "32x8x8";
    }
}

int run_steepest_batch(const int32_t* order, const BatchInst* inst, const int32_t* tile0, int count,
                       int64_t ntiles, int shape, bool packed, int32_t* asc, int32_t* desc, uint32_t* ext,
                       cudaStream_t s) {
    if (ntiles <= 0) return MSC_OK;
    switch (shape) {
        case 1: return launch_batch<Shape<16, 8, 16>>(order, inst, tile0, count, ntiles, packed, asc, desc, ext, s);
        case 2: return launch_batch<Shape<64, 4, 8>>(order, inst, tile0, count, ntiles, packed, asc, desc, ext, s);
        case 3: return launch_batch<Shape<16, 16, 8>>(order, inst, tile0, count, ntiles, packed, asc, desc, ext, s);
        default: return launch_batch<Tile>(order, inst, tile0, count, ntiles, packed, asc, desc, ext, s);
    }
}

int run_steepest_csr(const int32_t* order, const int32_t* row, const int32_t* col, int32_t n,
                     int32_t* asc, int32_t* desc, int32_t* status, cudaStream_t s) {
    if (n <= 0) return MSC_OK;
    const int64_t want = ceil_div((int64_t)n * kCsrLanes, 256);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)current_device().sms * 8));
    {
        TraceScope ts_("steepest.csr", s);
        k_steepest_csr<<<grid, 256, 0, s>>>(order, row, col, n, asc, desc, status);
    }
    MSC_LAUNCHED();
    return MSC_OK;
}

}  // namespace msc
