// Batched Morse-Smale segmentation (include/msc.h, msc_batch_*): the
// computation of msc_segment -- vertex order, steepest pointers (Alg. 1
// initialisation), path compression (Alg. 1 loop), dense cell ids -- for
// many independent grids packed into one vertex space, as one sequence of
// persistent kernels over all instances:
//
//   1. segmented onesweep sort: tiles never straddle two instances, ranks
//      are instance-local;
//   2. batched stencil: CTAs walk the tiles of every instance, pointers are
//      packed ids;
//   3. pointer jumping over the packed arrays (packed pointers never leave
//      their instance, so one compression serves all);
//   4. cell ids over the packed (asc, desc) pairs: pairs of instance i sort
//      before those of instance i+1, so instance i's dense ids are the
//      global ranks minus the number of pairs of earlier instances, found
//      by a binary search of off_i * total in the sorted pair keys;
//   5. a rebase pass turns packed ids into instance-local ones.
//
// A plan captures steps 1-5 once as a CUDA graph; the autotuner times the
// tile shape of step 2 and the active-list threshold of step 3.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "compress.cuh"
#include "msid.cuh"
#include "sort.cuh"
#include "steepest.cuh"

namespace msc {
namespace {

constexpr int kThreads = 256;
constexpr int kShapes = 4;
constexpr int kCtlWords = 64;  // [0] pair bound [1] 1 [2] cap [3] K [4] total cells

// Host-side description of a batch: packed offsets and tile tables.
struct Layout {
    int count = 0;
    int64_t total = 0;
    int64_t tiles = 0;  // sort tiles (kSortTile vertices, inside one instance)
    bool packed = true; // every instance has at most 2^27 vertices
    std::vector<int32_t> off, tile0, tile_seg;
    std::vector<BatchInst> inst;
    std::vector<int32_t> stile0[kShapes];
    int64_t stiles[kShapes] = {0, 0, 0, 0};
};

int make_layout(const msc_grid* grids, int count, Layout& L) {
    if (count <= 0 || !grids) return MSC_ERR_ARG;
    L.count = count;
    L.off.assign(count + 1, 0);
    L.tile0.assign(count + 1, 0);
    L.inst.assign(count, BatchInst{});
    for (int k = 0; k < kShapes; ++k) L.stile0[k].assign(count + 1, 0);
    int64_t off = 0, tiles = 0, st[kShapes] = {0, 0, 0, 0};
    for (int i = 0; i < count; ++i) {
        const msc_grid g = grids[i];
        if (g.nx <= 0 || g.ny <= 0 || g.nz <= 0) return MSC_ERR_ARG;
        const int64_t n = (int64_t)g.nx * g.ny * g.nz;
        if (n > INT32_MAX || off + n > INT32_MAX) return MSC_ERR_ARG;
        L.off[i] = (int32_t)off;
        L.tile0[i] = (int32_t)tiles;
        BatchInst& b = L.inst[i];
        b.nx = g.nx;
        b.ny = g.ny;
        b.nz = g.nz;
        b.off = (int32_t)off;
        b.vec = (g.nx % 4 == 0) && (off % 4 == 0);  // buffers are 256-byte aligned (checked on use)
        for (int k = 0; k < kShapes; ++k) {
            L.stile0[k][i] = (int32_t)st[k];
            st[k] += steepest_batch_tiles(k, g);
            if (st[k] > INT32_MAX) return MSC_ERR_ARG;
        }
        if (n > (int64_t(1) << 27)) L.packed = false;
        off += n;
        tiles += ceil_div(n, kSortTile);
    }
    L.off[count] = (int32_t)off;
    L.tile0[count] = (int32_t)tiles;
    for (int k = 0; k < kShapes; ++k) {
        L.stile0[k][count] = (int32_t)st[k];
        L.stiles[k] = st[k];
    }
    L.total = off;
    L.tiles = tiles;
    L.tile_seg.resize(tiles);
    for (int i = 0; i < count; ++i)
        for (int32_t t = L.tile0[i]; t < L.tile0[i + 1]; ++t) L.tile_seg[t] = i;
    return MSC_OK;
}

// Device pieces of the workspace.  The tables come first (uploaded in one
// copy), then the control words, then the largest of the stage scratches.
struct DevLayout {
    int32_t* off;
    int32_t* tile0;
    int32_t* tile_seg;
    BatchInst* inst;
    int32_t* stile0[kShapes];
    size_t table_bytes;  // bytes from the workspace start to the end of the tables
    uint32_t* ctl;       // kCtlWords
    uint32_t* ext;       // [count][2]
    int32_t* first;      // [count + 1]
    unsigned long long* checksum;  // [2]
    size_t stage_off;
};

template <typename C>
void carve_tables(C& c, const Layout& L, DevLayout* d) {
    int32_t* off = c.template take<int32_t>(L.count + 1);
    int32_t* tile0 = c.template take<int32_t>(L.count + 1);
    int32_t* tile_seg = c.template take<int32_t>(std::max<int64_t>(L.tiles, 1));
    BatchInst* inst = c.template take<BatchInst>(L.count);
    int32_t* st[kShapes];
    for (int k = 0; k < kShapes; ++k) st[k] = c.template take<int32_t>(L.count + 1);
    if (d) {
        d->off = off;
        d->tile0 = tile0;
        d->tile_seg = tile_seg;
        d->inst = inst;
        for (int k = 0; k < kShapes; ++k) d->stile0[k] = st[k];
    }
}

// Sizer with the Carver interface (pointers are meaningless).
struct SizeCarver {
    Sizer s;
    template <typename T>
    T* take(size_t count) {
        s.take<T>(count);
        return nullptr;
    }
};

size_t stage_bytes(const Layout& L) {
    Sizer sort, comp, ms;
    sort.take<int32_t>(std::max<int64_t>(L.total, 1));
    size_seg_sort_scratch(sort, L.count, L.tiles);
    size_compress_scratch(comp, L.total, 2);
    size_ms_scratch(ms, L.total);
    return std::max({sort.used, comp.used, ms.used});
}

size_t batch_bytes(const Layout& L) {
    SizeCarver c;
    carve_tables(c, L, nullptr);
    c.s.take<uint32_t>(kCtlWords);
    c.s.take<uint32_t>((size_t)2 * L.count);
    c.s.take<int32_t>(L.count + 1);
    c.s.take<unsigned long long>(2);
    return ((c.s.used + 255) & ~size_t(255)) + stage_bytes(L);
}

DevLayout carve_all(void* ws, size_t ws_bytes, const Layout& L) {
    Carver c(ws, ws_bytes);
    DevLayout d{};
    carve_tables(c, L, &d);
    d.table_bytes = c.used;
    d.ctl = c.take<uint32_t>(kCtlWords);
    d.ext = c.take<uint32_t>((size_t)2 * L.count);
    d.first = c.take<int32_t>(L.count + 1);
    d.checksum = c.take<unsigned long long>(2);
    d.stage_off = (c.used + 255) & ~size_t(255);
    return d;
}

// Copy the host tables into the workspace with one host-to-device copy.
int upload_tables(void* ws, const Layout& L, const DevLayout& d, cudaStream_t s) {
    std::vector<char> host(d.table_bytes, 0);
    auto put = [&](const void* dev, const void* src, size_t bytes) {
        const size_t at = static_cast<const char*>(dev) - static_cast<const char*>(ws);
        std::memcpy(host.data() + at, src, bytes);
    };
    put(d.off, L.off.data(), L.off.size() * 4);
    put(d.tile0, L.tile0.data(), L.tile0.size() * 4);
    if (L.tiles) put(d.tile_seg, L.tile_seg.data(), L.tile_seg.size() * 4);
    put(d.inst, L.inst.data(), L.inst.size() * sizeof(BatchInst));
    for (int k = 0; k < kShapes; ++k) put(d.stile0[k], L.stile0[k].data(), L.stile0[k].size() * 4);
    // pageable source: the call returns once the bytes are staged
    MSC_TRY(cudaMemcpyAsync(ws, host.data(), host.size(), cudaMemcpyHostToDevice, s));
    return MSC_OK;
}

// ctl[0] = sum over instances of min(n_i, minima_i * maxima_i): an upper
// bound on the distinct pairs (sizes the de-duplication table); ctl[1] = 1.
__global__ void k_batch_bound(const uint32_t* __restrict__ ext, const int32_t* __restrict__ off, int count,
                              uint32_t* ctl) {
    __shared__ unsigned long long s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    unsigned long long b = 0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const unsigned long long pairs = (unsigned long long)ext[2 * i] * ext[2 * i + 1];
        const unsigned long long n = (unsigned long long)(off[i + 1] - off[i]);
        b += pairs < n ? pairs : n;
    }
    atomicAdd(&s_sum, b);
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl[0] = (uint32_t)s_sum;  // <= total < 2^31
        ctl[1] = 1;
    }
}

// first[i] = #distinct pairs whose minimum lies before instance i (lower
// bound of off_i << sh among the sorted keys (asc << sh) | desc);
// num_cells[i] = first[i + 1] - first[i].
__device__ __forceinline__ int64_t lower_bound_u64(const unsigned long long* a, int64_t K,
                                                   unsigned long long x) {
    int64_t lo = 0, hi = K;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_batch_first(const unsigned long long* __restrict__ keys, const uint32_t* ctl,
                              const int32_t* __restrict__ off, int count, int sh, int32_t* first,
                              int32_t* num_cells) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int64_t K = ctl[3];
    const int64_t a = lower_bound_u64(keys, K, (unsigned long long)off[i] << sh);
    const int64_t b = i + 1 < count ? lower_bound_u64(keys, K, (unsigned long long)off[i + 1] << sh) : K;
    first[i] = (int32_t)a;
    num_cells[i] = (int32_t)(b - a);
}

// Packed ids -> instance-local ids, per sort tile (inside one instance).
constexpr int kRebasePer = kSortTile / kThreads;  // 16

__global__ void __launch_bounds__(kThreads) k_batch_rebase(const int32_t* __restrict__ tile_seg,
                                                           const int32_t* __restrict__ off,
                                                           const int32_t* __restrict__ tile0,
                                                           const int32_t* __restrict__ first, int64_t tiles,
                                                           int32_t* ms, int32_t* asc, int32_t* desc) {
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int i = tile_seg[t];
        const int32_t o = off[i], n = off[i + 1] - o, fr = first[i];
        const int64_t l0 = (t - tile0[i]) * kSortTile + threadIdx.x;
#pragma unroll
        for (int j = 0; j < kRebasePer; ++j) {
            const int64_t l = l0 + j * kThreads;
            if (l < n) {
                const int64_t v = o + l;
                ms[v] -= fr;
                asc[v] -= o;
                desc[v] -= o;
            }
        }
    }
}

// Order-sensitive checksum of the outputs (autotuner's equality check).
__global__ void k_batch_checksum(const int32_t* __restrict__ a, const int32_t* __restrict__ b,
                                 const int32_t* __restrict__ c, const int32_t* __restrict__ d, int64_t n,
                                 const int32_t* __restrict__ cells, int count, unsigned long long* out) {
    unsigned long long h = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long x = (unsigned long long)(uint32_t)a[v] | ((unsigned long long)(uint32_t)b[v] << 32);
        unsigned long long y = (unsigned long long)(uint32_t)c[v] | ((unsigned long long)(uint32_t)d[v] << 32);
        x = (x ^ (unsigned long long)v) * 0x9e3779b97f4a7c15ull;
        y = (y + (unsigned long long)v) * 0xc2b2ae3d27d4eb4full;
        h += (x ^ (x >> 29)) + (y ^ (y >> 31));
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        h += ((unsigned long long)(uint32_t)cells[i] + 1) * (0x100000001b3ull + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, h);
}

struct Buffers {
    const float* f;
    int32_t *order, *asc, *desc, *ms, *num_cells, *status;
};

struct Tune {
    int shape = 0;
    int build_shift = 3;
};

int run_batch(void* ws, size_t ws_bytes, const Layout& L, const DevLayout& d, const Buffers& B, const Tune& T,
              cudaStream_t s) {
    MSC_TRY(cudaMemsetAsync(B.status, 0, sizeof(int32_t), s));
    MSC_TRY(cudaMemsetAsync(d.ctl, 0, kCtlWords * sizeof(uint32_t), s));
    MSC_TRY(cudaMemsetAsync(d.ext, 0, (size_t)2 * L.count * sizeof(uint32_t), s));
    const int32_t total = (int32_t)L.total;
    // 1. instance-local order; asc / desc / ms double as the sort's ping-pong
    {
        Carver st(ws, ws_bytes);
        st.used = d.stage_off;
        int32_t* ib = st.take<int32_t>(std::max<int64_t>(L.total, 1));
        SortScratch sc = carve_seg_sort_scratch(st, L.count, L.tiles);
        SegTable t{d.off, d.tile0, d.tile_seg, L.count, L.total, L.tiles};
        int r = run_order_seg(B.f, t, B.order, reinterpret_cast<uint32_t*>(B.asc), B.desc,
                              reinterpret_cast<uint32_t*>(B.ms), ib, sc, B.status, s);
        if (r) return r;
    }
    // 2. steepest pointers (packed ids) + per-instance extrema counts
    int r = run_steepest_batch(B.order, d.inst, d.stile0[T.shape], L.count, L.stiles[T.shape], T.shape, L.packed,
                               B.asc, B.desc, d.ext, s);
    if (r) return r;
    {
        TraceScope ts_("batch.bound", s);
        k_batch_bound<<<1, kThreads, 0, s>>>(d.ext, d.off, L.count, d.ctl);
    }
    MSC_LAUNCHED();
    // 3. pointer jumping over the packed arrays
    {
        Carver st(ws, ws_bytes);
        st.used = d.stage_off;
        CompressScratch sc = carve_compress_scratch(st, L.total, 2);
        int32_t* arr[2] = {B.asc, B.desc};
        CompressTune ct;
        ct.build_shift = T.build_shift;
        ct.fill_lists = false;  // the tuned threshold
        ct.trusted = true;  // made by the batched stencil: in range, acyclic
        r = run_compress(arr, 2, total, sc, B.status, s, ct);
        if (r) return r;
    }
    // 4. packed cell ids, then per-instance first ranks and cell counts
    const unsigned long long* keys = nullptr;
    {
        Carver st(ws, ws_bytes);
        st.used = d.stage_off;
        MsScratch sc = carve_ms_scratch(st, L.total);
        sc.ctl = d.ctl;
        r = run_ms_id(B.asc, B.desc, total, B.ms, reinterpret_cast<int32_t*>(d.ctl + 4), sc, true, B.status, s,
                      &keys);
        if (r) return r;
    }
    {
        TraceScope ts_("batch.first", s);
        k_batch_first<<<(unsigned)ceil_div(L.count, kThreads), kThreads, 0, s>>>(
            keys, d.ctl, d.off, L.count, ms_pair_shift(L.total), d.first, B.num_cells);
    }
    MSC_LAUNCHED();
    // 5. instance-local ids
    {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(L.tiles, (int64_t)current_device().sms * 8));
        TraceScope ts_("batch.rebase", s);
        k_batch_rebase<<<grid, kThreads, 0, s>>>(d.tile_seg, d.off, d.tile0, d.first, L.tiles, B.ms, B.asc,
                                                 B.desc);
    }
    MSC_LAUNCHED();
    return MSC_OK;
}

// Autotuned settings, remembered per list of grids.
std::mutex g_tune_mu;
std::map<std::vector<int32_t>, Tune> g_tuned;

std::vector<int32_t> signature(const msc_grid* grids, int count) {
    std::vector<int32_t> sig((size_t)3 * count);
    for (int i = 0; i < count; ++i) {
        sig[3 * i] = grids[i].nx;
        sig[3 * i + 1] = grids[i].ny;
        sig[3 * i + 2] = grids[i].nz;
    }
    return sig;
}

Tune resolve(const msc_grid* grids, int count, const msc_tune* t) {
    Tune out;
    bool have = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned.find(signature(grids, count));
        if (it != g_tuned.end()) {
            out = it->second;
            have = true;
        }
    }
    if (!have) out = Tune();
    if (t && t->steepest_shape >= 0) out.shape = t->steepest_shape;
    if (t && t->build_shift > 0) out.build_shift = t->build_shift;
    return out;
}

bool tune_ok(const msc_tune* t) {
    if (!t) return true;
    return t->steepest_shape >= -1 && t->steepest_shape < kShapes && t->build_shift >= 0 && t->build_shift <= 30;
}

bool buffers_ok(const Buffers& B, void* ws) {
    if (!B.f || !B.order || !B.asc || !B.desc || !B.ms || !B.num_cells || !B.status || !ws) return false;
    const uintptr_t a = (uintptr_t)B.asc | (uintptr_t)B.desc;
    return (a & 15) == 0 && ((uintptr_t)ws & 255) == 0;
}

}  // namespace
}  // namespace msc

using namespace msc;

struct msc_batch_plan {
    Layout L;
    DevLayout d;
    Buffers B;
    Tune T;
    void* ws;
    size_t ws_bytes;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
};

extern "C" {

size_t msc_batch_workspace_bytes(const msc_grid* grids, int32_t count) {
    Layout L;
    if (make_layout(grids, count, L) != MSC_OK) return 0;
    return batch_bytes(L);
}

int msc_batch_segment(const msc_grid* grids, int32_t count, const float* f, int32_t* order, int32_t* asc,
                      int32_t* desc, int32_t* ms, int32_t* num_cells, void* ws, size_t ws_bytes,
                      const msc_tune* tune, int32_t* d_status, void* stream) {
    Layout L;
    int r = make_layout(grids, count, L);
    if (r) return r;
    const Buffers B{f, order, asc, desc, ms, num_cells, d_status};
    if (!buffers_ok(B, ws) || !tune_ok(tune)) return MSC_ERR_ARG;
    if (ws_bytes < batch_bytes(L)) return MSC_ERR_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const DevLayout d = carve_all(ws, ws_bytes, L);
    if ((r = upload_tables(ws, L, d, s))) return r;
    return run_batch(ws, ws_bytes, L, d, B, resolve(grids, count, tune), s);
}

int msc_batch_plan_create(const msc_grid* grids, int32_t count, const float* f, int32_t* order, int32_t* asc,
                          int32_t* desc, int32_t* ms, int32_t* num_cells, void* ws, size_t ws_bytes,
                          const msc_tune* tune, int32_t* d_status, void* stream, msc_batch_plan** out) {
    if (!out) return MSC_ERR_ARG;
    *out = nullptr;
    msc_batch_plan* p = new msc_batch_plan();
    int r = make_layout(grids, count, p->L);
    p->B = Buffers{f, order, asc, desc, ms, num_cells, d_status};
    if (!r && (!buffers_ok(p->B, ws) || !tune_ok(tune))) r = MSC_ERR_ARG;
    if (!r && ws_bytes < batch_bytes(p->L)) r = MSC_ERR_WS;
    if (r) {
        delete p;
        return r;
    }
    p->ws = ws;
    p->ws_bytes = ws_bytes;
    p->T = resolve(grids, count, tune);
    p->d = carve_all(ws, ws_bytes, p->L);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    r = upload_tables(ws, p->L, p->d, s);
    if (!r && cudaStreamSynchronize(s) != cudaSuccess) r = MSC_ERR_CUDA;
    if (r) {
        delete p;
        return r;
    }
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        delete p;
        return MSC_ERR_CUDA;
    }
    const unsigned long long before = launch_count();
    r = MSC_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) r = MSC_ERR_CUDA;
    if (!r) {
        const int rr = run_batch(ws, ws_bytes, p->L, p->d, p->B, p->T, cs);
        const cudaError_t e = cudaStreamEndCapture(cs, &p->graph);
        r = rr ? rr : (e != cudaSuccess ? MSC_ERR_CUDA : MSC_OK);
    }
    const unsigned long long captured = launch_count() - before;
    add_launches(-(long long)captured);  // counted again on every replay
    p->kernels = (int)captured;
    if (!r && cudaGraphInstantiate(&p->exec, p->graph, 0) != cudaSuccess) r = MSC_ERR_CUDA;
    cudaStreamDestroy(cs);
    if (r) {
        msc_batch_plan_destroy(p);
        return r;
    }
    *out = p;
    return MSC_OK;
}

int msc_batch_plan_launch(msc_batch_plan* p, void* stream) {
    if (!p || !p->exec) return MSC_ERR_ARG;
    if (cudaGraphLaunch(p->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) return MSC_ERR_CUDA;
    add_launches(p->kernels);
    return MSC_OK;
}

int msc_batch_plan_kernels(const msc_batch_plan* p) { return p ? p->kernels : 0; }

void msc_batch_plan_destroy(msc_batch_plan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    delete p;
}

int msc_batch_autotune(const msc_grid* grids, int32_t count, const float* f, int32_t* order, int32_t* asc,
                       int32_t* desc, int32_t* ms, int32_t* num_cells, void* ws, size_t ws_bytes,
                       int32_t* d_status, void* stream, int32_t reps, msc_tune* best, float* best_ms) {
    Layout L;
    int r = make_layout(grids, count, L);
    if (r) return r;
    const Buffers B{f, order, asc, desc, ms, num_cells, d_status};
    if (!buffers_ok(B, ws) || reps < 1) return MSC_ERR_ARG;
    if (ws_bytes < batch_bytes(L)) return MSC_ERR_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const DevLayout d = carve_all(ws, ws_bytes, L);
    if ((r = upload_tables(ws, L, d, s))) return r;
    cudaEvent_t e0, e1;
    MSC_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return MSC_ERR_CUDA;
    }
    bool have_ref = false;
    unsigned long long ref = 0;
    // time one candidate: warm-up, `reps` timed runs, checksum of the outputs
    auto measure = [&](const Tune& T, float* ms_out) -> int {
        int rr = run_batch(ws, ws_bytes, L, d, B, T, s);
        if (rr) return rr;
        if (cudaEventRecord(e0, s) != cudaSuccess) return MSC_ERR_CUDA;
        for (int i = 0; i < reps && !rr; ++i) rr = run_batch(ws, ws_bytes, L, d, B, T, s);
        if (rr) return rr;
        if (cudaEventRecord(e1, s) != cudaSuccess) return MSC_ERR_CUDA;
        if (cudaMemsetAsync(d.checksum, 0, sizeof(unsigned long long), s) != cudaSuccess) return MSC_ERR_CUDA;
        {
            TraceScope ts_("batch.checksum", s);
            k_batch_checksum<<<current_device().sms * 4, kThreads, 0, s>>>(order, asc, desc, ms, L.total, num_cells,
                                                                          L.count, d.checksum);
        }
        MSC_LAUNCHED();
        unsigned long long h = 0;
        int32_t st = 0;
        if (cudaMemcpyAsync(&h, d.checksum, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&st, d_status, sizeof st, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return MSC_ERR_CUDA;
        if (st != MSC_OK) return st;
        if (!have_ref) {
            ref = h;
            have_ref = true;
        } else if (h != ref) {
            return MSC_ERR_INTERNAL;  // a tuning changed the result
        }
        float t = 0.f;
        if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) return MSC_ERR_CUDA;
        *ms_out = t / reps;
        return MSC_OK;
    };
    Tune cur;
    float cur_ms = 0.f;
    r = measure(cur, &cur_ms);
    for (int k = 1; k < kShapes && !r; ++k) {  // tile shape, at the default threshold
        Tune t = cur;
        t.shape = k;
        float m = 0.f;
        r = measure(t, &m);
        if (!r && m < cur_ms) {
            cur = t;
            cur_ms = m;
        }
    }
    const int shifts[] = {2, 4, 5, 6};
    const int shape = cur.shape;
    for (int k = 0; k < 4 && !r; ++k) {  // active-list threshold, best shape
        Tune t;
        t.shape = shape;
        t.build_shift = shifts[k];
        float m = 0.f;
        r = measure(t, &m);
        if (!r && m < cur_ms) {
            cur = t;
            cur_ms = m;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r) return r;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tuned[signature(grids, count)] = cur;
    }
    if (best) {
        best->steepest_shape = cur.shape;
        best->build_shift = cur.build_shift;
    }
    if (best_ms) *best_ms = cur_ms;
    return MSC_OK;
}

}  // extern "C"
