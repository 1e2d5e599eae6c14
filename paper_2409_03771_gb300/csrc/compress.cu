// Path compression by pointer doubling (Alg. 1 compression loop): every
// active vertex v does u <- d[v], w <- d[u]; if u = w it is finished,
// otherwise d[v] <- w.  As in the paper the update is in place: a read of
// d[u] may already see this sweep's write, which only lengthens the jump.
//
// GPU form: one launch per sweep over all vertices (eight vertices per
// thread, lane-consecutive).  Each vertex follows up to kHops (4) hops per
// sweep (d[v] <- d[d[d[d[d[v]]]]]), so a sweep at least quintuples every
// pointer's reach for the same 8 bytes of pointer read and write per
// vertex; the extra reads mostly hit the cache.  Launched ceil(log5 n) + 2
// times.  Each sweep counts the vertices it changed; a sweep whose
// predecessor changed nothing returns at once, so no host synchronisation
// is needed.  A sweep also appends the vertices it changed to an active
// list (block-aggregated atomics) once the previous sweep's count is at
// most 1.5x the list's capacity (a vertex that did not move never moves
// again, so the count can only fall); when the changes still overflow the
// list, the next sweep walks all vertices instead.  The following sweeps
// walk only the list -- the GPU counterpart of the paper's per-thread
// active lists.  (With fill_lists off, the list is built only once at most
// n >> build_shift vertices changed, which never overflows.)  A pointer
// cycle is reported as MSC_ERR_NOT_CONVERGED: either a hop lands on its
// own vertex, or the last sweep still changes something.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "compress.cuh"

namespace msc {
namespace {

constexpr int kThreads = 256;

struct JumpArray {
    int32_t* p;
    JumpCtl* ctl;
    int32_t* list0;
    int32_t* list1;
    int64_t list_cap;  // entries of list0 and of list1
};

struct JumpPair {
    JumpArray a[2];
    int32_t n;
    uint32_t* roots;  // optional: roots[i] += #vertices of array i that point at themselves
};

#ifndef MSC_JUMP_HOPS
#define MSC_JUMP_HOPS 4
#endif
constexpr int kHops = MSC_JUMP_HOPS;  // pointer hops followed per vertex and sweep
constexpr int kPerThread = 8;  // vertices per thread and chunk
constexpr int kChunkV = kThreads * kPerThread;

// Up to kHops hops for each of a thread's vertices vid[j] (current
// pointers d[j]); bit j of the result is set when d[j] changed.  The hops
// advance all vertices together, so a thread keeps kPerThread independent
// gathers in flight instead of walking one chain at a time.  Every value
// read is an ancestor of the vertex on its path, so in-place reads of
// pointers already moved in this sweep only lengthen the jump: after s
// sweeps a vertex has advanced at least (kHops + 1)^s steps.  In a forest a
// hop always lands on a strict ancestor, so landing on the vertex itself
// can only happen on a pointer cycle (in-place jumping can collapse a
// cycle into such a self-loop, which would otherwise look converged).
//
// CHECKED = false (pointers made by the stencil kernels: in range and
// acyclic by construction, since order strictly increases along them)
// drops the per-hop range and cycle tests.
template <bool CHECKED>
__device__ __forceinline__ uint32_t jump_group(const int32_t* p, int32_t n, const int32_t (&vid)[kPerThread],
                                               int32_t (&d)[kPerThread], uint32_t valid, int32_t* status) {
    uint32_t live = 0, moved = 0;
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        if (!(valid >> j & 1u) || d[j] < 0) continue;
        if (CHECKED && (uint32_t)d[j] >= (uint32_t)n) {
            record_error(status, MSC_ERR_ARG);
            continue;
        }
        live |= 1u << j;
    }
#pragma unroll
    for (int h = 0; h < kHops; ++h) {
        if (h > 0 && !__any_sync(0xffffffffu, live)) break;  // the warp's chains all ended
        int32_t w[kPerThread];
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) w[j] = (live >> j & 1u) ? p[d[j]] : 0;
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) {
            if (!(live >> j & 1u)) continue;
            const int32_t u = d[j];
            if (w[j] == u) {
                live &= ~(1u << j);  // u is a root: done
            } else if (CHECKED && (uint32_t)w[j] >= (uint32_t)n) {
                record_error(status, MSC_ERR_ARG);  // out of range or inactive target
                live &= ~(1u << j);
            } else if (CHECKED && w[j] == vid[j]) {
                record_error(status, MSC_ERR_NOT_CONVERGED);
                live &= ~(1u << j);
            } else {
                d[j] = w[j];
                moved |= 1u << j;
            }
        }
    }
    return moved;
}

template <bool CHECKED>
__global__ void __launch_bounds__(kThreads) k_jump(const JumpPair pr, int step, uint32_t build_max,
                                                   int32_t* status) {
    const JumpArray A = blockIdx.y ? pr.a[1] : pr.a[0];
    const int32_t n = pr.n;
    int32_t* p = A.p;
    const uint32_t prev = step == 0 ? (uint32_t)n : A.ctl->cnt[step - 1];
    if (prev == 0) return;
    // the previous sweep's list is complete only if its changes fitted
    const bool from_list = step > 0 && A.ctl->built[step - 1] != 0 && (int64_t)prev <= A.list_cap;
    const bool build = prev <= build_max;
    if (build && blockIdx.x == 0 && threadIdx.x == 0) A.ctl->built[step] = 1u;
    int32_t* out_list = (step & 1) ? A.list1 : A.list0;
    const int32_t* in_list = (step & 1) ? A.list0 : A.list1;

    __shared__ uint32_t s_warp[kThreads / 32];
    __shared__ uint32_t s_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t total = from_list ? (int64_t)prev : (int64_t)n;
    const int64_t nchunks = (total + kChunkV - 1) / kChunkV;
    uint32_t changed_total = 0, roots_seen = 0;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        int32_t vid[kPerThread], d[kPerThread];
        uint32_t valid = 0, ch;
        // element j of the thread is vertex (or list entry) c*chunk + j*256 + tid:
        // the 32 lanes of every load, gather and store touch consecutive
        // vertices, whose pointers (and the pointers' pointers) are
        // neighbours, so each warp access covers few sectors
        if (!from_list) {
            const int64_t v0 = c * kChunkV + tid;
#pragma unroll
            for (int j = 0; j < kPerThread; ++j) {
                const int64_t v = v0 + (int64_t)j * kThreads;
                vid[j] = (int32_t)v;
                d[j] = v < n ? p[v] : -1;
                valid |= (v < n ? 1u : 0u) << j;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kPerThread; ++j) {
                const int64_t i = c * kChunkV + (int64_t)j * kThreads + tid;
                vid[j] = -1;
                if (i < total) {
                    const int32_t v = in_list[i];
                    MSC_GUARD((uint32_t)v < (uint32_t)n, status, -121) {
                        vid[j] = v;
                        valid |= 1u << j;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < kPerThread; ++j) d[j] = (valid >> j & 1u) ? p[vid[j]] : -1;
        }
        if (step == 0 && pr.roots) {  // the first sweep sees every pointer: count the roots
            uint32_t r = 0;
#pragma unroll
            for (int j = 0; j < kPerThread; ++j) r += (valid >> j & 1u) && d[j] == vid[j];
            roots_seen += r;
        }
        ch = jump_group<CHECKED>(p, n, vid, d, valid, status);
#pragma unroll
        for (int j = 0; j < kPerThread; ++j)
            if (ch >> j & 1u) p[vid[j]] = d[j];
        const uint32_t cnt = __popc(ch);
        changed_total += cnt;
        if (build) {  // append the changed vertices; trip count is block-uniform
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
                s_base = run ? atomicAdd(&A.ctl->cnt[step], run) : 0u;
            }
            __syncthreads();
            uint32_t off = s_base + s_warp[warp] + incl - cnt;
#pragma unroll
            for (int j = 0; j < kPerThread; ++j)
                if (ch & (1u << j)) {
                    if ((int64_t)off < A.list_cap) out_list[off] = vid[j];  // past it: the list is dropped
                    ++off;
                }
            __syncthreads();
        }
    }
    if (!build) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) changed_total += __shfl_xor_sync(0xffffffffu, changed_total, o);
        if (lane == 0 && changed_total) atomicAdd(&A.ctl->cnt[step], changed_total);
    }
    if (step == 0 && pr.roots) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) roots_seen += __shfl_xor_sync(0xffffffffu, roots_seen, o);
        if (lane == 0 && roots_seen) atomicAdd(&pr.roots[blockIdx.y], roots_seen);
    }
}

__global__ void k_jump_finish(const JumpPair pr, int count, int last, int32_t* status) {
    for (int i = 0; i < count; ++i)
        if (pr.a[i].ctl->cnt[last] != 0u) record_error(status, MSC_ERR_NOT_CONVERGED);
}

}  // namespace

// Sweeps for n vertices: enough for a path of n vertices at a (kHops+1)-fold
// advance per sweep, plus two; more are needed only by a pointer cycle.
int compress_steps(int64_t n) {
    int s = 0;
    for (int64_t reach = 1; reach < std::max<int64_t>(n, 2); reach *= (kHops + 1)) ++s;
    return std::min(kMaxJumpSteps, s + 2);
}

static int64_t list_capacity(int64_t n) { return n / 2 + 1; }

void size_compress_scratch(Sizer& s, int64_t n, int count) {
    s.take<JumpCtl>(count);
    s.take<int32_t>((size_t)count * 2 * list_capacity(n));
}

CompressScratch carve_compress_scratch(Carver& c, int64_t n, int count) {
    CompressScratch sc;
    sc.ctl = c.take<JumpCtl>(count);
    sc.list_cap = list_capacity(n);
    sc.lists = c.take<int32_t>((size_t)count * 2 * sc.list_cap);
    return sc;
}

int run_compress(int32_t* const* ptrs, int count, int32_t n, const CompressScratch& sc,
                 int32_t* status, cudaStream_t s, const CompressTune& tune) {
    if (n <= 0 || count < 1 || count > 2) return n < 0 ? MSC_ERR_ARG : MSC_OK;
    MSC_TRY(cudaMemsetAsync(sc.ctl, 0, sizeof(JumpCtl) * count, s));
    JumpPair pr{};
    pr.n = n;
    pr.roots = tune.roots;
    for (int i = 0; i < count; ++i) {
        pr.a[i].p = ptrs[i];
        pr.a[i].ctl = sc.ctl + i;
        pr.a[i].list0 = sc.lists + (size_t)i * 2 * sc.list_cap;
        pr.a[i].list1 = pr.a[i].list0 + sc.list_cap;
        pr.a[i].list_cap = sc.list_cap;
    }
    const int build_shift = std::max(1, std::min(tune.build_shift, 30));
    const int64_t fill_max = std::min<int64_t>(sc.list_cap + sc.list_cap / 2, UINT32_MAX);
    const uint32_t build_max = tune.fill_lists ? (uint32_t)fill_max : ((uint32_t)n >> build_shift);
    auto kern = tune.trusted ? k_jump<false> : k_jump<true>;
    int occ = 1;
    MSC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, 0));
    const int64_t chunks = ceil_div(n, kChunkV);
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(chunks, (int64_t)current_device().sms * std::max(occ, 1)));
    const int steps = compress_steps(n);
    for (int st = 0; st < steps; ++st) {
        {
            TraceScope ts_("compress.jump", s);
            kern<<<dim3(gx, count), kThreads, 0, s>>>(pr, st, build_max, status);
        }
        MSC_LAUNCHED();
    }
    {
        TraceScope ts_("compress.finish", s);
        k_jump_finish<<<1, 1, 0, s>>>(pr, count, steps - 1, status);
    }
    MSC_LAUNCHED();
    return MSC_OK;
}

}  // namespace msc

// ----------------------------------------------------------------------------
// msc_compress_noalloc: the same compression for callers that cannot
// allocate device memory.  Its scratch (the step counters and the two active
// lists) is this file-scope array, which every GPU that loads the library
// holds until the process exits.  The active list is built once at most
// n/16 vertices changed, so two lists of n_max/16 + 1 entries suffice.

namespace {

constexpr int64_t kNoAllocMaxN = MSC_NOALLOC_MAX_N;
constexpr int kNoAllocBuildShift = 4;
constexpr int64_t kNoAllocListCap = (kNoAllocMaxN >> kNoAllocBuildShift) + 1;
constexpr size_t kNoAllocCtlBytes = (sizeof(msc::JumpCtl) + 255) & ~size_t(255);
constexpr size_t kNoAllocBytes = kNoAllocCtlBytes + 2 * kNoAllocListCap * sizeof(int32_t);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch, looked up once per device with that
// device current (a host-side use of the symbol's name is not a device
// address).
int noalloc_scratch(void** out) {
    static void* addr[64] = {};
    static std::mutex mu;
    int dev = 0;
    MSC_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return MSC_ERR_ARG;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        MSC_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        addr[dev] = p;
    }
    *out = addr[dev];
    return MSC_OK;
}

}  // namespace

extern "C" MSC_API int msc_compress_noalloc(int32_t* ptr, int32_t n, int32_t* d_status, void* stream) {
    if (n < 0 || !d_status || (n > 0 && !ptr)) return MSC_ERR_ARG;
    if ((int64_t)n > kNoAllocMaxN) return MSC_ERR_TOO_LARGE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* base = nullptr;
    int r = noalloc_scratch(&base);
    if (r) return r;
    MSC_TRY(cudaMemsetAsync(d_status, 0, sizeof(int32_t), s));
    if (n == 0) return MSC_OK;
    msc::CompressScratch sc;
    sc.ctl = static_cast<msc::JumpCtl*>(base);  // zeroed by run_compress
    sc.list_cap = kNoAllocListCap;
    sc.lists = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(base) + kNoAllocCtlBytes);
    msc::CompressTune tune;
    tune.build_shift = kNoAllocBuildShift;
    tune.fill_lists = false;
    int32_t* arr[1] = {ptr};
    return msc::run_compress(arr, 1, n, sc, d_status, s, tune);
}
