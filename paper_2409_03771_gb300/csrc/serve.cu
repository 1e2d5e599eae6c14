// Request server with continuous batching (include/msc.h, msc_server_*).
//
// One scheduler thread owns admission.  Requests wait in a FIFO; the head
// is admitted when a slot is free and its device memory fits in the arena,
// so no request starves.  When the head is a small segmentation, the small
// segmentations among the next kLookAhead waiting requests join it (larger
// requests keep their places) and run as one batched launch over a packed
// copy of their inputs; every other request runs on its own.  A slot has
// two streams: requests of at least kBigRequest vertices -- the ones that
// set the tail latency -- run on the high-priority one, so that work
// overlapping them on other slots fills idle SMs instead of slowing them.
// Completion is signalled by a host function enqueued after the request's
// work on its stream (it only takes a mutex and notifies), and the
// scheduler then frees the slot; a request's outputs stay in the arena
// until msc_server_release.  CUDA work is issued outside the state lock.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace msc {
namespace {

constexpr int kMaxGroup = 256;        // requests in one batched launch
constexpr size_t kLookAhead = 64;     // waiting requests a group may be drawn from
constexpr int64_t kBigRequest = int64_t(1) << 24;  // vertices: high-priority stream
constexpr int64_t kGroupTotal = 1 << 28;  // vertices in one batched launch
constexpr size_t kAlign = 256;

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over the arena (offsets), coalescing on free.
class Arena {
   public:
    void reset(size_t bytes) {
        free_.clear();
        free_[0] = bytes;
        used_ = 0;
        cap_ = bytes;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = align_up(std::max<size_t>(bytes, 1));
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used_ += bytes;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align_up(std::max<size_t>(bytes, 1));
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t capacity() const { return cap_; }

   private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0, cap_ = 0;
};

struct Block {
    size_t off = 0, bytes = 0;
    int refs = 0;
};

struct Req {
    uint64_t ticket = 0;
    msc_job job{};
    int64_t n = 0;
    int status = MSC_PENDING;
    int32_t cells = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    Block* block = nullptr;
    int32_t *order = nullptr, *asc = nullptr, *desc = nullptr, *ms = nullptr, *label = nullptr;
    int group = 1;
    bool done = false;
    bool solo_only = false;  // its group failed: run it alone to get its own status
};

struct Slot {
    cudaStream_t stream = nullptr;     // low priority: batched and smaller requests
    cudaStream_t stream_hi = nullptr;  // high priority: requests of >= kBigRequest vertices
    int32_t* h_info = nullptr;  // pinned: [0] status, [1 + i] cells of request i
    bool busy = false;
};

struct Launch;

// Per-request device memory of a solo run.
size_t solo_bytes(const msc_job& j, int64_t n) {
    if (j.kind == MSC_JOB_SEGMENT)
        return 4 * align_up((size_t)n * 4) + 2 * kAlign + align_up(msc_workspace_bytes(MSC_OP_SEGMENT, n, 0));
    return align_up((size_t)n * 4) + kAlign + align_up(msc_workspace_bytes(MSC_OP_CC_MASK, n, 0));
}

}  // namespace
}  // namespace msc

using namespace msc;

struct msc_server {
    std::mutex mu;
    std::condition_variable cv;       // scheduler wake-ups
    std::condition_variable done_cv;  // waiters in msc_server_wait
    std::thread thread;
    bool stop = false;
    char* base = nullptr;
    Arena arena;
    uint64_t mem_version = 0, failed_version = ~0ull;
    int64_t group_max = 0;
    std::vector<Slot> slots;
    std::deque<Req*> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    std::vector<Launch*> completed;
    uint64_t next_ticket = 1;
    int running = 0, finished = 0;
    int big_running = 0;  // launches of >= kBigRequest vertices on the GPU
};

namespace msc {
namespace {

struct Launch {
    msc_server* srv;
    int slot;
    std::vector<Req*> reqs;
    Block* block;
    int host_error = MSC_OK;  // a launch that failed on the host
    double t_done = 0;
    bool hi = false;          // issued on the slot's high-priority stream
};

void CUDART_CB on_done(void* p) {  // CUDA host function: no CUDA calls here
    Launch* L = static_cast<Launch*>(p);
    std::lock_guard<std::mutex> lock(L->srv->mu);
    L->t_done = now_s();
    L->srv->completed.push_back(L);
    L->srv->cv.notify_all();
}

// Carve helpers over an arena block.
struct BlockCarver {
    char* p;
    size_t used = 0;
    template <typename T>
    T* take(size_t count) {
        T* r = reinterpret_cast<T*>(p + used);
        used += align_up(std::max<size_t>(count * sizeof(T), 1));
        return r;
    }
};

// Enqueue the work of an admitted launch on its slot (no lock held).
int issue(msc_server* S, Launch* L) {
    Slot& sl = S->slots[L->slot];
    cudaStream_t st = L->hi ? sl.stream_hi : sl.stream;
    BlockCarver c{S->base + L->block->off};
    const int k = (int)L->reqs.size();
    int r = MSC_OK;
    int32_t *status = nullptr, *cells = nullptr;
    if (k == 1 && L->reqs[0]->job.kind == MSC_JOB_CC_MASK) {
        Req* q = L->reqs[0];
        q->label = c.take<int32_t>(q->n);
        status = c.take<int32_t>(1);
        const size_t wsb = msc_workspace_bytes(MSC_OP_CC_MASK, q->n, 0);
        void* ws = c.take<char>(wsb);
        r = msc_cc_mask(static_cast<const uint8_t*>(q->job.input), q->job.g, q->job.conn, q->label, ws, wsb, status,
                        st);
    } else if (k == 1) {
        Req* q = L->reqs[0];
        q->order = c.take<int32_t>(q->n);
        q->asc = c.take<int32_t>(q->n);
        q->desc = c.take<int32_t>(q->n);
        q->ms = c.take<int32_t>(q->n);
        cells = c.take<int32_t>(1);
        status = c.take<int32_t>(1);
        const size_t wsb = msc_workspace_bytes(MSC_OP_SEGMENT, q->n, 0);
        void* ws = c.take<char>(wsb);
        r = msc_segment(static_cast<const float*>(q->job.input), q->job.g, q->order, q->asc, q->desc, q->ms, cells,
                        ws, wsb, status, st);
    } else {
        std::vector<msc_grid> grids(k);
        int64_t total = 0;
        for (int i = 0; i < k; ++i) {
            grids[i] = L->reqs[i]->job.g;
            total += L->reqs[i]->n;
        }
        float* f = c.take<float>(total);
        int32_t* order = c.take<int32_t>(total);
        int32_t* asc = c.take<int32_t>(total);
        int32_t* desc = c.take<int32_t>(total);
        int32_t* ms = c.take<int32_t>(total);
        cells = c.take<int32_t>(k);
        status = c.take<int32_t>(1);
        const size_t wsb = msc_batch_workspace_bytes(grids.data(), k);
        void* ws = c.take<char>(wsb);
        int64_t off = 0;
        for (int i = 0; i < k && r == MSC_OK; ++i) {
            Req* q = L->reqs[i];
            if (cudaMemcpyAsync(f + off, q->job.input, (size_t)q->n * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                r = MSC_ERR_CUDA;
            q->order = order + off;
            q->asc = asc + off;
            q->desc = desc + off;
            q->ms = ms + off;
            off += q->n;
        }
        if (r == MSC_OK)
            r = msc_batch_segment(grids.data(), k, f, order, asc, desc, ms, cells, ws, wsb, nullptr, status, st);
    }
    if (r == MSC_OK && cudaMemcpyAsync(sl.h_info, status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        r = MSC_ERR_CUDA;
    if (r == MSC_OK && cells &&
        cudaMemcpyAsync(sl.h_info + 1, cells, (size_t)k * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        r = MSC_ERR_CUDA;
    if (r == MSC_OK && cudaLaunchHostFunc(st, on_done, L) != cudaSuccess) r = MSC_ERR_CUDA;
    return r;
}

void finish(msc_server* S, Launch* L) {  // lock held
    Slot& sl = S->slots[L->slot];
    S->big_running -= L->hi;
    const int k = (int)L->reqs.size();
    if (k > 1 && L->host_error == MSC_OK && sl.h_info[0] != MSC_OK) {
        // A batched launch shares one status word: re-run its requests one
        // by one, ahead of the queue, so that each gets its own status.
        for (int i = k - 1; i >= 0; --i) {
            Req* q = L->reqs[i];
            q->solo_only = true;
            q->block = nullptr;
            q->order = q->asc = q->desc = q->ms = nullptr;
            S->queue.push_front(q);
        }
        S->arena.release(L->block->off, L->block->bytes);
        delete L->block;
        ++S->mem_version;
        sl.busy = false;
        S->running -= k;
        delete L;
        return;
    }
    for (int i = 0; i < k; ++i) {
        Req* q = L->reqs[i];
        q->status = L->host_error != MSC_OK ? L->host_error : sl.h_info[0];
        q->cells = (q->job.kind == MSC_JOB_SEGMENT && L->host_error == MSC_OK) ? sl.h_info[1 + i] : 0;
        q->t_done = L->t_done;
        q->done = true;
    }
    sl.busy = false;
    S->running -= k;
    S->finished += k;
    delete L;
}

int free_slot(msc_server* S) {
    for (size_t i = 0; i < S->slots.size(); ++i)
        if (!S->slots[i].busy) return (int)i;
    return -1;
}

bool groupable(const msc_server* S, const Req* q) {
    return q->job.kind == MSC_JOB_SEGMENT && q->n <= S->group_max && !q->solo_only;
}

// Pick the next launch from the head of the queue (lock held); nullptr if
// the head does not fit now.  A small segmentation at the head takes the
// small segmentations among the next kLookAhead requests with it.
Launch* admit(msc_server* S, int slot) {
    Req* head = S->queue.front();
    std::vector<size_t> take{0};  // queue positions
    size_t bytes = solo_bytes(head->job, head->n);
    auto group_bytes = [&](const std::vector<size_t>& pos) {
        std::vector<msc_grid> grids;
        int64_t total = 0;
        for (size_t i : pos) {
            grids.push_back(S->queue[i]->job.g);
            total += S->queue[i]->n;
        }
        const int k = (int)pos.size();
        return 5 * align_up((size_t)total * 4) + 2 * kAlign + align_up((size_t)k * 4) +
               align_up(msc_batch_workspace_bytes(grids.data(), k));
    };
    if (groupable(S, head)) {
        int64_t total = head->n;
        const size_t window = std::min(S->queue.size(), kLookAhead + 1);
        for (size_t i = 1; i < window && (int)take.size() < kMaxGroup; ++i) {
            Req* q = S->queue[i];
            if (!groupable(S, q) || total + q->n > kGroupTotal) continue;  // keeps its place
            take.push_back(i);
            total += q->n;
        }
        if (take.size() > 1) {
            bytes = group_bytes(take);
            // shrink the group until it fits (at least the head alone)
            while (bytes > S->arena.capacity() - S->arena.used() && take.size() > 1) {
                take.pop_back();
                bytes = take.size() == 1 ? solo_bytes(head->job, head->n) : group_bytes(take);
            }
        }
    }
    size_t off = 0;
    if (!S->arena.alloc(bytes, &off)) {
        if (take.size() == 1) return nullptr;
        take.resize(1);  // a fragmented arena: the head alone may still fit
        bytes = solo_bytes(head->job, head->n);
        if (!S->arena.alloc(bytes, &off)) return nullptr;
    }
    std::vector<Req*> reqs;
    for (size_t i : take) reqs.push_back(S->queue[i]);
    Block* b = new Block{off, bytes, (int)reqs.size()};
    Launch* L = new Launch{S, slot, reqs, b, MSC_OK, 0};
    L->hi = reqs.size() == 1 && head->n >= kBigRequest;
    S->big_running += L->hi;
    const double t = now_s();
    for (Req* q : reqs) {
        q->block = b;
        q->t_start = t;
        q->group = (int)reqs.size();
    }
    for (size_t j = take.size(); j-- > 0;) S->queue.erase(S->queue.begin() + (std::ptrdiff_t)take[j]);
    S->slots[slot].busy = true;
    S->running += (int)reqs.size();
    return L;
}

// Under light load (a short queue) a large request runs without newcomers:
// overlapping work would only slow the request that sets the tail latency.
// Under load the queue grows and everything overlaps for throughput.  The
// hold lifts when the large request completes or the queue grows (both
// wake the scheduler).
bool hold_back(const msc_server* S) {
#ifdef MSC_SERVE_NO_HOLD
    return false;
#else
    return S->big_running > 0 && S->queue.size() <= S->slots.size();
#endif
}

void scheduler(msc_server* S, int device) {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(S->mu);
    for (;;) {
        // every state in which the admission loop below admits nothing must
        // make this predicate false, or the thread would spin holding the
        // lock that the completion callbacks need
        S->cv.wait(lock, [&] {
            return (S->stop && S->running == 0) || !S->completed.empty() ||
                   (!S->stop && !S->queue.empty() && free_slot(S) >= 0 && S->failed_version != S->mem_version &&
                    !hold_back(S));
        });
        if (!S->completed.empty()) {
            for (Launch* L : S->completed) finish(S, L);
            S->completed.clear();
            S->done_cv.notify_all();
        }
        if (S->stop && S->running == 0) break;
        if (S->stop) continue;
        std::vector<Launch*> launches;
        int slot;
        while (!S->queue.empty() && (slot = free_slot(S)) >= 0 && !hold_back(S)) {
            Launch* L = admit(S, slot);
            if (!L) {
                S->failed_version = S->mem_version;  // retry after a release
                break;
            }
            launches.push_back(L);
        }
        if (launches.empty()) continue;
        lock.unlock();
        std::vector<Launch*> failed;
        for (Launch* L : launches) {
            const int r = issue(S, L);
            if (r != MSC_OK) {  // nothing will call on_done for it
                L->host_error = r;
                L->t_done = now_s();
                failed.push_back(L);
            }
        }
        lock.lock();
        for (Launch* L : failed) S->completed.push_back(L);
    }
}

void fill_result(const Req* q, msc_result* out) {
    out->status = q->status;
    out->num_cells = q->cells;
    out->n = q->n;
    const bool ok = q->done && q->status == MSC_OK;
    out->order = ok ? q->order : nullptr;
    out->asc = ok ? q->asc : nullptr;
    out->desc = ok ? q->desc : nullptr;
    out->ms = ok ? q->ms : nullptr;
    out->label = ok ? q->label : nullptr;
    out->t_submit = q->t_submit;
    out->t_start = q->t_start;
    out->t_done = q->t_done;
    out->group_size = q->group;
}

}  // namespace
}  // namespace msc

extern "C" {

msc_server* msc_server_create(size_t hbm_budget, int32_t slots, int64_t group_max_vertices) {
    if (hbm_budget < kAlign || slots < 1 || slots > 16 || group_max_vertices < 0) return nullptr;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return nullptr;
    auto S = std::make_unique<msc_server>();
    hbm_budget &= ~(kAlign - 1);
    if (cudaMalloc(&S->base, hbm_budget) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    S->arena.reset(hbm_budget);
    S->group_max = group_max_vertices;
    S->slots.resize(slots);
    int lo_prio = 0, hi_prio = 0;
    bool ok = cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio) == cudaSuccess;
    for (Slot& sl : S->slots) {
        ok = ok && cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking, lo_prio) == cudaSuccess;
        ok = ok && cudaStreamCreateWithPriority(&sl.stream_hi, cudaStreamNonBlocking, hi_prio) == cudaSuccess;
        ok = ok && cudaMallocHost(&sl.h_info, (1 + kMaxGroup) * sizeof(int32_t)) == cudaSuccess;
    }
    if (!ok) {
        for (Slot& sl : S->slots) {
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.stream_hi) cudaStreamDestroy(sl.stream_hi);
            if (sl.h_info) cudaFreeHost(sl.h_info);
        }
        cudaFree(S->base);
        return nullptr;
    }
    msc_server* s = S.release();
    s->thread = std::thread(scheduler, s, device);
    return s;
}

int msc_server_submit(msc_server* s, const msc_job* job, uint64_t* ticket) {
    if (!s || !job || !ticket) return MSC_ERR_ARG;
    const msc_grid g = job->g;
    if (g.nx <= 0 || g.ny <= 0 || g.nz <= 0 || !job->input) return MSC_ERR_ARG;
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    if (n > INT32_MAX) return MSC_ERR_ARG;
    if (job->kind != MSC_JOB_SEGMENT && job->kind != MSC_JOB_CC_MASK) return MSC_ERR_ARG;
    if (job->kind == MSC_JOB_CC_MASK && job->conn != 6 && job->conn != 14) return MSC_ERR_ARG;
    if (solo_bytes(*job, n) > s->arena.capacity()) return MSC_ERR_BUDGET;
    auto q = std::make_unique<Req>();
    q->job = *job;
    q->n = n;
    q->t_submit = now_s();
    std::lock_guard<std::mutex> lock(s->mu);
    q->ticket = s->next_ticket++;
    *ticket = q->ticket;
    s->queue.push_back(q.get());
    s->reqs.emplace(q->ticket, std::move(q));
    s->cv.notify_all();
    return MSC_OK;
}

int msc_server_poll(msc_server* s, uint64_t ticket, msc_result* out) {
    if (!s || !out) return MSC_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return MSC_ERR_ARG;
    fill_result(it->second.get(), out);
    return it->second->done ? MSC_OK : MSC_PENDING;
}

int msc_server_wait(msc_server* s, uint64_t ticket, double timeout_ms, msc_result* out) {
    if (!s || !out) return MSC_ERR_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return MSC_ERR_ARG;
    Req* q = it->second.get();
    auto ready = [&] { return q->done; };
    if (timeout_ms < 0)
        s->done_cv.wait(lock, ready);
    else
        s->done_cv.wait_for(lock, std::chrono::duration<double, std::milli>(timeout_ms), ready);
    fill_result(q, out);
    return q->done ? MSC_OK : MSC_PENDING;
}

int msc_server_release(msc_server* s, uint64_t ticket) {
    if (!s) return MSC_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return MSC_ERR_ARG;
    Req* q = it->second.get();
    if (!q->done) return MSC_PENDING;
    if (q->block && --q->block->refs == 0) {
        s->arena.release(q->block->off, q->block->bytes);
        delete q->block;
        ++s->mem_version;
        s->cv.notify_all();
    }
    s->reqs.erase(it);
    return MSC_OK;
}

int msc_server_stats(msc_server* s, size_t* arena_used, int32_t* queued, int32_t* running, int32_t* done) {
    if (!s) return MSC_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    if (arena_used) *arena_used = s->arena.used();
    if (queued) *queued = (int32_t)s->queue.size();
    if (running) *running = s->running;
    if (done) *done = s->finished;
    return MSC_OK;
}

void msc_server_destroy(msc_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        for (Req* q : s->queue) {  // never admitted: complete them as cancelled
            q->status = MSC_ERR_ARG;
            q->done = true;
        }
        s->queue.clear();
        s->cv.notify_all();
    }
    if (s->thread.joinable()) s->thread.join();  // returns once running work completed
    for (Slot& sl : s->slots) {
        cudaStreamSynchronize(sl.stream);
        cudaStreamSynchronize(sl.stream_hi);
        cudaStreamDestroy(sl.stream);
        cudaStreamDestroy(sl.stream_hi);
        cudaFreeHost(sl.h_info);
    }
    for (auto& kv : s->reqs) {
        Req* q = kv.second.get();
        if (q->block && --q->block->refs == 0) delete q->block;
    }
    cudaFree(s->base);
    delete s;
}

}  // extern "C"
