// Launch counting and optional per-kernel CUDA-event tracing.
//
// Every kernel launch of the library goes through a TraceScope: it bumps a
// process-wide launch counter and, while tracing is enabled, records a pair
// of CUDA events on the launching stream around the launch.  The events
// come from a pool that grows on demand and is recycled by msc_trace_reset.
// msc_trace_collect synchronises on the recorded events and reports, per
// label, the number of launches and the summed device time.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "msc_trace.h"

namespace msc {
namespace {

struct Rec {
    const char* label;
    cudaEvent_t a, b;
};

std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_on{0};
std::mutex g_mu;
std::vector<cudaEvent_t> g_pool;
size_t g_next = 0;
std::vector<Rec> g_recs;

cudaEvent_t take_event() {
    if (g_next == g_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        g_pool.push_back(e);
    }
    return g_pool[g_next++];
}

}  // namespace

TraceScope::TraceScope(const char* label, cudaStream_t s) : label_(label), stream_(s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_on.load(std::memory_order_relaxed)) return;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return;  // launches captured into a graph are not timed one by one
    std::lock_guard<std::mutex> lock(g_mu);
    a_ = take_event();
    b_ = take_event();
    if (a_ && b_) cudaEventRecord(a_, stream_);
}

TraceScope::~TraceScope() {
    if (!a_ || !b_) return;
    cudaEventRecord(b_, stream_);
    std::lock_guard<std::mutex> lock(g_mu);
    g_recs.push_back({label_, a_, b_});
}

void add_launches(long long k) {
    g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed);
}

unsigned long long launch_count() { return g_launches.load(); }

}  // namespace msc

using namespace msc;

extern "C" {

MSC_API unsigned long long msc_launch_count(void) { return g_launches.load(); }

MSC_API void msc_trace_enable(int on) { g_on.store(on ? 1 : 0); }

MSC_API void msc_trace_reset(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_recs.clear();
    g_next = 0;
}

MSC_API int msc_trace_collect(char* buf, size_t cap) {
    std::lock_guard<std::mutex> lock(g_mu);
    std::map<std::string, std::pair<long, double>> agg;
    for (const Rec& r : g_recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) return MSC_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return MSC_ERR_CUDA;
        auto& e = agg[r.label];
        e.first += 1;
        e.second += ms;
    }
    std::string out = "{";
    bool first = true;
    for (const auto& kv : agg) {
        char item[256];
        std::snprintf(item, sizeof item, "%s\"%s\": [%ld, %.6f]", first ? "" : ", ", kv.first.c_str(),
                      kv.second.first, kv.second.second);
        out += item;
        first = false;
    }
    out += "}";
    if (out.size() + 1 > cap) return MSC_ERR_ARG;
    std::memcpy(buf, out.c_str(), out.size() + 1);
    return MSC_OK;
}

}  // extern "C"
