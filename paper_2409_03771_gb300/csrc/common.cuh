// Internal helpers shared by the sm_103a kernels of the msc library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "msc.h"

namespace msc {

constexpr int kWarp = 32;

// ----------------------------------------------------------------------------
// device status word: the first error recorded wins
__device__ __forceinline__ void record_error(int32_t* status, int32_t code) {
    if (status) atomicCAS(status, MSC_OK, code);
}

// Debug builds (-DMSC_DEBUG_BOUNDS) check data-dependent addresses before
// the access: a violation records `code` in the status word and skips the
// access.  Release builds compile the check away.
#if defined(MSC_DEBUG_BOUNDS) || defined(MSC_GUARDS)
#define MSC_GUARD(cond, status, code) if (!(cond)) record_error((status), (code)); else
#else
#define MSC_GUARD(cond, status, code)
#endif

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_volatile_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.volatile.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int32_t ld_volatile_s32(const int32_t* p) {
    int32_t v;
    asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// ----------------------------------------------------------------------------
// host side
struct Device {
    int id = -1;
    int sms = 0;
    int max_smem_optin = 0;
};

// Counts one kernel launch and, while tracing is on, brackets it with CUDA
// events on its stream (see trace.cu).  Construct right before the launch
// and let it go out of scope right after.
class TraceScope {
   public:
    TraceScope(const char* label, cudaStream_t s);
    ~TraceScope();
    TraceScope(const TraceScope&) = delete;
    TraceScope& operator=(const TraceScope&) = delete;

   private:
    const char* label_;
    cudaStream_t stream_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};

// Launch counter adjustments: kernels recorded into a CUDA graph are
// counted when the graph is replayed, not when they are captured.
void add_launches(long long k);
unsigned long long launch_count();

// Properties of the current device (cached per device id).
const Device& current_device();

// Bump-pointer carving of a caller workspace (256-byte aligned pieces).
struct Carver {
    char* base;
    size_t used = 0;
    size_t cap;
    Carver(void* p, size_t bytes) : base(static_cast<char*>(p)), cap(bytes) {}
    template <typename T>
    T* take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        used = off + count * sizeof(T);
        return reinterpret_cast<T*>(base + off);
    }
    bool ok() const { return used <= cap; }
};

// Size-only twin of Carver, used by msc_workspace_bytes.
struct Sizer {
    size_t used = 0;
    template <typename T>
    void take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        used = off + count * sizeof(T);
    }
};

inline int ceil_log2(int64_t n) {
    int b = 0;
    while ((int64_t(1) << b) < n) ++b;
    return b;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

#define MSC_TRY(expr)                                  \
    do {                                               \
        if ((expr) != cudaSuccess) return MSC_ERR_CUDA; \
    } while (0)

#define MSC_LAUNCHED()                                    \
    do {                                                  \
        if (cudaPeekAtLastError() != cudaSuccess) {       \
            cudaGetLastError();                           \
            return MSC_ERR_CUDA;                          \
        }                                                 \
    } while (0)

}  // namespace msc
