// C ABI entry points (include/msc.h): argument checks, workspace carving,
// stage sequencing.  Every stage runs in the kernels of this directory.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "adjacency.cuh"
#include "cc.cuh"
#include "common.cuh"
#include "compress.cuh"
#include "msid.cuh"
#include "sort.cuh"
#include "steepest.cuh"
#include "tma.cuh"

namespace msc {

const Device& current_device() {
    static Device devs[64];
    static std::mutex mu;
    int id = 0;
    cudaGetDevice(&id);
    if (id < 0 || id >= 64) id = 0;
    Device& d = devs[id];
    if (d.id != id) {
        std::lock_guard<std::mutex> lock(mu);
        if (d.id != id) {
            int sms = 0, smem = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, id);
            cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, id);
            d.sms = sms > 0 ? sms : 1;
            d.max_smem_optin = smem;
            d.id = id;
        }
    }
    return d;
}

bool make_tensor_map_3d(CUtensorMap* map, const void* base, int elem_bytes, int nx, int ny, int nz,
                        int bx, int by, int bz) {
    using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<EncodeFn>(fn);
    });
    if (!encode) return false;
    if ((uintptr_t)base % 16 != 0) return false;
    const uint64_t pitch = (uint64_t)nx * elem_bytes;
    if (pitch % 16 != 0) return false;
    if (((uint64_t)bx * elem_bytes) % 16 != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {pitch, pitch * (uint64_t)ny};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_INT32;
    const CUresult r = encode(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

namespace {

constexpr size_t kCommonWords = 64;  // uint32 control words shared by all stages

// Workspaces are carved into 256-byte aligned pieces, some read with
// 16-byte loads: the base must be 256-byte aligned.
bool ws_aligned(const void* ws) { return ((uintptr_t)ws & 255) == 0; }

bool grid_ok(msc_grid g) {
    if (g.nx <= 0 || g.ny <= 0 || g.nz <= 0) return false;
    return (int64_t)g.nx * g.ny * g.nz <= (int64_t)INT32_MAX;
}

int64_t grid_n(msc_grid g) { return (int64_t)g.nx * g.ny * g.nz; }

void size_order(Sizer& s, int64_t n) {
    for (int i = 0; i < 2; ++i) {
        s.take<uint32_t>(std::max<int64_t>(n, 1));
        s.take<int32_t>(std::max<int64_t>(n, 1));
    }
    size_sort_scratch(s, n);
}

// Segment workspace: common words, then the largest of the three stages.
size_t segment_bytes(int64_t n) {
    Sizer common;
    common.take<uint32_t>(kCommonWords);
    Sizer sort, comp, ms;
    sort.take<int32_t>(std::max<int64_t>(n, 1));
    size_sort_scratch(sort, n);
    size_compress_scratch(comp, n, 2);
    size_ms_scratch(ms, n);
    return ((common.used + 255) & ~size_t(255)) + std::max({sort.used, comp.used, ms.used});
}

}  // namespace
}  // namespace msc

using namespace msc;

extern "C" {

const char* msc_status_string(int code) {
    switch (code) {
        case MSC_OK: return "ok";
        case MSC_ERR_ARG: return "invalid argument";
        case MSC_ERR_WS: return "workspace too small";
        case MSC_ERR_CUDA: return "CUDA error";
        case MSC_ERR_NAN: return "NaN in scalar field";
        case MSC_ERR_NOT_CONVERGED: return "pointer jumping did not converge (pointer cycle)";
        case MSC_ERR_BUDGET: return "request exceeds the memory budget";
        case MSC_ERR_INTERNAL: return "internal error";
        case MSC_ERR_TOO_LARGE: return "size exceeds a limit of the entry point";
        case MSC_PENDING: return "pending";
        default: return "unknown status";
    }
}

size_t msc_workspace_bytes(int op, int64_t n, int64_t nnz) {
    if (n < 0 || n > INT32_MAX) return 0;
    Sizer s;
    switch (op) {
        case MSC_OP_ORDER: size_order(s, n); return s.used;
        case MSC_OP_COMPRESS: size_compress_scratch(s, n, 1); return s.used;
        case MSC_OP_MS_ID:
            size_ms_scratch(s, n);
            return s.used;
        case MSC_OP_SEGMENT: return segment_bytes(n);
        case MSC_OP_CC_MASK: return 256;
        case MSC_OP_CC_MESH: return 256;
        case MSC_OP_ADJACENCY:
        case MSC_OP_EXTREMUM_GRAPH:
            if (!adjacency_size_ok(n)) return 0;
            size_adjacency_scratch(s, n, op == MSC_OP_EXTREMUM_GRAPH);
            return s.used;
        case MSC_OP_ADJACENCY_CSR:
        case MSC_OP_EXTREMUM_GRAPH_CSR:
            if (nnz < 0 || nnz > INT32_MAX) return 0;
            size_adjacency_csr_scratch(s, nnz, op == MSC_OP_EXTREMUM_GRAPH_CSR);
            return s.used;
        default: return 0;
    }
}

int msc_order(const float* f, int64_t n, int32_t* order, void* ws, size_t ws_bytes, int32_t* d_status,
              void* stream) {
    if (n < 0 || n > INT32_MAX || !d_status || (n > 0 && (!f || !order || !ws || !ws_aligned(ws))))
        return MSC_ERR_ARG;
    if (ws_bytes < msc_workspace_bytes(MSC_OP_ORDER, n, 0)) return MSC_ERR_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MSC_TRY(cudaMemsetAsync(d_status, 0, sizeof(int32_t), s));
    if (n == 0) return MSC_OK;
    Carver c(ws, ws_bytes);
    uint32_t* ka = c.take<uint32_t>(n);
    int32_t* ia = c.take<int32_t>(n);
    uint32_t* kb = c.take<uint32_t>(n);
    int32_t* ib = c.take<int32_t>(n);
    SortScratch sc = carve_sort_scratch(c, n);
    return run_order(f, n, order, ka, ia, kb, ib, sc, d_status, s);
}

int msc_steepest_grid(const int32_t* order, msc_grid g, int32_t* asc_ptr, int32_t* desc_ptr, void* stream) {
    if (!grid_ok(g) || !order || !asc_ptr || !desc_ptr) return MSC_ERR_ARG;
    return run_steepest_grid(order, g, asc_ptr, desc_ptr, nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

int msc_steepest_csr(const int32_t* order, const int32_t* row, const int32_t* col, int32_t n,
                     int32_t* asc_ptr, int32_t* desc_ptr, int32_t* d_status, void* stream) {
    if (n < 0 || !d_status || (n > 0 && (!order || !row || !col || !asc_ptr || !desc_ptr))) return MSC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MSC_TRY(cudaMemsetAsync(d_status, 0, sizeof(int32_t), s));
    return run_steepest_csr(order, row, col, n, asc_ptr, desc_ptr, d_status, s);
}

int msc_compress(int32_t* ptr, int32_t n, void* ws, size_t ws_bytes, int32_t* d_status, void* stream) {
    if (n < 0 || !d_status || (n > 0 && (!ptr || !ws || !ws_aligned(ws)))) return MSC_ERR_ARG;
    if (ws_bytes < msc_workspace_bytes(MSC_OP_COMPRESS, n, 0)) return MSC_ERR_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MSC_TRY(cudaMemsetAsync(d_status, 0, sizeof(int32_t), s));
    if (n == 0) return MSC_OK;
    Carver c(ws, ws_bytes);
    CompressScratch sc = carve_compress_scratch(c, n, 1);
    int32_t* arr[1] = {ptr};
    return run_compress(arr, 1, n, sc, d_status, s);
}

int msc_ms_id(const int32_t* asc, const int32_t* desc, int32_t n, int32_t* ms, int32_t* num_cells,
              void* ws, size_t ws_bytes, int32_t* d_status, void* stream) {
    if (n < 0 || !d_status || !num_cells || (n > 0 && (!asc || !desc || !ms || !ws || !ws_aligned(ws))))
        return MSC_ERR_ARG;
    if (ws_bytes < msc_workspace_bytes(MSC_OP_MS_ID, n, 0)) return MSC_ERR_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MSC_TRY(cudaMemsetAsync(d_status, 0, sizeof(int32_t), s));
    Carver c(ws, ws_bytes);
    MsScratch sc = carve_ms_scratch(c, n);
    return run_ms_id(asc, desc, n, ms, num_cells, sc, false, d_status, s);
}

int msc_segment(const float* f, msc_grid g, int32_t* order, int32_t* asc, int32_t* desc, int32_t* ms,
                int32_t* num_cells, void* ws, size_t ws_bytes, int32_t* d_status, void* stream) {
    if (!grid_ok(g) || !f || !order || !asc || !desc || !ms || !num_cells || !ws || !d_status || !ws_aligned(ws))
        return MSC_ERR_ARG;
    const int64_t n = grid_n(g);
    if (ws_bytes < segment_bytes(n)) return MSC_ERR_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MSC_TRY(cudaMemsetAsync(d_status, 0, sizeof(int32_t), s));
    Carver c(ws, ws_bytes);
    uint32_t* common = c.take<uint32_t>(kCommonWords);
    const size_t stage_off = c.used;
    MSC_TRY(cudaMemsetAsync(common, 0, kCommonWords * sizeof(uint32_t), s));
    // 1. order; the asc / desc / ms outputs double as the sort's ping-pong
    {
        Carver st(ws, ws_bytes);
        st.used = stage_off;
        int32_t* ib = st.take<int32_t>(n);
        SortScratch sc = carve_sort_scratch(st, n);
        int r = run_order(f, n, order, reinterpret_cast<uint32_t*>(asc), desc,
                          reinterpret_cast<uint32_t*>(ms), ib, sc, d_status, s);
        if (r) return r;
    }
    // 2. steepest pointers (the extrema are counted by the first jump sweep)
    int r = run_steepest_grid(order, g, asc, desc, nullptr, d_status, s);
    if (r) return r;
    // 3. pointer jumping on both arrays
    {
        Carver st(ws, ws_bytes);
        st.used = stage_off;
        CompressScratch sc = carve_compress_scratch(st, n, 2);
        int32_t* arr[2] = {asc, desc};
        CompressTune tune;
        tune.trusted = true;  // made by the stencil above: in range, acyclic
        tune.roots = common;  // common[0] = #minima (asc roots), common[1] = #maxima
        r = run_compress(arr, 2, (int32_t)n, sc, d_status, s, tune);
        if (r) return r;
    }
    // 4. dense Morse-Smale ids
    {
        Carver st(ws, ws_bytes);
        st.used = stage_off;
        MsScratch sc = carve_ms_scratch(st, n);
        sc.ctl = common;  // extrema counts from the steepest stage
        r = run_ms_id(asc, desc, (int32_t)n, ms, num_cells, sc, true, d_status, s);
    }
    return r;
}

int msc_cc_mask(const uint8_t* mask, msc_grid g, int32_t conn, int32_t* label, void* ws, size_t ws_bytes,
                int32_t* d_status, void* stream) {
    (void)ws;
    if (!grid_ok(g) || !mask || !label || !d_status || (conn != 6 && conn != 14)) return MSC_ERR_ARG;
    if (ws_bytes < msc_workspace_bytes(MSC_OP_CC_MASK, grid_n(g), 0)) return MSC_ERR_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MSC_TRY(cudaMemsetAsync(d_status, 0, sizeof(int32_t), s));
    return run_cc_mask(mask, g, conn, label, d_status, s);
}

int msc_cc_mesh(const int32_t* row, const int32_t* col, int32_t n, int32_t* label, void* ws, size_t ws_bytes,
                int32_t* d_status, void* stream) {
    if (n < 0 || !d_status || (n > 0 && (!row || !col || !label || !ws))) return MSC_ERR_ARG;
    if (ws_bytes < msc_workspace_bytes(MSC_OP_CC_MESH, n, 0)) return MSC_ERR_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MSC_TRY(cudaMemsetAsync(d_status, 0, sizeof(int32_t), s));
    if (n == 0) return MSC_OK;
    return run_cc_mesh(row, col, n, label, d_status, s, static_cast<int32_t*>(ws));
}

int msc_adjacency_grid(const int32_t* label, msc_grid g, int32_t conn, int32_t label_bound, int32_t* a,
                       int32_t* b, int64_t cap, int64_t* num_pairs, void* ws, size_t ws_bytes,
                       int32_t* d_status, void* stream) {
    if (!grid_ok(g) || !label || !num_pairs || !d_status || !ws || !ws_aligned(ws) ||
        (conn != 6 && conn != 14) || label_bound <= 0 || cap < 0 || (cap > 0 && (!a || !b)))
        return MSC_ERR_ARG;
    const int64_t n = grid_n(g);
    if (!adjacency_size_ok(n)) return MSC_ERR_TOO_LARGE;
    if (ws_bytes < msc_workspace_bytes(MSC_OP_ADJACENCY, n, 0)) return MSC_ERR_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MSC_TRY(cudaMemsetAsync(d_status, 0, sizeof(int32_t), s));
    return run_adjacency_grid(label, g, conn, label_bound, a, b, cap, num_pairs, ws, ws_bytes, d_status, s);
}

int msc_extremum_graph(const int32_t* label, const int32_t* order, msc_grid g, int32_t conn, int32_t label_bound,
                       int32_t sense, int32_t* a, int32_t* b, int32_t* saddle, int64_t cap, int64_t* num_arcs,
                       void* ws, size_t ws_bytes, int32_t* d_status, void* stream) {
    if (!grid_ok(g) || !label || !order || !num_arcs || !d_status || !ws || !ws_aligned(ws) ||
        (conn != 6 && conn != 14) || (sense != 1 && sense != -1) || label_bound <= 0 || cap < 0 ||
        (cap > 0 && (!a || !b || !saddle)))
        return MSC_ERR_ARG;
    const int64_t n = grid_n(g);
    if (!adjacency_size_ok(n)) return MSC_ERR_TOO_LARGE;
    if (ws_bytes < msc_workspace_bytes(MSC_OP_EXTREMUM_GRAPH, n, 0)) return MSC_ERR_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MSC_TRY(cudaMemsetAsync(d_status, 0, sizeof(int32_t), s));
    return run_adjacency_grid(label, g, conn, label_bound, a, b, cap, num_arcs, ws, ws_bytes, d_status, s, order,
                              sense, saddle);
}

int msc_adjacency_csr(const int32_t* label, const int32_t* row, const int32_t* col, int32_t n, int64_t nnz,
                      int32_t label_bound, int32_t* a, int32_t* b, int64_t cap, int64_t* num_pairs, void* ws,
                      size_t ws_bytes, int32_t* d_status, void* stream) {
    if (n < 0 || nnz < 0 || nnz > INT32_MAX || !num_pairs || !d_status || !ws || !ws_aligned(ws) ||
        label_bound <= 0 || cap < 0 || (cap > 0 && (!a || !b)) || (n > 0 && (!label || !row || (nnz > 0 && !col))))
        return MSC_ERR_ARG;
    if (ws_bytes < msc_workspace_bytes(MSC_OP_ADJACENCY_CSR, n, nnz)) return MSC_ERR_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MSC_TRY(cudaMemsetAsync(d_status, 0, sizeof(int32_t), s));
    return run_adjacency_csr(label, row, col, n, nnz, label_bound, a, b, cap, num_pairs, ws, ws_bytes, d_status, s);
}

int msc_extremum_graph_csr(const int32_t* label, const int32_t* order, const int32_t* row, const int32_t* col,
                           int32_t n, int64_t nnz, int32_t label_bound, int32_t sense, int32_t* a, int32_t* b,
                           int32_t* saddle, int64_t cap, int64_t* num_arcs, void* ws, size_t ws_bytes,
                           int32_t* d_status, void* stream) {
    if (n < 0 || nnz < 0 || nnz > INT32_MAX || !num_arcs || !d_status || !ws || !ws_aligned(ws) ||
        label_bound <= 0 || (sense != 1 && sense != -1) || cap < 0 || (cap > 0 && (!a || !b || !saddle)) ||
        (n > 0 && (!label || !order || !row || (nnz > 0 && !col))))
        return MSC_ERR_ARG;
    if (ws_bytes < msc_workspace_bytes(MSC_OP_EXTREMUM_GRAPH_CSR, n, nnz)) return MSC_ERR_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MSC_TRY(cudaMemsetAsync(d_status, 0, sizeof(int32_t), s));
    return run_adjacency_csr(label, row, col, n, nnz, label_bound, a, b, cap, num_arcs, ws, ws_bytes, d_status, s,
                             order, sense, saddle);
}

}  // extern "C"
