/*
 * msc.h -- C ABI of the GB300 (sm_103a) Morse-Smale segmentation and
 * connected-components library (arXiv 2409.03771, "Distributed Path
 * Compression for Piecewise Linear Morse-Smale Segmentations and Connected
 * Components"), single GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers named d_* or documented as "device" are CUDA device pointers;
 *    the caller owns every input, output and workspace buffer.  The library
 *    allocates nothing on these calls.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls only enqueue work: they are asynchronous on `stream`
 *    and return before the GPU has finished.
 *  - The return value reports host-side checks and launch errors:
 *    MSC_OK, MSC_ERR_ARG (null pointer, bad size, bad connectivity),
 *    MSC_ERR_WS (workspace smaller than msc_workspace_bytes), MSC_ERR_CUDA
 *    (a CUDA call or launch failed).
 *  - Errors found on the device are written to the caller's device status
 *    word `d_status` (int32): the call first resets it to MSC_OK, then the
 *    first error found wins (MSC_ERR_NAN, MSC_ERR_NOT_CONVERGED, MSC_ERR_ARG
 *    for an out-of-range pointer or CSR column, MSC_ERR_INTERNAL).  Read it
 *    after synchronising the stream.  Outputs are unspecified when it is
 *    not MSC_OK.  No device error traps or hangs the GPU: every device loop
 *    is bounded.
 *  - Workspace: a device buffer of at least msc_workspace_bytes(op, n, nnz)
 *    bytes, 256-byte aligned (a misaligned one returns MSC_ERR_ARG); its
 *    contents on entry do not matter and are clobbered.  Input and output
 *    arrays need only their element alignment.
 *  - Vertex ids of a regular grid are linear, x fastest:
 *    v = x + nx * (y + ny * z).  Sizes are limited to n < 2^31 vertices.
 *  - Outputs are deterministic: identical inputs give identical bytes.
 */
#ifndef MSC_H
#define MSC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MSC_API __attribute__((visibility("default")))
#else
#define MSC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define MSC_OK 0
#define MSC_ERR_ARG (-1)
#define MSC_ERR_WS (-2)
#define MSC_ERR_CUDA (-3)
#define MSC_ERR_NAN (-4)
#define MSC_ERR_NOT_CONVERGED (-5)
#define MSC_ERR_BUDGET (-6)
#define MSC_ERR_INTERNAL (-7)
#define MSC_ERR_TOO_LARGE (-8)
#define MSC_PENDING 1

/* Regular grid: vertices per axis. */
typedef struct {
    int32_t nx, ny, nz;
} msc_grid;

/* Operation ids for msc_workspace_bytes. */
enum {
    MSC_OP_ORDER = 1,
    MSC_OP_COMPRESS = 2,
    MSC_OP_MS_ID = 3,
    MSC_OP_SEGMENT = 4,
    MSC_OP_CC_MASK = 5,
    MSC_OP_CC_MESH = 6,
    MSC_OP_ADJACENCY = 7,
    MSC_OP_EXTREMUM_GRAPH = 8,
    MSC_OP_ADJACENCY_CSR = 9,
    MSC_OP_EXTREMUM_GRAPH_CSR = 10
};

/* Workspace bytes needed by `op` on n vertices (nnz CSR entries for
 * MSC_OP_CC_MESH and the two *_CSR ops, ignored otherwise).  0 for an
 * unknown op or bad size. */
MSC_API size_t msc_workspace_bytes(int op, int64_t n, int64_t nnz);

/* Human-readable name of a status code (static string). */
MSC_API const char* msc_status_string(int code);

/* Vertex order by Simulation of Simplicity (section "Preprocessing": sort
 * the vertices by scalar value, break ties by global id, and give every
 * vertex its index in the sorted array).
 *   f       device float32[n]: the scalar field.  -0.0 ties with +0.0;
 *           +-Inf are ordinary values; a NaN sets MSC_ERR_NAN.
 *   order   device int32[n] out: order[v] = #{u : (f[u], u) < (f[v], v)},
 *           a permutation of 0..n-1.
 * Method: LSD radix sort (four 8-bit digits) of order-preserving uint32
 * keys with a vertex-id payload, stable, ending in order[id] = position. */
MSC_API int msc_order(const float* f, int64_t n, int32_t* order, void* ws, size_t ws_bytes,
              int32_t* d_status, void* stream);

/* Steepest-descent and steepest-ascent pointers on the implicit Freudenthal
 * triangulation of a regular grid (Alg. 1 initialisation: every vertex
 * points at its largest neighbour; section "Ascending and Descending
 * Manifolds").  The link of a vertex holds the 14 neighbours at offsets
 * +-(1,0,0), +-(0,1,0), +-(0,0,1), +-(1,1,0), +-(1,0,1), +-(0,1,1),
 * +-(1,1,1) that lie inside the grid.
 *   order     device int32[n], a permutation of 0..n-1 (msc_order output).
 *   asc_ptr   device int32[n] out: the neighbour of smallest order, or v
 *             itself when v is a minimum.
 *   desc_ptr  device int32[n] out: the neighbour of largest order, or v
 *             itself when v is a maximum.
 * No workspace; no device-detected errors (order must be a permutation). */
MSC_API int msc_steepest_grid(const int32_t* order, msc_grid g, int32_t* asc_ptr, int32_t* desc_ptr,
                      void* stream);

/* The same over an explicit adjacency (the explicit-triangulation case):
 *   row  device int32[n+1], col device int32[row[n]]: CSR of a symmetric
 *        vertex adjacency; row[0] = 0.  A column outside [0, n) sets
 *        MSC_ERR_ARG in d_status. */
MSC_API int msc_steepest_csr(const int32_t* order, const int32_t* row, const int32_t* col, int32_t n,
                     int32_t* asc_ptr, int32_t* desc_ptr, int32_t* d_status, void* stream);

/* Path compression by pointer jumping, in place (Alg. 1 compression loop:
 * d[v] <- d[d[v]] until d[d[v]] = d[v]).  On return every active entry
 * holds the fixed point at the end of its pointer path.
 *   ptr  device int32[n], in/out.  Negative entries are inactive (the
 *        paper's -1 outside a feature mask) and are left as they are.
 *        An active entry pointing outside [0, n) or at an inactive entry
 *        sets MSC_ERR_ARG; a pointer cycle sets MSC_ERR_NOT_CONVERGED
 *        (every sweep advances each pointer by up to four hops; at most
 *        ceil(log5 n) + 2 sweeps are made). */
MSC_API int msc_compress(int32_t* ptr, int32_t n, void* ws, size_t ws_bytes, int32_t* d_status,
                 void* stream);

/* Path compression for callers that cannot allocate device memory.  The
 * paper has no counterpart.  Some callers must not call cudaMalloc: a
 * process whose device memory belongs to another allocator or to a fixed
 * budget (a serving runtime, a plugin inside a framework that owns the
 * device), or code that must not risk the device-wide synchronisation that
 * allocating and freeing can cause.  This entry point does what
 * msc_compress does, with the same arguments minus the workspace, and
 * allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine).  It is an ordinary host call that enqueues work on `stream`
 * (a memset, an occupancy query and about log5(n) + 3 kernel launches), so
 * it must not be made from a host function enqueued on a stream, where CUDA
 * calls are not allowed.
 *   n  at most MSC_NOALLOC_MAX_N; larger n returns MSC_ERR_TOO_LARGE.
 * Scratch: a static device array of about 2 MiB (step counters and two
 * active lists of MSC_NOALLOC_MAX_N / 16 + 1 entries), which every GPU that
 * loads libmsc holds until the process exits.  All calls share it and it
 * keeps the last call's contents (the counters are cleared on every call):
 * calls that overlap on the GPU -- on different streams, or on different
 * host threads without ordering -- race on it and must not be issued.
 * First call on a device: it looks up the array's device address
 * (cudaGetSymbolAddress with that device current), and with lazy module
 * loading (the CUDA default) that lookup and the first launches may load
 * the library's device code, which places the static array in device
 * memory -- a driver-side allocation that can synchronise.  So make one
 * warm-up call on each device (any n >= 1) before entering the context
 * that must not allocate, and before any stream capture. */
#define MSC_NOALLOC_MAX_N (1 << 22)
MSC_API int msc_compress_noalloc(int32_t* ptr, int32_t n, int32_t* d_status, void* stream);

/* Dense Morse-Smale cell ids (section "Ascending and Descending
 * Segmentation": vertices whose steepest descent and ascent end in the
 * same (minimum, maximum) pair form one cell).
 *   asc, desc  device int32[n]: per-vertex minimum and maximum labels,
 *              each in [0, n).
 *   ms         device int32[n] out: the index of (asc[v], desc[v]) among
 *              the distinct pairs sorted lexicographically, asc first.
 *   num_cells  device int32 out: the number of distinct pairs. */
MSC_API int msc_ms_id(const int32_t* asc, const int32_t* desc, int32_t n, int32_t* ms,
              int32_t* num_cells, void* ws, size_t ws_bytes, int32_t* d_status, void* stream);

/* The whole segmentation of a grid field: msc_order, steepest pointers,
 * path compression of both, Morse-Smale ids.  Outputs (device, n each):
 * order, asc (minimum label), desc (maximum label), ms; num_cells (device
 * int32).  Workspace: msc_workspace_bytes(MSC_OP_SEGMENT, n, 0). */
MSC_API int msc_segment(const float* f, msc_grid g, int32_t* order, int32_t* asc, int32_t* desc,
                int32_t* ms, int32_t* num_cells, void* ws, size_t ws_bytes, int32_t* d_status,
                void* stream);

/* Connected components of a feature mask on a regular grid (Alg. 3,
 * implicitly thresholded grid: label -1 off the mask).
 *   mask   device uint8[n]: nonzero = feature vertex.
 *   conn   6 (face neighbours) or 14 (the Freudenthal link).
 *   label  device int32[n] out: the smallest vertex id of the component
 *          (the paper labels with the largest; the partition is the same),
 *          -1 where mask is zero.
 * Method: union-find with min-label hooking, tile-local in shared memory,
 * then across tile faces, then pointer jumping to the roots. */
MSC_API int msc_cc_mask(const uint8_t* mask, msc_grid g, int32_t conn, int32_t* label, void* ws,
                size_t ws_bytes, int32_t* d_status, void* stream);

/* Connected components of an explicit mesh given as its vertex adjacency
 * (the explicit-CC variant of the Experiments section).
 *   row, col  device int32 CSR (row[n+1], col[row[n]]), symmetric.
 *   label     device int32[n] out: smallest vertex id of the component; a
 *             vertex with no edge labels itself.
 * Workspace: msc_workspace_bytes(MSC_OP_CC_MESH, n, nnz).  A column
 * outside [0, n) sets MSC_ERR_ARG in d_status.
 * Method: union-find with min-label hooking and subgraph sampling: every
 * vertex is first united with two of its neighbours, the most frequent
 * label of a sample names the dominant component, only vertices outside it
 * unite their remaining edges, and pointer jumping labels every vertex
 * with its root. */
MSC_API int msc_cc_mesh(const int32_t* row, const int32_t* col, int32_t n, int32_t* label, void* ws,
                size_t ws_bytes, int32_t* d_status, void* stream);

/* Adjacency of labelled regions: the connectivity preview of the
 * Morse-Smale complex built from its segmentations (section "Related Work",
 * Morse-Smale Complex) and the arcs of an extremum graph (Conclusion).  The
 * paper names both without defining an operation; this one is: every edge
 * (u, v) of the grid whose ends carry two different non-negative labels
 * gives the pair (min, max) of the two labels, and the result is the set of
 * distinct pairs in lexicographic order.  With asc or desc labels the pairs
 * are the minima or maxima whose manifolds touch; with cell ids, the cells
 * that share a boundary.
 *   label      device int32[n]: a label per vertex, negative = unlabelled.
 *   conn       14: the edges of the implicit triangulation (offsets
 *              (1,0,0), (0,1,0), (0,0,1), (1,1,0), (1,0,1), (0,1,1),
 *              (1,1,1)); 6: the face grid (the first three).
 *   label_bound  every label is below it (n for vertex-id labels, the cell
 *              count for cell ids; 1 .. 2^31-1).  A label at or above it
 *              sets MSC_ERR_ARG in d_status.  A tighter bound sorts fewer
 *              key bits: the pair key is lo * 2^s + hi, s = ceil(log2 bound).
 *   a, b       device int32[cap] out: the first min(cap, K) pairs, a < b.
 *   num_pairs  device int64 out: K, the number of distinct pairs (it may
 *              exceed cap; nothing is written past cap).
 * Workspace: msc_workspace_bytes(MSC_OP_ADJACENCY, n, 0), sized for 7n pair
 * keys (every edge of the 14-neighbour triangulation); n above
 * (2^31 - 1) / 7 returns MSC_ERR_TOO_LARGE.
 * Method: tiles of the grid, each de-duplicating its pair keys in a shared
 * hash set; radix sort of the tiles' keys; first key of every run. */
MSC_API int msc_adjacency_grid(const int32_t* label, msc_grid g, int32_t conn, int32_t label_bound,
                               int32_t* a, int32_t* b, int64_t cap, int64_t* num_pairs, void* ws,
                               size_t ws_bytes, int32_t* d_status, void* stream);

/* Arcs of the extremum graph with their saddles (Conclusion: the
 * segmentations make the extremum graph of a merge-tree computation
 * available; the paper defines neither the graph nor its saddles).  The
 * arcs are the region adjacency of msc_adjacency_grid applied to maximum
 * labels (sense = +1) or minimum labels (sense = -1).  Every edge between
 * two regions crosses at one of its ends: for maxima the end lower in the
 * order (a path from one maximum to the other through the edge comes down
 * to it), for minima the higher end.  The saddle of an arc is the crossing
 * vertex of its highest crossing edge (maxima) or of its lowest (minima).
 *   label      device int32[n]: desc labels (sense +1) or asc labels (-1)
 *              as msc_segment writes them, or any labels below
 *              label_bound (negative = unlabelled).
 *   order      device int32[n]: the vertex order (msc_order output, a
 *              permutation of 0..n-1; other values give unspecified
 *              saddles).
 *   conn, label_bound, cap: as for msc_adjacency_grid.
 *   a, b       device int32[cap] out: the first min(cap, K) arcs, a < b,
 *              in lexicographic order.
 *   saddle     device int32[cap] out: the arc's saddle vertex.
 *   num_arcs   device int64 out: K.
 * Workspace: msc_workspace_bytes(MSC_OP_EXTREMUM_GRAPH, n, 0) (7n keys
 * with their crossing vertices); n above (2^31 - 1) / 7 returns
 * MSC_ERR_TOO_LARGE.
 * Method: msc_adjacency_grid's, with each tile's shared set also keeping
 * the highest crossing of each key, the crossing vertices sorted with the
 * keys, and one atomic maximum per run of equal keys in a warp. */
MSC_API int msc_extremum_graph(const int32_t* label, const int32_t* order, msc_grid g, int32_t conn,
                               int32_t label_bound, int32_t sense, int32_t* a, int32_t* b, int32_t* saddle,
                               int64_t cap, int64_t* num_arcs, void* ws, size_t ws_bytes, int32_t* d_status,
                               void* stream);

/* The two operations above over an explicit mesh (the explicit
 * triangulation case), whose edges are the entries of a symmetric CSR
 * vertex adjacency, each taken from the row of its smaller end:
 *   row, col   device int32 CSR: row[n+1], col[nnz], row[0] = 0,
 *              row[n] = nnz.  A column outside [0, n) or a row range
 *              outside [0, nnz] sets MSC_ERR_ARG in d_status.
 *   nnz        the number of col entries (sizes the workspace; at most
 *              2^31 - 1).
 * Other arguments as for msc_adjacency_grid / msc_extremum_graph.
 * Workspace: msc_workspace_bytes(MSC_OP_ADJACENCY_CSR or
 * MSC_OP_EXTREMUM_GRAPH_CSR, n, nnz).
 * Method: a lane per vertex, the warp stepping through its rows together;
 * the keys (with their crossing vertices) are sorted and reduced as above. */
MSC_API int msc_adjacency_csr(const int32_t* label, const int32_t* row, const int32_t* col, int32_t n, int64_t nnz,
                              int32_t label_bound, int32_t* a, int32_t* b, int64_t cap, int64_t* num_pairs,
                              void* ws, size_t ws_bytes, int32_t* d_status, void* stream);
MSC_API int msc_extremum_graph_csr(const int32_t* label, const int32_t* order, const int32_t* row,
                                   const int32_t* col, int32_t n, int64_t nnz, int32_t label_bound, int32_t sense,
                                   int32_t* a, int32_t* b, int32_t* saddle, int64_t cap, int64_t* num_arcs,
                                   void* ws, size_t ws_bytes, int32_t* d_status, void* stream);

/* ---------------------------------------------------------------------
 * Batched segmentation.  The paper segments one grid at a time; a batch
 * applies the computation of msc_segment (Alg. 1 for both manifolds, then
 * the cell ids of section "Ascending and Descending Segmentation") to
 * `count` independent grids in one pass over a packed vertex space.
 * Grid i occupies ids [off_i, off_i + n_i) of every packed array, where
 * n_i = nx*ny*nz, off_0 = 0 and off_{i+1} = off_i + n_i; the total
 * sum n_i must stay below 2^31.  Every output is local to its instance and
 * is byte for byte what msc_segment returns for that grid alone:
 *   grids      host msc_grid[count] (read during the call only)
 *   f          device float32[total]
 *   order      device int32[total] out: rank of the vertex in its instance
 *   asc, desc  device int32[total] out: instance-local id of the vertex's
 *              minimum / maximum
 *   ms         device int32[total] out: instance-local dense cell id
 *   num_cells  device int32[count] out: cells of each instance
 * Workspace: msc_batch_workspace_bytes(grids, count).  Device errors go to
 * d_status as for msc_segment; a bad grid returns MSC_ERR_ARG. */

/* Tuning knobs of the batched path.  None changes any output. */
typedef struct {
    int32_t steepest_shape; /* stencil tile: 0 = 32x8x8, 1 = 16x8x16, 2 = 64x4x8,
                               3 = 16x16x8; -1 = tuned (msc_batch_autotune) or 0 */
    int32_t build_shift;    /* pointer jumping switches to an active list once at
                               most n >> build_shift pointers moved in a sweep
                               (1..30); 0 = tuned or 3 */
} msc_tune;

MSC_API size_t msc_batch_workspace_bytes(const msc_grid* grids, int32_t count);

/* One batched segmentation, enqueued as plain launches on `stream`.  The
 * instance tables are copied from host memory at the start of the call.
 * tune = NULL means { -1, 0 }. */
MSC_API int msc_batch_segment(const msc_grid* grids, int32_t count, const float* f, int32_t* order,
                              int32_t* asc, int32_t* desc, int32_t* ms, int32_t* num_cells, void* ws,
                              size_t ws_bytes, const msc_tune* tune, int32_t* d_status, void* stream);

/* The same batch captured once as a CUDA graph bound to these buffers.
 * Each msc_batch_plan_launch replays the whole batch (status reset
 * included) with one graph launch on `stream`; the inputs in f may change
 * between launches, the grids and buffers may not.  Creating the plan
 * copies the instance tables on `stream`, waits for that copy, and
 * captures on a private stream (it launches no kernel).  msc_batch_plan_kernels gives the kernels one
 * replay runs.  Destroy the plan before freeing its buffers. */
typedef struct msc_batch_plan msc_batch_plan;
MSC_API int msc_batch_plan_create(const msc_grid* grids, int32_t count, const float* f, int32_t* order,
                                  int32_t* asc, int32_t* desc, int32_t* ms, int32_t* num_cells,
                                  void* ws, size_t ws_bytes, const msc_tune* tune, int32_t* d_status,
                                  void* stream, msc_batch_plan** plan);
MSC_API int msc_batch_plan_launch(msc_batch_plan* plan, void* stream);
MSC_API int msc_batch_plan_kernels(const msc_batch_plan* plan);
MSC_API void msc_batch_plan_destroy(msc_batch_plan* plan);

/* Autotuner: times the batch under candidate tunings (tile shapes first,
 * then active-list thresholds for the best shape), `reps` timed runs each
 * after one warm-up, and checks that every candidate produces the same
 * outputs (a device checksum; a mismatch returns MSC_ERR_INTERNAL).  The
 * winner goes to *best (and its mean time in ms to *best_ms) and is
 * remembered for this list of grids: later calls with tune = NULL or
 * auto fields use it.  Synchronises `stream`. */
MSC_API int msc_batch_autotune(const msc_grid* grids, int32_t count, const float* f, int32_t* order,
                               int32_t* asc, int32_t* desc, int32_t* ms, int32_t* num_cells, void* ws,
                               size_t ws_bytes, int32_t* d_status, void* stream, int32_t reps,
                               msc_tune* best, float* best_ms);

/* ---------------------------------------------------------------------
 * Serving.  A server admits segmentation (msc_segment) and mask-CC
 * (msc_cc_mask) requests of mixed sizes, runs them with continuous
 * batching inside a fixed HBM budget and keeps each result on the device
 * until the caller releases it.  The paper has no serving layer; every
 * result is exactly what the single-request entry point returns for the
 * same input, alone or in any mix.
 *
 * Scheduling: a server thread takes requests in arrival order.  The head
 * of the queue is admitted when one of `slots` slots is free and its device
 * memory (outputs + workspace, from an arena of `hbm_budget` bytes
 * allocated at creation) fits, so no request starves.  When the head is a
 * segmentation of at most `group_max_vertices` vertices, the segmentations
 * of at most that size among the next 64 waiting requests are admitted
 * with it (larger requests keep their places) and run as one batched launch
 * (msc_batch_segment over a packed copy of their inputs); larger requests
 * and CC requests run on their own.  A batched launch that reports a
 * device error (e.g. a NaN in one field) is re-run request by request, so
 * every request gets the status it would get alone.  Work on different
 * slots overlaps on the GPU; each slot has a high-priority stream for
 * requests of at least 2^24 vertices and a low-priority one for the rest,
 * so that smaller work fills idle SMs around the large requests.  A
 * request that arrives while others run is admitted as soon as a slot and
 * memory free up.  Results stay in the arena until msc_server_release. */

#define MSC_JOB_SEGMENT 1
#define MSC_JOB_CC_MASK 2

typedef struct {
    int32_t kind;      /* MSC_JOB_SEGMENT or MSC_JOB_CC_MASK */
    msc_grid g;
    int32_t conn;      /* MSC_JOB_CC_MASK: 6 or 14 */
    const void* input; /* device float32[n] field (segment) or uint8[n] mask
                          (CC), owned by the caller, unchanged until the
                          request completes */
} msc_job;

typedef struct {
    int32_t status;      /* MSC_PENDING, MSC_OK or the request's error */
    int32_t num_cells;   /* segment: Morse-Smale cells; CC: 0 */
    int64_t n;           /* vertices */
    int32_t* order;      /* device, n entries, segment only (else NULL) */
    int32_t* asc;
    int32_t* desc;
    int32_t* ms;
    int32_t* label;      /* device, n entries, CC only (else NULL) */
    double t_submit;     /* host steady-clock seconds: submitted, */
    double t_start;      /* launched, */
    double t_done;       /* and seen complete */
    int32_t group_size;  /* requests that ran in the same launch */
} msc_result;

typedef struct msc_server msc_server;

/* hbm_budget: bytes of the result/workspace arena (allocated here; the
 * only allocation the server makes on the device).  slots: concurrent
 * streams (1..16).  group_max_vertices: size limit for batching several
 * segmentations into one launch (0 = never batch).  Returns NULL on a bad
 * argument or when the arena cannot be allocated. */
MSC_API msc_server* msc_server_create(size_t hbm_budget, int32_t slots, int64_t group_max_vertices);

/* Queue a request; *ticket identifies it.  Returns MSC_ERR_ARG for a bad
 * request and MSC_ERR_BUDGET when it could never fit the budget.  The
 * call only queues: it returns at once. */
MSC_API int msc_server_submit(msc_server* s, const msc_job* job, uint64_t* ticket);

/* Copy the request's state into *out: status MSC_PENDING while it waits
 * or runs.  msc_server_wait blocks up to timeout_ms (< 0: no limit) for
 * completion and returns the same as msc_server_poll. */
MSC_API int msc_server_poll(msc_server* s, uint64_t ticket, msc_result* out);
MSC_API int msc_server_wait(msc_server* s, uint64_t ticket, double timeout_ms, msc_result* out);

/* Free a completed request's device memory (its result pointers become
 * invalid).  MSC_PENDING if it has not completed, MSC_ERR_ARG for an
 * unknown ticket. */
MSC_API int msc_server_release(msc_server* s, uint64_t ticket);

/* Arena bytes in use and the number of requests queued, running, done. */
MSC_API int msc_server_stats(msc_server* s, size_t* arena_used, int32_t* queued, int32_t* running,
                             int32_t* done);

/* Waits for the running work, then frees the arena, the streams and every
 * result. */
MSC_API void msc_server_destroy(msc_server* s);

#ifdef __cplusplus
}
#endif

#endif /* MSC_H */
