/*
 * msc_oracle.c -- plain, sequential CPU oracle for Morse-Smale segmentation
 * by path compression and for connected components (arXiv 2409.03771).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library links, includes or calls
 * this file; only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark load it.  It shares no code, header, table or constant with
 * the CUDA path.  Every routine is the plain definition of what the GPU path
 * computes, written so that it can be checked against the paper by eye:
 * no blocking, no fusion, no reordering.
 *
 * Conventions (readings of the paper where it is silent):
 *   - vertex id of grid point (x,y,z) is x + nx*(y + ny*z), x fastest;
 *   - the implicit triangulation is the Freudenthal/Kuhn split, whose vertex
 *     link holds the 14 neighbours at offsets +-(1,0,0), +-(0,1,0), +-(0,0,1),
 *     +-(1,1,0), +-(1,0,1), +-(0,1,1), +-(1,1,1); out-of-grid offsets drop;
 *   - a vertex with no neighbour above it (below it) is a maximum (minimum)
 *     and points at itself;
 *   - connected-component labels are the SMALLEST vertex id of the component
 *     (the paper uses the largest; the partition is the same), -1 off-mask.
 *
 * Return codes: 0 ok, -1 bad argument, -4 NaN in the scalar field,
 * -5 a pointer walk did not reach a fixed point (cycle), -8 out of memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_NAN (-4)
#define OR_ERR_CYCLE (-5)
#define OR_ERR_OOM (-8)

/* ------------------------------------------------------------------------ */
/* Vertex order: Simulation of Simplicity by a global sort (section
 * "Preprocessing": sort by scalar value, ties broken by global id; the order
 * field holds each vertex's index in the sorted array).                     */

typedef struct {
    float f;
    int32_t id;
} or_key;

static int or_cmp_key(const void* a, const void* b) {
    const or_key* p = (const or_key*)a;
    const or_key* q = (const or_key*)b;
    /* IEEE '<': -0.0 and +0.0 compare equal and fall to the id tie-break. */
    if (p->f < q->f) return -1;
    if (q->f < p->f) return 1;
    return (p->id > q->id) - (p->id < q->id);
}

int32_t oracle_order(const float* f, int64_t n, int32_t* order) {
    if (n < 0 || n > INT32_MAX) return OR_ERR_ARG;
    for (int64_t v = 0; v < n; ++v)
        if (isnan(f[v])) return OR_ERR_NAN;
    or_key* k = (or_key*)malloc((size_t)(n > 0 ? n : 1) * sizeof(or_key));
    if (!k) return OR_ERR_OOM;
    for (int64_t v = 0; v < n; ++v) {
        k[v].f = f[v];
        k[v].id = (int32_t)v;
    }
    qsort(k, (size_t)n, sizeof(or_key), or_cmp_key);
    for (int64_t i = 0; i < n; ++i) order[k[i].id] = (int32_t)i;
    free(k);
    return OR_OK;
}

/* The order of one vertex, computed one by one by counting: order[v] is the
 * number of vertices u with (f[u], u) < (f[v], v).  Used for sampled checks
 * at sizes where the full sort is too slow to repeat.                      */
int64_t oracle_order_at(const float* f, int64_t n, int64_t v) {
    if (v < 0 || v >= n || isnan(f[v])) return OR_ERR_ARG;
    int64_t c = 0;
    const float fv = f[v];
    for (int64_t u = 0; u < n; ++u) {
        if (f[u] < fv || (!(fv < f[u]) && u < v)) ++c;
    }
    return c;
}

/* ------------------------------------------------------------------------ */
/* Steepest ascent / descent pointers (Alg. 1, initialisation: each vertex
 * points at its largest neighbour; the ascending manifold is the symmetric
 * case with the smallest neighbour).  Comparisons use the order field, which
 * makes f injective.                                                       */

static const int OR_FREUD[14][3] = {
    {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},  {0, 0, 1},
    {0, 0, -1}, {1, 1, 0},   {-1, -1, 0}, {1, 0, 1},  {-1, 0, -1},
    {0, 1, 1},  {0, -1, -1}, {1, 1, 1},   {-1, -1, -1}};

static const int OR_FACE6[6][3] = {{1, 0, 0},  {-1, 0, 0}, {0, 1, 0},
                                   {0, -1, 0}, {0, 0, 1},  {0, 0, -1}};

static int or_grid_ok(int32_t nx, int32_t ny, int32_t nz) {
    if (nx <= 0 || ny <= 0 || nz <= 0) return 0;
    return (int64_t)nx * ny * nz <= INT32_MAX;
}

int32_t oracle_steepest_grid(const int32_t* order, int32_t nx, int32_t ny,
                             int32_t nz, int32_t* asc_ptr, int32_t* desc_ptr) {
    if (!or_grid_ok(nx, ny, nz)) return OR_ERR_ARG;
    for (int32_t z = 0; z < nz; ++z)
        for (int32_t y = 0; y < ny; ++y)
            for (int32_t x = 0; x < nx; ++x) {
                const int64_t v = x + (int64_t)nx * (y + (int64_t)ny * z);
                int64_t hi = v, lo = v;
                for (int k = 0; k < 14; ++k) {
                    const int64_t xx = x + OR_FREUD[k][0];
                    const int64_t yy = y + OR_FREUD[k][1];
                    const int64_t zz = z + OR_FREUD[k][2];
                    if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny ||
                        zz >= nz)
                        continue;
                    const int64_t u = xx + (int64_t)nx * (yy + (int64_t)ny * zz);
                    if (order[u] > order[hi]) hi = u;
                    if (order[u] < order[lo]) lo = u;
                }
                desc_ptr[v] = (int32_t)hi;
                asc_ptr[v] = (int32_t)lo;
            }
    return OR_OK;
}

int32_t oracle_steepest_csr(const int32_t* order, const int32_t* row,
                            const int32_t* col, int32_t n, int32_t* asc_ptr,
                            int32_t* desc_ptr) {
    if (n < 0) return OR_ERR_ARG;
    for (int32_t v = 0; v < n; ++v) {
        int32_t hi = v, lo = v;
        for (int32_t e = row[v]; e < row[v + 1]; ++e) {
            const int32_t u = col[e];
            if (u < 0 || u >= n) return OR_ERR_ARG;
            if (order[u] > order[hi]) hi = u;
            if (order[u] < order[lo]) lo = u;
        }
        desc_ptr[v] = hi;
        asc_ptr[v] = lo;
    }
    return OR_OK;
}

/* (f, id) comparison: the order field's '<' without building it.           */
static int or_below(const float* f, int64_t a, int64_t b) {
    return f[a] < f[b] || (!(f[b] < f[a]) && a < b);
}

/* Steepest pointers of one vertex straight from f (sampled checks).        */
int32_t oracle_steepest_at(const float* f, int32_t nx, int32_t ny, int32_t nz,
                           int64_t v, int32_t* asc_ptr, int32_t* desc_ptr) {
    if (!or_grid_ok(nx, ny, nz)) return OR_ERR_ARG;
    const int64_t n = (int64_t)nx * ny * nz;
    if (v < 0 || v >= n) return OR_ERR_ARG;
    const int64_t x = v % nx, y = (v / nx) % ny, z = v / ((int64_t)nx * ny);
    int64_t hi = v, lo = v;
    for (int k = 0; k < 14; ++k) {
        const int64_t xx = x + OR_FREUD[k][0];
        const int64_t yy = y + OR_FREUD[k][1];
        const int64_t zz = z + OR_FREUD[k][2];
        if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz)
            continue;
        const int64_t u = xx + (int64_t)nx * (yy + (int64_t)ny * zz);
        if (isnan(f[u])) return OR_ERR_NAN;
        if (or_below(f, hi, u)) hi = u;
        if (or_below(f, u, lo)) lo = u;
    }
    *desc_ptr = (int32_t)hi;
    *asc_ptr = (int32_t)lo;
    return OR_OK;
}

/* The extrema reached from one vertex by walking the steepest paths
 * (definition of the ascending / descending manifold, section "Ascending
 * and Descending Manifolds").                                              */
int32_t oracle_labels_at(const float* f, int32_t nx, int32_t ny, int32_t nz,
                         int64_t v, int32_t* asc_label, int32_t* desc_label) {
    const int64_t n = (int64_t)nx * ny * nz;
    int32_t a, d, s;
    int64_t u = v, steps = 0;
    for (;;) { /* steepest ascent: follow the larger neighbour */
        s = oracle_steepest_at(f, nx, ny, nz, u, &a, &d);
        if (s) return s;
        if (d == u) break;
        u = d;
        if (++steps > n) return OR_ERR_CYCLE;
    }
    *desc_label = (int32_t)u;
    u = v;
    steps = 0;
    for (;;) { /* steepest descent */
        s = oracle_steepest_at(f, nx, ny, nz, u, &a, &d);
        if (s) return s;
        if (a == u) break;
        u = a;
        if (++steps > n) return OR_ERR_CYCLE;
    }
    *asc_label = (int32_t)u;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Path compression result: for every vertex, the fixed point reached by
 * following the pointer array (Alg. 1 compression loop; its result is the
 * end of the steepest path).  Negative entries are inactive (the paper's
 * -1 for vertices outside the feature mask, Alg. 3) and stay as they are.
 * A pointer out of range, or from an active entry to an inactive one, is a
 * bad argument; a walk longer than n steps is a cycle.                     */
int32_t oracle_walk(const int32_t* ptr, int64_t n, int32_t* label) {
    if (n < 0 || n > INT32_MAX) return OR_ERR_ARG;
    for (int64_t v = 0; v < n; ++v) {
        if (ptr[v] < 0) {
            label[v] = ptr[v];
            continue;
        }
        int64_t u = v, steps = 0;
        for (;;) {
            const int32_t p = ptr[u];
            if (p < 0 || p >= n) return OR_ERR_ARG;
            if (p == u) break;
            u = p;
            if (++steps > n) return OR_ERR_CYCLE;
        }
        label[v] = (int32_t)u;
    }
    return OR_OK;
}

/* The same result with memoisation: a walk stops at the first vertex whose
 * label is already known.  Checked against oracle_walk by the tests; used
 * where the plain walk is too slow (long paths on large grids).            */
int32_t oracle_walk_memo(const int32_t* ptr, int64_t n, int32_t* label) {
    if (n < 0 || n > INT32_MAX) return OR_ERR_ARG;
    const int32_t UNKNOWN = INT32_MIN;
    int32_t* stack = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!stack) return OR_ERR_OOM;
    for (int64_t v = 0; v < n; ++v) label[v] = UNKNOWN;
    for (int64_t v = 0; v < n; ++v) {
        if (label[v] != UNKNOWN) continue;
        if (ptr[v] < 0) {
            label[v] = ptr[v];
            continue;
        }
        int64_t top = 0, u = v;
        int32_t root;
        for (;;) {
            if (label[u] != UNKNOWN) {
                root = label[u];
                break;
            }
            const int32_t p = ptr[u];
            if (p < 0 || p >= n) {
                free(stack);
                return OR_ERR_ARG;
            }
            if (p == u) {
                root = (int32_t)u;
                break;
            }
            if (top > n) {
                free(stack);
                return OR_ERR_CYCLE;
            }
            stack[top++] = (int32_t)u;
            u = p;
        }
        while (top > 0) label[stack[--top]] = root;
        label[u] = root;
    }
    free(stack);
    return OR_OK;
}

/* One synchronous pointer-doubling round, out[v] = p[p[v]] (the two-array
 * variant the paper discusses next to Alg. 1, and the rule behind the
 * ghost-vertex table of Fig. 2).  Used only to replay that worked example. */
int32_t oracle_jump_sync(const int32_t* p, int64_t n, int32_t* out) {
    for (int64_t v = 0; v < n; ++v) {
        const int32_t u = p[v];
        if (u < 0) {
            out[v] = u;
            continue;
        }
        if (u >= n || p[u] < 0) return OR_ERR_ARG;
        out[v] = p[u];
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Morse-Smale cell id: vertices whose steepest descent and ascent end in the
 * same (minimum, maximum) pair form one cell (section "Ascending and
 * Descending Segmentation").  The dense id is the index of the vertex's
 * pair among the distinct pairs sorted lexicographically, minimum first.   */

typedef struct {
    int32_t a, d;
} or_pair;

static int or_cmp_pair(const void* x, const void* y) {
    const or_pair* p = (const or_pair*)x;
    const or_pair* q = (const or_pair*)y;
    if (p->a != q->a) return (p->a > q->a) - (p->a < q->a);
    return (p->d > q->d) - (p->d < q->d);
}

int32_t oracle_ms(const int32_t* asc, const int32_t* desc, int64_t n, int32_t* ms,
                  int32_t* num_cells) {
    if (n < 0 || n > INT32_MAX) return OR_ERR_ARG;
    or_pair* p = (or_pair*)malloc((size_t)(n > 0 ? n : 1) * sizeof(or_pair));
    if (!p) return OR_ERR_OOM;
    for (int64_t v = 0; v < n; ++v) {
        p[v].a = asc[v];
        p[v].d = desc[v];
    }
    qsort(p, (size_t)n, sizeof(or_pair), or_cmp_pair);
    int64_t k = 0; /* distinct pairs, in sorted order, packed to the front */
    for (int64_t i = 0; i < n; ++i)
        if (k == 0 || or_cmp_pair(&p[k - 1], &p[i]) != 0) p[k++] = p[i];
    for (int64_t v = 0; v < n; ++v) {
        or_pair key = {asc[v], desc[v]};
        int64_t lo = 0, hi = k; /* binary search for the pair's index */
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (or_cmp_pair(&p[mid], &key) < 0) lo = mid + 1;
            else hi = mid;
        }
        ms[v] = (int32_t)lo;
    }
    *num_cells = (int32_t)k;
    free(p);
    return OR_OK;
}

/* Full segmentation of a grid field: order, steepest pointers, walks to
 * the extrema, Morse-Smale ids.                                            */
int32_t oracle_segment_grid(const float* f, int32_t nx, int32_t ny, int32_t nz,
                            int32_t* order, int32_t* asc, int32_t* desc,
                            int32_t* ms, int32_t* num_cells) {
    if (!or_grid_ok(nx, ny, nz)) return OR_ERR_ARG;
    const int64_t n = (int64_t)nx * ny * nz;
    int32_t* ap = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* dp = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t s = (!ap || !dp) ? OR_ERR_OOM : OR_OK;
    if (!s) s = oracle_order(f, n, order);
    if (!s) s = oracle_steepest_grid(order, nx, ny, nz, ap, dp);
    if (!s) s = oracle_walk_memo(ap, n, asc);
    if (!s) s = oracle_walk_memo(dp, n, desc);
    if (!s) s = oracle_ms(asc, desc, n, ms, num_cells);
    free(ap);
    free(dp);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Connected components by breadth-first search (the ground truth for
 * Alg. 3, mirrored to the smallest id).  Seeds are scanned in increasing id
 * order, so the seed that opens a component is its smallest vertex id.     */

int32_t oracle_cc_grid(const uint8_t* mask, int32_t nx, int32_t ny, int32_t nz,
                       int32_t conn, int32_t* label) {
    if (!or_grid_ok(nx, ny, nz) || (conn != 6 && conn != 14)) return OR_ERR_ARG;
    const int64_t n = (int64_t)nx * ny * nz;
    const int (*off)[3] = conn == 6 ? OR_FACE6 : OR_FREUD;
    int32_t* queue = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!queue) return OR_ERR_OOM;
    for (int64_t v = 0; v < n; ++v) label[v] = -1;
    for (int64_t s = 0; s < n; ++s) {
        if (!mask[s] || label[s] != -1) continue;
        int64_t head = 0, tail = 0;
        label[s] = (int32_t)s;
        queue[tail++] = (int32_t)s;
        while (head < tail) {
            const int64_t w = queue[head++];
            const int64_t x = w % nx, y = (w / nx) % ny, z = w / ((int64_t)nx * ny);
            for (int k = 0; k < conn; ++k) {
                const int64_t xx = x + off[k][0], yy = y + off[k][1],
                              zz = z + off[k][2];
                if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny ||
                    zz >= nz)
                    continue;
                const int64_t u = xx + (int64_t)nx * (yy + (int64_t)ny * zz);
                if (mask[u] && label[u] == -1) {
                    label[u] = (int32_t)s;
                    queue[tail++] = (int32_t)u;
                }
            }
        }
    }
    free(queue);
    return OR_OK;
}

int32_t oracle_cc_csr(const int32_t* row, const int32_t* col, int32_t n,
                      int32_t* label) {
    if (n < 0) return OR_ERR_ARG;
    int32_t* queue = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!queue) return OR_ERR_OOM;
    for (int32_t v = 0; v < n; ++v) label[v] = -1;
    for (int32_t s = 0; s < n; ++s) {
        if (label[s] != -1) continue;
        int64_t head = 0, tail = 0;
        label[s] = s;
        queue[tail++] = s;
        while (head < tail) {
            const int32_t w = queue[head++];
            for (int32_t e = row[w]; e < row[w + 1]; ++e) {
                const int32_t u = col[e];
                if (u < 0 || u >= n) {
                    free(queue);
                    return OR_ERR_ARG;
                }
                if (label[u] == -1) {
                    label[u] = s;
                    queue[tail++] = u;
                }
            }
        }
    }
    free(queue);
    return OR_OK;
}

/* The component of one vertex, by BFS from it: its smallest id and its
 * size (sampled checks on grids too large to label in full).  A bitmap of
 * visited vertices keeps the memory at n/8 bytes plus the queue.           */
int32_t oracle_cc_grid_at(const uint8_t* mask, int32_t nx, int32_t ny,
                          int32_t nz, int32_t conn, int64_t v, int32_t* min_id,
                          int64_t* size) {
    if (!or_grid_ok(nx, ny, nz) || (conn != 6 && conn != 14)) return OR_ERR_ARG;
    const int64_t n = (int64_t)nx * ny * nz;
    if (v < 0 || v >= n) return OR_ERR_ARG;
    if (!mask[v]) {
        *min_id = -1;
        *size = 0;
        return OR_OK;
    }
    const int (*off)[3] = conn == 6 ? OR_FACE6 : OR_FREUD;
    uint8_t* seen = (uint8_t*)calloc((size_t)(n / 8 + 1), 1);
    int64_t cap = 1 << 20, head = 0, tail = 0;
    int32_t* queue = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
    if (!seen || !queue) {
        free(seen);
        free(queue);
        return OR_ERR_OOM;
    }
    int64_t best = v, count = 0;
    seen[v >> 3] |= (uint8_t)(1u << (v & 7));
    queue[tail++] = (int32_t)v;
    while (head < tail) {
        const int64_t w = queue[head++];
        if (w < best) best = w;
        const int64_t x = w % nx, y = (w / nx) % ny, z = w / ((int64_t)nx * ny);
        for (int k = 0; k < conn; ++k) {
            const int64_t xx = x + off[k][0], yy = y + off[k][1], zz = z + off[k][2];
            if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz)
                continue;
            const int64_t u = xx + (int64_t)nx * (yy + (int64_t)ny * zz);
            if (!mask[u] || (seen[u >> 3] >> (u & 7) & 1)) continue;
            seen[u >> 3] |= (uint8_t)(1u << (u & 7));
            if (tail == cap) {
                if (head > 0) { /* slide the live part of the queue down */
                    memmove(queue, queue + head, (size_t)(tail - head) * sizeof(int32_t));
                    tail -= head;
                    head = 0;
                }
                if (tail == cap) {
                    cap *= 2;
                    int32_t* q2 = (int32_t*)realloc(queue, (size_t)cap * sizeof(int32_t));
                    if (!q2) {
                        free(seen);
                        free(queue);
                        return OR_ERR_OOM;
                    }
                    queue = q2;
                }
            }
            queue[tail++] = (int32_t)u;
        }
        ++count;
    }
    free(seen);
    free(queue);
    *min_id = (int32_t)best;
    *size = count;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Adjacency of labelled regions (the preview of the Morse-Smale complex
 * assembled from the segmentations, Related Work; the extremum graph named
 * as future work in the Conclusion): every edge (u, v) of the implicit
 * triangulation (conn 14) or of the face grid (conn 6) whose endpoints carry
 * two different non-negative labels contributes the pair (min, max) of the
 * two labels.  Output: the distinct pairs in lexicographic order, written to
 * a_out / b_out (caller-provided, cap entries) and counted in *count.  When
 * more than cap distinct pairs exist, *count holds their number and nothing
 * beyond cap is written.                                                    */

static int or_cmp_u64(const void* x, const void* y) {
    const uint64_t a = *(const uint64_t*)x, b = *(const uint64_t*)y;
    return a < b ? -1 : a > b;
}

int oracle_adjacency_grid(const int32_t* label, int32_t nx, int32_t ny, int32_t nz, int conn,
                          int32_t* a_out, int32_t* b_out, int64_t cap, int64_t* count) {
    if (!or_grid_ok(nx, ny, nz) || !label || !count || (conn != 6 && conn != 14) || cap < 0) return OR_ERR_ARG;
    const int (*off)[3] = conn == 6 ? OR_FACE6 : OR_FREUD;
    const int64_t n = (int64_t)nx * ny * nz;
    /* every edge once: only the offsets that come first in the table of each
     * +- pair (the even entries) are followed from each vertex */
    int64_t m = 0, mcap = 1024;
    uint64_t* pairs = (uint64_t*)malloc((size_t)mcap * sizeof(uint64_t));
    if (!pairs) return OR_ERR_OOM;
    for (int64_t v = 0; v < n; ++v) {
        const int64_t x = v % nx, y = (v / nx) % ny, z = v / ((int64_t)nx * ny);
        for (int k = 0; k < conn; k += 2) {
            const int64_t xx = x + off[k][0], yy = y + off[k][1], zz = z + off[k][2];
            if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) continue;
            const int64_t u = xx + (int64_t)nx * (yy + (int64_t)ny * zz);
            const int32_t a = label[v], b = label[u];
            if (a < 0 || b < 0 || a == b) continue;
            if (m == mcap) {
                mcap *= 2;
                uint64_t* p2 = (uint64_t*)realloc(pairs, (size_t)mcap * sizeof(uint64_t));
                if (!p2) {
                    free(pairs);
                    return OR_ERR_OOM;
                }
                pairs = p2;
            }
            const uint32_t lo = (uint32_t)(a < b ? a : b), hi = (uint32_t)(a < b ? b : a);
            pairs[m++] = ((uint64_t)lo << 32) | hi;
        }
    }
    qsort(pairs, (size_t)m, sizeof(uint64_t), or_cmp_u64);
    int64_t k = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (i > 0 && pairs[i] == pairs[i - 1]) continue;
        if (k < cap) {
            a_out[k] = (int32_t)(pairs[i] >> 32);
            b_out[k] = (int32_t)(uint32_t)pairs[i];
        }
        ++k;
    }
    free(pairs);
    *count = k;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Arcs of the extremum graph with their saddles (Conclusion: the extremum
 * graph that the segmentations make computable).  `label` holds maximum
 * labels (sense = +1) or minimum labels (sense = -1) and `order` the vertex
 * order.  Every edge (u, v) between two different non-negative labels a, b
 * crosses from one region into the other at a level: for maxima the lower
 * of its two ends in the order (a path between the two maxima through this
 * edge must come down to it), for minima the higher.  The saddle of the
 * pair (min(a,b), max(a,b)) is the end vertex with the highest such level
 * over all of the pair's edges for maxima, the lowest for minima.  Output:
 * the distinct pairs in lexicographic order with their saddle vertex; cap
 * and *count as for oracle_adjacency_grid.                                  */

typedef struct {
    uint64_t key;  /* lo << 32 | hi */
    int32_t level; /* order of the crossing vertex */
    int32_t vertex;
} or_arc;

static int or_cmp_arc(const void* x, const void* y) {
    const or_arc* p = (const or_arc*)x;
    const or_arc* q = (const or_arc*)y;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return (p->level > q->level) - (p->level < q->level);
}

int oracle_extremum_graph(const int32_t* label, const int32_t* order, int32_t nx, int32_t ny, int32_t nz,
                          int conn, int sense, int32_t* a_out, int32_t* b_out, int32_t* saddle_out,
                          int64_t cap, int64_t* count) {
    if (!or_grid_ok(nx, ny, nz) || !label || !order || !count || (conn != 6 && conn != 14) ||
        (sense != 1 && sense != -1) || cap < 0)
        return OR_ERR_ARG;
    const int (*off)[3] = conn == 6 ? OR_FACE6 : OR_FREUD;
    const int64_t n = (int64_t)nx * ny * nz;
    int64_t m = 0, mcap = 1024;
    or_arc* arcs = (or_arc*)malloc((size_t)mcap * sizeof(or_arc));
    if (!arcs) return OR_ERR_OOM;
    for (int64_t v = 0; v < n; ++v) {
        const int64_t x = v % nx, y = (v / nx) % ny, z = v / ((int64_t)nx * ny);
        for (int k = 0; k < conn; k += 2) { /* each edge once */
            const int64_t xx = x + off[k][0], yy = y + off[k][1], zz = z + off[k][2];
            if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) continue;
            const int64_t u = xx + (int64_t)nx * (yy + (int64_t)ny * zz);
            const int32_t la = label[v], lb = label[u];
            if (la < 0 || lb < 0 || la == lb) continue;
            if (m == mcap) {
                mcap *= 2;
                or_arc* p2 = (or_arc*)realloc(arcs, (size_t)mcap * sizeof(or_arc));
                if (!p2) {
                    free(arcs);
                    return OR_ERR_OOM;
                }
                arcs = p2;
            }
            const int lower_is_v = order[v] < order[u];
            /* maxima: the crossing vertex is the lower end; minima: the higher */
            const int64_t w = (sense > 0) == lower_is_v ? v : u;
            const uint32_t lo = (uint32_t)(la < lb ? la : lb), hi = (uint32_t)(la < lb ? lb : la);
            arcs[m].key = ((uint64_t)lo << 32) | hi;
            arcs[m].level = order[w];
            arcs[m].vertex = (int32_t)w;
            ++m;
        }
    }
    qsort(arcs, (size_t)m, sizeof(or_arc), or_cmp_arc);
    int64_t k = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (i > 0 && arcs[i].key == arcs[i - 1].key) continue;
        /* the run of this key is sorted by level: its last entry is the
         * highest crossing, its first the lowest */
        int64_t j = i;
        while (j + 1 < m && arcs[j + 1].key == arcs[i].key) ++j;
        if (k < cap) {
            a_out[k] = (int32_t)(arcs[i].key >> 32);
            b_out[k] = (int32_t)(uint32_t)arcs[i].key;
            saddle_out[k] = sense > 0 ? arcs[j].vertex : arcs[i].vertex;
        }
        ++k;
    }
    free(arcs);
    *count = k;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* The same two operations over an explicit mesh (the explicit-triangulation
 * case): the edges are the CSR entries (row[n+1], col[row[n]]), symmetric;
 * each edge is taken from the row of its smaller end.  order may be NULL
 * for the plain adjacency; with order, saddle_out receives each pair's
 * crossing vertex as in oracle_extremum_graph.                              */

int oracle_adjacency_csr(const int32_t* label, const int32_t* order, const int32_t* row, const int32_t* col,
                         int32_t n, int sense, int32_t* a_out, int32_t* b_out, int32_t* saddle_out, int64_t cap,
                         int64_t* count) {
    if (n < 0 || !label || !row || !col || !count || cap < 0 || (order && sense != 1 && sense != -1))
        return OR_ERR_ARG;
    int64_t m = 0, mcap = 1024;
    or_arc* arcs = (or_arc*)malloc((size_t)mcap * sizeof(or_arc));
    if (!arcs) return OR_ERR_OOM;
    for (int32_t v = 0; v < n; ++v) {
        for (int32_t e = row[v]; e < row[v + 1]; ++e) {
            const int32_t u = col[e];
            if (u < 0 || u >= n) {
                free(arcs);
                return OR_ERR_ARG;
            }
            if (u <= v) continue; /* each edge from its smaller end */
            const int32_t la = label[v], lb = label[u];
            if (la < 0 || lb < 0 || la == lb) continue;
            if (m == mcap) {
                mcap *= 2;
                or_arc* p2 = (or_arc*)realloc(arcs, (size_t)mcap * sizeof(or_arc));
                if (!p2) {
                    free(arcs);
                    return OR_ERR_OOM;
                }
                arcs = p2;
            }
            const uint32_t lo = (uint32_t)(la < lb ? la : lb), hi = (uint32_t)(la < lb ? lb : la);
            arcs[m].key = ((uint64_t)lo << 32) | hi;
            if (order) {
                const int lower_is_v = order[v] < order[u];
                const int32_t w = (sense > 0) == lower_is_v ? v : u;
                arcs[m].level = order[w];
                arcs[m].vertex = w;
            } else {
                arcs[m].level = 0;
                arcs[m].vertex = 0;
            }
            ++m;
        }
    }
    qsort(arcs, (size_t)m, sizeof(or_arc), or_cmp_arc);
    int64_t k = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (i > 0 && arcs[i].key == arcs[i - 1].key) continue;
        int64_t j = i;
        while (j + 1 < m && arcs[j + 1].key == arcs[i].key) ++j;
        if (k < cap) {
            a_out[k] = (int32_t)(arcs[i].key >> 32);
            b_out[k] = (int32_t)(uint32_t)arcs[i].key;
            if (order && saddle_out) saddle_out[k] = sense > 0 ? arcs[j].vertex : arcs[i].vertex;
        }
        ++k;
    }
    free(arcs);
    *count = k;
    return OR_OK;
}
