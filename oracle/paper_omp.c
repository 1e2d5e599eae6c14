/*
 * paper_omp.c -- CPU baseline: the paper's shared-memory method on all host
 * cores with OpenMP (arXiv 2409.03771).
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY, and not the oracle: it is the
 * method the paper runs inside each rank, restated for one shared-memory
 * process, so that the GPU figures have the paper's own method on this
 * box's host cores beside them.  Only the tests and the CPU-baseline leg of
 * the benchmark load it.  It shares no code with the CUDA path or with
 * msc_oracle.c (the tests compare it with the oracle).
 *
 *   - Segmentation (Alg. 1, one rank, no ghost vertices): every vertex
 *     points at its steepest neighbour (a vertex with none points at
 *     itself); then each thread takes a contiguous block of vertices as its
 *     list of active vertices and repeats, over the list, u = d[v],
 *     w = d[u] (an atomic read: another thread may be moving u), drop v when
 *     u = w, else d[v] = w -- in place, until its list is empty.  Once for
 *     the descending pointers, once for the ascending ones.
 *   - Connected components (Alg. 3, mirrored to the smallest id, which the
 *     library and the oracle use): every feature vertex points at the
 *     smallest id among itself and its feature neighbours, path compression
 *     as above, then stitching -- for every feature vertex v and feature
 *     neighbour u with d[u] < d[v], d[d[v]] = d[u] -- and path compression
 *     again.  One stitching pass can lose a merge when two threads hook the
 *     same root, so stitching and compression repeat until a stitching pass
 *     changes nothing; the result is the smallest id of every component.
 *   - The vertex order (the paper's preprocessing, done by TTK) and the
 *     dense Morse-Smale cell ids (not in the paper) come from parallel LSD
 *     radix sorts, so that the baseline produces every output of the GPU
 *     path: order by (f, id), cell id = rank of (asc, desc) among the
 *     distinct pairs.
 *
 * Grid vertex ids are x + nx * (y + ny * z); the triangulation's link is the
 * 14 Freudenthal offsets, the face grid's the 6 axis offsets.
 * Return codes: 0 ok, -1 bad argument, -4 NaN, -8 out of memory.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PO_OK 0
#define PO_ERR_ARG (-1)
#define PO_ERR_NAN (-4)
#define PO_ERR_OOM (-8)

static const int po_link14[14][3] = {
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},   {0, 0, -1},  {1, 1, 0},
    {-1, -1, 0}, {1, 0, 1}, {-1, 0, -1}, {0, 1, 1}, {0, -1, -1}, {1, 1, 1},  {-1, -1, -1}};

int po_threads(void) { return omp_get_max_threads(); }

static double po_now(void) { return omp_get_wtime(); }

/* ------------------------------------------------------------------------ */
/* Parallel stable LSD radix sort of (key, value) by the low `bits` bits of
 * the key, 8 bits per pass; each thread counts and moves a contiguous block.
 * Returns 1 when the result is in the second pair of buffers.               */

static int po_radix_u64(uint64_t* k0, int32_t* v0, uint64_t* k1, int32_t* v1, int64_t n, int bits) {
    const int passes = (bits + 7) / 8;
    const int T = omp_get_max_threads();
    int64_t* cnt = (int64_t*)calloc((size_t)T * 256, sizeof(int64_t));
    if (!cnt) return -1;
    uint64_t *ka = k0, *kb = k1;
    int32_t *va = v0, *vb = v1;
    for (int p = 0; p < passes; ++p) {
        const int sh = 8 * p;
#pragma omp parallel num_threads(T)
        {
            const int t = omp_get_thread_num();
            const int64_t b = n * t / T, e = n * (t + 1) / T;
            int64_t* c = cnt + (size_t)t * 256;
            memset(c, 0, 256 * sizeof(int64_t));
            for (int64_t i = b; i < e; ++i) c[(ka[i] >> sh) & 255u]++;
#pragma omp barrier
#pragma omp single
            {
                int64_t run = 0;
                for (int d = 0; d < 256; ++d)
                    for (int u = 0; u < T; ++u) {
                        const int64_t x = cnt[(size_t)u * 256 + d];
                        cnt[(size_t)u * 256 + d] = run;
                        run += x;
                    }
            }
            for (int64_t i = b; i < e; ++i) {
                const int64_t q = c[(ka[i] >> sh) & 255u]++;
                kb[q] = ka[i];
                vb[q] = va[i];
            }
        }
        uint64_t* tk = ka;
        ka = kb;
        kb = tk;
        int32_t* tv = va;
        va = vb;
        vb = tv;
    }
    free(cnt);
    return passes & 1;
}

static inline uint32_t po_fkey(float x) {
    uint32_t u;
    memcpy(&u, &x, sizeof(u));
    if (u == 0x80000000u) u = 0u; /* -0.0 equals +0.0 */
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

/* order[v] = position of v when the vertices are sorted by (f, id). */
int po_order(const float* f, int64_t n, int32_t* order) {
    if (n < 0 || n > INT32_MAX) return PO_ERR_ARG;
    uint64_t* k0 = (uint64_t*)malloc((size_t)n * 8 + 8);
    uint64_t* k1 = (uint64_t*)malloc((size_t)n * 8 + 8);
    int32_t* v0 = (int32_t*)malloc((size_t)n * 4 + 4);
    int32_t* v1 = (int32_t*)malloc((size_t)n * 4 + 4);
    if (!k0 || !k1 || !v0 || !v1) {
        free(k0), free(k1), free(v0), free(v1);
        return PO_ERR_OOM;
    }
    int nan = 0;
#pragma omp parallel for reduction(| : nan) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        nan |= f[i] != f[i];
        k0[i] = po_fkey(f[i]);
        v0[i] = (int32_t)i;
    }
    int rc = PO_OK;
    if (nan) {
        rc = PO_ERR_NAN;
    } else {
        const int alt = po_radix_u64(k0, v0, k1, v1, n, 32);
        if (alt < 0) {
            rc = PO_ERR_OOM;
        } else {
            const int32_t* ids = alt ? v1 : v0;
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) order[ids[i]] = (int32_t)i;
        }
    }
    free(k0), free(k1), free(v0), free(v1);
    return rc;
}

/* Steepest pointers over the 14-neighbour link (Alg. 1 initialisation). */
int po_steepest_grid(const int32_t* order, int32_t nx, int32_t ny, int32_t nz, int32_t* asc, int32_t* desc) {
    if (nx <= 0 || ny <= 0 || nz <= 0) return PO_ERR_ARG;
    const int64_t n = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
        const int64_t x = v % nx, y = (v / nx) % ny, z = v / ((int64_t)nx * ny);
        int64_t up = v, dn = v;
        int32_t oup = order[v], odn = order[v];
        for (int k = 0; k < 14; ++k) {
            const int64_t xx = x + po_link14[k][0], yy = y + po_link14[k][1], zz = z + po_link14[k][2];
            if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) continue;
            const int64_t u = xx + (int64_t)nx * (yy + (int64_t)ny * zz);
            if (order[u] > oup) {
                oup = order[u];
                up = u;
            }
            if (order[u] < odn) {
                odn = order[u];
                dn = u;
            }
        }
        desc[v] = (int32_t)up;
        asc[v] = (int32_t)dn;
    }
    return PO_OK;
}

/* Alg. 1's path compression: per-thread lists of active vertices, in place.
 * Negative entries are inactive. */
void po_compress(int32_t* d, int64_t n) {
#pragma omp parallel
    {
        const int t = omp_get_thread_num(), T = omp_get_num_threads();
        const int64_t b = n * t / T, e = n * (t + 1) / T;
        int32_t* act = (int32_t*)malloc((size_t)(e - b) * 4 + 4);
        int64_t na = 0;
        for (int64_t v = b; v < e; ++v) {
            const int32_t p = __atomic_load_n(&d[v], __ATOMIC_RELAXED);
            if (p >= 0 && p != v) act[na++] = (int32_t)v;
        }
        while (na > 0) {
            int64_t keep = 0;
            for (int64_t i = 0; i < na; ++i) {
                const int32_t v = act[i];
                const int32_t u = __atomic_load_n(&d[v], __ATOMIC_RELAXED);
                const int32_t w = __atomic_load_n(&d[u], __ATOMIC_RELAXED);
                if (u == w) continue; /* v points at a root: done */
                __atomic_store_n(&d[v], w, __ATOMIC_RELAXED);
                act[keep++] = v;
            }
            na = keep;
        }
        free(act);
    }
}

/* Dense cell ids: rank of (asc[v], desc[v]) among the distinct pairs. */
int po_ms(const int32_t* asc, const int32_t* desc, int64_t n, int32_t* ms, int32_t* num_cells) {
    if (n < 0 || n > INT32_MAX) return PO_ERR_ARG;
    int b = 0;
    while (((int64_t)1 << b) < n) ++b;
    uint64_t* k0 = (uint64_t*)malloc((size_t)n * 8 + 8);
    uint64_t* k1 = (uint64_t*)malloc((size_t)n * 8 + 8);
    int32_t* v0 = (int32_t*)malloc((size_t)n * 4 + 4);
    int32_t* v1 = (int32_t*)malloc((size_t)n * 4 + 4);
    const int T = omp_get_max_threads();
    int64_t* part = (int64_t*)calloc((size_t)T + 1, sizeof(int64_t));
    if (!k0 || !k1 || !v0 || !v1 || !part) {
        free(k0), free(k1), free(v0), free(v1), free(part);
        return PO_ERR_OOM;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        k0[i] = ((uint64_t)(uint32_t)asc[i] << b) | (uint32_t)desc[i];
        v0[i] = (int32_t)i;
    }
    const int alt = po_radix_u64(k0, v0, k1, v1, n, 2 * b);
    const uint64_t* ks = alt ? k1 : k0;
    const int32_t* vs = alt ? v1 : v0;
    /* heads of runs of equal keys, counted per thread block, then ranked */
#pragma omp parallel num_threads(T)
    {
        const int t = omp_get_thread_num();
        const int64_t lo = n * t / T, hi = n * (t + 1) / T;
        int64_t c = 0;
        for (int64_t i = lo; i < hi; ++i) c += i == 0 || ks[i] != ks[i - 1];
        part[t + 1] = c;
#pragma omp barrier
#pragma omp single
        for (int u = 0; u < T; ++u) part[u + 1] += part[u];
        int64_t r = part[t] - 1;
        for (int64_t i = lo; i < hi; ++i) {
            r += i == 0 || ks[i] != ks[i - 1];
            ms[vs[i]] = (int32_t)r;
        }
    }
    *num_cells = (int32_t)part[T];
    free(k0), free(k1), free(v0), free(v1), free(part);
    return PO_OK;
}

/* The whole segmentation; secs[4] = seconds of order, steepest, the two
 * path compressions, cell ids. */
int po_segment_grid(const float* f, int32_t nx, int32_t ny, int32_t nz, int32_t* order, int32_t* asc,
                    int32_t* desc, int32_t* ms, int32_t* num_cells, double* secs) {
    if (nx <= 0 || ny <= 0 || nz <= 0) return PO_ERR_ARG;
    const int64_t n = (int64_t)nx * ny * nz;
    double t0 = po_now();
    int rc = po_order(f, n, order);
    if (rc) return rc;
    double t1 = po_now();
    po_steepest_grid(order, nx, ny, nz, asc, desc);
    double t2 = po_now();
    po_compress(desc, n);
    po_compress(asc, n);
    double t3 = po_now();
    rc = po_ms(asc, desc, n, ms, num_cells);
    double t4 = po_now();
    if (secs) {
        secs[0] = t1 - t0;
        secs[1] = t2 - t1;
        secs[2] = t3 - t2;
        secs[3] = t4 - t3;
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Connected components (Alg. 3, mirrored to the smallest id).              */

/* Stitching for one edge (v, u): hook v's target under u's target when u's
 * is smaller (labels only ever decrease, so no cycle forms).  Returns 1 when
 * a root moved. */
static inline int po_hook(int32_t* d, int32_t dv, int64_t u) {
    const int32_t du = __atomic_load_n(&d[u], __ATOMIC_RELAXED);
    if (du < 0 || du >= dv) return 0;
    const int32_t cur = __atomic_load_n(&d[dv], __ATOMIC_RELAXED);
    if (du >= cur) return 0;
    __atomic_store_n(&d[dv], du, __ATOMIC_RELAXED);
    return 1;
}

/* label[v] = smallest id of v's component of the mask (6 or 14
 * neighbours), -1 off the mask. */
int po_cc_grid(const uint8_t* mask, int32_t nx, int32_t ny, int32_t nz, int32_t conn, int32_t* label) {
    if (nx <= 0 || ny <= 0 || nz <= 0 || (conn != 6 && conn != 14)) return PO_ERR_ARG;
    const int64_t n = (int64_t)nx * ny * nz;
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
#define PO_GRID_NEIGHBOURS(BODY)                                                                   \
    {                                                                                              \
        const int64_t x = v % nx, y = (v / nx) % ny, z = v / sz;                                   \
        for (int j = 0; j < conn; ++j) {                                                           \
            const int64_t xx = x + po_link14[j][0], yy = y + po_link14[j][1], zz = z + po_link14[j][2]; \
            if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) continue;          \
            const int64_t u = xx * sx + yy * sy + zz * sz;                                         \
            if (!mask[u]) continue;                                                                \
            BODY                                                                                   \
        }                                                                                          \
    }
    /* every feature vertex points at the smallest id among itself and its
     * feature neighbours */
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
        if (!mask[v]) {
            label[v] = -1;
            continue;
        }
        int64_t m = v;
        PO_GRID_NEIGHBOURS(if (u < m) m = u;)
        label[v] = (int32_t)m;
    }
    po_compress(label, n);
    for (;;) {
        int64_t moved = 0;
#pragma omp parallel for reduction(+ : moved) schedule(static)
        for (int64_t v = 0; v < n; ++v) {
            const int32_t dv = __atomic_load_n(&label[v], __ATOMIC_RELAXED);
            if (dv < 0) continue;
            PO_GRID_NEIGHBOURS(moved += po_hook(label, dv, u);)
        }
        if (!moved) break;
        po_compress(label, n);
    }
#undef PO_GRID_NEIGHBOURS
    return PO_OK;
}

/* Components of an explicit graph (symmetric CSR); isolated vertices label
 * themselves. */
int po_cc_csr(const int32_t* row, const int32_t* col, int32_t n, int32_t* label) {
    if (n < 0) return PO_ERR_ARG;
    int bad = 0;
#pragma omp parallel for reduction(| : bad) schedule(static)
    for (int64_t v = 0; v < n; ++v) {
        int64_t m = v;
        for (int32_t e = row[v]; e < row[v + 1]; ++e) {
            const int32_t u = col[e];
            if (u < 0 || u >= n) {
                bad = 1;
                continue;
            }
            if (u < m) m = u;
        }
        label[v] = (int32_t)m;
    }
    if (bad) return PO_ERR_ARG;
    po_compress(label, n);
    for (;;) {
        int64_t moved = 0;
#pragma omp parallel for reduction(+ : moved) schedule(static)
        for (int64_t v = 0; v < n; ++v) {
            const int32_t dv = __atomic_load_n(&label[v], __ATOMIC_RELAXED);
            for (int32_t e = row[v]; e < row[v + 1]; ++e) moved += po_hook(label, dv, col[e]);
        }
        if (!moved) break;
        po_compress(label, n);
    }
    return PO_OK;
}

/* Seconds of a full connected-components call, for the benchmark. */
double po_wtime(void) { return po_now(); }
