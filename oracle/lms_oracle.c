/*
 * lms_oracle.c - plain, slow, single-threaded FP64 reference for Laplacian
 * mesh smoothing (LMS) and its vertex orderings.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  It shares no code with the
 * CUDA library and must never be called from the product path.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no -ffast-math): every
 * floating-point operation below is one IEEE-754 round-to-nearest operation
 * in the order written.
 *
 * What each function follows (Aupy, Park & Raghavan, "Locality-Aware
 * Laplacian Mesh Smoothing"):
 *   or_triangle_quality / or_vertex_quality / or_mesh_quality - Section 3.2:
 *       edge-length ratio (shortest over longest edge) per triangle, the mean
 *       over the triangles attached to a vertex, the mean over all |V|
 *       vertices (Algorithm 1 divides the summed quality by |V|).
 *   or_jacobi_sweep - Eq. 1 applied to every interior vertex from the old
 *       positions (simultaneous update; boundary vertices keep their place).
 *   or_inplace_sweep - Algorithm 1's inner loop: interior vertices visited in
 *       a given sequence, each moved by Eq. 1 using the current positions.
 *   or_smooth - Algorithm 1's outer loop with the stopping rule of Section
 *       5.1 (stop once the global quality improves by less than a criterion)
 *       and an iteration cap (Section 3.2 notes that one exists).
 *   or_order_random / or_order_bfs / or_order_rdr - the orderings compared in
 *       Section 5.2: a seeded random permutation, breadth-first search, and
 *       the Reuse Distance Reducing ordering of Algorithm 2.
 *   or_relabel - storing the mesh under an ordering (the node array of the
 *       Section 5.2.3 footnote, relabelled).
 *   or_color_greedy - first-fit colouring of the interior vertices in
 *       storage order; the sequence "colour by colour, storage order inside a
 *       colour" is the in-place sweep that a coloured Gauss-Seidel reproduces.
 *   or_order_rbfs - the reversed breadth-first order (BFS visit order read
 *       backwards) that Section 2 reports from Munson and Hovland's study.
 *   or_order_brdr - a blocked variant of Algorithm 2 that is not in the paper:
 *       the BFS order cut into blocks of consecutive positions, Algorithm 2
 *       applied to each block's own subgraph, blocks kept in BFS order.
 *   or_block_sequence - an order for Algorithm 1's in-place sweep that is not
 *       in the paper: the storage order cut into tiles of consecutive
 *       positions, the tiles coloured first-fit (ascending tile index) so that
 *       no two tiles of one colour share an edge between interior vertices,
 *       and the interior vertices visited by (tile colour, tile, vertex
 *       colour, storage position).  Tiles of one colour, and the vertices of
 *       one colour inside a tile, are independent, so a parallel sweep that
 *       runs them together equals the sequential sweep in this order.
 *   or_access_trace / or_reuse_distances / or_quantile - Section 2.2's reuse
 *       distance over the data accesses of one sweep (Fig. 3: a vertex, then
 *       its neighbours), and the quantiles of Table 2 (the X quantile is the
 *       smallest value with at least a fraction X of the population at or
 *       below it).
 *
 * Readings where the paper is silent (the same list is kept with the design
 * notes):
 *   - neighbour sums run left to right over the stored row, x and y
 *     separately, starting from 0.0; the mean is one IEEE division by the
 *     neighbour count;
 *   - a triangle whose longest edge has length 0 has quality 0; a vertex with
 *     no triangle has quality 0 and still counts in |V|;
 *   - the quality mean of a vertex sums its triangles in ascending triangle id;
 *     the mesh mean sums vertices in ascending id;
 *   - RDR sort key is (quality, vertex id) ascending; neighbour lists include
 *     boundary vertices; l[0] is the first (worst-quality) member of l;
 *     vertices never reached are appended in ascending id at the end;
 *   - BFS starts at vertex 0, visits neighbours in ascending id and restarts
 *     at the smallest unvisited id when the queue empties;
 *   - RANDOM is a Fisher-Yates shuffle driven by splitmix64 (Steele, Lea &
 *     Flood, OOPSLA 2014) seeded with the given seed;
 *   - the stopping rule stops after sweep k when Q_k >= goal or
 *     Q_k - Q_{k-1} < tol (a signed difference);
 *   - the access trace of a sweep visits the interior vertices in the given
 *     sequence; for each it lists the vertex itself (optional) and then its
 *     stored row; an element is a vertex.  Two measures of the distance
 *     between consecutive accesses to one element: the number of distinct
 *     elements accessed in between (Section 2.2, Fig. 1) and the number of
 *     accesses in between (Table 2's maxima exceed the vertex count, which
 *     only this measure allows).  First accesses have no reuse distance and
 *     are left out of the population;
 *   - the quantile index is k = ceil(X * m) in double precision, clamped to
 *     [1, m], over the m sorted distances (the k-th smallest is returned).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_OOM -2

/* ---------------------------------------------------------------- quality */

/* Section 3.2: shortest edge length divided by longest edge length. */
static double triangle_quality(const double* xy, int32_t a, int32_t b, int32_t c) {
    const int32_t v[3] = {a, b, c};
    double len[3];
    for (int e = 0; e < 3; ++e) {
        int32_t p = v[e], q = v[(e + 1) % 3];
        double dx = xy[2 * q] - xy[2 * p];
        double dy = xy[2 * q + 1] - xy[2 * p + 1];
        len[e] = sqrt(dx * dx + dy * dy);
    }
    double lo = len[0], hi = len[0];
    for (int e = 1; e < 3; ++e) {
        if (len[e] < lo) lo = len[e];
        if (len[e] > hi) hi = len[e];
    }
    if (hi == 0.0) return 0.0;
    return lo / hi;
}

int or_triangle_quality(int32_t ntri, const int32_t* tri, const double* xy, double* q_t) {
    if (ntri < 0 || (ntri > 0 && (!tri || !xy || !q_t))) return OR_ERR_ARG;
    for (int32_t t = 0; t < ntri; ++t)
        q_t[t] = triangle_quality(xy, tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]);
    return OR_OK;
}

/* Section 3.2: a vertex's quality is the mean quality of its triangles. */
int or_vertex_quality(int32_t n, int32_t ntri, const int32_t* tri, const double* xy, double* q_v) {
    if (n <= 0 || ntri < 0 || !xy || !q_v || (ntri > 0 && !tri)) return OR_ERR_ARG;
    double* sum = (double*)calloc((size_t)n, sizeof(double));
    int32_t* cnt = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    if (!sum || !cnt) { free(sum); free(cnt); return OR_ERR_OOM; }
    for (int32_t t = 0; t < ntri; ++t) {               /* ascending triangle id */
        double q = triangle_quality(xy, tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]);
        for (int k = 0; k < 3; ++k) {
            int32_t v = tri[3 * t + k];
            sum[v] = sum[v] + q;
            cnt[v] += 1;
        }
    }
    for (int32_t v = 0; v < n; ++v) q_v[v] = cnt[v] > 0 ? sum[v] / (double)cnt[v] : 0.0;
    free(sum); free(cnt);
    return OR_OK;
}

/* Algorithm 1: the global quality is the summed vertex quality over |V|. */
int or_mesh_quality(int32_t n, int32_t ntri, const int32_t* tri, const double* xy, double* Q) {
    if (!Q) return OR_ERR_ARG;
    double* q_v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!q_v) return OR_ERR_OOM;
    int rc = or_vertex_quality(n, ntri, tri, xy, q_v);
    if (rc == OR_OK) {
        double s = 0.0;
        for (int32_t v = 0; v < n; ++v) s = s + q_v[v];
        *Q = s / (double)n;
    }
    free(q_v);
    return rc;
}

/* ---------------------------------------------------------------- sweeps */

/* Eq. 1 for vertex v, reading positions from src: mean of the neighbours. */
static void laplacian_point(const int32_t* row_ptr, const int32_t* col_idx, const double* src,
                            int32_t v, double* px, double* py) {
    double sx = 0.0, sy = 0.0;
    int32_t N = row_ptr[v + 1] - row_ptr[v];
    for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
        int32_t u = col_idx[e];
        sx = sx + src[2 * u];
        sy = sy + src[2 * u + 1];
    }
    *px = sx / (double)N;
    *py = sy / (double)N;
}

/* One simultaneous (Jacobi) sweep: dst = Eq. 1 of src on interior vertices, src elsewhere. */
int or_jacobi_sweep(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                    const double* src, double* dst) {
    if (n <= 0 || !row_ptr || !col_idx || !is_boundary || !src || !dst || src == dst) return OR_ERR_ARG;
    for (int32_t v = 0; v < n; ++v) {
        if (is_boundary[v]) {
            dst[2 * v] = src[2 * v];
            dst[2 * v + 1] = src[2 * v + 1];
        } else {
            laplacian_point(row_ptr, col_idx, src, v, &dst[2 * v], &dst[2 * v + 1]);
        }
    }
    return OR_OK;
}

/* Algorithm 1's inner loop: visit seq[0..nseq) in order, smoothing each interior vertex in place. */
int or_inplace_sweep(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                     int32_t nseq, const int32_t* seq, double* xy) {
    if (n <= 0 || !row_ptr || !col_idx || !is_boundary || !xy || nseq < 0 || (nseq > 0 && !seq)) return OR_ERR_ARG;
    for (int32_t i = 0; i < nseq; ++i) {
        int32_t v = seq[i];
        if (v < 0 || v >= n) return OR_ERR_ARG;
        if (is_boundary[v]) continue;
        double px, py;
        laplacian_point(row_ptr, col_idx, xy, v, &px, &py);
        xy[2 * v] = px;
        xy[2 * v + 1] = py;
    }
    return OR_OK;
}

/*
 * Algorithm 1 with the stopping rule.  mode 0: Jacobi sweeps; mode 1: in-place
 * sweeps over seq.  tol < 0: exactly max_iters sweeps, no quality.  Otherwise
 * Q_0 is computed first and after sweep k the loop stops when Q_k >= goal or
 * Q_k - Q_{k-1} < tol.  q_hist (optional, max_iters + 1 entries) receives
 * Q_0..Q_k.  *iters receives the number of sweeps done.
 */
int or_smooth(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
              int32_t ntri, const int32_t* tri, double* xy, int32_t max_iters, int32_t mode,
              int32_t nseq, const int32_t* seq, double tol, double goal, int32_t* iters, double* q_hist) {
    if (n <= 0 || !xy || !iters || max_iters < 0 || (mode != 0 && mode != 1)) return OR_ERR_ARG;
    if (tol >= 0.0 && (ntri <= 0 || !tri)) return OR_ERR_ARG;
    double* tmp = NULL;
    if (mode == 0) {
        tmp = (double*)malloc(sizeof(double) * 2 * (size_t)n);
        if (!tmp) return OR_ERR_OOM;
    }
    double q_prev = 0.0;
    int rc = OR_OK;
    if (tol >= 0.0) {
        rc = or_mesh_quality(n, ntri, tri, xy, &q_prev);
        if (rc != OR_OK) goto done;
        if (q_hist) q_hist[0] = q_prev;
    }
    *iters = 0;
    for (int32_t k = 1; k <= max_iters; ++k) {
        if (mode == 0) {
            rc = or_jacobi_sweep(n, row_ptr, col_idx, is_boundary, xy, tmp);
            if (rc != OR_OK) goto done;
            memcpy(xy, tmp, sizeof(double) * 2 * (size_t)n);
        } else {
            rc = or_inplace_sweep(n, row_ptr, col_idx, is_boundary, nseq, seq, xy);
            if (rc != OR_OK) goto done;
        }
        *iters = k;
        if (tol >= 0.0) {
            double q;
            rc = or_mesh_quality(n, ntri, tri, xy, &q);
            if (rc != OR_OK) goto done;
            if (q_hist) q_hist[k] = q;
            if (q >= goal || q - q_prev < tol) break;
            q_prev = q;
        }
    }
done:
    free(tmp);
    return rc;
}

/* ------------------------------------------------------------- orderings */

static uint64_t splitmix64(uint64_t* state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* RANDOM: Fisher-Yates over 0..n-1, new_to_old[k] = original id stored at position k. */
int or_order_random(int32_t n, uint64_t seed, int32_t* new_to_old) {
    if (n <= 0 || !new_to_old) return OR_ERR_ARG;
    for (int32_t i = 0; i < n; ++i) new_to_old[i] = i;
    uint64_t st = seed;
    for (int32_t i = n - 1; i >= 1; --i) {
        int32_t j = (int32_t)(splitmix64(&st) % (uint64_t)(i + 1));
        int32_t t = new_to_old[i]; new_to_old[i] = new_to_old[j]; new_to_old[j] = t;
    }
    return OR_OK;
}

static int cmp_int32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* BFS: visit order of a breadth-first search from vertex 0, neighbours by ascending id. */
int or_order_bfs(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t* new_to_old) {
    if (n <= 0 || !row_ptr || !col_idx || !new_to_old) return OR_ERR_ARG;
    uint8_t* seen = (uint8_t*)calloc((size_t)n, 1);
    int32_t* nb = (int32_t*)malloc(sizeof(int32_t) * 64);
    if (!seen || !nb) { free(seen); free(nb); return OR_ERR_OOM; }
    int32_t nb_cap = 64, head = 0, tail = 0;
    for (int32_t root = 0; root < n; ++root) {
        if (seen[root]) continue;
        seen[root] = 1;
        new_to_old[tail++] = root;
        while (head < tail) {
            int32_t v = new_to_old[head++];
            int32_t len = row_ptr[v + 1] - row_ptr[v];
            if (len > nb_cap) {
                int32_t* g = (int32_t*)realloc(nb, sizeof(int32_t) * (size_t)len);
                if (!g) { free(seen); free(nb); return OR_ERR_OOM; }
                nb = g; nb_cap = len;
            }
            memcpy(nb, col_idx + row_ptr[v], sizeof(int32_t) * (size_t)len);
            qsort(nb, (size_t)len, sizeof(int32_t), cmp_int32);
            for (int32_t e = 0; e < len; ++e) {
                int32_t u = nb[e];
                if (!seen[u]) { seen[u] = 1; new_to_old[tail++] = u; }
            }
        }
    }
    free(seen); free(nb);
    return OR_OK;
}

/* Reversed BFS: the BFS visit order read from its last vertex to its first. */
int or_order_rbfs(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t* new_to_old) {
    if (n <= 0 || !new_to_old) return OR_ERR_ARG;
    int32_t* fwd = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!fwd) return OR_ERR_OOM;
    int rc = or_order_bfs(n, row_ptr, col_idx, fwd);
    if (rc == OR_OK)
        for (int32_t k = 0; k < n; ++k) new_to_old[k] = fwd[n - 1 - k];
    free(fwd);
    return rc;
}

/* RDR sort key: (quality, id) ascending */
static const double* g_key_q;
static int key_less(int32_t a, int32_t b) {
    if (g_key_q[a] < g_key_q[b]) return 1;
    if (g_key_q[a] > g_key_q[b]) return 0;
    return a < b;
}
static int cmp_key(const void* pa, const void* pb) {
    int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
    if (a == b) return 0;
    return key_less(a, b) ? -1 : 1;
}

/* l <- unprocessed neighbours of v sorted by increasing quality; returns |l| */
static int32_t unprocessed_neighbours(const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* processed,
                                      int32_t v, int32_t* l) {
    int32_t m = 0;
    for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
        if (!processed[col_idx[e]]) l[m++] = col_idx[e];
    qsort(l, (size_t)m, sizeof(int32_t), cmp_key);
    return m;
}

/*
 * Algorithm 2 (Reuse Distance Reducing ordering).  q_v: per-vertex quality.
 * For every interior vertex i in increasing quality that is not processed yet:
 * order i if needed, mark it processed, then walk: l = its unprocessed
 * neighbours by increasing quality; order the members of l not yet ordered;
 * mark l[0] processed and continue from l[0] until l is empty.
 */
int or_order_rdr(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                 const double* q_v, int32_t* new_to_old) {
    if (n <= 0 || !row_ptr || !col_idx || !is_boundary || !q_v || !new_to_old) return OR_ERR_ARG;
    int32_t max_deg = 0;
    for (int32_t v = 0; v < n; ++v)
        if (row_ptr[v + 1] - row_ptr[v] > max_deg) max_deg = row_ptr[v + 1] - row_ptr[v];
    uint8_t* processed = (uint8_t*)calloc((size_t)n, 1);
    uint8_t* sorted = (uint8_t*)calloc((size_t)n, 1);
    int32_t* interior = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* l = (int32_t*)malloc(sizeof(int32_t) * (size_t)(max_deg + 1));
    if (!processed || !sorted || !interior || !l) {
        free(processed); free(sorted); free(interior); free(l);
        return OR_ERR_OOM;
    }
    g_key_q = q_v;
    int32_t ni = 0;
    for (int32_t v = 0; v < n; ++v)
        if (!is_boundary[v]) interior[ni++] = v;
    qsort(interior, (size_t)ni, sizeof(int32_t), cmp_key);

    int32_t next_num = 0;
    for (int32_t ii = 0; ii < ni; ++ii) {
        int32_t i = interior[ii];
        if (processed[i]) continue;
        if (!sorted[i]) {
            new_to_old[next_num++] = i;
            sorted[i] = 1;
        }
        processed[i] = 1;
        int32_t m = unprocessed_neighbours(row_ptr, col_idx, processed, i, l);
        while (m > 0) {
            for (int32_t j = 0; j < m; ++j) {
                if (!sorted[l[j]]) {
                    new_to_old[next_num++] = l[j];
                    sorted[l[j]] = 1;
                }
            }
            int32_t w = l[0];
            processed[w] = 1;
            m = unprocessed_neighbours(row_ptr, col_idx, processed, w, l);
        }
    }
    for (int32_t v = 0; v < n; ++v)            /* vertices no walk reached */
        if (!sorted[v]) { new_to_old[next_num++] = v; sorted[v] = 1; }
    free(processed); free(sorted); free(interior); free(l);
    return next_num == n ? OR_OK : OR_ERR_ARG;
}

/* ----------------------------------------------------------- relabelling */

/*
 * Store the mesh under an ordering: new row k is the old row new_to_old[k]
 * with every id mapped to its new position; entry order inside a row is kept.
 */
int or_relabel(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const int32_t* new_to_old,
               int32_t* out_row_ptr, int32_t* out_col_idx) {
    if (n <= 0 || !row_ptr || !col_idx || !new_to_old || !out_row_ptr || !out_col_idx) return OR_ERR_ARG;
    int32_t* old_to_new = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!old_to_new) return OR_ERR_OOM;
    for (int32_t k = 0; k < n; ++k) old_to_new[new_to_old[k]] = k;
    out_row_ptr[0] = 0;
    for (int32_t k = 0; k < n; ++k) {
        int32_t v = new_to_old[k];
        int32_t len = row_ptr[v + 1] - row_ptr[v];
        for (int32_t e = 0; e < len; ++e) out_col_idx[out_row_ptr[k] + e] = old_to_new[col_idx[row_ptr[v] + e]];
        out_row_ptr[k + 1] = out_row_ptr[k] + len;
    }
    free(old_to_new);
    return OR_OK;
}

/* ------------------------------------------------------------- colouring */

/*
 * First-fit colouring of the interior vertices, visited in storage order
 * new_to_old[0..n): each gets the smallest colour not used by an interior
 * neighbour coloured before it.  colour[] is indexed by original id; boundary
 * vertices get -1.  Returns the number of colours in *ncolours.
 */
int or_color_greedy(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                    const int32_t* new_to_old, int32_t* colour, int32_t* ncolours) {
    if (n <= 0 || !row_ptr || !col_idx || !is_boundary || !new_to_old || !colour || !ncolours) return OR_ERR_ARG;
    int32_t max_deg = 0;
    for (int32_t v = 0; v < n; ++v)
        if (row_ptr[v + 1] - row_ptr[v] > max_deg) max_deg = row_ptr[v + 1] - row_ptr[v];
    uint8_t* used = (uint8_t*)calloc((size_t)max_deg + 2, 1);
    if (!used) return OR_ERR_OOM;
    for (int32_t v = 0; v < n; ++v) colour[v] = -1;
    int32_t nc = 0;
    for (int32_t k = 0; k < n; ++k) {
        int32_t v = new_to_old[k];
        if (is_boundary[v]) continue;
        memset(used, 0, (size_t)max_deg + 2);
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            int32_t c = colour[col_idx[e]];
            if (c >= 0 && c <= max_deg) used[c] = 1;
        }
        int32_t c = 0;
        while (used[c]) ++c;
        colour[v] = c;
        if (c + 1 > nc) nc = c + 1;
    }
    free(used);
    *ncolours = nc;
    return OR_OK;
}

/*
 * The in-place sequence a coloured Gauss-Seidel sweep reproduces: interior
 * vertices sorted by (colour, storage position).  seq receives original ids;
 * returns the count in *nseq.
 */
int or_color_sequence(int32_t n, const uint8_t* is_boundary, const int32_t* new_to_old, const int32_t* colour,
                      int32_t ncolours, int32_t* seq, int32_t* nseq) {
    if (n <= 0 || !is_boundary || !new_to_old || !colour || !seq || !nseq || ncolours < 0) return OR_ERR_ARG;
    int32_t m = 0;
    for (int32_t c = 0; c < ncolours; ++c)
        for (int32_t k = 0; k < n; ++k) {
            int32_t v = new_to_old[k];
            if (!is_boundary[v] && colour[v] == c) seq[m++] = v;
        }
    *nseq = m;
    return OR_OK;
}

/*
 * Block order of the in-place sweep (see the file header).  Storage position k
 * lies in tile k / tile; colour[] is a proper colouring of the interior
 * vertices by original id (-1 = boundary), e.g. or_color_greedy's.  Outputs:
 * tile_colour[ceil(n / tile)] (tiles without interior vertices get colour 0),
 * *ntile_colours, and seq (original ids of the interior vertices in block
 * order) with its length in *nseq.
 */
int or_block_sequence(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                      const int32_t* new_to_old, const int32_t* colour, int32_t ncolours, int32_t tile,
                      int32_t* tile_colour, int32_t* ntile_colours, int32_t* seq, int32_t* nseq) {
    if (n <= 0 || !row_ptr || !col_idx || !is_boundary || !new_to_old || !colour || ncolours < 0 || tile < 1 ||
        !tile_colour || !ntile_colours || !seq || !nseq)
        return OR_ERR_ARG;
    const int32_t ntiles = (int32_t)(((int64_t)n + tile - 1) / tile);
    int32_t* pos = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    uint8_t* used = (uint8_t*)calloc((size_t)ntiles + 1, 1);
    if (!pos || !used) {
        free(pos);
        free(used);
        return OR_ERR_OOM;
    }
    for (int32_t k = 0; k < n; ++k) pos[new_to_old[k]] = k;
    for (int32_t t = 0; t < ntiles; ++t) tile_colour[t] = -1;
    int32_t nt = 0;
    for (int32_t t = 0; t < ntiles; ++t) {
        /* colours of the already coloured tiles that share an interior-interior edge with tile t */
        memset(used, 0, (size_t)ntiles + 1);
        const int32_t k1 = (int32_t)((int64_t)(t + 1) * tile < n ? (t + 1) * tile : n);
        for (int32_t k = t * tile; k < k1; ++k) {
            const int32_t v = new_to_old[k];
            if (is_boundary[v]) continue;
            for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
                const int32_t u = col_idx[e];
                if (is_boundary[u]) continue;
                const int32_t tu = pos[u] / tile;
                if (tu != t && tile_colour[tu] >= 0) used[tile_colour[tu]] = 1;
            }
        }
        int32_t c = 0;
        while (used[c]) ++c;
        tile_colour[t] = c;
        if (c + 1 > nt) nt = c + 1;
    }
    int32_t m = 0;
    for (int32_t tc = 0; tc < nt; ++tc)
        for (int32_t t = 0; t < ntiles; ++t) {
            if (tile_colour[t] != tc) continue;
            const int32_t k1 = (int32_t)((int64_t)(t + 1) * tile < n ? (t + 1) * tile : n);
            for (int32_t c = 0; c < ncolours; ++c)
                for (int32_t k = t * tile; k < k1; ++k) {
                    const int32_t v = new_to_old[k];
                    if (!is_boundary[v] && colour[v] == c) seq[m++] = v;
                }
        }
    free(pos);
    free(used);
    *ntile_colours = nt;
    *nseq = m;
    return OR_OK;
}

/*
 * The data accesses of one sweep over the interior vertices of seq (original
 * ids, in visiting order): for each, the vertex itself when with_vertex != 0,
 * then the entries of its stored row.  trace receives original ids; *len the
 * count.  trace may be NULL to count only.
 */
int or_access_trace(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                    int32_t nseq, const int32_t* seq, int32_t with_vertex, int32_t* trace, int64_t* len) {
    if (n <= 0 || !row_ptr || !col_idx || !is_boundary || nseq < 0 || (nseq > 0 && !seq) || !len) return OR_ERR_ARG;
    int64_t t = 0;
    for (int32_t k = 0; k < nseq; ++k) {
        int32_t v = seq[k];
        if (v < 0 || v >= n) return OR_ERR_ARG;
        if (is_boundary[v]) continue;
        if (with_vertex) {
            if (trace) trace[t] = v;
            ++t;
        }
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            if (trace) trace[t] = col_idx[e];
            ++t;
        }
    }
    *len = t;
    return OR_OK;
}

/*
 * Reuse distances of a trace over elements 0..n-1, by direct inspection: for
 * the access at time t to element x whose previous access was at time p, the
 * accesses at times p+1 .. t-1 are walked and either counted (measure 1) or
 * their distinct elements counted (measure 0).  dist receives one value per
 * access that has a previous access, in trace order; *m their count.
 */
int or_reuse_distances(int64_t len, const int32_t* trace, int32_t n, int32_t measure, int64_t* dist, int64_t* m) {
    if (len < 0 || (len > 0 && !trace) || n <= 0 || (measure != 0 && measure != 1) || !m) return OR_ERR_ARG;
    int64_t* last = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int64_t* stamp = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    if (!last || !stamp) { free(last); free(stamp); return OR_ERR_OOM; }
    for (int32_t i = 0; i < n; ++i) { last[i] = -1; stamp[i] = -1; }
    int64_t cnt = 0;
    for (int64_t t = 0; t < len; ++t) {
        int32_t x = trace[t];
        if (x < 0 || x >= n) { free(last); free(stamp); return OR_ERR_ARG; }
        int64_t p = last[x];
        if (p >= 0) {
            int64_t d = 0;
            for (int64_t s = p + 1; s < t; ++s) {
                if (measure == 1) { ++d; continue; }
                if (stamp[trace[s]] != t) { stamp[trace[s]] = t; ++d; }
            }
            if (dist) dist[cnt] = d;
            ++cnt;
        }
        last[x] = t;
    }
    free(last); free(stamp);
    *m = cnt;
    return OR_OK;
}

static int cmp_int64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

/* Table 2's X quantile of m values: the k-th smallest, k = ceil(X * m) clamped to [1, m]. */
int or_quantile(int64_t m, const int64_t* values, double X, int64_t* out) {
    if (m <= 0 || !values || !out || !(X >= 0.0 && X <= 1.0)) return OR_ERR_ARG;
    int64_t* s = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
    if (!s) return OR_ERR_OOM;
    memcpy(s, values, sizeof(int64_t) * (size_t)m);
    qsort(s, (size_t)m, sizeof(int64_t), cmp_int64);
    double km = ceil(X * (double)m);
    int64_t k = (int64_t)km;
    if (k < 1) k = 1;
    if (k > m) k = m;
    *out = s[k - 1];
    free(s);
    return OR_OK;
}

static int cmp_int32_asc(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/*
 * Block RDR.  bfs = the BFS order (or_order_bfs); block j = the vertices at
 * BFS positions [j*block, (j+1)*block).  For each block in turn: its interior
 * vertices by increasing (quality, id) are the walk seeds; a walk from vertex i
 * orders i if needed, marks it processed, and repeatedly lists i's unprocessed
 * neighbours that lie in the same block by increasing (quality, id), orders the
 * ones not yet ordered, and continues from the first of them; block members no
 * walk ordered follow in ascending id.  With block >= n this is Algorithm 2;
 * with block = 1 it is the BFS order.
 */
int or_order_brdr(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                  const double* q_v, int32_t block, int32_t* new_to_old) {
    if (n <= 0 || !row_ptr || !col_idx || !is_boundary || !q_v || !new_to_old || block <= 0) return OR_ERR_ARG;
    int32_t max_deg = 0;
    for (int32_t v = 0; v < n; ++v)
        if (row_ptr[v + 1] - row_ptr[v] > max_deg) max_deg = row_ptr[v + 1] - row_ptr[v];
    int32_t* bfs = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* blk = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* seeds = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* l = (int32_t*)malloc(sizeof(int32_t) * (size_t)(max_deg + 1));
    uint8_t* processed = (uint8_t*)calloc((size_t)n, 1);
    uint8_t* sorted = (uint8_t*)calloc((size_t)n, 1);
    if (!bfs || !blk || !seeds || !l || !processed || !sorted) {
        free(bfs); free(blk); free(seeds); free(l); free(processed); free(sorted);
        return OR_ERR_OOM;
    }
    int rc = or_order_bfs(n, row_ptr, col_idx, bfs);
    if (rc != OR_OK) {
        free(bfs); free(blk); free(seeds); free(l); free(processed); free(sorted);
        return rc;
    }
    for (int32_t k = 0; k < n; ++k) blk[bfs[k]] = k / block;
    g_key_q = q_v;
    int32_t next_num = 0;
    for (int32_t start = 0; start < n; start += block) {
        const int32_t end = start + block < n ? start + block : n, j = start / block;
        int32_t ns = 0;
        for (int32_t k = start; k < end; ++k)
            if (!is_boundary[bfs[k]]) seeds[ns++] = bfs[k];
        qsort(seeds, (size_t)ns, sizeof(int32_t), cmp_key);
        for (int32_t si = 0; si < ns; ++si) {
            int32_t i = seeds[si];
            if (processed[i]) continue;
            if (!sorted[i]) { new_to_old[next_num++] = i; sorted[i] = 1; }
            processed[i] = 1;
            for (;;) {
                int32_t m = 0;   /* unprocessed neighbours of i in block j, by increasing key */
                for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
                    if (!processed[col_idx[e]] && blk[col_idx[e]] == j) l[m++] = col_idx[e];
                if (m == 0) break;
                qsort(l, (size_t)m, sizeof(int32_t), cmp_key);
                for (int32_t t = 0; t < m; ++t)
                    if (!sorted[l[t]]) { new_to_old[next_num++] = l[t]; sorted[l[t]] = 1; }
                i = l[0];
                processed[i] = 1;
            }
        }
        /* members no walk reached, ascending id */
        int32_t nl = 0;
        for (int32_t k = start; k < end; ++k)
            if (!sorted[bfs[k]]) seeds[nl++] = bfs[k];
        qsort(seeds, (size_t)nl, sizeof(int32_t), cmp_int32_asc);
        for (int32_t t = 0; t < nl; ++t) { new_to_old[next_num++] = seeds[t]; sorted[seeds[t]] = 1; }
    }
    free(bfs); free(blk); free(seeds); free(l); free(processed); free(sorted);
    return OR_OK;
}
