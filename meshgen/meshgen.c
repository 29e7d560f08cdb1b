/*
 * meshgen.c - seeded synthetic 2D triangle meshes.
 *
 * Input generator only: it holds none of the smoothing, quality or ordering
 * arithmetic of the method.  Both the oracle-side tests and the CUDA path take
 * their inputs from here.
 *
 * The paper measures on nine Triangle-generated meshes of 0.3-0.4M vertices
 * with average degree ~6 (Section 5.1, Table 1).  Those files are not
 * available, so this module builds stand-ins with the same structure:
 *
 *   1. an s x s grid on [0,1]^2 (optionally graded in x: spacing grows
 *      linearly 1x -> 10x across the domain);
 *   2. every cell split into two triangles along a random diagonal;
 *   3. interior vertices jittered by U(-j, j) x the local spacing per axis;
 *   4. a fraction of the interior edges flipped (in a seeded random order,
 *      when the quad is strictly convex, the new diagonal is absent and the
 *      degrees stay in range);
 *   5. a fraction of the triangles split at their centroid (skipped when a
 *      corner would exceed degree 12).
 *
 * All randomness comes from splitmix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), consumed in this fixed order:
 * diagonals (cells row-major), jitter (interior vertices by id, x then y),
 * edge shuffle, triangle shuffle.  Compile with -ffp-contract=off so that x86
 * and Arm hosts produce identical coordinates.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MG_OK 0
#define MG_ERR_ARG -1
#define MG_ERR_OOM -2

typedef struct {
    int32_t n;          /* vertices */
    int32_t n_grid;     /* grid vertices (ids [0, n_grid)); centroid vertices follow */
    int32_t ntri;       /* triangles */
    int64_t nnz;        /* CSR entries = 2 x edges */
    int32_t nflips;     /* flips performed */
    int32_t nsplits;    /* splits performed */
    double* xy;         /* [2n] x0 y0 x1 y1 ... */
    int32_t* row_ptr;   /* [n+1] */
    int32_t* col_idx;   /* [nnz], each row ascending */
    uint8_t* is_boundary; /* [n] 1 = on the border of the square */
    int32_t* tri;       /* [3 ntri] counter-clockwise corners (before jitter) */
} mg_mesh;

static inline uint64_t sm64_next(uint64_t* s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform double in [0,1) with 53 random bits */
static inline double sm64_unit(uint64_t* s) {
    return (double)(sm64_next(s) >> 11) * (1.0 / 9007199254740992.0);
}

/* uniform double in [0,1): exported so callers can draw side lengths etc. */
double mg_unit(uint64_t* state) { return sm64_unit(state); }
uint64_t mg_next(uint64_t* state) { return sm64_next(state); }

static double orient(const double* xy, int32_t a, int32_t b, int32_t c) {
    double ax = xy[2 * a], ay = xy[2 * a + 1];
    double bx = xy[2 * b] - ax, by = xy[2 * b + 1] - ay;
    double cx = xy[2 * c] - ax, cy = xy[2 * c + 1] - ay;
    return bx * cy - by * cx;
}

/* corner index of vertex v in triangle t, or -1 */
static inline int corner_of(const int32_t* tri, int32_t t, int32_t v) {
    if (tri[3 * t] == v) return 0;
    if (tri[3 * t + 1] == v) return 1;
    if (tri[3 * t + 2] == v) return 2;
    return -1;
}

/*
 * Find a triangle containing the edge (a, b) by walking the fan of a (both
 * directions, since boundary fans are open).  Returns the triangle or -1.
 * nbr[3t+k] is the triangle across the edge opposite corner k.
 */
static int32_t find_edge(const int32_t* tri, const int32_t* nbr, const int32_t* vt,
                         int32_t a, int32_t b) {
    int32_t t0 = vt[a];
    if (t0 < 0) return -1;
    int32_t t = t0;
    for (int guard = 0; guard < 64; ++guard) {           /* counter-clockwise */
        if (corner_of(tri, t, b) >= 0) return t;
        int k = corner_of(tri, t, a);
        /* triangle (a, p, q): the next one CCW around a is across edge (a, q), opposite p */
        int32_t nt = nbr[3 * t + (k + 1) % 3];
        if (nt < 0 || nt == t0) break;
        t = nt;
    }
    t = t0;
    for (int guard = 0; guard < 64; ++guard) {           /* clockwise */
        int k = corner_of(tri, t, a);
        int32_t nt = nbr[3 * t + (k + 2) % 3];           /* across edge (a, p), opposite q */
        if (nt < 0 || nt == t0) break;
        t = nt;
        if (corner_of(tri, t, b) >= 0) return t;
    }
    return -1;
}

static void set_nbr(int32_t* tri, int32_t* nbr, int32_t t, int32_t old_t, int32_t new_t) {
    if (t < 0) return;
    for (int k = 0; k < 3; ++k)
        if (nbr[3 * t + k] == old_t) { nbr[3 * t + k] = new_t; return; }
    (void)tri;
}

void mg_free(mg_mesh* m) {
    if (!m) return;
    free(m->xy); free(m->row_ptr); free(m->col_idx); free(m->is_boundary); free(m->tri);
    memset(m, 0, sizeof(*m));
}

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/*
 * Build a mesh.  side >= 3.  graded != 0: x-spacing h_i proportional to
 * 1 + 9 i / (side - 2).  jitter: fraction of the local spacing (0.3 in all
 * workloads).  flip_frac / split_frac: 0.10 / 0.05 in the flipped workloads.
 */
int mg_generate(int32_t side, int32_t graded, double jitter, double flip_frac, double split_frac,
                uint64_t seed, mg_mesh* out) {
    if (!out || side < 3 || side > 46000) return MG_ERR_ARG;
    memset(out, 0, sizeof(*out));
    const int64_t s = side;
    const int64_t n_grid = s * s;
    const int64_t ncell = (s - 1) * (s - 1);
    const int64_t t_grid = 2 * ncell;
    const int64_t max_split = (int64_t)(split_frac * (double)t_grid) + 1;
    const int64_t n_cap = n_grid + max_split;
    const int64_t t_cap = t_grid + 2 * max_split;
    if (n_cap > INT32_MAX / 2 || 3 * t_cap > INT32_MAX) return MG_ERR_ARG;

    uint64_t rng = seed;
    double* xy = (double*)malloc(sizeof(double) * 2 * n_cap);
    int32_t* tri = (int32_t*)malloc(sizeof(int32_t) * 3 * t_cap);
    int32_t* nbr = (int32_t*)malloc(sizeof(int32_t) * 3 * t_grid);
    int32_t* vt = (int32_t*)malloc(sizeof(int32_t) * n_cap);
    int32_t* deg = (int32_t*)calloc(n_cap, sizeof(int32_t));
    uint8_t* bnd = (uint8_t*)calloc(n_cap, 1);
    double* xs = (double*)malloc(sizeof(double) * s);
    double* hx = (double*)malloc(sizeof(double) * s);
    uint8_t* diag = (uint8_t*)malloc(ncell);
    if (!xy || !tri || !nbr || !vt || !deg || !bnd || !xs || !hx || !diag) goto oom;

    /* 1. grid coordinates */
    if (graded) {
        double H = 0.0;
        for (int64_t i = 0; i + 1 < s; ++i) { hx[i] = 1.0 + 9.0 * (double)i / (double)(s - 2); H += hx[i]; }
        for (int64_t i = 0; i + 1 < s; ++i) hx[i] = hx[i] / H;
        xs[0] = 0.0;
        for (int64_t i = 1; i < s; ++i) xs[i] = xs[i - 1] + hx[i - 1];
        xs[s - 1] = 1.0;
    } else {
        for (int64_t i = 0; i + 1 < s; ++i) hx[i] = 1.0 / (double)(s - 1);
        for (int64_t i = 0; i < s; ++i) xs[i] = (double)i / (double)(s - 1);
    }
    const double hy = 1.0 / (double)(s - 1);
    for (int64_t j = 0; j < s; ++j)
        for (int64_t i = 0; i < s; ++i) {
            int64_t v = j * s + i;
            xy[2 * v] = xs[i];
            xy[2 * v + 1] = (double)j / (double)(s - 1);
            bnd[v] = (i == 0 || j == 0 || i == s - 1 || j == s - 1);
        }

    /* 2. random diagonals; triangles counter-clockwise, ids 2*cell + {0,1} */
    for (int64_t c = 0; c < ncell; ++c) diag[c] = (uint8_t)(sm64_next(&rng) & 1u);
    for (int64_t j = 0; j + 1 < s; ++j)
        for (int64_t i = 0; i + 1 < s; ++i) {
            int64_t c = j * (s - 1) + i;
            int32_t v00 = (int32_t)(j * s + i), v10 = v00 + 1;
            int32_t v01 = (int32_t)((j + 1) * s + i), v11 = v01 + 1;
            int32_t* t0 = tri + 6 * c;
            if (diag[c] == 0) {
                t0[0] = v00; t0[1] = v10; t0[2] = v11;
                t0[3] = v00; t0[4] = v11; t0[5] = v01;
            } else {
                t0[0] = v00; t0[1] = v10; t0[2] = v01;
                t0[3] = v10; t0[4] = v11; t0[5] = v01;
            }
        }

    /* 3. jitter interior vertices */
    for (int64_t j = 1; j + 1 < s; ++j)
        for (int64_t i = 1; i + 1 < s; ++i) {
            int64_t v = j * s + i;
            double hloc = 0.5 * (hx[i - 1] + hx[i]);
            double ux = sm64_unit(&rng), uy = sm64_unit(&rng);
            xy[2 * v] += (2.0 * ux - 1.0) * jitter * hloc;
            xy[2 * v + 1] += (2.0 * uy - 1.0) * jitter * hy;
        }

    /* triangle adjacency (grid structure), vertex -> one incident triangle, degrees */
    for (int64_t t = 0; t < 3 * t_grid; ++t) nbr[t] = -1;
    for (int64_t v = 0; v < n_cap; ++v) vt[v] = -1;
    {
        /* generic matching through each vertex's incident triangles (<= 8 on a grid) */
        int32_t* cnt = (int32_t*)calloc(n_grid + 1, sizeof(int32_t));
        int32_t* inc = (int32_t*)malloc(sizeof(int32_t) * 3 * t_grid);
        if (!cnt || !inc) { free(cnt); free(inc); goto oom; }
        for (int64_t t = 0; t < t_grid; ++t)
            for (int k = 0; k < 3; ++k) cnt[tri[3 * t + k] + 1]++;
        for (int64_t v = 0; v < n_grid; ++v) cnt[v + 1] += cnt[v];
        int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * n_grid);
        if (!fill) { free(cnt); free(inc); goto oom; }
        memcpy(fill, cnt, sizeof(int32_t) * n_grid);
        for (int64_t t = 0; t < t_grid; ++t)
            for (int k = 0; k < 3; ++k) inc[fill[tri[3 * t + k]]++] = (int32_t)t;
        free(fill);
        for (int64_t t = 0; t < t_grid; ++t)
            for (int k = 0; k < 3; ++k) {
                int32_t a = tri[3 * t + (k + 1) % 3], b = tri[3 * t + (k + 2) % 3];
                for (int32_t e = cnt[a]; e < cnt[a + 1]; ++e) {
                    int32_t u = inc[e];
                    if (u != t && corner_of(tri, u, b) >= 0) { nbr[3 * t + k] = u; break; }
                }
            }
        for (int64_t v = 0; v < n_grid; ++v) vt[v] = cnt[v] < cnt[v + 1] ? inc[cnt[v]] : -1;
        free(cnt); free(inc);
    }
    for (int64_t j = 0; j < s; ++j)
        for (int64_t i = 0; i < s; ++i) {
            int64_t v = j * s + i;
            int d = 0;
            if (i > 0) d++;
            if (i + 1 < s) d++;
            if (j > 0) d++;
            if (j + 1 < s) d++;
            /* diagonals of the up to four cells around (i,j) that touch it */
            if (i > 0 && j > 0 && diag[(j - 1) * (s - 1) + (i - 1)] == 0) d++;         /* cell SW: v11 */
            if (i + 1 < s && j + 1 < s && diag[j * (s - 1) + i] == 0) d++;             /* cell NE: v00 */
            if (i + 1 < s && j > 0 && diag[(j - 1) * (s - 1) + i] == 1) d++;           /* cell SE: v01 */
            if (i > 0 && j + 1 < s && diag[j * (s - 1) + (i - 1)] == 1) d++;           /* cell NW: v10 */
            deg[v] = d;
        }

    /* 4. flips over the sorted interior-edge list, shuffled */
    int32_t nflips = 0;
    if (flip_frac > 0.0) {
        int64_t e_int = 2 * (s - 1) * (s - 2) + ncell;
        int64_t* edges = (int64_t*)malloc(sizeof(int64_t) * e_int);
        if (!edges) goto oom;
        int64_t ne = 0;
        for (int64_t j = 0; j < s; ++j)
            for (int64_t i = 0; i < s; ++i) {
                int64_t a = j * s + i;
                /* candidates b > a in ascending order: a+1, a+s-1, a+s, a+s+1 */
                if (i + 1 < s && !(j == 0 || j == s - 1)) edges[ne++] = (a << 32) | (a + 1);
                if (i > 0 && j + 1 < s && diag[j * (s - 1) + (i - 1)] == 1) edges[ne++] = (a << 32) | (a + s - 1);
                if (j + 1 < s && !(i == 0 || i == s - 1)) edges[ne++] = (a << 32) | (a + s);
                if (i + 1 < s && j + 1 < s && diag[j * (s - 1) + i] == 0) edges[ne++] = (a << 32) | (a + s + 1);
            }
        for (int64_t i = ne - 1; i >= 1; --i) {
            int64_t r = (int64_t)(sm64_next(&rng) % (uint64_t)(i + 1));
            int64_t tmp = edges[i]; edges[i] = edges[r]; edges[r] = tmp;
        }
        int64_t nf = (int64_t)(flip_frac * (double)ne);
        for (int64_t f = 0; f < nf; ++f) {
            int32_t a = (int32_t)(edges[f] >> 32), b = (int32_t)(edges[f] & 0xffffffff);
            int32_t t1 = find_edge(tri, nbr, vt, a, b);
            if (t1 < 0) continue;
            int ka = corner_of(tri, t1, a), kb = corner_of(tri, t1, b);
            int k1 = 3 - ka - kb;                       /* corner opposite the edge */
            int32_t c = tri[3 * t1 + k1];
            int32_t p = tri[3 * t1 + (k1 + 1) % 3], q = tri[3 * t1 + (k1 + 2) % 3];
            int32_t t2 = nbr[3 * t1 + k1];
            if (t2 < 0) continue;
            int kp2 = corner_of(tri, t2, p), kq2 = corner_of(tri, t2, q);
            int k2 = 3 - kp2 - kq2;
            int32_t d = tri[3 * t2 + k2];
            /* quad c, p, d, q must be strictly convex */
            if (!(orient(xy, c, p, d) > 0.0 && orient(xy, p, d, q) > 0.0 &&
                  orient(xy, d, q, c) > 0.0 && orient(xy, q, c, p) > 0.0)) continue;
            if (find_edge(tri, nbr, vt, c, d) >= 0) continue;
            if (deg[p] - 1 < (bnd[p] ? 2 : 4) || deg[q] - 1 < (bnd[q] ? 2 : 4)) continue;
            if (deg[c] + 1 > 11 || deg[d] + 1 > 11) continue;
            /* old t1 = (c,p,q): A across (q,c), B across (c,p); old t2 = (d,q,p): C across (p,d), D across (d,q) */
            int32_t A = nbr[3 * t1 + (k1 + 1) % 3];
            int32_t B = nbr[3 * t1 + (k1 + 2) % 3];
            int32_t C = nbr[3 * t2 + (k2 + 1) % 3];
            int32_t D = nbr[3 * t2 + (k2 + 2) % 3];
            /* new t1 = (c,p,d), new t2 = (d,q,c) */
            tri[3 * t1] = c; tri[3 * t1 + 1] = p; tri[3 * t1 + 2] = d;
            nbr[3 * t1] = C; nbr[3 * t1 + 1] = t2; nbr[3 * t1 + 2] = B;
            tri[3 * t2] = d; tri[3 * t2 + 1] = q; tri[3 * t2 + 2] = c;
            nbr[3 * t2] = A; nbr[3 * t2 + 1] = t1; nbr[3 * t2 + 2] = D;
            set_nbr(tri, nbr, A, t1, t2);
            set_nbr(tri, nbr, C, t2, t1);
            vt[p] = t1; vt[c] = t1; vt[q] = t2; vt[d] = t2;
            deg[p]--; deg[q]--; deg[c]++; deg[d]++;
            nflips++;
        }
        free(edges);
    }

    /* 5. centroid splits over a shuffled triangle list */
    int64_t n = n_grid, T = t_grid;
    int32_t nsplits = 0;
    if (split_frac > 0.0) {
        int32_t* order = (int32_t*)malloc(sizeof(int32_t) * t_grid);
        if (!order) goto oom;
        for (int64_t t = 0; t < t_grid; ++t) order[t] = (int32_t)t;
        for (int64_t i = t_grid - 1; i >= 1; --i) {
            int64_t r = (int64_t)(sm64_next(&rng) % (uint64_t)(i + 1));
            int32_t tmp = order[i]; order[i] = order[r]; order[r] = tmp;
        }
        int64_t ns = (int64_t)(split_frac * (double)t_grid);
        for (int64_t k = 0; k < ns; ++k) {
            int32_t t = order[k];
            int32_t a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
            if (deg[a] + 1 > 12 || deg[b] + 1 > 12 || deg[c] + 1 > 12) continue;
            int32_t p = (int32_t)n++;
            xy[2 * p] = (xy[2 * a] + xy[2 * b] + xy[2 * c]) / 3.0;
            xy[2 * p + 1] = (xy[2 * a + 1] + xy[2 * b + 1] + xy[2 * c + 1]) / 3.0;
            bnd[p] = 0;
            tri[3 * t + 2] = p;                                        /* (a, b, p) */
            tri[3 * T] = b; tri[3 * T + 1] = c; tri[3 * T + 2] = p; T++;  /* (b, c, p) */
            tri[3 * T] = c; tri[3 * T + 1] = a; tri[3 * T + 2] = p; T++;  /* (c, a, p) */
            deg[a]++; deg[b]++; deg[c]++; deg[p] = 3;
            nsplits++;
        }
        free(order);
    }

    /* 6. CSR from the triangles: rows ascending, duplicates removed */
    {
        int64_t* start = (int64_t*)calloc(n + 1, sizeof(int64_t));
        if (!start) goto oom;
        for (int64_t t = 0; t < T; ++t)
            for (int k = 0; k < 3; ++k) start[tri[3 * t + k] + 1] += 2;
        for (int64_t v = 0; v < n; ++v) start[v + 1] += start[v];
        int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * start[n]);
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
        int32_t* row_ptr = (int32_t*)malloc(sizeof(int32_t) * (n + 1));
        if (!tmp || !fill || !row_ptr) { free(start); free(tmp); free(fill); free(row_ptr); goto oom; }
        memcpy(fill, start, sizeof(int64_t) * (n + 1));
        for (int64_t t = 0; t < T; ++t)
            for (int k = 0; k < 3; ++k) {
                int32_t a = tri[3 * t + k];
                tmp[fill[a]++] = tri[3 * t + (k + 1) % 3];
                tmp[fill[a]++] = tri[3 * t + (k + 2) % 3];
            }
        int64_t nnz = 0;
        row_ptr[0] = 0;
        for (int64_t v = 0; v < n; ++v) {
            int32_t* r = tmp + start[v];
            int64_t len = start[v + 1] - start[v];
            qsort(r, (size_t)len, sizeof(int32_t), cmp_i32);
            for (int64_t e = 0; e < len; ++e)
                if (e == 0 || r[e] != r[e - 1]) tmp[nnz++] = r[e];
            row_ptr[v + 1] = (int32_t)nnz;
        }
        free(start); free(fill);
        int32_t* col_idx = (int32_t*)realloc(tmp, sizeof(int32_t) * (nnz > 0 ? nnz : 1));
        if (!col_idx) { free(tmp); free(row_ptr); goto oom; }
        out->row_ptr = row_ptr;
        out->col_idx = col_idx;
        out->nnz = nnz;
    }

    out->n = (int32_t)n;
    out->n_grid = (int32_t)n_grid;
    out->ntri = (int32_t)T;
    out->nflips = nflips;
    out->nsplits = nsplits;
    out->xy = (double*)realloc(xy, sizeof(double) * 2 * n);
    out->tri = (int32_t*)realloc(tri, sizeof(int32_t) * 3 * T);
    out->is_boundary = (uint8_t*)realloc(bnd, (size_t)n);
    free(nbr); free(vt); free(deg); free(xs); free(hx); free(diag);
    return MG_OK;

oom:
    free(xy); free(tri); free(nbr); free(vt); free(deg); free(bnd); free(xs); free(hx); free(diag);
    mg_free(out);
    return MG_ERR_OOM;
}
