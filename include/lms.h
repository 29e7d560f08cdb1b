/*
 * lms.h - C ABI of liblms: GB300 Laplacian mesh smoothing with
 * locality-aware vertex orderings.
 *
 * Method: Aupy, Park & Raghavan, "Locality-Aware Laplacian Mesh Smoothing".
 *   - smoothing step: Eq. 1 (a vertex moves to the mean of its N mesh
 *     neighbours), applied to interior vertices only (Algorithm 1);
 *   - quality: Section 3.2 (edge-length ratio of a triangle, mean over a
 *     vertex's triangles, mean over all |V| vertices);
 *   - stopping rule: Section 5.1 (stop once the global quality improves by
 *     less than a criterion, 5e-6 in the paper) plus an iteration cap
 *     (Section 3.2);
 *   - orderings: original, random, breadth-first, and the Reuse Distance
 *     Reducing ordering of Algorithm 2 (Section 4.2), compared in Section 5.2.
 *
 * Conventions for every entry point:
 *   - ids are int32, vertices 0..n-1 in the caller's (original) labelling;
 *   - coordinates are interleaved doubles: xy[2v] = x, xy[2v+1] = y;
 *   - inputs are host pointers and are copied; the caller keeps ownership;
 *     outputs go to caller-allocated host buffers;
 *   - every int-returning call returns LMS_OK (0) or a negative LMS_ERR_*;
 *     lms_error_string() gives a message;
 *   - device work is issued on the CUDA stream given at creation (NULL = the
 *     legacy default stream); calls that return host data synchronise that
 *     stream first;
 *   - a handle is not thread-safe; distinct handles are independent.
 *
 * Entry points marked [host] do no device work and need no GPU.
 */
#ifndef LMS_H
#define LMS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LMS_OK 0
#define LMS_ERR_ARG (-1)          /* NULL pointer, bad enum, n <= 0, out-of-range index, non-finite coordinate */
#define LMS_ERR_CSR (-2)          /* row_ptr not monotone / not starting at 0, id out of range, self-loop,
                                     duplicate entry, or adjacency not symmetric */
#define LMS_ERR_ISOLATED (-3)     /* interior vertex with no neighbour: Eq. 1 would divide by zero */
#define LMS_ERR_NO_TRIANGLES (-4) /* quality, RDR or a stopping rule requested without triangles */
#define LMS_ERR_CUDA (-5)         /* a CUDA runtime call failed */
#define LMS_ERR_OOM (-6)          /* host or device allocation failed */
#define LMS_ERR_TIMEOUT (-7)      /* a bounded device-side wait gave up */
#define LMS_ERR_STATE (-8)        /* call not valid in the handle's current state */

/* precision of the stored coordinates and of the sweep arithmetic */
#define LMS_FP64 0 /* double2 coordinates, FP64 sums and division (results equal the FP64 sequential sums) */
#define LMS_FP32 1 /* float2 coordinates relative to the bounding-box centre, scaled by the larger box
                      side; compensated (Kahan) FP32 neighbour sums, mean by a correctly rounded
                      division by the count (lms_selftest_div32); quality reduced in FP64 */

/* vertex orderings (Section 5.2.1 compares ORI, BFS and RDR; Fig. 1 adds a random one) */
#define LMS_ORI 0    /* original order: identity permutation */
#define LMS_RANDOM 1 /* Fisher-Yates shuffle driven by splitmix64(seed) */
#define LMS_BFS 2    /* breadth-first visit order from vertex 0, neighbours by ascending id,
                        restarting at the smallest unvisited id */
#define LMS_RDR 3    /* Algorithm 2: walks from the worst-quality interior vertex, appending
                        unordered neighbours by increasing (quality, id) */
#define LMS_RBFS 4   /* reversed BFS: the LMS_BFS visit order read backwards (the ordering Section 2
                        reports from Munson and Hovland's study) */
#define LMS_BRDR 5   /* block RDR, a data-parallel variant of Algorithm 2 that is not in the paper: the
                        LMS_BFS order cut into blocks of LMS_BRDR_BLOCK consecutive positions, Algorithm 2
                        applied to each block's own subgraph (walks never leave the block; members no
                        walk reached follow in ascending id), blocks kept in BFS order.  Every reuse
                        stays within about two blocks, as for BFS, while most are as short as RDR's */
#define LMS_BRDR_BLOCK 4096

/* reuse-distance measures (lms_reuse_profile) */
#define LMS_REUSE_DISTINCT 0 /* distinct elements accessed between two accesses to one element (Section 2.2) */
#define LMS_REUSE_ACCESSES 1 /* accesses between them (the measure Table 2's maxima imply) */

/* sweep modes */
#define LMS_JACOBI 0     /* all interior vertices read the previous sweep's positions (ping-pong) */
#define LMS_COLORED_GS 1 /* in place, colour by colour of a first-fit colouring of the interior vertices
                            in storage order; equals Algorithm 1's sequential in-place sweep taken in
                            (colour, storage position) order */
#define LMS_INPLACE_STATIC 2 /* the paper's parallel form (Section 5.1): Algorithm 1 in place with the
                                storage order divided evenly into contiguous blocks, one GPU thread per
                                block (lms_set_inplace_split); neighbours are read as they are at that
                                moment, so results depend on timing - except with one thread, which is
                                the sequential in-place sweep in storage order */
#define LMS_BLOCK_GS 3 /* not in the paper: block Gauss-Seidel - Algorithm 1 in place in the block order
                          of lms_block_order (tiles of lms_set_block_tile consecutive positions of the
                          ordering), tiles of one tile colour swept at the same time, colour groups
                          inside a tile one after another; deterministic, equal to the sequential
                          in-place sweep in that order */

/* sweep kernels */
#define LMS_KERNEL_DIRECT 0 /* one thread per vertex; CSR and positions loaded through L1; rows read `chunk`
                               entries at a time (all ids, then all gathers, then the sums) */
#define LMS_KERNEL_STAGED 1 /* tile CSR brought to shared memory by TMA bulk copies one tile ahead; neighbour
                               positions gathered edge-parallel into shared memory, then summed per vertex */
#define LMS_KERNEL_SELL 2   /* batched only: SELL-C-sigma work layout - inside every tile the interior vertices
                               sorted by degree into slices of 32 whose neighbour ids are stored
                               column-major; one lane per slot, coalesced id loads, no row offsets */
#define LMS_KERNEL_PACKED 3 /* batched only: one thread per vertex; one 32-bit word per vertex packs its row's
                               offset within its mesh, its neighbour count and its boundary flag, so a
                               thread learns its row from one load; needs meshes of fewer than 2^22 CSR
                               entries and rows of at most 63 entries */

/* where the FP64 sweep's arithmetic runs (lms_set_fp64_arith); every choice gives the IEEE
   round-to-nearest sums and quotients, so results are identical */
#define LMS_FP64_ARITH_FPU 0      /* FP64 instructions: adds, and the table-driven division */
#define LMS_FP64_ARITH_INT_ADDS 1 /* neighbour sums on the integer pipes, division on the FP64 unit */
#define LMS_FP64_ARITH_INT 2      /* sums and division on the integer pipes; zero or subnormal operands,
                                     exponent gaps above 9 in a sum, the top binade and subnormal results
                                     go to the FP64 unit */
#define LMS_FP64_ARITH_MIXED2 3   /* division on the integer pipes; the add of every even row position
                                     there too, the others on the FP64 unit (both pipes busy at once) */
#define LMS_FP64_ARITH_MIXED3 4   /* as LMS_FP64_ARITH_MIXED2 with every third row position (the default:
                                     fastest on GB300) */

typedef struct lms_mesh_s* lms_handle;
typedef struct lms_batch_s* lms_batch;

/* one mesh of a batch; all pointers are host pointers, copied by lms_batch_create */
typedef struct {
    int32_t n;                   /* vertices */
    const int32_t* row_ptr;      /* [n+1] CSR offsets, row_ptr[0] = 0 */
    const int32_t* col_idx;      /* [row_ptr[n]] symmetric adjacency, no self-loops or duplicates */
    const double* xy;            /* [2n] coordinates */
    const uint8_t* is_boundary;  /* [n] nonzero = fixed vertex */
    int32_t ntri;                /* triangles (may be 0 when tri is NULL) */
    const int32_t* tri;          /* [3 ntri] corner ids, or NULL */
} lms_mesh_desc;

/* Text for a status code (static storage). [host] */
const char* lms_error_string(int status);

/*
 * Route the library's device allocations through caller-supplied functions
 * (for example a framework's caching allocator).  alloc(bytes, stream, ctx)
 * returns a device pointer or NULL; release(ptr, ctx) frees it.  Passing NULL
 * for both restores cudaMalloc/cudaFree.  Affects handles created afterwards;
 * a handle frees with the functions it allocated with.  [host]
 */
int lms_set_device_allocator(void* (*alloc)(size_t bytes, void* stream, void* ctx),
                             void (*release)(void* ptr, void* ctx), void* ctx);

/*
 * Check a mesh without creating anything.  Returns LMS_OK, LMS_ERR_ARG,
 * LMS_ERR_CSR or LMS_ERR_ISOLATED; tri may be NULL when ntri == 0. [host]
 */
int lms_validate(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                 int32_t ntri, const int32_t* tri);

/*
 * Vertex ordering on the host (Section 4.2, Algorithm 2; Section 5.2.1).
 * q_v: [n] per-vertex quality (Section 3.2), required for LMS_RDR and LMS_BRDR and ignored
 * otherwise.  new_to_old: [n] output, new_to_old[k] = original id stored at
 * position k; always a permutation (Theorem 1; vertices no RDR walk reaches
 * are appended in ascending id).  [host]
 */
int lms_order_host(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                   const double* q_v, int ordering, uint64_t seed, int32_t* new_to_old);

/*
 * Reuse-distance profile of one sweep (Section 2.2, Fig. 1, Table 2).  The
 * trace visits the interior vertices in storage order new_to_old (NULL: the
 * identity) and lists, for each, the vertex itself when with_vertex != 0 and
 * then its stored row (the access pattern of Fig. 3); elements are vertices.
 * Every access that repeats an element gets a reuse distance (measure =
 * LMS_REUSE_DISTINCT or LMS_REUSE_ACCESSES); first accesses get none.
 * Outputs (each may be NULL): out_q[i] = the q[i] quantile for i < nq, the
 * ceil(q[i] m)-th smallest of the m distances (clamped to [1, m]; -1 when m = 0;
 * q[i] in [0, 1]); *mean; *n_accesses = trace length; *n_reuses = m;
 * hist[33]: hist[0] counts distance 0, hist[b] distances in [2^(b-1), 2^b).
 * Cost O(T log T) time and 8 T bytes for a trace of T accesses (T < 2^32).
 * Returns LMS_ERR_ARG (NULL input, bad enum, q outside [0, 1], new_to_old not a
 * permutation), LMS_ERR_CSR or LMS_ERR_OOM.  [host]
 */
int lms_reuse_profile(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                      const int32_t* new_to_old, int32_t with_vertex, int32_t measure, int32_t nq, const double* q,
                      int64_t* out_q, double* mean, int64_t* n_accesses, int64_t* n_reuses, int64_t* hist);

/*
 * First-fit colouring of the interior vertices visited in storage order
 * new_to_old.  colour: [n] output indexed by original id (-1 for boundary
 * vertices); *ncolours receives the colour count.  [host]
 */
int lms_color_host(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                   const int32_t* new_to_old, int32_t* colour, int32_t* ncolours);

/*
 * Block order of Algorithm 1's in-place sweep (not in the paper; the sequential form of a block
 * Gauss-Seidel): the storage order new_to_old cut into tiles of `tile` consecutive positions; tiles
 * coloured first-fit in ascending tile index so that no two tiles of one colour share an edge between
 * interior vertices (tile_colour: [ceil(n / tile)] output; tiles without interior vertices get 0;
 * *ntile_colours the count); order: [n] output receiving the interior vertices (original ids) by
 * (tile colour, tile, colour of lms_color_host's colouring, storage position), *n_order their count.
 * Tiles of one colour, and one colour's vertices inside a tile, are independent, so sweeping them at
 * the same time equals the in-place sweep in this order.  LMS_ERR_ARG, LMS_ERR_OOM.  [host]
 */
int lms_block_order(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                    const int32_t* new_to_old, int32_t tile, int32_t* tile_colour, int32_t* ntile_colours,
                    int32_t* order, int32_t* n_order);

/*
 * Diagnostic of the LMS_BLOCK_GS tables: builds them for storage order new_to_old and tile as a handle
 * does, and walks them in the device sweep's launch order (tile colour, tile, colour group, table
 * order), writing the visited interior vertices (original ids) to seq ([n]), their count to *nseq and
 * the number of launches of one sweep to *n_launches (the one-CTA-per-tile form of tiles below 65,536
 * positions: one launch per tile colour; tiles from 65,536 up run one launch per non-empty (tile colour,
 * vertex colour) range instead, in the same order).  Equals lms_block_order's order.  LMS_ERR_ARG,
 * LMS_ERR_OOM.  [host]
 */
int lms_block_walk(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                   const int32_t* new_to_old, int32_t tile, int32_t* seq, int32_t* nseq, int32_t* n_launches);

/*
 * Split a batch of k independent meshes between `ranks` GPUs by whole meshes, balanced by vertex count
 * (the paper splits one mesh's vertices evenly between threads, Section 5.1; meshes of a batch share no
 * vertex, so whole meshes need no exchange between GPUs).  Longest-processing-time rule: meshes taken by
 * vertex count, largest first (ties by index), each to the rank with the smallest load so far (ties to
 * the lowest rank).  Every mesh lands on exactly one rank and the most loaded rank exceeds the least
 * loaded by at most the largest mesh.  n_vertices: [k] counts (>= 1); rank_of: [k] output; load: [ranks]
 * output of vertices per rank (may be NULL).  Deterministic.  LMS_ERR_ARG (NULL, k < 1, ranks < 1, a count
 * < 1).  [host]
 */
int lms_partition_meshes(int32_t k, const int32_t* n_vertices, int32_t ranks, int32_t* rank_of, int64_t* load);

/*
 * Create a smoothing handle: validates the mesh (as lms_validate), copies it
 * to the device and stores the coordinates in `precision`.  The initial
 * ordering is LMS_ORI.  tri may be NULL (ntri = 0); quality, LMS_RDR and the
 * stopping rule then return LMS_ERR_NO_TRIANGLES.  cuda_stream: a
 * cudaStream_t or NULL.
 */
int lms_create(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* xy,
               const uint8_t* is_boundary, int32_t ntri, const int32_t* tri, int precision,
               void* cuda_stream, lms_handle* out);

/*
 * Store the mesh under an ordering (Section 4.2 / 5.2.1) and relabel the
 * device CSR, coordinates and triangles.  Where the permutation is computed:
 * LMS_BFS and LMS_RBFS on the device (level-synchronous search, equal to the
 * sequential one); LMS_BRDR on the device (rows of at most 64 entries; longer
 * rows use the host implementation, with the same result); LMS_RDR keys on the
 * device (Section 3.2 qualities of the current coordinates, FP64) and its walk
 * on the host; LMS_RANDOM and LMS_ORI on the host.  Rows keep their entry
 * order, so Jacobi results do not depend on the ordering.  seed is used by
 * LMS_RANDOM.  Synchronous; lms_last_reorder_ms reports the time taken.
 */
int lms_reorder(lms_handle h, int ordering, uint64_t seed);

/*
 * Smooth: up to max_iters sweeps of `mode` (Eq. 1 on every interior vertex).
 * tol < 0: exactly max_iters sweeps (asynchronous; *iters_done = max_iters).
 * tol >= 0: Algorithm 1 with the Section 5.1 rule - Q_0 is computed first and
 * the loop stops after sweep k when Q_k - Q_{k-1} < tol (signed), or at
 * max_iters; synchronous.  The last sweep also records the largest vertex
 * displacement (see lms_last_stats).  iters_done may be NULL.
 */
int lms_smooth(lms_handle h, int32_t max_iters, int mode, double tol, int32_t* iters_done);

/*
 * Sweep kernel of a handle: LMS_KERNEL_DIRECT (default; one thread per vertex - FP32 Jacobi runs on the
 * persistent work-queue sweep over 128- to 512-vertex tiles chosen by mesh size, as do the colour passes of
 * FP32 coloured GS (128-vertex tiles), rows read 4 entries at a time; the other sweeps on a
 * one-pass grid, FP64 rows read 4 entries at a time; tile ignored) or LMS_KERNEL_STAGED (tile = vertices
 * per work item, a multiple of 32 up to 4096; the handle's initial tile is 512 for FP32 and 256 for FP64);
 * block = 128 or 256 threads (the work-queue sweep always uses 128).  Results do not depend on the choice
 * beyond FP32 rounding.
 */
int lms_set_launch(lms_handle h, int32_t kernel, int32_t block, int32_t tile);

/* Tile of LMS_BLOCK_GS sweeps in storage positions (tile >= 1), or 0 to choose it by mesh size (about
   eight tiles per SM, within 128..1024).  The sweep's result depends on the tile
   (it fixes the order).  Tiles below 65,536 positions run one CTA per tile on the ordering's layout; from
   65,536 up the mesh moves to a layout sorted by (tile colour, vertex colour, ordering position) and each
   (tile colour, vertex colour) range is one in-place launch, as coloured GS runs its colours - the same
   order, so the same results either way.  lms_get_block_tile returns the tile the next sweep uses.
   [host] */
int lms_set_block_tile(lms_handle h, int32_t tile);

/* How LMS_BLOCK_GS sweeps read positions.  on = 0 (default): through L1 from global memory.  on = 1: each
   CTA copies its tile, the tile's halo (the neighbours of its interior vertices outside the tile), the
   tile's rows as shared-memory indices and its vertex list into shared memory, sweeps the tile's colour
   groups there and writes back the tile's interior vertices - used whenever the largest tile with its
   halo fits in one CTA's shared memory (and needs fewer than 65,536 positions), else the sweep reads
   global memory.  Results are the same either way (the same in-place order); on GB300 the staged form
   was slower on every measured mesh (shared memory sized for the largest tile limits the CTAs per SM).
   [host]  LMS_ERR_ARG. */
int lms_set_block_staging(lms_handle h, int32_t on);
int lms_get_block_tile(lms_handle h, int32_t* tile);

/* Where the arithmetic of FP64 Jacobi and coloured GS sweeps (Eq. 1) runs: LMS_FP64_ARITH_* (default
   LMS_FP64_ARITH_MIXED3).  GB300 executes FP64 instructions at a little over one lane per clock per SM and
   32-bit integer instructions at up to 64 or 128, so moving part of the correctly rounded arithmetic to
   integer instructions keeps both busy.  Results do not depend on the choice.  LMS_ERR_ARG for another
   value.  [host] */
int lms_set_fp64_arith(lms_handle h, int32_t mode);

/* Global mesh quality Q (Section 3.2, FP64 reduction) of the current coordinates. */
int lms_quality(lms_handle h, double* Q);

/* Current coordinates in the original labelling: [2n] doubles (FP32 storage is mapped back exactly
   as x = c + s * x_hat in FP64; before any sweep the values passed in are returned unchanged). */
int lms_get_coords(lms_handle h, double* xy);

/* Replace the coordinates ([2n], original labelling); the ordering is kept.  The copy is issued on the
   handle's stream: a page-locked xy must stay valid until that stream has reached it (any call that
   returns host data synchronises it). */
int lms_set_coords(lms_handle h, const double* xy);

/* Current ordering: [n] new_to_old. */
int lms_get_permutation(lms_handle h, int32_t* new_to_old);

/* Colouring used by LMS_COLORED_GS for the current ordering ([n], original labelling, -1 = boundary).
   Computed on first use. */
int lms_get_colors(lms_handle h, int32_t* colour, int32_t* ncolours);

/* Device CSR of the current storage layout, downloaded: row_ptr [n+1], col_idx [nnz]; the layout's
   new_to_old [n] goes to storage_new_to_old when it is not NULL.  After lms_reorder the layout is the
   ordering's; after an LMS_COLORED_GS sweep it is the coloured layout (interior vertices grouped by
   colour, each group in the ordering's order, then the boundary vertices). */
int lms_get_csr(lms_handle h, int32_t* row_ptr, int32_t* col_idx, int32_t* storage_new_to_old);

/* Statistics of the last lms_smooth: largest vertex displacement of its final sweep (original units),
   device time in ms, Q before and after (NaN when no stopping rule ran).  Any pointer may be NULL. */
int lms_last_stats(lms_handle h, double* max_disp, double* ms, double* q_first, double* q_last);

/* The displacement check and device time of the last lms_smooth alone: the same as lms_last_stats with
   q_first and q_last left out (max_disp = largest vertex displacement of the final sweep in original
   units, ms = device time).  Any pointer may be NULL. */
int lms_last_error_stats(lms_handle h, double* max_disp, double* ms);

/* Number of GPU threads (contiguous blocks of the storage order) of LMS_INPLACE_STATIC sweeps; 0 = one
   per resident thread slot of the device (the default), 1 = the sequential Algorithm 1.  [host] */
int lms_set_inplace_split(lms_handle h, int32_t threads);

/* Wall time of the last lms_reorder in ms: computing the ordering (RDR: device quality keys + host
   walk; BFS / reversed BFS: device search + copy of the permutation to the host; RANDOM: host shuffle)
   and building the relabelled layout on the device.  NaN before the first lms_reorder.  [host] */
int lms_last_reorder_ms(lms_handle h, double* ordering_ms, double* layout_ms);

/* Free a handle and its device memory (NULL is ignored). */
void lms_destroy(lms_handle h);

/*
 * FP64 Jacobi sweeps that allocate no device memory.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc (code running inside another framework's memory pool or
 * under a fixed device-memory budget, services that forbid allocations on their steady-state path).
 * All buffers are the caller's DEVICE pointers: row_ptr [n+1] and col_idx [row_ptr[n]] (CSR, as for
 * lms_create), is_boundary [n] (nonzero = fixed), xy [2n] interleaved positions (input; receives the
 * result), xy_tmp [2n] work buffer (needs no initial contents; must not overlap xy, else LMS_ERR_ARG).
 * Runs `iters` sweeps on cuda_stream (NULL = legacy default stream), asynchronously: in each sweep every
 * interior vertex moves to the mean of its neighbours' positions and boundary vertices stay put.  Results
 * equal lms_smooth's FP64 Jacobi bit for bit (sums in stored row order, one IEEE division).  The mesh is
 * not validated.
 * The sweeps' only scratch - one work-queue counter per sweep - is a fixed 4 KB array inside the library
 * that every GPU loading the library holds until the process exits.  Hence:
 *   - iters is limited to 1024 per call (LMS_ERR_ARG beyond, with a message);
 *   - the first call on a device looks up that array's address (and makes the driver load the library's
 *     device code), so make it once before any stream capture; the address is kept for the process, so
 *     after a cudaDeviceReset of a device this entry point must not be used on that device again;
 *   - every call shares the array: calls whose work overlaps on the GPU (other streams, other threads)
 *     race and give wrong results; serialise them.
 */
int lms_jacobi_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                       double* xy, double* xy_tmp, int32_t iters, void* cuda_stream);

/*
 * Bounds checks of debug builds.  A library built with -DLMS_CHECKS tests every neighbour id against
 * the vertex count before a sweep or ordering kernel uses it, counts each failure on the device and
 * skips that access.  *enabled = 1 in such a build (0 otherwise, where the count is always 0);
 * *violations = failures since the last reset; reset != 0 clears the count.  Any pointer may be NULL.
 */
int lms_debug_checks(int32_t* enabled, uint64_t* violations, int32_t reset);

/* Text of the last CUDA error seen by this thread (empty if none). [host] */
const char* lms_last_error_detail(void);

/*
 * Diagnostic of the FP64 sweep's division: q[i] = s[i] / d[i] (d[i] >= 1) computed on the device by the
 * same table-driven routine the sweep uses (reciprocal RN(1/d), product, one fused correction).  Every
 * q[i] must equal the IEEE quotient.  Host arrays of `count` entries.
 */
int lms_selftest_div64(int32_t count, const double* s, const int32_t* d, double* q);

/*
 * Diagnostic of the FP32 sweeps' mean: q[i] = s[i] / d[i] (1 <= d[i] <= 64) computed on the device by
 * the routine every FP32 sweep uses (rounded reciprocal, product, one fused correction).  For finite s[i]
 * with |s[i]| >= 2^-100, and for zeros, q[i] must equal the IEEE round-to-nearest quotient; below 2^-100
 * it is within one ulp of it.  Host arrays of `count` entries.  LMS_ERR_ARG (negative count, NULL, d[i]
 * < 1), LMS_ERR_CUDA.
 */
int lms_selftest_div32(int32_t count, const float* s, const int32_t* d, float* q);

/*
 * Diagnostics of the FP64 sweep's integer-pipe arithmetic (LMS_FP64_ARITH_INT): s[i] = a[i] + b[i] and
 * q[i] = s[i] / d[i] (1 <= d[i]) computed on the device by those routines.  Every result must equal the
 * IEEE round-to-nearest sum or quotient.  Finite inputs; host arrays of `count` entries.  LMS_ERR_ARG
 * (negative count, NULL, d[i] < 1), LMS_ERR_CUDA.
 */
int lms_selftest_add64(int32_t count, const double* a, const double* b, double* s);
int lms_selftest_divint64(int32_t count, const double* s, const int32_t* d, double* q);

/*
 * Self-test of the bounded device-side waits (the tile-copy waits of the staged kernel): one device
 * thread waits on an mbarrier phase that nothing completes, gives up after about wait_us microseconds
 * (1 .. 2,000,000; counted in cycles of the top SM clock, so longer at lower clocks) and records the
 * expiry, which the host reports as LMS_ERR_TIMEOUT - the status a real expired wait returns.  The CUDA
 * context stays usable.  Returns LMS_ERR_TIMEOUT on success of the self-test, LMS_ERR_ARG, LMS_ERR_CUDA.
 */
int lms_selftest_timeout(int32_t wait_us);

/*
 * Batched FP32 smoothing of many independent meshes in one persistent
 * work-queue kernel per sweep.  Each mesh is stored under `ordering`
 * (computed as lms_reorder does), normalised by its own bounding box, and cut
 * into vertex tiles that never cross a mesh boundary; CTAs pull tiles from a
 * device counter.  Launch parameters come from the autotuner unless set with
 * lms_batch_set_config.
 */
int lms_batch_create(int32_t k, const lms_mesh_desc* meshes, int ordering, uint64_t seed, void* cuda_stream,
                     lms_batch* out);

/* `iters` Jacobi sweeps of every mesh, recorded once into a CUDA graph and replayed (asynchronous).  The
   graph holds two independent chains of sweeps over two halves of the meshes, so one half's sweep tail
   overlaps the other half's work; lms_batch_last_launches counts both chains' launches. */
int lms_batch_smooth(lms_batch b, int32_t iters);

/* Coordinates of mesh `mesh` in its original labelling ([2 n_mesh] doubles).  Returns LMS_ERR_TIMEOUT
   when a sweep since the batch's creation gave up a bounded wait (its results are then unreliable). */
int lms_batch_get_coords(lms_batch b, int32_t mesh, double* xy);

/* All meshes' coordinates, concatenated in mesh order, original labelling ([2 sum n] doubles). */
int lms_batch_get_all_coords(lms_batch b, double* xy);

/* Replace all meshes' coordinates (concatenated as above); the orderings are kept.  Asynchronous: xy must
   stay valid until the stream has read it, and a non-finite value is reported as LMS_ERR_ARG by the next
   lms_batch_get_coords / lms_batch_get_all_coords. */
int lms_batch_set_all_coords(lms_batch b, const double* xy);

/*
 * End-to-end batched smoothing from and to host memory: xy_in ([2 * n_total] FP64, the meshes'
 * original orders concatenated, as for lms_batch_set_all_coords) -> `iters` Jacobi sweeps -> xy_out
 * (same layout, as lms_batch_get_all_coords).  The meshes are split into `groups` runs of whole meshes
 * whose vertex counts ramp up and down by a factor of 4 (1 : 4 : 16 : ... : 4 : 1); each group's input
 * copy, sweeps and output copy are ordered, and the copies of one group overlap the sweeps of the others
 * (two copy streams; groups alternate between the caller's stream and a second compute stream, so one
 * group's last sweeps overlap the next group's first), so only the first input and the last output copy
 * are exposed.  The
 * result equals lms_batch_set_all_coords + lms_batch_smooth(iters) + lms_batch_get_all_coords bit for
 * bit, and afterwards the batch holds it as after those calls.  The copies overlap only when xy_in and
 * xy_out are page-locked.  groups in [1, k] (the SELL kernel always uses 1).  Synchronous.  Returns
 * LMS_ERR_ARG (NULL, bad counts, or a non-finite input value), LMS_ERR_CUDA.
 */
int lms_batch_run(lms_batch b, const double* xy_in, double* xy_out, int32_t iters, int32_t groups);

/* Totals: vertices, interior vertices, CSR entries, tiles (any pointer may be NULL). [no device work] */
int lms_batch_info(lms_batch b, int64_t* n_total, int64_t* n_interior, int64_t* nnz_total, int32_t* n_tiles);

/*
 * Launch configuration of the batched sweep: kernel = LMS_KERNEL_*, block =
 * threads per CTA (128/256/512; staged: 128 or 256), chunk = row entries read
 * per step (direct: 1 to 6, or 8; staged: 1; SELL: 1, 4 or 8), tile =
 * vertices per work item, a multiple of 128 (staged: at most 4096; SELL: the
 * degree-sorting window sigma), ctas_per_sm = resident CTAs of the persistent
 * grid (0 = as many as fit).  lms_batch_autotune times the candidates on the
 * batch (without changing its coordinates), keeps the fastest and returns it;
 * results are cached in the file named by the LMS_AUTOTUNE_CACHE environment
 * variable when it is set.  Any output pointer may be NULL.
 */
int lms_batch_get_config(lms_batch b, int32_t* kernel, int32_t* block, int32_t* chunk, int32_t* tile,
                         int32_t* ctas_per_sm);
int lms_batch_set_config(lms_batch b, int32_t kernel, int32_t block, int32_t chunk, int32_t tile, int32_t ctas_per_sm);
int lms_batch_autotune(lms_batch b, int32_t* kernel, int32_t* block, int32_t* chunk, int32_t* tile,
                       int32_t* ctas_per_sm);

/*
 * Chains of the sweep graph of lms_batch_smooth: the meshes are cut into `chains` runs of whole meshes
 * with about equal vertex counts, and each run's sweeps form an independent chain of launches in one
 * CUDA graph, so the end of one chain's sweep overlaps the other chains' work.  1 to 8 (default 2; the
 * SELL kernel always uses 1); results do not depend on it.  lms_batch_autotune times 1 to 4 chains on
 * the chosen launch configuration and keeps the fastest.  [no device work]  LMS_ERR_ARG.
 */
int lms_batch_set_chains(lms_batch b, int32_t chains);
int lms_batch_get_chains(lms_batch b, int32_t* chains);

/*
 * Storage layout of a batch.  window = 0 stores every mesh in its ordering's sequence.  window > 0 (a
 * multiple of 32, at most 65536) cuts each mesh's ordering sequence into runs of `window` consecutive
 * positions and stores every run sorted by (boundary vertices first, then ascending neighbour count),
 * stable inside equal keys: a vertex moves at most window - 1 places, and the threads of one warp get
 * rows of about one length.  The ordering itself (lms_batch_get_permutation), the coordinates the batch
 * holds and every Jacobi result are unchanged (Eq. 1 sums each row in its stored entry order, whatever
 * the storage position).  Synchronous; rebuilds the tile tables and drops captured sweep graphs.
 * lms_batch_autotune stores the batch under the ordering itself (window 0).  LMS_ERR_ARG (NULL, bad
 * window), LMS_ERR_OOM, LMS_ERR_CUDA.
 */
int lms_batch_set_layout(lms_batch b, int32_t window);
int lms_batch_get_layout(lms_batch b, int32_t* window);

/* Ordering of mesh `mesh` of a batch ([n_mesh] new_to_old, local ids).  LMS_RANDOM uses seed + mesh. */
int lms_batch_get_permutation(lms_batch b, int32_t mesh, int32_t* new_to_old);

/* Kernel launches issued by the last lms_batch_smooth / lms_smooth. [no device work] */
int lms_batch_last_launches(lms_batch b, int64_t* launches);
int lms_last_launches(lms_handle h, int64_t* launches);

void lms_batch_destroy(lms_batch b);

#ifdef __cplusplus
}
#endif

#endif /* LMS_H */
