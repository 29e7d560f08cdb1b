// lms_internal.h - declarations shared by the host code (lms_host.cpp), the
// C-ABI layer (lms_capi.cpp) and the CUDA kernels (lms_kernels.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "lms.h"

namespace lms {

// ----------------------------------------------------------------- host side

// Structural checks of a CSR mesh (see lms_validate in lms.h).
int validate_mesh(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                  int32_t ntri, const int32_t* tri);

// Orderings (Section 4.2 / Algorithm 2, Section 5.2.1).  new_to_old[k] = original id at position k.
int order_vertices(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                   const double* q_v, int ordering, uint64_t seed, int32_t* new_to_old);

// First-fit colouring of interior vertices in storage order; colour indexed by original id.
int colour_vertices(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                    const int32_t* new_to_old, int32_t* colour, int32_t* ncolours);

// Block order of the in-place sweep (see lms_block_order in lms.h).  vertex_colour ([n], by original id)
// and nvertex_colours, when given, receive the first-fit vertex colouring the order uses.
int block_order(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                const int32_t* new_to_old, int32_t tile, int32_t* tile_colour, int32_t* ntile_colours,
                int32_t* order, int32_t* n_order, int32_t* vertex_colour = nullptr,
                int32_t* nvertex_colours = nullptr);

// Tables of a block Gauss-Seidel sweep (LMS_BLOCK_GS) for storage order new_to_old: verts = storage
// positions of the interior vertices in block order; per listed tile (a tile holding interior vertices,
// in block order) ncolours + 1 offsets of its vertex-colour groups in verts (groups[t * (ncolours + 1)
// + c]); tiles of tile colour c are the listed tiles [tc_ofs[c], tc_ofs[c + 1]).
struct BlockTables {
    std::vector<int32_t> verts, groups, tc_ofs;
    int32_t ncolours = 1;
};
int block_tables(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                 const int32_t* new_to_old, int32_t tile, BlockTables& out);

// Shared-memory tables of the staged block Gauss-Seidel sweep, built from BlockTables for the same storage
// order and tile: per listed tile its position range [x, y) and halo range [z, w) in `halo` (storage
// positions of the neighbours of its interior vertices outside the tile, in first-seen order); per entry
// of BlockTables::verts the start of its row in `lcol` (lrow, one more entry than verts), and in lcol each
// row's neighbours, in stored row order, as indices into the tile's shared-memory copy: position p of the
// tile -> p - x, halo vertex j -> (y - x) + j.  max_slots = largest (y - x) + (w - z) over the tiles.
struct BlockStageTables {
    std::vector<int32_t> tile_info;  // 4 ints per listed tile: x, y, z, w
    std::vector<int32_t> halo, lrow;
    std::vector<uint16_t> lcol;
    int32_t max_slots = 0;
    int32_t max_verts = 0;    // largest count of interior vertices in a tile
    int32_t max_entries = 0;  // largest count of lcol entries of a tile
};
// Returns LMS_ERR_ARG when a tile with its halo needs 65,536 slots or more (16-bit local indices).
int block_stage_tables(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const int32_t* new_to_old,
                       int32_t tile, const BlockTables& bt, BlockStageTables& out);

// Set the message reported with LMS_ERR_CUDA and friends (thread-local).
void set_error_detail(const std::string& s);
const std::string& error_detail();

// ------------------------------------------------------------- device side

constexpr int kMaxRecipDeg = 64;  // reciprocal table size for the exact FP64 division
// The device reciprocal table (SweepArgs::recip) holds kRecipTableDoubles 8-byte slots: RN(1/d) for
// d = 0..kMaxRecipDeg, then the integer division's words floor((2^64 - 1) / d) as (high, low) uint32
// pairs for d = 0..kMaxRecipDeg (read as a uint32 array from slot kMaxRecipDeg + 1).
constexpr int kRecipTableDoubles = 2 * (kMaxRecipDeg + 1);

// State shared by the sweep, quality and stop-check kernels of one handle.
struct DevState {
    double q_prev;                 // Q of the previous sweep
    double q_cur;                  // Q of the latest sweep (or of lms_quality)
    double q_first;                // Q_0
    unsigned long long disp2[2];   // max squared displacement, by sweep parity (bits of a double >= 0)
    int32_t stop;                  // set by the stop check once the rule fires
    int32_t k;                     // sweeps completed under the stopping rule
    int32_t iters_at_stop;         // sweep index at which the rule fired
    int32_t err;                   // nonzero: a device-side check failed
};

struct SweepArgs {
    const int32_t* row_ptr;
    const int32_t* col_idx;
    const uint32_t* bnd_bits;      // bit v set = boundary (NULL: every vertex in range is interior)
    const void* src;               // double2 / float2 positions read
    void* dst;                     // positions written (== src for the in-place coloured sweep)
    int32_t v_begin, v_end;        // vertex range of a static launch
    const int32_t* order;          // static launch: thread i handles vertex order[i] (NULL: vertex i)
    int32_t n_vertices;            // vertices addressable by col_idx (bounds checks of debug builds)
    const int2* items;             // work-queue tiles (batched)
    int32_t n_items;
    int32_t* queue;                // work-queue counter for this sweep
    const DevState* state;         // stop flag (NULL: never stop)
    unsigned long long* disp2;     // max squared displacement accumulator (NULL: off)
    const double* recip;           // [kMaxRecipDeg+1] RN(1/d) for the FP64 exact division
};

// Block Gauss-Seidel sweep (k_block_gs): one CTA per tile of one tile colour; inside a tile the vertex
// colours run one after another, separated by block barriers; positions updated in place.  Tiles of one
// colour share no edge between interior vertices, so a launch equals the in-place sweep over its tiles
// in block order (lms_block_order).
struct BlockGsArgs {
    const int32_t* row_ptr;
    const int32_t* col_idx;
    void* xy;                      // double2 / float2 positions, updated in place
    const int32_t* verts;          // storage positions of the interior vertices in block order
    const int32_t* group_ofs;      // [listed tile][ncolours + 1]: offsets of the tile's colour groups in verts
    int32_t ncolours;
    int32_t tile_begin;            // listed tile handled by block 0 of this launch
    int32_t n_vertices;            // vertices addressable by col_idx (bounds checks of debug builds)
    const DevState* state;         // stop flag (NULL: never stop)
    unsigned long long* disp2;     // max squared displacement (NULL: off)
    const double* recip;           // FP64 reciprocal table
};
cudaError_t launch_block_gs(int precision, const BlockGsArgs& a, int32_t n_tiles, cudaStream_t stream);

// Staged block Gauss-Seidel (k_block_gs_staged): as k_block_gs, but each CTA copies its tile and the
// tile's halo into shared memory, sweeps the colour groups there and writes back the tile's interior
// vertices.  Tables from BlockStageTables.
struct BlockGsStagedArgs {
    void* xy;                      // double2 / float2 positions, updated in place
    const int4* tile_info;         // per listed tile: first, end position; first, end halo entry
    const int32_t* halo;
    const int32_t* verts;          // storage positions of the interior vertices in block order
    const int32_t* lrow;           // per verts entry: first local neighbour index in lcol (+1 entry)
    const uint16_t* lcol;          // local neighbour indices into the tile's shared-memory copy
    const int32_t* group_ofs;      // [listed tile][ncolours + 1]: offsets of the tile's colour groups in verts
    int32_t ncolours;
    int32_t tile_begin;            // listed tile handled by block 0 of this launch
    int32_t max_slots;             // shared-memory positions per CTA (largest tile + halo)
    int32_t max_verts;             // largest interior vertex count of a tile
    int32_t max_entries;           // largest local-row entry count of a tile
    const DevState* state;         // stop flag (NULL: never stop)
    unsigned long long* disp2;     // max squared displacement (NULL: off)
    const double* recip;           // FP64 reciprocal table
};
cudaError_t launch_block_gs_staged(int precision, const BlockGsStagedArgs& a, int32_t n_tiles, cudaStream_t stream);
// bytes of dynamic shared memory per CTA of k_block_gs_staged
size_t block_gs_staged_smem(int precision, int32_t max_slots, int32_t max_verts, int32_t max_entries);

// Tile-staged sweep (lms_staged.cu): items[i] = (first vertex, end vertex, first CSR entry, end entry)
// of a tile; tiles never cross a mesh or a colour range.  row_ptr, col_idx and bnd_bits must have at
// least 8 readable padding entries past their ends (copies are rounded to 16 bytes).
struct StagedArgs {
    const int32_t* row_ptr;
    const int32_t* col_idx;
    const uint32_t* bnd_bits;      // NULL: every vertex of every tile is interior
    const void* src;
    void* dst;
    const int4* items;
    int32_t n_items;
    int32_t* queue;                // tile counter of this launch (zeroed before it)
    int32_t tile_cap;              // max vertices per tile
    int32_t e_cap;                 // max CSR entries per tile
    int32_t n_vertices;            // vertices addressable by col_idx (bounds checks of debug builds)
    const DevState* state;         // stop flag (NULL: never stop)
    unsigned long long* disp2;     // max squared displacement (NULL: off)
    const double* recip;           // FP64 reciprocal table
    int32_t* err;                  // set to 1 when a bounded wait expired
};
size_t staged_smem_bytes(int precision, int32_t tile_cap, int32_t e_cap);
// One thread waits (bounded by bound_cycles) on an mbarrier phase that never completes; sets *err = 1.
cudaError_t launch_wait_selftest(long long bound_cycles, int32_t* err, cudaStream_t stream);
cudaError_t launch_sweep_staged(int precision, bool in_place, const StagedArgs& a, int grid, int block,
                                cudaStream_t stream);
int staged_occupancy(int precision, bool in_place, int block, int32_t tile_cap, int32_t e_cap);

// Breadth-first orderings of k graphs on the device (k_bfs).  Graph g holds vertices
// [voff[g], voff[g+1]) (voff NULL: one graph of n_total vertices) and its CSR uses global ids;
// out[voff[g] + p] = global id at queue position p.  pos and parent are [n_total] scratch.
struct BfsArgs {
    const int32_t* row_ptr;
    const int32_t* col_idx;
    const int32_t* voff;
    int32_t k;
    int32_t n_total;
    int32_t* out;
    int32_t* pos;
    int32_t* parent;
};
int bfs_cluster_size(int32_t max_graph_vertices);
cudaError_t launch_bfs(const BfsArgs& a, int cluster, cudaStream_t stream);

// Block RDR on the device (k_block_rdr): blocks[b] = (graph's first vertex v0, first and end BFS
// position of the block within the graph, unused); bfs / bfs_pos = a BfsArgs out / pos pair; out receives
// the new_to_old (global ids) at the same places as bfs.  cap = a power of two >= the largest block.
struct BrdrArgs {
    const int32_t* row_ptr;
    const int32_t* col_idx;
    const uint8_t* is_boundary;
    const double* q;
    const int32_t* bfs;
    const int32_t* bfs_pos;
    const int4* blocks;
    int32_t n_blocks;
    int32_t cap;
    int32_t n_total;               // vertices addressable by col_idx (bounds checks of debug builds)
    int32_t* out;
};
size_t block_rdr_smem(int32_t cap);
cudaError_t launch_block_rdr(const BrdrArgs& a, int sms, cudaStream_t stream);
int block_rdr_max_degree();  // rows longer than this need the host implementation

// Failed bounds checks counted by each kernel source in debug builds (-DLMS_CHECKS; 0 otherwise).
unsigned long long check_violations_kernels(bool reset);
unsigned long long check_violations_orderings(bool reset);
unsigned long long check_violations_noalloc(bool reset);
unsigned long long check_violations_staged(bool reset);
bool checks_enabled();

// Launchers (all asynchronous on `stream`; return cudaError_t of the launch).
// fp64_arith: LMS_FP64_ARITH_* (where the FP64 sums and means run; ignored for FP32)
cudaError_t launch_sweep(int precision, bool in_place, const SweepArgs& a, int block, int fp64_arith,
                         cudaStream_t stream);
// The paper's static-schedule in-place sweep over [0, a.v_end) split into `threads` contiguous blocks
// (k_inplace_static); positions in a.dst, updated in place.
cudaError_t launch_inplace_static(int precision, const SweepArgs& a, int32_t threads, cudaStream_t stream);
// Batched FP32 sweep over a SELL-C-sigma work layout (see k_batch_sell).
struct SellArgs {
    const int32_t* col;            // column-major neighbour ids per slice, -1 past a slot's row
    const int2* slice;             // per slice: (first entry, slice degree)
    const int32_t* slot;           // per slot (32 per slice): storage position of the vertex, -1 = empty
    const void* src;
    void* dst;
    const int2* items;             // per tile: [first slice, end slice)
    int32_t n_items;
    int32_t* queue;
};
cudaError_t launch_batch_sell(const SellArgs& a, int block, int chunk, int grid, cudaStream_t stream);
int batch_sell_occupancy(int block, int chunk);

// Batched FP32 sweep over packed rows (k_batch_sweep_packed): row_words[v] = (first id pair of v's row -
// first id pair of v's mesh) | neighbour count << kPackedDegreeShift | boundary << 31; id_pairs holds every
// row padded to an even length with -1.  A batch can use it when every mesh has fewer than 2^22 id pairs
// and every row at most kMaxPackedDegree entries.
constexpr int kPackedDegreeShift = 22;
constexpr int32_t kPackedOffsetMask = (1 << kPackedDegreeShift) - 1;
constexpr int32_t kPackedDegreeMask = 63;
constexpr int kMaxPackedDegree = 63;
struct PackedArgs {
    const int32_t* row_words;
    const int2* id_pairs;
    const void* src;               // float2 positions read
    void* dst;                     // float2 positions written
    const int2* items;             // work-queue tiles (first vertex, end vertex)
    const int32_t* items_pbase;    // per tile: first id pair of the tile's mesh
    int32_t n_items;
    int32_t* queue;                // work-queue counter for this sweep
    int32_t n_vertices;            // vertices addressable by the ids (bounds checks of debug builds)
};
// chunk = ids per step: 2, 4 or 6
cudaError_t launch_batch_sweep_packed(const PackedArgs& a, int block, int chunk, int grid, cudaStream_t stream);
int batch_packed_occupancy(int block, int chunk);  // resident CTAs per SM (0 on error)
// Single-mesh FP32 Jacobi sweep over packed rows (k_sweep_packed_mesh): row_words[v] = (first id pair of v's row
// - block_pbase[v >> kPackedBlockShift]) | neighbour count << kPackedDegreeShift | boundary << 31, with
// block_pbase[b] = first id pair of the rows of storage positions [b << kPackedBlockShift, ...); id_pairs
// holds every interior row, farthest neighbour first, padded to an even length with -1.  Rows of at most
// kMaxPackedDegree entries.
constexpr int kPackedBlockShift = 12;
struct PackedMeshArgs {
    const int32_t* row_words;
    const int32_t* block_pbase;
    const int2* id_pairs;
    const void* src;               // float2 positions read
    void* dst;                     // float2 positions written
    const int2* items;             // work-queue tiles (first vertex, end vertex)
    int32_t n_items;
    int32_t* queue;                // work-queue counter for this launch
    int32_t n_vertices;            // vertices addressable by the ids (bounds checks of debug builds)
    const DevState* state;         // stop flag (NULL: never stop)
    unsigned long long* disp2;     // max squared displacement (NULL: off)
};
cudaError_t launch_sweep_packed_mesh(const PackedMeshArgs& a, int block, int grid, cudaStream_t stream);
int sweep_packed_mesh_occupancy(int block);  // resident CTAs per SM (0 on error)

// out[2 pstart[v] ...] = row v of (row_ptr, col_idx) padded with -1 to 2 (pstart[v + 1] - pstart[v]) ids
cudaError_t launch_pad_rows(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const int32_t* pstart,
                            int32_t* out, cudaStream_t stream);
// Orders every row's entries by decreasing |u - v| (stable); rows of at most kMaxPackedDegree entries.
// row_ptr may carry the boundary flag in bit 31.
cudaError_t launch_sort_rows_far_first(int32_t n, const int32_t* row_ptr, int32_t* col_idx, cudaStream_t stream);

// batched work-queue sweep, rows read `chunk` (1 to 6, or 8) entries at a time
cudaError_t launch_batch_sweep(const SweepArgs& a, int block, int chunk, int grid, cudaStream_t stream);
int batch_sweep_occupancy(int block, int chunk);  // resident CTAs per SM (0 on error)

cudaError_t launch_tri_quality_exact(int32_t ntri, const int32_t* tri, const double* xy64, double* q_t,
                                     cudaStream_t stream);
cudaError_t launch_vertex_quality_exact(int32_t n, const int32_t* vt_ptr, const int32_t* vt_idx,
                                        const double* q_t, double* q_v, cudaStream_t stream);
// Per-sweep quality: partial sums of w_t * q_t over a fixed grid of nblocks, then a fixed-order finish.
constexpr int kQualityBlocks = 1024;
// w: per-triangle weights, double for FP64 positions and float for FP32 positions.
cudaError_t launch_quality_partials(int precision, int32_t ntri, const int32_t* tri, const void* xy,
                                    const void* w, double* partials, const DevState* state,
                                    cudaStream_t stream);
// Q = (sum of partials) / n.  mode 0: store into q_cur; mode 1: Q_0 (q_first = q_prev = q_cur = Q).
cudaError_t launch_quality_finish(const double* partials, double n, DevState* state, int mode, cudaStream_t stream);
// Stop check after a sweep (Section 5.1 rule + iteration cap); skipped once the rule has fired.
cudaError_t launch_stop_check(const double* partials, double n, DevState* state, double tol, double goal,
                              int32_t max_iters, cudaStream_t stream);

cudaError_t launch_gather_rows(int32_t n, const int32_t* new_to_old, const int32_t* rp_src, const int32_t* ci_src,
                               const int32_t* rp_dst, int32_t* ci_dst, const int32_t* map, cudaStream_t stream);
// batched CSR: set bit 31 of row_ptr[v] for boundary vertices (read back with & 0x7fffffff)
cudaError_t launch_flag_boundary_rows(int32_t n, const uint32_t* bits, int32_t* row_ptr, cudaStream_t stream);
cudaError_t launch_map_ids(int64_t count, const int32_t* map, const int32_t* src, int32_t* dst,
                           cudaStream_t stream);
cudaError_t launch_boundary_bits(int32_t n, const int32_t* new_to_old, const uint8_t* bnd_orig, uint32_t* bits,
                                 cudaStream_t stream);
// dst[k] = src[perm[k]] for 16-byte (double2) or 8-byte (float2) elements
cudaError_t launch_gather_xy(int precision, int32_t n, const int32_t* perm, const void* src, void* dst,
                             cudaStream_t stream);
// original-order FP64 input -> storage-order positions: dst[k] = f(src[new_to_old[k]])
// precision FP32: normalised with (cx, cy, inv_s); item_mesh/item ranges give per-mesh constants when given
cudaError_t launch_load_xy(int precision, int32_t n, const int32_t* new_to_old, const double* src_orig, void* dst,
                           double cx, double cy, double inv_s, cudaStream_t stream);
// storage-order positions -> original-order FP64: dst[new_to_old[k]] = g(src[k]); FP32 boundary vertices
// are taken from fixed_xy (original order) when it is given
cudaError_t launch_store_xy(int precision, int32_t n, const int32_t* new_to_old, const void* src, double* dst_orig,
                            double cx, double cy, double s, const uint8_t* bnd_orig, const double* fixed_xy,
                            cudaStream_t stream);
// batched: per-tile mesh constants (tile t covers items[t], belongs to mesh item_mesh[t])
// writes both ping-pong buffers; sets *bad to 1 when an input coordinate is not finite
cudaError_t launch_batch_load_xy(int32_t n_items, const int2* items, const int32_t* item_mesh,
                                 const int32_t* new_to_old, const double* src_orig, float2* dst0, float2* dst1,
                                 const double* mesh_cs, int32_t* bad, cudaStream_t stream);
cudaError_t launch_batch_store_xy(int32_t n_items, const int2* items, const int32_t* item_mesh,
                                  const int32_t* new_to_old, const float2* src, double* dst_orig,
                                  const double* mesh_cs, const uint32_t* bnd_bits, const double* fixed_xy,
                                  cudaStream_t stream);

// Diagnostic: q[i] = s[i] / d[i] by the FP32 sweeps' mean (mean_f32 with c = 0).
cudaError_t launch_div32_selftest(int32_t count, const float* s, const int32_t* d, float* q, cudaStream_t stream);
// Diagnostic: s[i] = RN(a[i] + b[i]) by the integer-pipe addition of the FP64 sweep (add_rn_int).
cudaError_t launch_add_selftest(int32_t count, const double* a, const double* b, double* s, cudaStream_t stream);
// Diagnostic: q[i] = s[i] / d[i] by the integer-pipe division of LMS_FP64_ARITH_INT (div_rn_int).
cudaError_t launch_divint_selftest(int32_t count, const double* s, const int32_t* d, const double* recip, double* q,
                                   cudaStream_t stream);
// Diagnostic: q[i] = s[i] / d[i] by the table-driven exact division used in the FP64 sweep.
cudaError_t launch_div_selftest(int32_t count, const double* s, const int32_t* d, const double* recip, double* q,
                                cudaStream_t stream);

}  // namespace lms
