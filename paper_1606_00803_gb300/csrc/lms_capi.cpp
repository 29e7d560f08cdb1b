// lms_capi.cpp - the C ABI of liblms (declared in include/lms.h): handles,
// device memory, storage layouts, CUDA-graph capture of sweep loops, the
// Section 5.1 stopping rule, device orderings (BFS, block RDR), the batched
// work-queue path, its autotuner and the pipelined end-to-end batch call.
//
// Storage layouts.  A handle keeps the mesh in one storage order at a time:
//   - the ordering's layout (lms_reorder): position k holds original vertex
//     new_to_old[k]; Jacobi and the in-place static sweep run here (the
//     latter moves the mesh back here after a coloured Gauss-Seidel);
//   - the coloured layout (first LMS_COLORED_GS sweep after a reorder): the
//     interior vertices sorted by (colour, position in the ordering), then the
//     boundary vertices; each colour is one contiguous range, so one colour
//     pass reads its rows and writes its positions contiguously, and its
//     neighbour gathers stay inside the ordering's locality window of every
//     other colour.  Jacobi results do not depend on the layout (rows keep
//     their entry order), so Jacobi also runs on the coloured layout.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <functional>
#include <map>
#include <mutex>
#include <sstream>
#include <thread>
#include <vector>

#include "lms_internal.h"

using lms::DevState;
using lms::SweepArgs;

namespace {

struct Allocator {
    void* (*alloc)(size_t, void*, void*) = nullptr;
    void (*release)(void*, void*) = nullptr;
    void* ctx = nullptr;
};
std::mutex g_alloc_mu;
Allocator g_alloc;

#define LMS_CUDA(call)                                                                           \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            lms::set_error_detail(std::string(#call) + ": " + cudaGetErrorString(e_));           \
            return e_ == cudaErrorMemoryAllocation ? LMS_ERR_OOM : LMS_ERR_CUDA;                 \
        }                                                                                        \
    } while (0)

#define LMS_TRY(expr)             \
    do {                          \
        int rc_ = (expr);         \
        if (rc_ != LMS_OK) return rc_; \
    } while (0)

// Device allocations of one handle, released together.
struct Arena {
    Allocator al;
    cudaStream_t stream = nullptr;
    std::vector<void*> ptrs;

    int get(void** out, size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        if (bytes == 0) bytes = 256;
        void* p = nullptr;
        if (al.alloc) {
            p = al.alloc(bytes, stream, al.ctx);
            if (!p) return LMS_ERR_OOM;
        } else {
            cudaError_t e = cudaMalloc(&p, bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                lms::set_error_detail(std::string("cudaMalloc: ") + cudaGetErrorString(e));
                return LMS_ERR_OOM;
            }
        }
        ptrs.push_back(p);
        *out = p;
        return LMS_OK;
    }
    template <typename T>
    int get(T** out, size_t count) {
        return get(reinterpret_cast<void**>(out), count * sizeof(T));
    }
    void release_all() {
        for (void* p : ptrs) {
            if (al.release)
                al.release(p, al.ctx);
            else
                cudaFree(p);
        }
        ptrs.clear();
    }
};

struct GraphCache {
    std::map<std::string, cudaGraphExec_t> execs;
    std::map<std::string, int64_t> kernels;
    void clear() {
        for (auto& kv : execs) cudaGraphExecDestroy(kv.second);
        execs.clear();
        kernels.clear();
    }
};

int64_t count_kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return -1;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return -1;
    int64_t k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

// Record `body` (issuing work on the capture stream) into an executable graph.
template <typename F>
int capture(cudaStream_t cap, F&& body, cudaGraphExec_t* exec, int64_t* kernels) {
    LMS_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    int rc = body(cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (rc != LMS_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) {
        lms::set_error_detail(std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
        return LMS_ERR_CUDA;
    }
    *kernels = count_kernel_nodes(g);
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        lms::set_error_detail(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        return LMS_ERR_CUDA;
    }
    return LMS_OK;
}

int check_launch(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return LMS_OK;
    lms::set_error_detail(std::string(what) + ": " + cudaGetErrorString(e));
    return LMS_ERR_CUDA;
}

bool all_finite(const double* xy, int64_t count) {
    for (int64_t i = 0; i < count; ++i)
        if (!std::isfinite(xy[i])) return false;
    return true;
}

// Bounding box centre and scale (the larger side; 1 for a degenerate box).
void bbox(const double* xy, int32_t n, double* cx, double* cy, double* s) {
    double x0 = xy[0], x1 = xy[0], y0 = xy[1], y1 = xy[1];
    for (int32_t v = 1; v < n; ++v) {
        x0 = std::min(x0, xy[2 * v]);
        x1 = std::max(x1, xy[2 * v]);
        y0 = std::min(y0, xy[2 * v + 1]);
        y1 = std::max(y1, xy[2 * v + 1]);
    }
    *cx = 0.5 * (x0 + x1);
    *cy = 0.5 * (y0 + y1);
    double side = std::max(x1 - x0, y1 - y0);
    *s = side > 0.0 ? side : 1.0;
}

// Vertex -> triangle incidence, rows in ascending triangle id.
void build_incidence(int32_t n, int32_t ntri, const int32_t* tri, std::vector<int32_t>& ptr,
                     std::vector<int32_t>& idx) {
    ptr.assign(n + 1, 0);
    for (int64_t i = 0; i < 3 * int64_t(ntri); ++i) ptr[tri[i] + 1]++;
    for (int32_t v = 0; v < n; ++v) ptr[v + 1] += ptr[v];
    idx.resize(std::max<int64_t>(1, 3 * int64_t(ntri)));
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (int32_t t = 0; t < ntri; ++t)
        for (int c = 0; c < 3; ++c) idx[fill[tri[3 * t + c]]++] = t;
}

// w_t = sum over t's corners of 1 / (number of triangles at the corner)
void build_weights(int32_t ntri, const int32_t* tri, const std::vector<int32_t>& ptr, std::vector<double>& w) {
    w.resize(std::max<int32_t>(1, ntri));
    for (int32_t t = 0; t < ntri; ++t) {
        double s = 0.0;
        for (int c = 0; c < 3; ++c) {
            int32_t v = tri[3 * t + c];
            s += 1.0 / double(ptr[v + 1] - ptr[v]);
        }
        w[t] = s;
    }
}

// RN(1/d), then the (high, low) words of floor((2^64 - 1) / d), d = 0..kMaxRecipDeg (lms_internal.h)
std::vector<double> recip_table() {
    std::vector<double> r(lms::kRecipTableDoubles, 0.0);
    for (int d = 1; d <= lms::kMaxRecipDeg; ++d) r[d] = 1.0 / double(d);
    std::vector<uint32_t> words(2 * (lms::kMaxRecipDeg + 1), 0u);
    for (int d = 1; d <= lms::kMaxRecipDeg; ++d) {
        const uint64_t m = ~0ull / uint64_t(d);
        words[2 * d] = uint32_t(m >> 32);
        words[2 * d + 1] = uint32_t(m);
    }
    std::memcpy(r.data() + lms::kMaxRecipDeg + 1, words.data(), 4 * words.size());
    return r;
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Storage layouts of a mesh handle: the ordering's own, colour-major (coloured GS), and block-range
// (the block Gauss-Seidel with tiles of at least kBlockRangeTile positions).
constexpr int kLayoutOrdering = 0, kLayoutColoured = 1, kLayoutBlockRanges = 2;
// Block Gauss-Seidel tiles from this size up run on the block-range layout, one range per (tile colour,
// vertex colour); smaller tiles run one CTA per tile on the ordering layout.
constexpr int32_t kBlockRangeTile = 65536;

}  // namespace

// ------------------------------------------------------------------ handle

struct lms_mesh_s {
    Arena arena;
    cudaStream_t stream = nullptr;      // caller's stream (work runs here)
    cudaStream_t cap = nullptr;         // private stream used only to record graphs
    int precision = LMS_FP64;
    int32_t n = 0, ntri = 0, nnz = 0;
    // host copies, original labelling
    std::vector<int32_t> rp, ci, tri;
    std::vector<uint8_t> bnd;
    // orderings
    std::vector<int32_t> user_perm;     // the ordering (new_to_old)
    std::vector<int32_t> perm;          // current storage layout (new_to_old)
    int gs_layout = kLayoutOrdering;    // storage layout kind (kLayout*)
    int32_t gs_layout_tile = 0;         // tile of the block-range layout
    bool colours_valid = false;
    std::vector<int32_t> colour;        // by original id
    int32_t ncolours = 0;
    // in-place range layouts: range r occupies storage [range_ofs[r], range_ofs[r+1]); coloured layout: one
    // range per colour; block-range layout: one per non-empty (tile colour, vertex colour) pair, in order
    std::vector<int32_t> range_ofs;
    double cx = 0, cy = 0, scale = 1;   // FP32 normalisation
    // device, original labelling
    int32_t *d_rp0 = nullptr, *d_ci0 = nullptr, *d_tri0 = nullptr, *d_vt_ptr = nullptr, *d_vt_idx = nullptr;
    uint8_t* d_bnd0 = nullptr;
    double* d_w = nullptr;              // per-triangle quality weights: doubles (FP64) or floats (FP32)
    // device, current layout
    int32_t *d_rp = nullptr, *d_ci = nullptr, *d_tri = nullptr, *d_perm = nullptr, *d_tmp = nullptr;
    uint32_t* d_bits = nullptr;
    void* d_xy[2] = {nullptr, nullptr};
    int cur = 0;
    void* d_xy_swap = nullptr;          // layout changes
    double* d_xy64 = nullptr;           // FP64 staging in original order (input / output / RDR keys)
    double* d_pristine = nullptr;       // FP32: caller's last coordinates, original order (boundary rows
                                        // stay valid after sweeps: boundary vertices never move)
    bool pristine_valid = false;
    double *d_qt = nullptr, *d_qv = nullptr, *d_partials = nullptr, *d_recip = nullptr;
    DevState* d_state = nullptr;
    DevState* h_state = nullptr;        // pinned
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // sweep launch configuration and tile tables (staged kernel)
    int kernel = LMS_KERNEL_DIRECT, block = 256, tile = 512;
    std::vector<int32_t> rp_cur;        // row offsets of the current layout (host copy)
    int4* d_items4 = nullptr;           // tiles over [0, n), then tiles of each colour range
    int64_t items_cap = 0;
    int32_t n_items_all = 0;
    std::vector<int32_t> item_col_ofs;  // range r: tiles [n_items_all + ofs[r], n_items_all + ofs[r+1])
    int32_t e_cap = 0;
    int32_t* d_rpf = nullptr;           // row offsets of the current layout with the boundary flag in bit 31
    int32_t* d_order = nullptr;         // FP64: thread -> vertex map of the one-thread-per-vertex sweeps
    int2* d_items2 = nullptr;           // FP32 work-queue tiles over [0, n), then over each colour's range
    int64_t items2_cap = 0;
    int32_t n_items2 = 0;               // tiles over [0, n)
    std::vector<int32_t> item2_col_ofs; // range r: tiles [n_items2 + ofs[r], n_items2 + ofs[r+1])
    // FP32 packed rows of the current layout (Jacobi, k_sweep_packed_mesh); pk_ok false when a row is too long
    bool pk_ok = false;
    int32_t *d_pk_rw = nullptr, *d_pk_bbase = nullptr;
    int2* d_pk_pairs = nullptr;
    int64_t pk_pairs_cap = 0;
    int32_t* d_queue = nullptr;         // one tile counter per work-queue launch of a graph
    int32_t queue_slots = 0;
    int32_t slot_next = 0;              // next counter while a graph is recorded
    int32_t* d_err = nullptr;           // set by a kernel whose bounded wait expired
    int sms = 0;
    GraphCache graphs;
    int64_t last_launches = 0;
    bool stats_pending = false;
    int last_disp_slot = 0;
    double last_disp = NAN, last_ms = NAN, q_first = NAN, q_last = NAN;
    double reorder_ms[2] = {NAN, NAN};  // last lms_reorder: ordering, relabelled layout
    int32_t inplace_threads = 0;        // LMS_INPLACE_STATIC split (0: one thread per resident slot)
    // LMS_BLOCK_GS tables for the ordering layout (rebuilt after a reorder or a tile change)
    int32_t block_tile_req = 0;         // requested tile (0: by mesh size)
    int32_t block_tile = 0;             // tile of the current tables
    bool block_valid = false;
    int32_t block_ncolours = 0;         // vertex colours (group slots per tile)
    std::vector<int32_t> block_tc_ofs;  // tile colour c: listed tiles [ofs[c], ofs[c+1])
    int32_t* d_blk_verts = nullptr;
    int32_t* d_blk_groups = nullptr;
    int64_t blk_verts_cap = 0, blk_groups_cap = 0;
    // staged block Gauss-Seidel tables (tile + halo in shared memory); used when block_staged and they fit
    // (off by default: slower than reading through L1 on the measured meshes)
    bool block_staged = false;
    bool st_valid = false;
    int32_t st_max_slots = 0, st_max_verts = 0, st_max_entries = 0;
    int4* d_st_tile = nullptr;
    int32_t *d_st_halo = nullptr, *d_st_lrow = nullptr;
    uint16_t* d_st_lcol = nullptr;
    int64_t st_tile_cap = 0, st_halo_cap = 0, st_lrow_cap = 0, st_lcol_cap = 0;
    int32_t fp64_arith = LMS_FP64_ARITH_MIXED3;  // where FP64 sums and means run (fastest on GB300)

    ~lms_mesh_s() {
        if (stream) cudaStreamSynchronize(stream);
        graphs.clear();
        arena.release_all();
        if (h_state) cudaFreeHost(h_state);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (cap) cudaStreamDestroy(cap);
    }
};

namespace {

// Breadth-first orderings on the device (k_bfs) of k graphs with vertex offsets voff (host; NULL:
// one graph of n vertices) over the device CSR rp/ci with global ids.  With q != NULL (device vertex
// qualities) and is_boundary (device flags), each BFS order is then cut into blocks of LMS_BRDR_BLOCK
// positions and reordered by block RDR (k_block_rdr).  out (host, [n]) receives the global new_to_old.
// Scratch comes from the allocator and is released before returning.
int device_order(const Allocator& al, cudaStream_t s, int sms, const int32_t* rp, const int32_t* ci, int32_t n,
                 int32_t k, const int64_t* voff, const double* q, const uint8_t* is_boundary, int32_t* out) {
    Arena tmp;
    tmp.al = al;
    tmp.stream = s;
    lms::BfsArgs a{};
    int32_t* d_voff = nullptr;
    int32_t* d_brdr = nullptr;
    int4* d_blocks = nullptr;
    const int32_t graphs = voff ? k : 1;
    std::vector<int32_t> v32(graphs + 1);
    for (int32_t g = 0; g <= graphs; ++g) v32[g] = voff ? int32_t(voff[g]) : (g == 0 ? 0 : n);
    int32_t largest = 0;
    for (int32_t g = 0; g < graphs; ++g) largest = std::max(largest, v32[g + 1] - v32[g]);
    std::vector<int4> blocks;
    if (q)
        for (int32_t g = 0; g < graphs; ++g)
            for (int32_t st = 0; st < v32[g + 1] - v32[g]; st += LMS_BRDR_BLOCK)
                blocks.push_back(make_int4(v32[g], st, std::min(v32[g + 1] - v32[g], st + LMS_BRDR_BLOCK), 0));
    int rc;
    if ((rc = tmp.get(&a.out, n)) || (rc = tmp.get(&a.pos, n)) || (rc = tmp.get(&a.parent, n)) ||
        (voff && (rc = tmp.get(&d_voff, k + 1))) || (q && (rc = tmp.get(&d_brdr, n))) ||
        (q && (rc = tmp.get(&d_blocks, blocks.size())))) {
        tmp.release_all();
        return rc;
    }
    a.row_ptr = rp;
    a.col_idx = ci;
    a.voff = d_voff;
    a.k = graphs;
    a.n_total = n;
    cudaError_t e = voff ? cudaMemcpyAsync(d_voff, v32.data(), 4 * size_t(k + 1), cudaMemcpyHostToDevice, s)
                         : cudaSuccess;
    if (!e) e = lms::launch_bfs(a, lms::bfs_cluster_size(largest), s);
    const int32_t* result = a.out;
    if (!e && q) {
        lms::BrdrArgs b{};
        b.row_ptr = rp;
        b.col_idx = ci;
        b.is_boundary = is_boundary;
        b.q = q;
        b.bfs = a.out;
        b.bfs_pos = a.pos;
        b.blocks = d_blocks;
        b.n_blocks = int32_t(blocks.size());
        b.n_total = n;
        b.cap = 1;
        while (b.cap < std::min(largest, int32_t(LMS_BRDR_BLOCK))) b.cap <<= 1;
        b.out = d_brdr;
        e = cudaMemcpyAsync(d_blocks, blocks.data(), sizeof(int4) * blocks.size(), cudaMemcpyHostToDevice, s);
        if (!e) e = lms::launch_block_rdr(b, sms, s);
        result = d_brdr;
    }
    if (!e) e = cudaMemcpyAsync(out, result, 4 * size_t(n), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    tmp.release_all();
    if (e) {
        lms::set_error_detail(std::string(q ? "device block RDR: " : "device BFS: ") + cudaGetErrorString(e));
        return LMS_ERR_CUDA;
    }
    return LMS_OK;
}

int max_row(const int32_t* rp, int64_t n) {
    int32_t m = 0;
    for (int64_t v = 0; v < n; ++v) m = std::max(m, rp[v + 1] - rp[v]);
    return m;
}

// Move the mesh to storage order `perm_new` (new_to_old): CSR rows gathered from the original
// ones with ids mapped, triangles mapped, boundary bits, positions carried over.
int apply_layout(lms_mesh_s* h, const std::vector<int32_t>& perm_new) {
    const int32_t n = h->n;
    std::vector<int32_t> old_inv(n), rel(n), new_inv(n), rp(n + 1);
    for (int32_t k = 0; k < n; ++k) old_inv[h->perm[k]] = k;
    for (int32_t k = 0; k < n; ++k) {
        rel[k] = old_inv[perm_new[k]];
        new_inv[perm_new[k]] = k;
    }
    rp[0] = 0;
    for (int32_t k = 0; k < n; ++k) rp[k + 1] = rp[k] + (h->rp[perm_new[k] + 1] - h->rp[perm_new[k]]);
    cudaStream_t s = h->stream;
    LMS_CUDA(cudaMemcpyAsync(h->d_perm, perm_new.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    LMS_CUDA(cudaMemcpyAsync(h->d_tmp, new_inv.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    LMS_CUDA(cudaMemcpyAsync(h->d_rp, rp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s));
    LMS_TRY(check_launch(lms::launch_gather_rows(n, h->d_perm, h->d_rp0, h->d_ci0, h->d_rp, h->d_ci, h->d_tmp, s),
                         "gather_rows"));
    if (h->ntri > 0)
        LMS_TRY(check_launch(lms::launch_map_ids(3 * int64_t(h->ntri), h->d_tmp, h->d_tri0, h->d_tri, s), "map_ids"));
    LMS_TRY(check_launch(lms::launch_boundary_bits(n, h->d_perm, h->d_bnd0, h->d_bits, s), "boundary_bits"));
    // positions: swap <- cur[rel], then both ping-pong buffers <- swap
    LMS_CUDA(cudaMemcpyAsync(h->d_tmp, rel.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    LMS_TRY(check_launch(lms::launch_gather_xy(h->precision, n, h->d_tmp, h->d_xy[h->cur], h->d_xy_swap, s),
                         "gather_xy"));
    const size_t vb = (h->precision == LMS_FP64 ? 16 : 8) * size_t(n);
    LMS_CUDA(cudaMemcpyAsync(h->d_xy[0], h->d_xy_swap, vb, cudaMemcpyDeviceToDevice, s));
    LMS_CUDA(cudaMemcpyAsync(h->d_xy[1], h->d_xy_swap, vb, cudaMemcpyDeviceToDevice, s));
    h->cur = 0;
    // the host vectors above must outlive the asynchronous copies
    LMS_CUDA(cudaStreamSynchronize(s));
    h->perm = perm_new;
    h->rp_cur.swap(rp);
    h->graphs.clear();
    return LMS_OK;
}

// Tile tables of the current layout: tiles of `tile` vertices over [0, n) (Jacobi), then, in the
// coloured layout, tiles over each colour's range (one coloured-GS launch per colour).
// Packed rows of the current layout for the FP32 work-queue Jacobi sweep (k_sweep_packed_mesh): the rows copied,
// farthest neighbour first, into the id-pair array padded to even length; one word per vertex with the
// row's first pair relative to its block of 4,096 positions, its neighbour count and its boundary flag.
// Leaves pk_ok false (the older row-offset kernel runs) when a row has more than kMaxPackedDegree entries.
int build_packed_mesh(lms_mesh_s* h) {
    h->pk_ok = false;
    if (h->precision != LMS_FP32) return LMS_OK;
    const int32_t n = h->n;
    const int32_t nb = (n + (1 << lms::kPackedBlockShift) - 1) >> lms::kPackedBlockShift;
    std::vector<int32_t> ps(size_t(n) + 1, 0), rw(n), bb(nb);
    for (int32_t v = 0; v < n; ++v) {
        const int32_t d = h->rp_cur[v + 1] - h->rp_cur[v];
        if (d > lms::kMaxPackedDegree) return LMS_OK;
        ps[v + 1] = ps[v] + (h->bnd[h->perm[v]] ? 0 : (d + 1) / 2);
    }
    for (int32_t v = 0; v < n; ++v) {
        const int32_t d = h->rp_cur[v + 1] - h->rp_cur[v];
        rw[v] = (ps[v] - ps[(v >> lms::kPackedBlockShift) << lms::kPackedBlockShift]) | (d << lms::kPackedDegreeShift) |
                (h->bnd[h->perm[v]] ? int32_t(0x80000000u) : 0);
    }
    for (int32_t b = 0; b < nb; ++b) bb[b] = ps[size_t(b) << lms::kPackedBlockShift];
    const int64_t P = ps[n];
    if (!h->d_pk_rw) {
        LMS_TRY(h->arena.get(&h->d_pk_rw, std::max(1, n)));
        LMS_TRY(h->arena.get(&h->d_pk_bbase, std::max(1, nb)));
    }
    if (P + 1 > h->pk_pairs_cap) {  // every layout of these rows needs at most (nnz + n) / 2 pairs
        const int64_t cap = std::max<int64_t>(P + 1, (int64_t(h->nnz) + n) / 2 + 1);
        LMS_TRY(h->arena.get(&h->d_pk_pairs, size_t(cap)));
        h->pk_pairs_cap = cap;
    }
    Arena tmp;
    tmp.al = h->arena.al;
    tmp.stream = h->stream;
    int32_t *d_ps = nullptr, *d_ci = nullptr;
    int rc = tmp.get(&d_ps, size_t(n) + 1);
    if (!rc) rc = tmp.get(&d_ci, size_t(std::max(1, h->nnz)));
    if (rc) {
        tmp.release_all();
        return rc;
    }
    cudaError_t e = cudaMemcpyAsync(d_ps, ps.data(), sizeof(int32_t) * (size_t(n) + 1), cudaMemcpyHostToDevice, h->stream);
    if (!e) e = cudaMemcpyAsync(d_ci, h->d_ci, sizeof(int32_t) * size_t(h->nnz), cudaMemcpyDeviceToDevice, h->stream);
    if (!e) e = lms::launch_sort_rows_far_first(n, h->d_rp, d_ci, h->stream);
    if (!e) e = lms::launch_pad_rows(n, h->d_rp, d_ci, d_ps, reinterpret_cast<int32_t*>(h->d_pk_pairs), h->stream);
    if (!e) e = cudaMemcpyAsync(h->d_pk_rw, rw.data(), sizeof(int32_t) * size_t(n), cudaMemcpyHostToDevice, h->stream);
    if (!e) e = cudaMemcpyAsync(h->d_pk_bbase, bb.data(), sizeof(int32_t) * size_t(nb), cudaMemcpyHostToDevice, h->stream);
    if (!e) e = cudaStreamSynchronize(h->stream);
    tmp.release_all();
    if (e) {
        lms::set_error_detail(std::string("packed rows: ") + cudaGetErrorString(e));
        return LMS_ERR_CUDA;
    }
    h->pk_ok = true;
    return LMS_OK;
}

int build_items(lms_mesh_s* h) {
    std::vector<int4> items;
    int32_t e_cap = 0;
    auto add = [&](int32_t lo, int32_t hi) {
        for (int32_t v = lo; v < hi; v += h->tile) {
            const int32_t vb = std::min(hi, v + h->tile);
            items.push_back(make_int4(v, vb, h->rp_cur[v], h->rp_cur[vb]));
            e_cap = std::max(e_cap, h->rp_cur[vb] - h->rp_cur[v]);
        }
    };
    add(0, h->n);
    h->n_items_all = int32_t(items.size());
    h->item_col_ofs.assign(1, 0);
    const int32_t nranges = h->gs_layout == kLayoutOrdering ? 0 : int32_t(h->range_ofs.size()) - 1;
    for (int32_t r = 0; r < nranges; ++r) {
        add(h->range_ofs[r], h->range_ofs[r + 1]);
        h->item_col_ofs.push_back(int32_t(items.size()) - h->n_items_all);
    }
    if (int64_t(items.size()) > h->items_cap) {
        const int64_t cap = int64_t(items.size()) + 64;
        LMS_TRY(h->arena.get(&h->d_items4, cap));
        h->items_cap = cap;
    }
    LMS_CUDA(cudaMemcpyAsync(h->d_items4, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice,
                             h->stream));
    // FP32 work queue: tiles and row offsets carrying the boundary flag.  Jacobi tiles: the largest of
    // 512, 256, 128 vertices that still gives every resident CTA of the queue kernel four tiles (a mesh of
    // ~1M vertices is latency-bound and sweeps 28% faster in 128-vertex tiles; from ~5M vertices up the
    // larger tiles win by a few per cent).  A colour range holds a seventh of the mesh or so, so its tiles
    // are 128 vertices (one 128-thread round each; 5-28% faster colour passes than 512).
    const int64_t resident = int64_t(std::max(1, lms::batch_sweep_occupancy(128, 4))) * std::max(1, h->sms);
    int32_t kQueueTile = 512;
    while (kQueueTile > 128 && (int64_t(h->n) + kQueueTile - 1) / kQueueTile < 4 * resident) kQueueTile >>= 1;
    constexpr int32_t kColourTile = 128;
    std::vector<int2> items2;
    for (int32_t v = 0; v < h->n; v += kQueueTile) items2.push_back(make_int2(v, std::min(h->n, v + kQueueTile)));
    const int32_t n_all2 = int32_t(items2.size());
    h->item2_col_ofs.assign(1, 0);
    for (int32_t r = 0; r < nranges; ++r) {
        for (int32_t v = h->range_ofs[r]; v < h->range_ofs[r + 1]; v += kColourTile)
            items2.push_back(make_int2(v, std::min(h->range_ofs[r + 1], v + kColourTile)));
        h->item2_col_ofs.push_back(int32_t(items2.size()) - n_all2);
    }
    if (int64_t(items2.size()) > h->items2_cap) {
        const int64_t cap = int64_t(items2.size()) + 16;
        LMS_TRY(h->arena.get(&h->d_items2, cap));
        h->items2_cap = cap;
    }
    LMS_CUDA(cudaMemcpyAsync(h->d_items2, items2.data(), sizeof(int2) * items2.size(), cudaMemcpyHostToDevice,
                             h->stream));
    h->n_items2 = n_all2;
    LMS_CUDA(cudaMemcpyAsync(h->d_rpf, h->d_rp, sizeof(int32_t) * size_t(h->n + 1), cudaMemcpyDeviceToDevice,
                             h->stream));
    LMS_TRY(check_launch(lms::launch_flag_boundary_rows(h->n, h->d_bits, h->d_rpf, h->stream), "flag_rows"));
    // FP64 one-thread-per-vertex sweeps: inside windows of kOrderWindow storage positions (never crossing
    // a range of an in-place layout), threads take the interior vertices by decreasing degree, then the boundary ones, so
    // the lanes of a warp run rows of one length (the FP64 pipe issues a warp's add for every lane, idle
    // or not).  Each vertex's arithmetic is unchanged, so results are too.
    std::vector<int32_t> order;
    if (h->precision == LMS_FP64) {
        constexpr int32_t kOrderWindow = 1024;
        order.resize(h->n);
        std::vector<int32_t> cuts{0, h->n};
        if (nranges > 0) cuts.insert(cuts.end() - 1, h->range_ofs.begin() + 1, h->range_ofs.end());
        std::sort(cuts.begin(), cuts.end());
        cuts.erase(std::unique(cuts.begin(), cuts.end()), cuts.end());
        std::vector<int32_t> count;
        for (size_t c = 0; c + 1 < cuts.size(); ++c)
            for (int32_t w0 = cuts[c]; w0 < cuts[c + 1]; w0 += kOrderWindow) {
                const int32_t w1 = std::min(cuts[c + 1], w0 + kOrderWindow);
                int32_t maxd = 0;
                for (int32_t k = w0; k < w1; ++k) maxd = std::max(maxd, h->rp_cur[k + 1] - h->rp_cur[k]);
                // bucket = maxd - degree for interior vertices (largest first), maxd + 1 for boundary ones
                count.assign(maxd + 3, 0);
                auto bucket = [&](int32_t k) {
                    return h->bnd[h->perm[k]] ? maxd + 1 : maxd - (h->rp_cur[k + 1] - h->rp_cur[k]);
                };
                for (int32_t k = w0; k < w1; ++k) ++count[bucket(k) + 1];
                for (int32_t b = 0; b + 1 < int32_t(count.size()); ++b) count[b + 1] += count[b];
                for (int32_t k = w0; k < w1; ++k) order[w0 + count[bucket(k)]++] = k;
            }
        LMS_CUDA(cudaMemcpyAsync(h->d_order, order.data(), sizeof(int32_t) * size_t(h->n), cudaMemcpyHostToDevice,
                                 h->stream));
    }
    LMS_CUDA(cudaStreamSynchronize(h->stream));
    h->e_cap = e_cap;
    h->graphs.clear();
    return build_packed_mesh(h);
}

int ensure_queue(lms_mesh_s* h, int32_t slots) {
    if (slots <= h->queue_slots) return LMS_OK;
    const int32_t want = std::max<int32_t>(slots, 256);
    LMS_TRY(h->arena.get(&h->d_queue, want));
    h->queue_slots = want;
    return LMS_OK;
}

// The block Gauss-Seidel on the block-range layout (tiles of kBlockRangeTile positions or more).
int32_t block_tile_for(const lms_mesh_s* h);
bool block_range_form(const lms_mesh_s* h) { return block_tile_for(h) >= kBlockRangeTile; }

// Work-queue counters one sweep uses: one per launch.
int queue_slots_per_sweep(lms_mesh_s* h, int mode) {
    if (mode == LMS_BLOCK_GS && !block_range_form(h)) return std::max<int>(1, int(h->block_tc_ofs.size()) - 1);
    if (mode == LMS_COLORED_GS || mode == LMS_BLOCK_GS) return std::max<int>(1, int(h->range_ofs.size()) - 1);
    return 1;
}

// FP32 Jacobi and coloured GS with the direct kernel run on the work-queue sweep (rows in chunks of 4).
bool uses_queue_sweep(const lms_mesh_s* h, int mode) {
    return h->kernel == LMS_KERNEL_DIRECT && h->precision == LMS_FP32 && (mode == LMS_JACOBI || mode == LMS_COLORED_GS);
}

// Current positions as FP64 in the original labelling, in d_xy64.
int positions_fp64_original(lms_mesh_s* h) {
    if (h->precision == LMS_FP32 && h->pristine_valid) {
        LMS_CUDA(cudaMemcpyAsync(h->d_xy64, h->d_pristine, 16 * size_t(h->n), cudaMemcpyDeviceToDevice, h->stream));
        return LMS_OK;
    }
    return check_launch(lms::launch_store_xy(h->precision, h->n, h->d_perm, h->d_xy[h->cur], h->d_xy64, h->cx,
                                             h->cy, h->scale, h->d_bnd0, h->d_pristine, h->stream),
                        "store_xy");
}

int ensure_colours(lms_mesh_s* h) {
    if (h->colours_valid) return LMS_OK;
    h->colour.assign(h->n, -1);
    LMS_TRY(lms::colour_vertices(h->n, h->rp.data(), h->ci.data(), h->bnd.data(), h->user_perm.data(),
                                 h->colour.data(), &h->ncolours));
    h->colours_valid = true;
    return LMS_OK;
}

// Tile of the block Gauss-Seidel: the requested one, else about eight tiles per SM, at most 1,024
// positions (on the 18.4M-vertex mesh in the BFS order larger tiles were slower: 0.66 / 0.75 / 0.80 ms
// per FP32 sweep at 1,024 / 2,048 / 4,096; RDR 3.48 ms at 1,024).  From kBlockRangeTile up the sweep
// runs on the block-range layout (RDR, FP32: 0.99 / 0.66 / 0.54 / 0.46 ms per sweep at 2^20 / 2^21 /
// 2^22 / 2^23 positions; coloured GS 0.39).
int32_t block_tile_for(const lms_mesh_s* h) {
    if (h->block_tile_req > 0) return h->block_tile_req;
    const int64_t want = int64_t(h->n) / (int64_t(h->sms) * 8);
    return int32_t(std::min<int64_t>(1024, std::max<int64_t>(128, want)));
}

// LMS_BLOCK_GS tables for the current ordering (lms::block_tables), uploaded.
int ensure_block_tables(lms_mesh_s* h) {
    const int32_t tile = block_tile_for(h);
    if (h->block_valid && h->block_tile == tile) return LMS_OK;
    lms::BlockTables bt;
    LMS_TRY(lms::block_tables(h->n, h->rp.data(), h->ci.data(), h->bnd.data(), h->user_perm.data(), tile, bt));
    if (bt.verts.empty()) bt.verts.assign(1, 0);
    if (bt.groups.empty()) bt.groups.assign(size_t(bt.ncolours) + 1, 0);
    if (int64_t(bt.verts.size()) > h->blk_verts_cap) {
        LMS_TRY(h->arena.get(&h->d_blk_verts, bt.verts.size()));
        h->blk_verts_cap = int64_t(bt.verts.size());
    }
    if (int64_t(bt.groups.size()) > h->blk_groups_cap) {
        LMS_TRY(h->arena.get(&h->d_blk_groups, bt.groups.size()));
        h->blk_groups_cap = int64_t(bt.groups.size());
    }
    LMS_CUDA(cudaMemcpyAsync(h->d_blk_verts, bt.verts.data(), sizeof(int32_t) * bt.verts.size(),
                             cudaMemcpyHostToDevice, h->stream));
    LMS_CUDA(cudaMemcpyAsync(h->d_blk_groups, bt.groups.data(), sizeof(int32_t) * bt.groups.size(),
                             cudaMemcpyHostToDevice, h->stream));
    // shared-memory tables of the staged kernel, when a tile with its halo fits in a CTA's shared memory
    h->st_valid = false;
    lms::BlockStageTables st;
    int dev = 0, smem_max = 0;
    if (h->block_staged && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
        lms::block_stage_tables(h->n, h->rp.data(), h->ci.data(), h->user_perm.data(), tile, bt, st) == LMS_OK &&
        lms::block_gs_staged_smem(h->precision, st.max_slots, st.max_verts, st.max_entries) + 2048 <= size_t(smem_max)) {
        if (st.tile_info.empty()) st.tile_info.assign(4, 0);
        if (st.halo.empty()) st.halo.assign(1, 0);
        if (st.lcol.empty()) st.lcol.assign(1, 0);
        const int64_t ntile = int64_t(st.tile_info.size() / 4);
        if (ntile > h->st_tile_cap) {
            LMS_TRY(h->arena.get(&h->d_st_tile, size_t(ntile)));
            h->st_tile_cap = ntile;
        }
        if (int64_t(st.halo.size()) > h->st_halo_cap) {
            LMS_TRY(h->arena.get(&h->d_st_halo, st.halo.size()));
            h->st_halo_cap = int64_t(st.halo.size());
        }
        if (int64_t(st.lrow.size()) > h->st_lrow_cap) {
            LMS_TRY(h->arena.get(&h->d_st_lrow, st.lrow.size()));
            h->st_lrow_cap = int64_t(st.lrow.size());
        }
        if (int64_t(st.lcol.size()) > h->st_lcol_cap) {
            LMS_TRY(h->arena.get(&h->d_st_lcol, st.lcol.size()));
            h->st_lcol_cap = int64_t(st.lcol.size());
        }
        LMS_CUDA(cudaMemcpyAsync(h->d_st_tile, st.tile_info.data(), sizeof(int32_t) * st.tile_info.size(),
                                 cudaMemcpyHostToDevice, h->stream));
        LMS_CUDA(cudaMemcpyAsync(h->d_st_halo, st.halo.data(), sizeof(int32_t) * st.halo.size(), cudaMemcpyHostToDevice,
                                 h->stream));
        LMS_CUDA(cudaMemcpyAsync(h->d_st_lrow, st.lrow.data(), sizeof(int32_t) * st.lrow.size(), cudaMemcpyHostToDevice,
                                 h->stream));
        LMS_CUDA(cudaMemcpyAsync(h->d_st_lcol, st.lcol.data(), sizeof(uint16_t) * st.lcol.size(), cudaMemcpyHostToDevice,
                                 h->stream));
        h->st_max_slots = st.max_slots;
        h->st_max_verts = st.max_verts;
        h->st_max_entries = st.max_entries;
        h->st_valid = true;
    }
    LMS_CUDA(cudaStreamSynchronize(h->stream));  // the host tables die here
    h->block_tc_ofs = bt.tc_ofs;
    h->block_ncolours = bt.ncolours;
    h->block_tile = tile;
    h->block_valid = true;
    h->graphs.clear();  // captured sweeps hold the old tables' pointers and launch counts
    return LMS_OK;
}

// The ordering's own layout (after an in-place sweep moved the mesh to a range layout).
int ensure_ordering_layout(lms_mesh_s* h) {
    if (h->gs_layout == kLayoutOrdering) return LMS_OK;
    LMS_TRY(apply_layout(h, h->user_perm));
    h->gs_layout = kLayoutOrdering;
    h->range_ofs.clear();
    return build_items(h);
}

// Range layout: the interior vertices grouped by key[v] (0 .. nkeys - 1; stable in the ordering's
// position), one range per non-empty key in ascending key order, then the boundary vertices (key -1).
int apply_range_layout(lms_mesh_s* h, const std::vector<int32_t>& key_by_pos, int32_t nkeys, int kind) {
    const int32_t n = h->n;
    std::vector<int32_t> start(size_t(nkeys) + 1, 0);
    for (int32_t k = 0; k < n; ++k)
        if (key_by_pos[k] >= 0) ++start[key_by_pos[k] + 1];
    for (int32_t c = 0; c < nkeys; ++c) start[c + 1] += start[c];
    std::vector<int32_t> fill(start.begin(), start.end()), p(n);
    int32_t tail = start[nkeys];
    for (int32_t k = 0; k < n; ++k) {
        const int32_t c = key_by_pos[k];
        p[c >= 0 ? fill[c]++ : tail++] = h->user_perm[k];
    }
    h->range_ofs.assign(1, 0);
    for (int32_t c = 0; c < nkeys; ++c)
        if (start[c + 1] > start[c]) h->range_ofs.push_back(start[c + 1]);
    LMS_TRY(apply_layout(h, p));
    h->gs_layout = kind;
    return build_items(h);
}

int ensure_coloured_layout(lms_mesh_s* h) {
    if (h->gs_layout == kLayoutColoured) return LMS_OK;
    LMS_TRY(ensure_colours(h));
    std::vector<int32_t> key(h->n);
    for (int32_t k = 0; k < h->n; ++k) key[k] = h->colour[h->user_perm[k]];
    return apply_range_layout(h, key, h->ncolours, kLayoutColoured);
}

// Block-range layout of the block Gauss-Seidel with tile `tile`: interior vertices by (tile colour, vertex
// colour, ordering position).  Tiles of one tile colour share no edge between interior vertices and a
// colour's vertices inside a tile are independent, so sweeping the ranges one after another, each range
// in one step, is the in-place sweep in lms_block_order's (tile colour, tile, vertex colour, position)
// order.
int ensure_block_range_layout(lms_mesh_s* h, int32_t tile) {
    if (h->gs_layout == kLayoutBlockRanges && h->gs_layout_tile == tile) return LMS_OK;
    LMS_TRY(ensure_colours(h));
    const int32_t n = h->n;
    const int64_t ntiles = (int64_t(n) + tile - 1) / tile;
    std::vector<int32_t> tile_colour(static_cast<size_t>(ntiles)), order(n), key(n);
    int32_t ntc = 0, n_order = 0;
    LMS_TRY(lms::block_order(n, h->rp.data(), h->ci.data(), h->bnd.data(), h->user_perm.data(), tile,
                             tile_colour.data(), &ntc, order.data(), &n_order));
    for (int32_t k = 0; k < n; ++k) {
        const int32_t c = h->colour[h->user_perm[k]];
        key[k] = c < 0 ? -1 : tile_colour[k / tile] * h->ncolours + c;
    }
    LMS_TRY(apply_range_layout(h, key, ntc * h->ncolours, kLayoutBlockRanges));
    h->gs_layout_tile = tile;
    return LMS_OK;
}

SweepArgs sweep_args(lms_mesh_s* h, int src, int dst) {
    SweepArgs a{};
    a.row_ptr = h->d_rp;
    a.col_idx = h->d_ci;
    a.bnd_bits = h->d_bits;
    a.src = h->d_xy[src];
    a.dst = h->d_xy[dst];
    a.v_begin = 0;
    a.v_end = h->n;
    a.n_vertices = h->n;
    a.recip = h->d_recip;
    return a;
}

// One sweep issued on stream s.  k1 = 1-based sweep index (selects the displacement slot);
// base = buffer holding sweep 0.  Jacobi: reads buf[(base + k1 - 1) & 1], writes the other.
int issue_sweep(lms_mesh_s* h, int mode, int base, int k1, bool disp, bool stoppable, cudaStream_t s) {
    const int src = (base + k1 - 1) & 1;
    // on the block-range layout the block Gauss-Seidel sweeps its ranges exactly as coloured GS does
    if (mode == LMS_BLOCK_GS && h->gs_layout == kLayoutBlockRanges) mode = LMS_COLORED_GS;
    const int32_t nranges = h->gs_layout == kLayoutOrdering ? 0 : int32_t(h->range_ofs.size()) - 1;
    if (mode == LMS_BLOCK_GS && h->block_staged && h->st_valid) {  // one launch per tile colour, staged
        lms::BlockGsStagedArgs a{};
        a.xy = h->d_xy[base];
        a.tile_info = h->d_st_tile;
        a.halo = h->d_st_halo;
        a.verts = h->d_blk_verts;
        a.lrow = h->d_st_lrow;
        a.lcol = h->d_st_lcol;
        a.group_ofs = h->d_blk_groups;
        a.ncolours = h->block_ncolours;
        a.max_slots = h->st_max_slots;
        a.max_verts = h->st_max_verts;
        a.max_entries = h->st_max_entries;
        a.state = stoppable ? h->d_state : nullptr;
        a.disp2 = disp ? &h->d_state->disp2[k1 & 1] : nullptr;
        a.recip = h->d_recip;
        for (size_t c = 0; c + 1 < h->block_tc_ofs.size(); ++c) {
            a.tile_begin = h->block_tc_ofs[c];
            LMS_TRY(check_launch(
                lms::launch_block_gs_staged(h->precision, a, h->block_tc_ofs[c + 1] - h->block_tc_ofs[c], s),
                "block_gs_staged"));
        }
        return LMS_OK;
    }
    if (mode == LMS_BLOCK_GS) {  // one launch per tile colour, in place
        lms::BlockGsArgs a{};
        a.row_ptr = h->d_rp;
        a.col_idx = h->d_ci;
        a.xy = h->d_xy[base];
        a.verts = h->d_blk_verts;
        a.group_ofs = h->d_blk_groups;
        a.ncolours = h->block_ncolours;
        a.n_vertices = h->n;
        a.state = stoppable ? h->d_state : nullptr;
        a.disp2 = disp ? &h->d_state->disp2[k1 & 1] : nullptr;
        a.recip = h->d_recip;
        for (size_t c = 0; c + 1 < h->block_tc_ofs.size(); ++c) {
            a.tile_begin = h->block_tc_ofs[c];
            LMS_TRY(check_launch(lms::launch_block_gs(h->precision, a, h->block_tc_ofs[c + 1] - h->block_tc_ofs[c], s),
                                 "block_gs"));
        }
        return LMS_OK;
    }
    if (mode == LMS_INPLACE_STATIC) {
        SweepArgs a = sweep_args(h, base, base);
        a.state = stoppable ? h->d_state : nullptr;
        a.disp2 = disp ? &h->d_state->disp2[k1 & 1] : nullptr;
        const int32_t threads = h->inplace_threads > 0 ? h->inplace_threads : std::min(h->n, h->sms * 2048);
        return check_launch(lms::launch_inplace_static(h->precision, a, threads, s), "inplace_static");
    }
    if (h->kernel == LMS_KERNEL_STAGED) {
        lms::StagedArgs a{};
        a.row_ptr = h->d_rp;
        a.col_idx = h->d_ci;
        a.recip = h->d_recip;
        a.err = h->d_err;
        a.tile_cap = h->tile;
        a.e_cap = h->e_cap;
        a.n_vertices = h->n;
        a.state = stoppable ? h->d_state : nullptr;
        a.disp2 = disp ? &h->d_state->disp2[k1 & 1] : nullptr;
        const int occ = std::max(1, lms::staged_occupancy(h->precision, mode != LMS_JACOBI, h->block, h->tile, h->e_cap));
        const int ranges = mode == LMS_JACOBI ? 1 : nranges;
        for (int32_t c = 0; c < ranges; ++c) {
            if (mode == LMS_JACOBI) {
                a.bnd_bits = h->d_bits;
                a.src = h->d_xy[src];
                a.dst = h->d_xy[src ^ 1];
                a.items = h->d_items4;
                a.n_items = h->n_items_all;
            } else {
                a.bnd_bits = nullptr;  // every vertex of a range is interior
                a.src = h->d_xy[base];
                a.dst = h->d_xy[base];
                a.items = h->d_items4 + h->n_items_all + h->item_col_ofs[c];
                a.n_items = h->item_col_ofs[c + 1] - h->item_col_ofs[c];
            }
            if (h->slot_next >= h->queue_slots) return LMS_ERR_STATE;
            a.queue = h->d_queue + h->slot_next++;
            const int grid = std::max(1, std::min(occ * h->sms, a.n_items));
            LMS_TRY(check_launch(lms::launch_sweep_staged(h->precision, mode != LMS_JACOBI, a, grid, h->block, s),
                                 "staged_sweep"));
        }
        return LMS_OK;
    }
    if (uses_queue_sweep(h, mode) && mode == LMS_JACOBI && h->pk_ok) {
        // packed rows, one launch over all tiles.  Coloured GS keeps the row-offset kernel below: over the
        // 4096 x 4096 mesh in the RDR ordering its colour passes ran 1% slower on packed rows, while Jacobi
        // ran 9% faster.
        constexpr int kBlock = 128;
        lms::PackedMeshArgs a{};
        a.row_words = h->d_pk_rw;
        a.block_pbase = h->d_pk_bbase;
        a.id_pairs = h->d_pk_pairs;
        a.src = h->d_xy[src];
        a.dst = h->d_xy[src ^ 1];
        a.items = h->d_items2;
        a.n_items = h->n_items2;
        if (h->slot_next >= h->queue_slots) return LMS_ERR_STATE;
        a.queue = h->d_queue + h->slot_next++;
        a.n_vertices = h->n;
        a.state = stoppable ? h->d_state : nullptr;
        a.disp2 = disp ? &h->d_state->disp2[k1 & 1] : nullptr;
        const int occ = std::max(1, lms::sweep_packed_mesh_occupancy(kBlock));
        const int grid = std::max(1, std::min(occ * h->sms, a.n_items));
        return check_launch(lms::launch_sweep_packed_mesh(a, kBlock, grid, s), "packed_sweep");
    }
    if (uses_queue_sweep(h, mode)) {
        constexpr int kChunk = 4, kBlock = 128;
        const int occ = std::max(1, lms::batch_sweep_occupancy(kBlock, kChunk));
        // Jacobi: one launch over [0, n) from one buffer into the other.  In-place sweeps: one launch per
        // range, in place - a range's vertices are never neighbours of one another, so no launch reads a
        // position it writes.
        const int ranges = mode == LMS_JACOBI ? 1 : nranges;
        for (int32_t c = 0; c < ranges; ++c) {
            SweepArgs a = mode == LMS_JACOBI ? sweep_args(h, src, src ^ 1) : sweep_args(h, base, base);
            a.row_ptr = h->d_rpf;
            if (mode == LMS_JACOBI) {
                a.items = h->d_items2;
                a.n_items = h->n_items2;
            } else {
                a.items = h->d_items2 + h->n_items2 + h->item2_col_ofs[c];
                a.n_items = h->item2_col_ofs[c + 1] - h->item2_col_ofs[c];
            }
            if (h->slot_next >= h->queue_slots) return LMS_ERR_STATE;
            a.queue = h->d_queue + h->slot_next++;
            a.state = stoppable ? h->d_state : nullptr;
            a.disp2 = disp ? &h->d_state->disp2[k1 & 1] : nullptr;
            const int grid = std::max(1, std::min(occ * h->sms, a.n_items));
            LMS_TRY(check_launch(lms::launch_batch_sweep(a, kBlock, kChunk, grid, s), "queue_sweep"));
        }
        return LMS_OK;
    }
    if (mode == LMS_JACOBI) {
        SweepArgs a = sweep_args(h, src, src ^ 1);
        a.state = stoppable ? h->d_state : nullptr;
        a.disp2 = disp ? &h->d_state->disp2[k1 & 1] : nullptr;
        a.order = h->precision == LMS_FP64 ? h->d_order : nullptr;
        return check_launch(lms::launch_sweep(h->precision, false, a, h->block, h->fp64_arith, s), "sweep");
    }
    for (int32_t c = 0; c < nranges; ++c) {
        SweepArgs a = sweep_args(h, base, base);
        a.order = h->precision == LMS_FP64 ? h->d_order : nullptr;
        a.bnd_bits = nullptr;  // every vertex of a range is interior
        a.v_begin = h->range_ofs[c];
        a.v_end = h->range_ofs[c + 1];
        a.state = stoppable ? h->d_state : nullptr;
        a.disp2 = disp ? &h->d_state->disp2[k1 & 1] : nullptr;
        LMS_TRY(check_launch(lms::launch_sweep(h->precision, true, a, h->block, h->fp64_arith, s), "sweep"));
    }
    return LMS_OK;
}

int get_graph(lms_mesh_s* h, const std::string& key, const std::function<int(cudaStream_t)>& body,
              cudaGraphExec_t* exec, int64_t* kernels) {
    auto it = h->graphs.execs.find(key);
    if (it != h->graphs.execs.end()) {
        *exec = it->second;
        *kernels = h->graphs.kernels[key];
        return LMS_OK;
    }
    LMS_TRY(capture(h->cap, body, exec, kernels));
    h->graphs.execs[key] = *exec;
    h->graphs.kernels[key] = *kernels;
    return LMS_OK;
}

int finish_stats(lms_mesh_s* h) {
    if (!h->stats_pending) return LMS_OK;
    LMS_CUDA(cudaStreamSynchronize(h->stream));
    DevState st;
    LMS_CUDA(cudaMemcpy(&st, h->d_state, sizeof(DevState), cudaMemcpyDeviceToHost));
    double d2 = 0.0;
    std::memcpy(&d2, &st.disp2[h->last_disp_slot], sizeof(double));
    h->last_disp = std::sqrt(d2) * (h->precision == LMS_FP32 ? h->scale : 1.0);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess) h->last_ms = ms;
    int32_t kerr = 0;
    LMS_CUDA(cudaMemcpy(&kerr, h->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
    h->stats_pending = false;
    if (st.err != 0 || kerr != 0) {
        lms::set_error_detail("a bounded wait on a tile copy expired");
        return LMS_ERR_TIMEOUT;
    }
    return LMS_OK;
}

}  // namespace

// ---------------------------------------------------------------- C ABI

extern "C" {

int lms_set_device_allocator(void* (*alloc)(size_t, void*, void*), void (*release)(void*, void*), void* ctx) {
    if ((alloc == nullptr) != (release == nullptr)) return LMS_ERR_ARG;
    std::lock_guard<std::mutex> g(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.release = release;
    g_alloc.ctx = ctx;
    return LMS_OK;
}

int lms_create(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* xy,
               const uint8_t* is_boundary, int32_t ntri, const int32_t* tri, int precision, void* cuda_stream,
               lms_handle* out) {
    if (!out || !xy || (precision != LMS_FP64 && precision != LMS_FP32)) return LMS_ERR_ARG;
    *out = nullptr;
    LMS_TRY(lms::validate_mesh(n, row_ptr, col_idx, is_boundary, ntri, tri));
    if (!all_finite(xy, 2 * int64_t(n))) return LMS_ERR_ARG;

    auto h = new (std::nothrow) lms_mesh_s();
    if (!h) return LMS_ERR_OOM;
    auto fail = [&](int rc) {
        delete h;
        return rc;
    };
    {
        std::lock_guard<std::mutex> g(g_alloc_mu);
        h->arena.al = g_alloc;
    }
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->arena.stream = h->stream;
    h->precision = precision;
    h->n = n;
    h->ntri = ntri;
    h->nnz = row_ptr[n];
    h->rp.assign(row_ptr, row_ptr + n + 1);
    h->ci.assign(col_idx, col_idx + h->nnz);
    h->bnd.assign(is_boundary, is_boundary + n);
    for (auto& b : h->bnd) b = b ? 1 : 0;
    if (ntri > 0) h->tri.assign(tri, tri + 3 * int64_t(ntri));
    h->user_perm.resize(n);
    for (int32_t i = 0; i < n; ++i) h->user_perm[i] = i;
    h->perm = h->user_perm;
    bbox(xy, n, &h->cx, &h->cy, &h->scale);

    std::vector<int32_t> vt_ptr, vt_idx;
    std::vector<double> w;
    build_incidence(n, ntri, h->tri.data(), vt_ptr, vt_idx);
    build_weights(ntri, h->tri.data(), vt_ptr, w);

    cudaError_t e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        lms::set_error_detail(std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
        return fail(LMS_ERR_CUDA);
    }
    if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&h->h_state), sizeof(DevState)) != cudaSuccess)
        return fail(LMS_ERR_CUDA);

    Arena& A = h->arena;
    const size_t vb = (precision == LMS_FP64 ? 16 : 8) * size_t(n);
    const int64_t t3 = std::max<int64_t>(1, 3 * int64_t(ntri));
    int rc = LMS_OK;
    if ((rc = A.get(&h->d_rp0, n + 1)) || (rc = A.get(&h->d_ci0, std::max(1, h->nnz))) ||
        (rc = A.get(&h->d_tri0, t3)) || (rc = A.get(&h->d_vt_ptr, n + 1)) || (rc = A.get(&h->d_vt_idx, t3)) ||
        (rc = A.get(&h->d_bnd0, n)) || (rc = A.get(&h->d_w, std::max(1, ntri))) || (rc = A.get(&h->d_rp, n + 1 + 8)) || (rc = A.get(&h->d_rpf, n + 1 + 8)) ||
        (rc = A.get(&h->d_ci, h->nnz + 8)) || (rc = A.get(&h->d_order, precision == LMS_FP64 ? n : 1)) ||
        (rc = A.get(&h->d_tri, t3)) || (rc = A.get(&h->d_perm, n)) ||
        (rc = A.get(&h->d_tmp, n)) || (rc = A.get(&h->d_bits, (n + 31) / 32 + 8)) || (rc = A.get(&h->d_err, 1)) ||
        (rc = A.get(&h->d_xy[0], vb)) || (rc = A.get(&h->d_xy[1], vb)) || (rc = A.get(&h->d_xy_swap, vb)) ||
        (rc = A.get(&h->d_xy64, 2 * size_t(n))) || (rc = A.get(&h->d_qt, std::max(1, ntri))) ||
        (rc = A.get(&h->d_qv, n)) || (rc = A.get(&h->d_partials, lms::kQualityBlocks)) ||
        (rc = A.get(&h->d_recip, lms::kRecipTableDoubles)) || (rc = A.get(&h->d_state, 1)))
        return fail(rc);
    if (precision == LMS_FP32 && (rc = A.get(&h->d_pristine, 2 * size_t(n)))) return fail(rc);

    cudaStream_t s = h->stream;
    auto recip = recip_table();
    std::vector<float> wf(w.begin(), w.end());  // FP32 handles: weights rounded to float
    std::vector<int32_t> ident(n);
    for (int32_t i = 0; i < n; ++i) ident[i] = i;
    auto up = [&](void* dst, const void* src, size_t bytes) {
        return bytes == 0 ? cudaSuccess : cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    };
    if (up(h->d_rp0, h->rp.data(), 4 * size_t(n + 1)) || up(h->d_ci0, h->ci.data(), 4 * size_t(h->nnz)) ||
        up(h->d_tri0, h->tri.data(), 12 * size_t(ntri)) || up(h->d_vt_ptr, vt_ptr.data(), 4 * size_t(n + 1)) ||
        up(h->d_vt_idx, vt_idx.data(), 12 * size_t(ntri)) || up(h->d_bnd0, h->bnd.data(), size_t(n)) ||
        up(h->d_w, precision == LMS_FP64 ? static_cast<const void*>(w.data()) : static_cast<const void*>(wf.data()),
           (precision == LMS_FP64 ? 8 : 4) * size_t(ntri)) ||
        up(h->d_recip, recip.data(), 8 * recip.size()) ||
        up(h->d_perm, ident.data(), 4 * size_t(n)) || up(h->d_rp, h->rp.data(), 4 * size_t(n + 1)) ||
        up(h->d_ci, h->ci.data(), 4 * size_t(h->nnz)) || up(h->d_tri, h->tri.data(), 12 * size_t(ntri)) ||
        up(h->d_xy64, xy, 16 * size_t(n)) || cudaMemsetAsync(h->d_state, 0, sizeof(DevState), s) ||
        cudaMemsetAsync(h->d_err, 0, sizeof(int32_t), s) || cudaMemsetAsync(h->d_bits, 0, 4 * size_t((n + 31) / 32 + 8), s) ||
        cudaMemsetAsync(h->d_rp + n + 1, 0, 4 * 8, s) || cudaMemsetAsync(h->d_ci + h->nnz, 0, 4 * 8, s)) {
        lms::set_error_detail(std::string("upload: ") + cudaGetErrorString(cudaGetLastError()));
        return fail(LMS_ERR_CUDA);
    }
    if ((rc = check_launch(lms::launch_boundary_bits(n, h->d_perm, h->d_bnd0, h->d_bits, s), "boundary_bits")))
        return fail(rc);
    const double inv_s = 1.0 / h->scale;
    for (int b = 0; b < 2; ++b)
        if ((rc = check_launch(lms::launch_load_xy(precision, n, h->d_perm, h->d_xy64, h->d_xy[b], h->cx, h->cy,
                                                   inv_s, s),
                               "load_xy")))
            return fail(rc);
    if (precision == LMS_FP32) {
        if (cudaMemcpyAsync(h->d_pristine, h->d_xy64, 16 * size_t(n), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return fail(LMS_ERR_CUDA);
        h->pristine_valid = true;
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        lms::set_error_detail(std::string("create: ") + cudaGetErrorString(e));
        return fail(LMS_ERR_CUDA);
    }
    {
        int dev = 0;
        cudaDeviceProp prop;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
            return fail(LMS_ERR_CUDA);
        h->sms = prop.multiProcessorCount;
    }
    if (precision == LMS_FP64) h->tile = 256;
    h->rp_cur = h->rp;
    if ((rc = build_items(h))) return fail(rc);
    *out = h;
    return LMS_OK;
}

int lms_reorder(lms_handle h, int ordering, uint64_t seed) {
    if (!h || ordering < LMS_ORI || ordering > LMS_BRDR) return LMS_ERR_ARG;
    if ((ordering == LMS_RDR || ordering == LMS_BRDR) && h->ntri == 0) return LMS_ERR_NO_TRIANGLES;
    LMS_TRY(finish_stats(h));
    LMS_CUDA(cudaStreamSynchronize(h->stream));  // earlier work does not count towards the ordering time
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<double> q;
    if (ordering == LMS_RDR || ordering == LMS_BRDR) {
        // keys: Section 3.2 vertex qualities of the current positions, FP64, original labels
        LMS_TRY(positions_fp64_original(h));
        LMS_TRY(check_launch(lms::launch_tri_quality_exact(h->ntri, h->d_tri0, h->d_xy64, h->d_qt, h->stream),
                             "tri_quality"));
        LMS_TRY(check_launch(
            lms::launch_vertex_quality_exact(h->n, h->d_vt_ptr, h->d_vt_idx, h->d_qt, h->d_qv, h->stream),
            "vertex_quality"));
        q.resize(h->n);
        LMS_CUDA(cudaMemcpyAsync(q.data(), h->d_qv, 8 * size_t(h->n), cudaMemcpyDeviceToHost, h->stream));
        LMS_CUDA(cudaStreamSynchronize(h->stream));
    }
    std::vector<int32_t> p(h->n);
    if (ordering == LMS_BFS || ordering == LMS_RBFS) {
        // level-synchronous search on the device, equal to the sequential one
        LMS_TRY(device_order(h->arena.al, h->stream, h->sms, h->d_rp0, h->d_ci0, h->n, 1, nullptr, nullptr, nullptr,
                             p.data()));
        if (ordering == LMS_RBFS) std::reverse(p.begin(), p.end());
    } else if (ordering == LMS_BRDR && max_row(h->rp.data(), h->n) <= lms::block_rdr_max_degree()) {
        // device BFS, then Algorithm 2 inside each block on the device, keys already in d_qv
        LMS_TRY(device_order(h->arena.al, h->stream, h->sms, h->d_rp0, h->d_ci0, h->n, 1, nullptr, h->d_qv, h->d_bnd0,
                             p.data()));
    } else {
        LMS_TRY(lms::order_vertices(h->n, h->rp.data(), h->ci.data(), h->bnd.data(), q.empty() ? nullptr : q.data(),
                                    ordering, seed, p.data()));
    }
    const auto t1 = std::chrono::steady_clock::now();
    h->user_perm = p;
    h->colours_valid = false;
    h->block_valid = false;
    h->gs_layout = kLayoutOrdering;
    h->range_ofs.clear();
    LMS_TRY(apply_layout(h, p));
    LMS_TRY(build_items(h));
    LMS_CUDA(cudaStreamSynchronize(h->stream));
    const auto t2 = std::chrono::steady_clock::now();
    h->reorder_ms[0] = std::chrono::duration<double, std::milli>(t1 - t0).count();
    h->reorder_ms[1] = std::chrono::duration<double, std::milli>(t2 - t1).count();
    return LMS_OK;
}

int lms_set_inplace_split(lms_handle h, int32_t threads) {
    if (!h || threads < 0) return LMS_ERR_ARG;
    LMS_TRY(finish_stats(h));
    h->inplace_threads = threads;
    h->graphs.clear();
    return LMS_OK;
}

int lms_last_reorder_ms(lms_handle h, double* ordering_ms, double* layout_ms) {
    if (!h) return LMS_ERR_ARG;
    if (ordering_ms) *ordering_ms = h->reorder_ms[0];
    if (layout_ms) *layout_ms = h->reorder_ms[1];
    return LMS_OK;
}

int lms_set_launch(lms_handle h, int32_t kernel, int32_t block, int32_t tile) {
    if (!h) return LMS_ERR_ARG;
    if (kernel == LMS_KERNEL_STAGED) {
        if ((block != 128 && block != 256) || tile < 32 || tile > 4096 || (tile % 32) != 0) return LMS_ERR_ARG;
    } else if (kernel == LMS_KERNEL_DIRECT) {
        if (block != 128 && block != 256) return LMS_ERR_ARG;
    } else {
        return LMS_ERR_ARG;
    }
    LMS_TRY(finish_stats(h));
    const int old_tile = h->tile;
    h->kernel = kernel;
    h->block = block;
    if (kernel == LMS_KERNEL_STAGED) h->tile = tile;
    if (h->tile != old_tile) LMS_TRY(build_items(h));
    if (kernel == LMS_KERNEL_STAGED &&
        lms::staged_occupancy(h->precision, false, h->block, h->tile, h->e_cap) <= 0) {
        lms::set_error_detail("tile does not fit in shared memory");
        return LMS_ERR_ARG;
    }
    h->graphs.clear();
    return LMS_OK;
}

int lms_set_block_tile(lms_handle h, int32_t tile) {
    if (!h || tile < 0) return LMS_ERR_ARG;
    LMS_TRY(finish_stats(h));
    if (tile != h->block_tile_req) {
        h->block_tile_req = tile;
        h->graphs.clear();
    }
    return LMS_OK;
}

int lms_set_block_staging(lms_handle h, int32_t on) {
    if (!h || (on != 0 && on != 1)) return LMS_ERR_ARG;
    if (h->block_staged != (on != 0)) {
        h->block_staged = on != 0;
        h->block_valid = false;  // the staged tables are built with the block tables when staging is on
        h->graphs.clear();
    }
    return LMS_OK;
}

int lms_get_block_tile(lms_handle h, int32_t* tile) {
    if (!h || !tile) return LMS_ERR_ARG;
    *tile = block_tile_for(h);
    return LMS_OK;
}

int lms_set_fp64_arith(lms_handle h, int32_t mode) {
    if (!h || mode < LMS_FP64_ARITH_FPU || mode > LMS_FP64_ARITH_MIXED3) return LMS_ERR_ARG;
    LMS_TRY(finish_stats(h));
    if (mode != h->fp64_arith) h->graphs.clear();
    h->fp64_arith = mode;
    return LMS_OK;
}

int lms_smooth(lms_handle h, int32_t max_iters, int mode, double tol, int32_t* iters_done) {
    if (!h || max_iters < 0 ||
        (mode != LMS_JACOBI && mode != LMS_COLORED_GS && mode != LMS_INPLACE_STATIC && mode != LMS_BLOCK_GS) ||
        std::isnan(tol))
        return LMS_ERR_ARG;
    if (tol >= 0.0 && h->ntri == 0) return LMS_ERR_NO_TRIANGLES;
    LMS_TRY(finish_stats(h));
    if (mode == LMS_COLORED_GS) LMS_TRY(ensure_coloured_layout(h));
    if (mode == LMS_BLOCK_GS && block_range_form(h)) {
        LMS_TRY(ensure_block_range_layout(h, block_tile_for(h)));
    } else if (mode == LMS_INPLACE_STATIC || mode == LMS_BLOCK_GS) {
        LMS_TRY(ensure_ordering_layout(h));
        if (mode == LMS_BLOCK_GS) LMS_TRY(ensure_block_tables(h));
    }
    if (iters_done) *iters_done = 0;
    h->q_first = h->q_last = NAN;
    h->last_disp = NAN;
    if (max_iters == 0) return LMS_OK;
    cudaStream_t s = h->stream;
    const int base = h->cur;
    const double nd = double(h->n);

    if (tol < 0.0) {
        std::string key = "fixed/" + std::to_string(mode) + "/" + std::to_string(max_iters) + "/" + std::to_string(base);
        key += "/" + std::to_string(h->kernel) + "/" + std::to_string(h->block) + "/" + std::to_string(h->tile);
        cudaGraphExec_t exec;
        int64_t kernels = 0;
        const int32_t slots = max_iters * queue_slots_per_sweep(h, mode);
        LMS_TRY(ensure_queue(h, slots));
        LMS_TRY(get_graph(h, key,
                          [&](cudaStream_t cs) -> int {
                              h->slot_next = 0;
                              LMS_CUDA(cudaMemsetAsync(h->d_state, 0, sizeof(DevState), cs));
                              LMS_CUDA(cudaMemsetAsync(h->d_queue, 0, sizeof(int32_t) * slots, cs));
                              for (int32_t k = 1; k <= max_iters; ++k)
                                  LMS_TRY(issue_sweep(h, mode, base, k, k == max_iters, false, cs));
                              return LMS_OK;
                          },
                          &exec, &kernels));
        LMS_CUDA(cudaEventRecord(h->ev0, s));
        LMS_CUDA(cudaGraphLaunch(exec, s));
        LMS_CUDA(cudaEventRecord(h->ev1, s));
        h->last_launches = kernels;
        h->last_disp_slot = max_iters & 1;
        h->stats_pending = true;
        if (mode == LMS_JACOBI) h->cur = (base + max_iters) & 1;
        h->pristine_valid = false;
        if (iters_done) *iters_done = max_iters;
        return LMS_OK;
    }

    // Algorithm 1 with the Section 5.1 rule: Q_0, then chunks of sweeps each followed by the
    // quality reduction and the stop check, replayed from one graph until the rule fires.
    constexpr int32_t kChunk = 8;
    DevState init{};
    *h->h_state = init;
    LMS_CUDA(cudaEventRecord(h->ev0, s));
    LMS_CUDA(cudaMemcpyAsync(h->d_state, h->h_state, sizeof(DevState), cudaMemcpyHostToDevice, s));
    LMS_TRY(check_launch(lms::launch_quality_partials(h->precision, h->ntri, h->d_tri, h->d_xy[base], h->d_w,
                                                      h->d_partials, nullptr, s),
                         "quality"));
    LMS_TRY(check_launch(lms::launch_quality_finish(h->d_partials, nd, h->d_state, 1, s), "quality_finish"));
    int64_t launches = 2;
    char tol_hex[64];
    std::snprintf(tol_hex, sizeof(tol_hex), "%a", tol);
    std::string key = "stop/" + std::to_string(mode) + "/" + std::to_string(base) + "/" + std::to_string(max_iters) +
                      "/" + tol_hex + "/" + std::to_string(h->kernel) + "/" + std::to_string(h->block) + "/" +
                      std::to_string(h->tile);
    cudaGraphExec_t exec;
    int64_t kernels = 0;
    const int32_t slots = kChunk * queue_slots_per_sweep(h, mode);
    LMS_TRY(ensure_queue(h, slots));
    LMS_TRY(get_graph(h, key,
                      [&](cudaStream_t cs) -> int {
                          h->slot_next = 0;
                          LMS_CUDA(cudaMemsetAsync(h->d_queue, 0, sizeof(int32_t) * slots, cs));
                          for (int32_t i = 0; i < kChunk; ++i) {
                              const int k1 = 1 + i;  // chunks start at odd sweep indices (kChunk is even)
                              LMS_TRY(issue_sweep(h, mode, base, k1, true, true, cs));
                              const void* xy = h->d_xy[mode == LMS_JACOBI ? ((base + k1) & 1) : base];
                              LMS_TRY(check_launch(lms::launch_quality_partials(h->precision, h->ntri, h->d_tri, xy,
                                                                                h->d_w, h->d_partials, h->d_state, cs),
                                                   "quality"));
                              LMS_TRY(check_launch(lms::launch_stop_check(h->d_partials, nd, h->d_state, tol,
                                                                          INFINITY, max_iters, cs),
                                                   "stop_check"));
                          }
                          return LMS_OK;
                      },
                      &exec, &kernels));
    int32_t done = 0;
    for (int32_t launched = 0; launched < max_iters; launched += kChunk) {
        LMS_CUDA(cudaGraphLaunch(exec, s));
        launches += kernels;
        LMS_CUDA(cudaMemcpyAsync(h->h_state, h->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, s));
        LMS_CUDA(cudaStreamSynchronize(s));
        if (h->h_state->stop) {
            done = h->h_state->iters_at_stop;
            break;
        }
    }
    LMS_CUDA(cudaEventRecord(h->ev1, s));
    LMS_CUDA(cudaStreamSynchronize(s));
    if (h->h_state->err) return LMS_ERR_TIMEOUT;
    if (!h->h_state->stop) {
        lms::set_error_detail("stopping rule did not terminate within max_iters");
        return LMS_ERR_STATE;
    }
    h->last_launches = launches;
    h->q_first = h->h_state->q_first;
    h->q_last = h->h_state->q_cur;
    h->last_disp_slot = done & 1;
    h->stats_pending = true;
    if (mode == LMS_JACOBI) h->cur = (base + done) & 1;
    h->pristine_valid = false;
    if (iters_done) *iters_done = done;
    return finish_stats(h);
}

int lms_quality(lms_handle h, double* Q) {
    if (!h || !Q) return LMS_ERR_ARG;
    if (h->ntri == 0) return LMS_ERR_NO_TRIANGLES;
    LMS_TRY(finish_stats(h));
    cudaStream_t s = h->stream;
    LMS_TRY(check_launch(lms::launch_quality_partials(h->precision, h->ntri, h->d_tri, h->d_xy[h->cur], h->d_w,
                                                      h->d_partials, nullptr, s),
                         "quality"));
    LMS_TRY(check_launch(lms::launch_quality_finish(h->d_partials, double(h->n), h->d_state, 0, s), "quality_finish"));
    LMS_CUDA(cudaMemcpyAsync(h->h_state, h->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    LMS_CUDA(cudaStreamSynchronize(s));
    *Q = h->h_state->q_cur;
    return LMS_OK;
}

int lms_get_coords(lms_handle h, double* xy) {
    if (!h || !xy) return LMS_ERR_ARG;
    LMS_TRY(finish_stats(h));
    LMS_TRY(positions_fp64_original(h));
    LMS_CUDA(cudaMemcpyAsync(xy, h->d_xy64, 16 * size_t(h->n), cudaMemcpyDeviceToHost, h->stream));
    LMS_CUDA(cudaStreamSynchronize(h->stream));
    return LMS_OK;
}

int lms_set_coords(lms_handle h, const double* xy) {
    if (!h || !xy) return LMS_ERR_ARG;
    if (!all_finite(xy, 2 * int64_t(h->n))) return LMS_ERR_ARG;
    LMS_TRY(finish_stats(h));
    cudaStream_t s = h->stream;
    LMS_CUDA(cudaMemcpyAsync(h->d_xy64, xy, 16 * size_t(h->n), cudaMemcpyHostToDevice, s));
    for (int b = 0; b < 2; ++b)
        LMS_TRY(check_launch(lms::launch_load_xy(h->precision, h->n, h->d_perm, h->d_xy64, h->d_xy[b], h->cx, h->cy,
                                                 1.0 / h->scale, s),
                             "load_xy"));
    if (h->precision == LMS_FP32) {
        LMS_CUDA(cudaMemcpyAsync(h->d_pristine, h->d_xy64, 16 * size_t(h->n), cudaMemcpyDeviceToDevice, s));
        h->pristine_valid = true;
    }
    h->cur = 0;
    return LMS_OK;
}

int lms_get_permutation(lms_handle h, int32_t* new_to_old) {
    if (!h || !new_to_old) return LMS_ERR_ARG;
    std::memcpy(new_to_old, h->user_perm.data(), sizeof(int32_t) * h->n);
    return LMS_OK;
}

int lms_get_colors(lms_handle h, int32_t* colour, int32_t* ncolours) {
    if (!h || !colour || !ncolours) return LMS_ERR_ARG;
    LMS_TRY(ensure_colours(h));
    std::memcpy(colour, h->colour.data(), sizeof(int32_t) * h->n);
    *ncolours = h->ncolours;
    return LMS_OK;
}

int lms_get_csr(lms_handle h, int32_t* row_ptr, int32_t* col_idx, int32_t* storage_new_to_old) {
    if (!h || !row_ptr || (!col_idx && h->nnz > 0)) return LMS_ERR_ARG;
    LMS_TRY(finish_stats(h));
    LMS_CUDA(cudaMemcpyAsync(row_ptr, h->d_rp, 4 * size_t(h->n + 1), cudaMemcpyDeviceToHost, h->stream));
    if (h->nnz > 0)
        LMS_CUDA(cudaMemcpyAsync(col_idx, h->d_ci, 4 * size_t(h->nnz), cudaMemcpyDeviceToHost, h->stream));
    LMS_CUDA(cudaStreamSynchronize(h->stream));
    if (storage_new_to_old) std::memcpy(storage_new_to_old, h->perm.data(), sizeof(int32_t) * h->n);
    return LMS_OK;
}

int lms_last_stats(lms_handle h, double* max_disp, double* ms, double* q_first, double* q_last) {
    if (!h) return LMS_ERR_ARG;
    LMS_TRY(finish_stats(h));
    if (max_disp) *max_disp = h->last_disp;
    if (ms) *ms = h->last_ms;
    if (q_first) *q_first = h->q_first;
    if (q_last) *q_last = h->q_last;
    return LMS_OK;
}

int lms_last_error_stats(lms_handle h, double* max_disp, double* ms) {
    return lms_last_stats(h, max_disp, ms, nullptr, nullptr);
}

int lms_last_launches(lms_handle h, int64_t* launches) {
    if (!h || !launches) return LMS_ERR_ARG;
    *launches = h->last_launches;
    return LMS_OK;
}

namespace {
int selftest_div(int32_t count, const double* s, const int32_t* d, double* q, bool integer) {
    if (count < 0 || (count > 0 && (!s || !d || !q))) return LMS_ERR_ARG;
    for (int32_t i = 0; i < count; ++i)
        if (d[i] < 1) return LMS_ERR_ARG;
    if (count == 0) return LMS_OK;
    Arena A;
    double *ds = nullptr, *dq = nullptr, *dr = nullptr;
    int32_t* dd = nullptr;
    int rc = LMS_OK;
    if ((rc = A.get(&ds, count)) || (rc = A.get(&dq, count)) || (rc = A.get(&dr, lms::kRecipTableDoubles)) ||
        (rc = A.get(&dd, count))) {
        A.release_all();
        return rc;
    }
    auto recip = recip_table();
    cudaError_t e = cudaMemcpy(ds, s, 8 * size_t(count), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dd, d, 4 * size_t(count), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dr, recip.data(), 8 * recip.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = integer ? lms::launch_divint_selftest(count, ds, dd, dr, dq, nullptr)
                    : lms::launch_div_selftest(count, ds, dd, dr, dq, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(q, dq, 8 * size_t(count), cudaMemcpyDeviceToHost);
    A.release_all();
    if (e != cudaSuccess) {
        lms::set_error_detail(std::string("selftest: ") + cudaGetErrorString(e));
        return LMS_ERR_CUDA;
    }
    return LMS_OK;
}
}  // namespace

int lms_selftest_div64(int32_t count, const double* s, const int32_t* d, double* q) {
    return selftest_div(count, s, d, q, false);
}

int lms_selftest_div32(int32_t count, const float* s, const int32_t* d, float* q) {
    if (count < 0 || (count > 0 && (!s || !d || !q))) return LMS_ERR_ARG;
    for (int32_t i = 0; i < count; ++i)
        if (d[i] < 1) return LMS_ERR_ARG;
    if (count == 0) return LMS_OK;
    Arena A;
    float *ds = nullptr, *dq = nullptr;
    int32_t* dd = nullptr;
    int rc = LMS_OK;
    if ((rc = A.get(&ds, count)) || (rc = A.get(&dq, count)) || (rc = A.get(&dd, count))) {
        A.release_all();
        return rc;
    }
    cudaError_t e = cudaMemcpy(ds, s, 4 * size_t(count), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dd, d, 4 * size_t(count), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = lms::launch_div32_selftest(count, ds, dd, dq, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(q, dq, 4 * size_t(count), cudaMemcpyDeviceToHost);
    A.release_all();
    if (e != cudaSuccess) {
        lms::set_error_detail(std::string("selftest: ") + cudaGetErrorString(e));
        return LMS_ERR_CUDA;
    }
    return LMS_OK;
}

int lms_selftest_divint64(int32_t count, const double* s, const int32_t* d, double* q) {
    return selftest_div(count, s, d, q, true);
}

int lms_selftest_add64(int32_t count, const double* a, const double* b, double* s) {
    if (count < 0 || (count > 0 && (!a || !b || !s))) return LMS_ERR_ARG;
    if (count == 0) return LMS_OK;
    Arena A;
    double *da = nullptr, *db = nullptr, *ds = nullptr;
    int rc = LMS_OK;
    if ((rc = A.get(&da, count)) || (rc = A.get(&db, count)) || (rc = A.get(&ds, count))) {
        A.release_all();
        return rc;
    }
    cudaError_t e = cudaMemcpy(da, a, 8 * size_t(count), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(db, b, 8 * size_t(count), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = lms::launch_add_selftest(count, da, db, ds, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(s, ds, 8 * size_t(count), cudaMemcpyDeviceToHost);
    A.release_all();
    if (e != cudaSuccess) {
        lms::set_error_detail(std::string("selftest: ") + cudaGetErrorString(e));
        return LMS_ERR_CUDA;
    }
    return LMS_OK;
}

int lms_selftest_timeout(int32_t wait_us) {
    if (wait_us < 1 || wait_us > 2000000) return LMS_ERR_ARG;
    int dev = 0, khz = 0;
    LMS_CUDA(cudaGetDevice(&dev));
    LMS_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    const long long bound = static_cast<long long>(wait_us) * std::max(khz, 1) / 1000;  // cycles at the top clock
    Arena A;
    int32_t* d_err = nullptr;
    LMS_TRY(A.get(&d_err, 1));
    int32_t err = 0;
    cudaError_t e = cudaMemset(d_err, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = lms::launch_wait_selftest(bound, d_err, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(&err, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost);
    A.release_all();
    if (e != cudaSuccess) {
        lms::set_error_detail(std::string("wait selftest: ") + cudaGetErrorString(e));
        return LMS_ERR_CUDA;
    }
    if (err) {
        lms::set_error_detail("bounded device wait expired (self-test)");
        return LMS_ERR_TIMEOUT;
    }
    return LMS_OK;
}

int lms_debug_checks(int32_t* enabled, uint64_t* violations, int32_t reset) {
    if (enabled) *enabled = lms::checks_enabled() ? 1 : 0;
    const unsigned long long v = lms::check_violations_kernels(reset != 0) +
                                 lms::check_violations_orderings(reset != 0) +
                                 lms::check_violations_noalloc(reset != 0) +
                                 lms::check_violations_staged(reset != 0);
    if (violations) *violations = v;
    return LMS_OK;
}

const char* lms_last_error_detail(void) { return lms::error_detail().c_str(); }

void lms_destroy(lms_handle h) { delete h; }

}  // extern "C"

// ------------------------------------------------------------------ batch

struct lms_batch_s {
    Arena arena;
    cudaStream_t stream = nullptr, cap = nullptr;
    int32_t k = 0;
    int64_t n_total = 0, n_int = 0, nnz_total = 0;
    std::vector<int64_t> voff;          // vertex offset of each mesh (k+1)
    std::vector<int32_t> perm;          // global new_to_old of the storage layout
    std::vector<int32_t> order_perm;    // global new_to_old of the ordering (lms_batch_get_permutation)
    std::vector<uint8_t> bnd_store;     // boundary flag per storage position
    int32_t window = 0;                 // degree-grouping window of the storage layout (0: the ordering)
    std::vector<int32_t> rp;            // relabelled global row offsets (host copy, for the tile table)
    std::vector<double> cs;             // per mesh (cx, cy, inv_s, s)
    int32_t *d_rp = nullptr, *d_ci = nullptr, *d_perm = nullptr, *d_item_mesh = nullptr, *d_queue = nullptr;
    // d_rp: relabelled row offsets with the boundary flag in bit 31 (row_ptr[v] | boundary(v) << 31)
    int32_t* d_err = nullptr;           // set by a kernel whose bounded wait expired
    uint32_t* d_bits = nullptr;
    int2* d_items = nullptr;
    int4* d_items4 = nullptr;           // (first vertex, end vertex, first entry, end entry)
    int32_t* d_item_pbase = nullptr;    // per tile: first id pair of the tile's mesh (packed kernel)
    int32_t* d_rw = nullptr;            // packed row words (LMS_KERNEL_PACKED)
    int2* d_pairs = nullptr;            // rows padded to even length, read as id pairs (LMS_KERNEL_PACKED)
    int64_t pairs_cap = 0;
    std::vector<int32_t> pstart;        // first id pair of each storage position's row (host copy)
    bool packed_ok = false;             // every mesh < 2^22 id pairs and every row <= kMaxPackedDegree entries
    int32_t e_cap = 0;                  // max CSR entries of a tile
    // SELL-C-sigma work layout (built on demand for the current tile size)
    int32_t* d_sell_col = nullptr;
    int2* d_sell_slice = nullptr;
    int32_t* d_sell_slot = nullptr;
    int2* d_sell_items = nullptr;
    int64_t sell_col_cap = 0, sell_slice_cap = 0, sell_items_cap = 0;
    int32_t sell_n_items = 0;
    int sell_sigma = 0;                 // tile size the SELL tables were built for (0 = none)
    float2* d_xy[3] = {nullptr, nullptr, nullptr};  // ping-pong + autotune scratch
    double* d_xy64 = nullptr;           // FP64 staging, original order
    double* d_fixed = nullptr;          // caller's last coordinates, original order (boundary values)
    double* d_cs = nullptr;
    int cur = 0;
    int32_t queue_slots = 0;
    // launch configuration
    int kernel = LMS_KERNEL_DIRECT, block = 128, chunk = 4, tile = 512, ctas_per_sm = 0;
    int chains = 2;                     // parallel chains of sweeps in a lms_batch_smooth graph
    bool configured = false;
    int32_t n_items = 0;
    int items_tile = 0;                 // tile size the item table was built for
    int2* d_items_cap = nullptr;
    int32_t* d_item_mesh_cap = nullptr;
    int64_t items_capacity = 0;
    GraphCache graphs;
    int64_t last_launches = 0;
    int sms = 0;
    // lms_batch_run: copy streams, a second compute stream and per-group events
    cudaStream_t s_in = nullptr, s_out = nullptr, s_c2 = nullptr;
    cudaEvent_t ev_join = nullptr;
    // lms_batch_smooth: capture streams and fork/join events of the parallel sweep chains
    std::vector<cudaStream_t> cap_extra;
    std::vector<cudaEvent_t> ev_extra;
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_in, ev_done;
    cudaEvent_t ev_start = nullptr;

    ~lms_batch_s() {
        if (stream) cudaStreamSynchronize(stream);
        if (s_in) cudaStreamSynchronize(s_in);
        if (s_out) cudaStreamSynchronize(s_out);
        if (s_c2) cudaStreamSynchronize(s_c2);
        graphs.clear();
        arena.release_all();
        for (cudaEvent_t e : ev_in) cudaEventDestroy(e);
        for (cudaEvent_t e : ev_done) cudaEventDestroy(e);
        if (ev_start) cudaEventDestroy(ev_start);
        if (ev_join) cudaEventDestroy(ev_join);
        if (ev_fork) cudaEventDestroy(ev_fork);
        for (cudaEvent_t e : ev_extra) cudaEventDestroy(e);
        for (cudaStream_t st : cap_extra) cudaStreamDestroy(st);
        if (s_c2) cudaStreamDestroy(s_c2);
        if (s_in) cudaStreamDestroy(s_in);
        if (s_out) cudaStreamDestroy(s_out);
        if (cap) cudaStreamDestroy(cap);
    }
};

namespace {

int batch_build_items(lms_batch_s* b, int tile) {
    if (b->items_tile == tile) return LMS_OK;
    std::vector<int2> items;
    std::vector<int4> items4;
    std::vector<int32_t> im, ieb;
    int32_t e_cap = 0;
    for (int32_t m = 0; m < b->k; ++m)
        for (int64_t v = b->voff[m]; v < b->voff[m + 1]; v += tile) {
            const int32_t va = int32_t(v), vb = int32_t(std::min<int64_t>(v + tile, b->voff[m + 1]));
            items.push_back(make_int2(va, vb));
            items4.push_back(make_int4(va, vb, b->rp[va], b->rp[vb]));
            e_cap = std::max(e_cap, b->rp[vb] - b->rp[va]);
            im.push_back(m);
            ieb.push_back(b->pstart.empty() ? 0 : b->pstart[b->voff[m]]);
        }
    if (int64_t(items.size()) > b->items_capacity) return LMS_ERR_STATE;
    LMS_CUDA(cudaMemcpyAsync(b->d_item_pbase, ieb.data(), sizeof(int32_t) * ieb.size(), cudaMemcpyHostToDevice,
                             b->stream));
    LMS_CUDA(cudaMemcpyAsync(b->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, b->stream));
    LMS_CUDA(cudaMemcpyAsync(b->d_items4, items4.data(), sizeof(int4) * items4.size(), cudaMemcpyHostToDevice,
                             b->stream));
    LMS_CUDA(cudaMemcpyAsync(b->d_item_mesh, im.data(), sizeof(int32_t) * im.size(), cudaMemcpyHostToDevice, b->stream));
    LMS_CUDA(cudaStreamSynchronize(b->stream));
    b->n_items = int32_t(items.size());
    b->items_tile = tile;
    b->e_cap = e_cap;
    b->graphs.clear();
    return LMS_OK;
}

// SELL-C-sigma tables for sorting windows of `sigma` vertices (the tiles).  Reads the relabelled CSR and
// boundary bits back from the device.
int batch_build_sell(lms_batch_s* b, int sigma) {
    if (b->sell_sigma == sigma) return LMS_OK;
    const int32_t N = int32_t(b->n_total);
    const int64_t E = b->nnz_total;
    std::vector<int32_t> ci(std::max<int64_t>(1, E));
    std::vector<uint32_t> bits((N + 31) / 32);
    LMS_CUDA(cudaMemcpyAsync(ci.data(), b->d_ci, 4 * size_t(E), cudaMemcpyDeviceToHost, b->stream));
    LMS_CUDA(cudaMemcpyAsync(bits.data(), b->d_bits, 4 * bits.size(), cudaMemcpyDeviceToHost, b->stream));
    LMS_CUDA(cudaStreamSynchronize(b->stream));
    const std::vector<int32_t>& rp = b->rp;
    std::vector<int32_t> col;
    std::vector<int2> slices, items;
    std::vector<int32_t> slots;
    col.reserve(size_t(E * 1.1) + 64);
    std::vector<std::pair<int32_t, int32_t>> verts;  // (-degree, position): stable by position
    for (int32_t m = 0; m < b->k; ++m)
        for (int64_t t0 = b->voff[m]; t0 < b->voff[m + 1]; t0 += sigma) {
            const int64_t t1 = std::min<int64_t>(t0 + sigma, b->voff[m + 1]);
            verts.clear();
            for (int64_t v = t0; v < t1; ++v)
                if (!((bits[v >> 5] >> (v & 31)) & 1u)) verts.push_back({-(rp[v + 1] - rp[v]), int32_t(v)});
            if (verts.empty()) continue;
            std::stable_sort(verts.begin(), verts.end());
            const int32_t first_slice = int32_t(slices.size());
            for (size_t s0 = 0; s0 < verts.size(); s0 += 32) {
                const size_t s1 = std::min(verts.size(), s0 + 32);
                const int32_t deg = -verts[s0].first;  // largest in the slice
                const int64_t base = int64_t(col.size());
                if (base + 32 * int64_t(deg) >= INT32_MAX) return LMS_ERR_ARG;
                slices.push_back(make_int2(int32_t(base), deg));
                col.resize(col.size() + 32 * size_t(deg), -1);
                for (size_t l = 0; l < 32; ++l) {
                    if (s0 + l < s1) {
                        const int32_t v = verts[s0 + l].second;
                        slots.push_back(v);
                        for (int32_t j = 0; j < rp[v + 1] - rp[v]; ++j) col[base + 32 * j + l] = ci[rp[v] + j];
                    } else {
                        slots.push_back(-1);
                    }
                }
            }
            items.push_back(make_int2(first_slice, int32_t(slices.size())));
        }
    if (int64_t(col.size()) > b->sell_col_cap) {
        LMS_TRY(b->arena.get(&b->d_sell_col, col.size() + 64));
        b->sell_col_cap = int64_t(col.size()) + 64;
    }
    if (int64_t(slices.size()) > b->sell_slice_cap) {
        LMS_TRY(b->arena.get(&b->d_sell_slice, slices.size() + 16));
        LMS_TRY(b->arena.get(&b->d_sell_slot, 32 * (slices.size() + 16)));
        b->sell_slice_cap = int64_t(slices.size()) + 16;
    }
    if (int64_t(items.size()) > b->sell_items_cap) {
        LMS_TRY(b->arena.get(&b->d_sell_items, items.size() + 16));
        b->sell_items_cap = int64_t(items.size()) + 16;
    }
    LMS_CUDA(cudaMemcpyAsync(b->d_sell_col, col.data(), 4 * col.size(), cudaMemcpyHostToDevice, b->stream));
    LMS_CUDA(cudaMemcpyAsync(b->d_sell_slice, slices.data(), sizeof(int2) * slices.size(), cudaMemcpyHostToDevice,
                             b->stream));
    LMS_CUDA(cudaMemcpyAsync(b->d_sell_slot, slots.data(), 4 * slots.size(), cudaMemcpyHostToDevice, b->stream));
    LMS_CUDA(cudaMemcpyAsync(b->d_sell_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice,
                             b->stream));
    LMS_CUDA(cudaStreamSynchronize(b->stream));
    b->sell_n_items = int32_t(items.size());
    b->sell_sigma = sigma;
    b->graphs.clear();
    return LMS_OK;
}

// Packed rows of the current layout (LMS_KERNEL_PACKED): every interior row copied into the id-pair array
// padded to an even length, and per vertex one word with the row's first pair relative to its mesh's,
// its neighbour count and the boundary flag.  Leaves packed_ok false (and the kernel unavailable) when a
// mesh has 2^22 id pairs or more or a row more than kMaxPackedDegree entries.  The tile table's per-tile
// mesh pair bases come from pstart: rebuild the tile table after this.
int batch_build_row_words(lms_batch_s* b) {
    b->packed_ok = false;
    b->pstart.clear();
    const int32_t N = int32_t(b->n_total);
    std::vector<int32_t> ps(size_t(N) + 1, 0), rw(N);
    for (int32_t v = 0; v < N; ++v) {
        const int32_t d = b->rp[v + 1] - b->rp[v];
        if (d > lms::kMaxPackedDegree) return LMS_OK;
        ps[v + 1] = ps[v] + (b->bnd_store[v] ? 0 : (d + 1) / 2);
    }
    for (int32_t m = 0; m < b->k; ++m) {
        const int32_t v0 = int32_t(b->voff[m]), v1 = int32_t(b->voff[m + 1]);
        if (ps[v1] - ps[v0] > lms::kPackedOffsetMask) return LMS_OK;
        for (int32_t v = v0; v < v1; ++v)
            rw[v] = (ps[v] - ps[v0]) | ((b->rp[v + 1] - b->rp[v]) << lms::kPackedDegreeShift) |
                    (b->bnd_store[v] ? int32_t(0x80000000u) : 0);
    }
    const int64_t P = ps[N];
    if (!b->d_rw) LMS_TRY(b->arena.get(&b->d_rw, std::max(1, N)));
    if (P + 1 > b->pairs_cap) {
        // sized for the largest padding any layout of these rows can need: one pair per vertex beyond E / 2
        const int64_t cap = std::max<int64_t>(P + 1, (b->nnz_total + b->n_total) / 2 + 1);
        LMS_TRY(b->arena.get(&b->d_pairs, size_t(cap)));
        b->pairs_cap = cap;
    }
    Arena tmp;
    tmp.al = b->arena.al;
    tmp.stream = b->stream;
    int32_t* d_ps = nullptr;
    if (int rc = tmp.get(&d_ps, size_t(N) + 1)) return rc;
    cudaError_t e = cudaMemcpyAsync(d_ps, ps.data(), sizeof(int32_t) * (size_t(N) + 1), cudaMemcpyHostToDevice, b->stream);
    if (!e) e = cudaMemcpyAsync(b->d_rw, rw.data(), sizeof(int32_t) * size_t(N), cudaMemcpyHostToDevice, b->stream);
    if (!e) e = lms::launch_pad_rows(N, b->d_rp, b->d_ci, d_ps, reinterpret_cast<int32_t*>(b->d_pairs), b->stream);
    if (!e) e = cudaStreamSynchronize(b->stream);
    tmp.release_all();
    if (e) {
        lms::set_error_detail(std::string("packed rows: ") + cudaGetErrorString(e));
        return LMS_ERR_CUDA;
    }
    b->pstart.swap(ps);
    b->packed_ok = true;
    return LMS_OK;
}

lms::PackedArgs batch_packed_args(lms_batch_s* b, int src, int dst, int slot) {
    lms::PackedArgs a{};
    a.row_words = b->d_rw;
    a.id_pairs = b->d_pairs;
    a.src = b->d_xy[src];
    a.dst = b->d_xy[dst];
    a.items = b->d_items;
    a.items_pbase = b->d_item_pbase;
    a.n_items = b->n_items;
    a.queue = b->d_queue + slot;
    a.n_vertices = int32_t(b->n_total);
    return a;
}

lms::StagedArgs batch_staged_args(lms_batch_s* b, int src, int dst, int slot) {
    lms::StagedArgs a{};
    a.row_ptr = b->d_rp;
    a.col_idx = b->d_ci;
    a.bnd_bits = b->d_bits;
    a.src = b->d_xy[src];
    a.dst = b->d_xy[dst];
    a.items = b->d_items4;
    a.n_items = b->n_items;
    a.queue = b->d_queue + slot;
    a.tile_cap = b->items_tile;
    a.e_cap = b->e_cap;
    a.n_vertices = int32_t(b->n_total);
    a.err = b->d_err;
    return a;
}

SweepArgs batch_args(lms_batch_s* b, int src, int dst, int slot) {
    SweepArgs a{};
    a.row_ptr = b->d_rp;
    a.col_idx = b->d_ci;
    a.bnd_bits = b->d_bits;
    a.src = b->d_xy[src];
    a.dst = b->d_xy[dst];
    a.items = b->d_items;
    a.n_items = b->n_items;
    a.queue = b->d_queue + slot;
    a.v_end = int32_t(b->n_total);
    a.n_vertices = int32_t(b->n_total);
    return a;
}

int batch_occupancy(lms_batch_s* b) {
    if (b->kernel == LMS_KERNEL_SELL) return lms::batch_sell_occupancy(b->block, b->chunk);
    if (b->kernel == LMS_KERNEL_PACKED) return lms::batch_packed_occupancy(b->block, b->chunk);
    if (b->kernel == LMS_KERNEL_STAGED)
        return lms::staged_occupancy(LMS_FP32, false, b->block, b->items_tile, b->e_cap);
    return lms::batch_sweep_occupancy(b->block, b->chunk);
}

// one sweep of the batch on stream s: reads buffer src, writes dst, counts tiles in queue slot `slot`
// one sweep over the tiles [i0, i1) of the item table (direct and staged kernels; meshes never share a
// tile, so a range of tiles is a range of whole meshes when it starts and ends at mesh boundaries)
int batch_issue_range(lms_batch_s* b, int src, int dst, int slot, int grid, cudaStream_t s, int32_t i0, int32_t i1) {
    if (b->kernel == LMS_KERNEL_STAGED) {
        lms::StagedArgs a = batch_staged_args(b, src, dst, slot);
        a.items += i0;
        a.n_items = i1 - i0;
        return check_launch(lms::launch_sweep_staged(LMS_FP32, false, a, grid, b->block, s), "staged_sweep");
    }
    if (b->kernel == LMS_KERNEL_PACKED) {
        lms::PackedArgs a = batch_packed_args(b, src, dst, slot);
        a.items += i0;
        a.items_pbase += i0;
        a.n_items = i1 - i0;
        return check_launch(lms::launch_batch_sweep_packed(a, b->block, b->chunk, grid, s), "batch_sweep_packed");
    }
    SweepArgs a = batch_args(b, src, dst, slot);
    a.items += i0;
    a.n_items = i1 - i0;
    return check_launch(lms::launch_batch_sweep(a, b->block, b->chunk, grid, s), "batch_sweep");
}

int batch_issue(lms_batch_s* b, int src, int dst, int slot, int grid, cudaStream_t s) {
    if (b->kernel == LMS_KERNEL_SELL) {
        lms::SellArgs a{};
        a.col = b->d_sell_col;
        a.slice = b->d_sell_slice;
        a.slot = b->d_sell_slot;
        a.src = b->d_xy[src];
        a.dst = b->d_xy[dst];
        a.items = b->d_sell_items;
        a.n_items = b->sell_n_items;
        a.queue = b->d_queue + slot;
        return check_launch(lms::launch_batch_sell(a, b->block, b->chunk, grid, s), "sell_sweep");
    }
    if (b->kernel == LMS_KERNEL_STAGED)
        return check_launch(lms::launch_sweep_staged(LMS_FP32, false, batch_staged_args(b, src, dst, slot), grid,
                                                     b->block, s),
                            "staged_sweep");
    if (b->kernel == LMS_KERNEL_PACKED)
        return check_launch(lms::launch_batch_sweep_packed(batch_packed_args(b, src, dst, slot), b->block, b->chunk,
                                                           grid, s),
                            "batch_sweep_packed");
    return check_launch(lms::launch_batch_sweep(batch_args(b, src, dst, slot), b->block, b->chunk, grid, s),
                        "batch_sweep");
}

int batch_grid(lms_batch_s* b) {
    int occ = batch_occupancy(b);
    if (occ <= 0) occ = 1;
    int per_sm = b->ctas_per_sm > 0 ? std::min(b->ctas_per_sm, occ) : occ;
    return std::max(1, per_sm * b->sms);
}

int ensure_queue(lms_batch_s* b, int32_t slots) {
    if (slots <= b->queue_slots) return LMS_OK;
    int32_t want = std::max<int32_t>(slots, 64);
    LMS_TRY(b->arena.get(&b->d_queue, want));
    b->queue_slots = want;
    b->graphs.clear();
    return LMS_OK;
}

std::string autotune_key(lms_batch_s* b) {
    cudaDeviceProp p;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&p, dev);
    auto bucket = [](int64_t x) {
        int l = 0;
        while (x > 1) {
            x >>= 1;
            ++l;
        }
        return l;
    };
    std::ostringstream os;
    os << "v12|" << p.name << "|fp32|jacobi|n2^" << bucket(b->n_total) << "|nnz2^" << bucket(b->nnz_total);
    std::string s = os.str();
    for (auto& c : s)
        if (c == ' ') c = '_';
    return s;
}

// Storage layout of the batch for degree-grouping window `window`: the ordering's sequence of each mesh
// cut into runs of `window` consecutive positions (never crossing a mesh), each run stably sorted by
// (boundary first, then ascending row length).  window = 0 keeps the ordering itself.  A warp's 32
// threads then take rows of about one length, so a warp's row loop ends with its rows instead of
// running to the longest of 32 mixed rows; positions move at most window - 1 places, so the ordering's
// locality is kept.  Jacobi results do not depend on the storage order (rows keep their entry order).
void layout_for_window(const lms_batch_s* b, int32_t window, const std::vector<int32_t>& deg_orig,
                       const std::vector<uint8_t>& bnd_orig, std::vector<int32_t>& out) {
    out = b->order_perm;
    if (window <= 0) return;
    std::vector<std::pair<int32_t, int32_t>> key;  // (class, position in the run): stable by position
    for (int32_t m = 0; m < b->k; ++m)
        for (int64_t t0 = b->voff[m]; t0 < b->voff[m + 1]; t0 += window) {
            const int64_t t1 = std::min<int64_t>(t0 + window, b->voff[m + 1]);
            key.clear();
            for (int64_t i = t0; i < t1; ++i) {
                const int32_t v = b->order_perm[i];
                key.push_back({bnd_orig[v] ? -1 : deg_orig[v], int32_t(i)});
            }
            std::stable_sort(key.begin(), key.end(),
                             [](const std::pair<int32_t, int32_t>& x, const std::pair<int32_t, int32_t>& y) {
                                 return x.first < y.first;
                             });
            for (int64_t i = t0; i < t1; ++i) out[i] = b->order_perm[key[i - t0].second];
        }
}

// Move the batch from its current storage layout to the layout of `window` on the device: rows gathered
// with their entry order kept and ids renamed, boundary bits and row flags rebuilt, both position buffers
// permuted (the coordinates the batch holds are kept); tile tables rebuilt and captured graphs dropped.
int batch_relayout(lms_batch_s* b, int32_t window) {
    if (window == b->window) return LMS_OK;
    const int32_t N = int32_t(b->n_total);
    const int64_t E = b->nnz_total;
    std::vector<int32_t> deg_orig(N);
    std::vector<uint8_t> bnd_orig(N);
    for (int32_t i = 0; i < N; ++i) {
        deg_orig[b->perm[i]] = b->rp[i + 1] - b->rp[i];
        bnd_orig[b->perm[i]] = b->bnd_store[i];
    }
    std::vector<int32_t> np;
    layout_for_window(b, window, deg_orig, bnd_orig, np);
    // q[i] = current storage position of the vertex placed at i; qinv its inverse
    std::vector<int32_t> inv_cur(N), q(N), qinv(N), rp_new(N + 1, 0);
    std::vector<uint8_t> bnd_new(N);
    for (int32_t i = 0; i < N; ++i) inv_cur[b->perm[i]] = i;
    for (int32_t i = 0; i < N; ++i) {
        q[i] = inv_cur[np[i]];
        qinv[q[i]] = i;
        rp_new[i + 1] = rp_new[i] + (b->rp[q[i] + 1] - b->rp[q[i]]);
        bnd_new[i] = b->bnd_store[q[i]];
    }
    cudaStream_t s = b->stream;
    LMS_CUDA(cudaStreamSynchronize(s));
    Arena tmp;
    tmp.al = b->arena.al;
    tmp.stream = s;
    int32_t *d_rp_old = nullptr, *d_ci_old = nullptr, *d_q = nullptr, *d_qinv = nullptr;
    uint8_t* d_bnd_old = nullptr;
    int rc = LMS_OK;
    if ((rc = tmp.get(&d_rp_old, N + 1)) || (rc = tmp.get(&d_ci_old, std::max<int64_t>(1, E))) ||
        (rc = tmp.get(&d_q, N)) || (rc = tmp.get(&d_qinv, N)) || (rc = tmp.get(&d_bnd_old, N))) {
        tmp.release_all();
        return rc;
    }
    cudaError_t e = cudaMemcpyAsync(d_rp_old, b->rp.data(), 4 * size_t(N + 1), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(d_ci_old, b->d_ci, 4 * size_t(E), cudaMemcpyDeviceToDevice, s);
    if (!e) e = cudaMemcpyAsync(d_q, q.data(), 4 * size_t(N), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(d_qinv, qinv.data(), 4 * size_t(N), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(d_bnd_old, b->bnd_store.data(), size_t(N), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(b->d_rp, rp_new.data(), 4 * size_t(N + 1), cudaMemcpyHostToDevice, s);
    if (!e) e = lms::launch_gather_rows(N, d_q, d_rp_old, d_ci_old, b->d_rp, b->d_ci, d_qinv, s);
    if (!e) e = cudaMemsetAsync(b->d_bits, 0, 4 * size_t((N + 31) / 32), s);
    if (!e) e = lms::launch_boundary_bits(N, d_q, d_bnd_old, b->d_bits, s);
    if (!e) e = lms::launch_flag_boundary_rows(N, b->d_bits, b->d_rp, s);
    for (int buf = 0; buf < 2 && !e; ++buf) {
        e = lms::launch_gather_xy(LMS_FP32, N, d_q, b->d_xy[buf], b->d_xy[2], s);
        if (!e) e = cudaMemcpyAsync(b->d_xy[buf], b->d_xy[2], sizeof(float2) * size_t(N), cudaMemcpyDeviceToDevice, s);
    }
    if (!e) e = cudaMemcpyAsync(b->d_perm, np.data(), 4 * size_t(N), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaStreamSynchronize(s);
    tmp.release_all();
    if (e) {
        lms::set_error_detail(std::string("batch layout: ") + cudaGetErrorString(e));
        return LMS_ERR_CUDA;
    }
    b->rp.swap(rp_new);
    b->perm.swap(np);
    b->bnd_store.swap(bnd_new);
    b->window = window;
    b->graphs.clear();
    b->items_tile = 0;
    b->sell_sigma = 0;
    LMS_TRY(batch_build_row_words(b));
    LMS_TRY(batch_build_items(b, b->tile));
    if (b->kernel == LMS_KERNEL_SELL) LMS_TRY(batch_build_sell(b, b->tile));
    if (b->kernel == LMS_KERNEL_PACKED && !b->packed_ok) b->kernel = LMS_KERNEL_DIRECT;
    return LMS_OK;
}

}  // namespace

extern "C" {

int lms_batch_create(int32_t k, const lms_mesh_desc* meshes, int ordering, uint64_t seed, void* cuda_stream,
                     lms_batch* out) {
    if (!out || !meshes || k <= 0 || ordering < LMS_ORI || ordering > LMS_BRDR) return LMS_ERR_ARG;
    *out = nullptr;
    // validate in parallel
    std::vector<int> status(k, LMS_OK);
    {
        std::atomic<int32_t> next(0);
        unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        for (unsigned t = 0; t < nt; ++t)
            pool.emplace_back([&]() {
                for (int32_t m; (m = next++) < k;) {
                    const lms_mesh_desc& d = meshes[m];
                    int rc = lms::validate_mesh(d.n, d.row_ptr, d.col_idx, d.is_boundary, d.ntri, d.tri);
                    if (rc == LMS_OK && (!d.xy || !all_finite(d.xy, 2 * int64_t(d.n)))) rc = LMS_ERR_ARG;
                    if (rc == LMS_OK && (ordering == LMS_RDR || ordering == LMS_BRDR) && (d.ntri <= 0 || !d.tri)) rc = LMS_ERR_NO_TRIANGLES;
                    status[m] = rc;
                }
            });
        for (auto& th : pool) th.join();
    }
    for (int rc : status)
        if (rc != LMS_OK) return rc;

    auto b = new (std::nothrow) lms_batch_s();
    if (!b) return LMS_ERR_OOM;
    auto fail = [&](int rc) {
        delete b;
        return rc;
    };
    {
        std::lock_guard<std::mutex> g(g_alloc_mu);
        b->arena.al = g_alloc;
    }
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->arena.stream = b->stream;
    b->k = k;
    b->voff.assign(k + 1, 0);
    std::vector<int64_t> eoff(k + 1, 0), toff(k + 1, 0);
    for (int32_t m = 0; m < k; ++m) {
        b->voff[m + 1] = b->voff[m] + meshes[m].n;
        eoff[m + 1] = eoff[m] + meshes[m].row_ptr[meshes[m].n];
        toff[m + 1] = toff[m] + ((ordering == LMS_RDR || ordering == LMS_BRDR) ? meshes[m].ntri : 0);
        for (int32_t v = 0; v < meshes[m].n; ++v) b->n_int += meshes[m].is_boundary[v] ? 0 : 1;
    }
    b->n_total = b->voff[k];
    b->nnz_total = eoff[k];
    if (b->n_total >= INT32_MAX || b->nnz_total >= INT32_MAX || toff[k] * 3 >= INT32_MAX) return fail(LMS_ERR_ARG);
    const int32_t N = int32_t(b->n_total), E = int32_t(b->nnz_total), T = int32_t(toff[k]);
    cudaDeviceProp prop;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return fail(LMS_ERR_CUDA);
    b->sms = prop.multiProcessorCount;
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) return fail(LMS_ERR_CUDA);

    // concatenated original arrays (global ids)
    std::vector<int32_t> rp0(N + 1), ci0(std::max(1, E)), tri0(std::max<int64_t>(3, 3 * int64_t(T)));
    std::vector<uint8_t> bnd0(N);
    std::vector<double> xy0(2 * size_t(N));
    b->cs.assign(4 * size_t(k), 0.0);
    for (int32_t m = 0; m < k; ++m) {
        const lms_mesh_desc& d = meshes[m];
        const int32_t vo = int32_t(b->voff[m]), eo = int32_t(eoff[m]);
        for (int32_t v = 0; v < d.n; ++v) {
            rp0[vo + v] = eo + d.row_ptr[v];
            bnd0[vo + v] = d.is_boundary[v] ? 1 : 0;
        }
        for (int32_t e = 0; e < d.row_ptr[d.n]; ++e) ci0[eo + e] = vo + d.col_idx[e];
        if (ordering == LMS_RDR || ordering == LMS_BRDR)
            for (int64_t i = 0; i < 3 * int64_t(d.ntri); ++i) tri0[3 * toff[m] + i] = vo + d.tri[i];
        std::memcpy(xy0.data() + 2 * size_t(vo), d.xy, 16 * size_t(d.n));
        double cx, cy, s;
        bbox(d.xy, d.n, &cx, &cy, &s);
        b->cs[4 * m] = cx;
        b->cs[4 * m + 1] = cy;
        b->cs[4 * m + 2] = 1.0 / s;
        b->cs[4 * m + 3] = s;
    }
    rp0[N] = E;

    Arena& A = b->arena;
    Arena orig;  // original-label copies, released once the relabelled arrays exist
    orig.al = b->arena.al;
    orig.stream = b->stream;
    int32_t *d_rp0 = nullptr, *d_ci0 = nullptr, *d_inv = nullptr;
    uint8_t* d_bnd0 = nullptr;
    auto fail_orig = [&](int rc) {
        if (b->stream) cudaStreamSynchronize(b->stream);
        orig.release_all();
        return fail(rc);
    };
    int max_items = 0;
    for (int32_t m = 0; m < k; ++m) max_items += (meshes[m].n + 127) / 128;
    b->items_capacity = max_items;
    int rc = LMS_OK;
    if ((rc = A.get(&b->d_rp, N + 1 + 8)) || (rc = A.get(&b->d_ci, E + 8)) || (rc = A.get(&b->d_perm, N)) ||
        (rc = A.get(&b->d_bits, (N + 31) / 32 + 8)) || (rc = A.get(&b->d_err, 2)) ||
        (rc = A.get(&b->d_items4, max_items)) || (rc = A.get(&b->d_xy[0], N)) || (rc = A.get(&b->d_xy[1], N)) ||
        (rc = A.get(&b->d_xy[2], N)) || (rc = A.get(&b->d_xy64, 2 * size_t(N))) || (rc = A.get(&b->d_fixed, 2 * size_t(N))) ||
        (rc = A.get(&b->d_cs, 4 * size_t(k))) ||
        (rc = A.get(&b->d_items, max_items)) || (rc = A.get(&b->d_item_mesh, max_items)) ||
        (rc = A.get(&b->d_item_pbase, max_items)) ||
        (rc = ensure_queue(b, 64)) || (rc = orig.get(&d_rp0, N + 1)) || (rc = orig.get(&d_ci0, std::max(1, E))) ||
        (rc = orig.get(&d_inv, N)) || (rc = orig.get(&d_bnd0, N)))
        return fail_orig(rc);
    cudaStream_t s = b->stream;
    if (cudaMemsetAsync(b->d_err, 0, 2 * sizeof(int32_t), s) || cudaMemsetAsync(b->d_bits, 0, 4 * ((N + 31) / 32 + 8), s) ||
        cudaMemsetAsync(b->d_rp, 0, 4 * size_t(N + 1 + 8), s) || cudaMemsetAsync(b->d_ci, 0, 4 * size_t(E + 8), s) ||
        cudaMemcpyAsync(d_rp0, rp0.data(), 4 * size_t(N + 1), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(d_ci0, ci0.data(), 4 * size_t(E), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(d_bnd0, bnd0.data(), size_t(N), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(b->d_xy64, xy0.data(), 16 * size_t(N), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(b->d_fixed, xy0.data(), 16 * size_t(N), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(b->d_cs, b->cs.data(), 32 * size_t(k), cudaMemcpyHostToDevice, s))
        return fail_orig(LMS_ERR_CUDA);

    // RDR keys: Section 3.2 vertex qualities in FP64 on the device (block RDR keeps them there when its
    // walks run on the device)
    std::vector<double> q;
    Arena keys;
    keys.al = b->arena.al;
    keys.stream = s;
    double* d_qv_keep = nullptr;
    bool brdr_device = false;
    if (ordering == LMS_BRDR) {
        int32_t max_deg = 0;
        for (int32_t m = 0; m < k; ++m) max_deg = std::max(max_deg, max_row(meshes[m].row_ptr, meshes[m].n));
        brdr_device = max_deg <= lms::block_rdr_max_degree();
        if (brdr_device && (rc = keys.get(&d_qv_keep, N))) return fail_orig(rc);
    }
    if (ordering == LMS_RDR || ordering == LMS_BRDR) {
        std::vector<int32_t> vt_ptr, vt_idx;
        build_incidence(N, T, tri0.data(), vt_ptr, vt_idx);
        int32_t *d_tri = nullptr, *d_vp = nullptr, *d_vi = nullptr;
        double *d_qt = nullptr, *d_qv = nullptr;
        Arena tmp;
        tmp.al = b->arena.al;
        tmp.stream = s;
        if ((rc = tmp.get(&d_tri, 3 * size_t(T))) || (rc = tmp.get(&d_vp, N + 1)) ||
            (rc = tmp.get(&d_vi, 3 * size_t(T))) || (rc = tmp.get(&d_qt, T)) || (rc = tmp.get(&d_qv, N))) {
            tmp.release_all();
            keys.release_all();
            return fail_orig(rc);
        }
        q.resize(N);
        cudaError_t e = cudaMemcpyAsync(d_tri, tri0.data(), 12 * size_t(T), cudaMemcpyHostToDevice, s);
        if (!e) e = cudaMemcpyAsync(d_vp, vt_ptr.data(), 4 * size_t(N + 1), cudaMemcpyHostToDevice, s);
        if (!e) e = cudaMemcpyAsync(d_vi, vt_idx.data(), 12 * size_t(T), cudaMemcpyHostToDevice, s);
        if (!e) e = lms::launch_tri_quality_exact(T, d_tri, b->d_xy64, d_qt, s);
        if (!e) e = lms::launch_vertex_quality_exact(N, d_vp, d_vi, d_qt, d_qv, s);
        if (!e && d_qv_keep) e = cudaMemcpyAsync(d_qv_keep, d_qv, 8 * size_t(N), cudaMemcpyDeviceToDevice, s);
        if (!e) e = cudaMemcpyAsync(q.data(), d_qv, 8 * size_t(N), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        tmp.release_all();
        if (e) {
            keys.release_all();
            lms::set_error_detail(std::string("batch quality: ") + cudaGetErrorString(e));
            return fail_orig(LMS_ERR_CUDA);
        }
    }
    // per-mesh orderings: breadth-first ones on the device (one search per mesh), the others on
    // host threads
    b->perm.resize(N);
    if (ordering == LMS_BFS || ordering == LMS_RBFS || (ordering == LMS_BRDR && brdr_device)) {
        rc = device_order(b->arena.al, s, b->sms, d_rp0, d_ci0, N, k, b->voff.data(),
                          ordering == LMS_BRDR ? d_qv_keep : nullptr, ordering == LMS_BRDR ? d_bnd0 : nullptr,
                          b->perm.data());
        keys.release_all();
        if (rc) return fail_orig(rc);
        if (ordering == LMS_RBFS)
            for (int32_t m = 0; m < k; ++m) std::reverse(b->perm.begin() + b->voff[m], b->perm.begin() + b->voff[m + 1]);
    } else {
        std::atomic<int32_t> next(0);
        unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        for (unsigned t = 0; t < nt; ++t)
            pool.emplace_back([&]() {
                std::vector<int32_t> p;
                for (int32_t m; (m = next++) < k;) {
                    const lms_mesh_desc& d = meshes[m];
                    p.resize(d.n);
                    const int64_t vo = b->voff[m];
                    int r = lms::order_vertices(d.n, d.row_ptr, d.col_idx, d.is_boundary,
                                                q.empty() ? nullptr : q.data() + vo, ordering, seed + uint64_t(m),
                                                p.data());
                    status[m] = r;
                    for (int32_t i = 0; i < d.n; ++i) b->perm[vo + i] = int32_t(vo + p[i]);
                }
            });
        for (auto& th : pool) th.join();
    }
    for (int r : status)
        if (r != LMS_OK) return fail_orig(r);
    // relabel on the device
    int32_t max_deg_all = 0;
    for (int32_t m = 0; m < k; ++m) max_deg_all = std::max(max_deg_all, max_row(meshes[m].row_ptr, meshes[m].n));
    std::vector<int32_t> inv(N);
    std::vector<int32_t>& rp = b->rp;
    rp.assign(N + 1, 0);
    for (int32_t i = 0; i < N; ++i) inv[b->perm[i]] = i;
    for (int32_t i = 0; i < N; ++i) rp[i + 1] = rp[i] + (rp0[b->perm[i] + 1] - rp0[b->perm[i]]);
    cudaError_t e = cudaMemcpyAsync(b->d_perm, b->perm.data(), 4 * size_t(N), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(d_inv, inv.data(), 4 * size_t(N), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(b->d_rp, rp.data(), 4 * size_t(N + 1), cudaMemcpyHostToDevice, s);
    if (!e) e = lms::launch_gather_rows(N, b->d_perm, d_rp0, d_ci0, b->d_rp, b->d_ci, d_inv, s);
    if (!e) e = lms::launch_boundary_bits(N, b->d_perm, d_bnd0, b->d_bits, s);
    // rows farthest neighbour first (storage distance): a row's first chunk of gathers then holds the
    // references most likely to miss L1, so their latency overlaps the rest of the row (FP32 Kahan sums, so
    // the order moves results by rounding only; rows longer than kMaxPackedDegree keep their order)
    if (!e && max_deg_all <= lms::kMaxPackedDegree) e = lms::launch_sort_rows_far_first(N, b->d_rp, b->d_ci, s);
    if (!e) e = lms::launch_flag_boundary_rows(N, b->d_bits, b->d_rp, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) {
        lms::set_error_detail(std::string("batch relabel: ") + cudaGetErrorString(e));
        return fail_orig(LMS_ERR_CUDA);
    }
    orig.release_all();
    b->order_perm = b->perm;
    b->bnd_store.resize(N);
    for (int32_t i = 0; i < N; ++i) b->bnd_store[i] = bnd0[b->perm[i]];
    if ((rc = batch_build_row_words(b)) || (rc = batch_build_items(b, b->tile))) return fail(rc);
    e = lms::launch_batch_load_xy(b->n_items, b->d_items, b->d_item_mesh, b->d_perm, b->d_fixed, b->d_xy[0],
                                  b->d_xy[1], b->d_cs, b->d_err + 1, s);
    if (e) return fail(check_launch(e, "batch_load_xy"));
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(LMS_ERR_CUDA);
    *out = b;
    return LMS_OK;
}

int lms_batch_get_config(lms_batch b, int32_t* kernel, int32_t* block, int32_t* chunk, int32_t* tile,
                         int32_t* ctas_per_sm) {
    if (!b) return LMS_ERR_ARG;
    if (kernel) *kernel = b->kernel;
    if (block) *block = b->block;
    if (chunk) *chunk = b->chunk;
    if (tile) *tile = b->tile;
    if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm > 0 ? std::min(b->ctas_per_sm, batch_occupancy(b)) : batch_occupancy(b);
    return LMS_OK;
}

int lms_batch_set_config(lms_batch b, int32_t kernel, int32_t block, int32_t chunk, int32_t tile, int32_t ctas_per_sm) {
    if (!b) return LMS_ERR_ARG;
    if (block != 128 && block != 256 && block != 512) return LMS_ERR_ARG;
    if (tile < 128 || tile > 65536 || (tile % 128) != 0 || ctas_per_sm < 0) return LMS_ERR_ARG;
    switch (kernel) {
        case LMS_KERNEL_DIRECT:
            if (chunk < 1 || chunk > 8 || chunk == 7) return LMS_ERR_ARG;
            break;
        case LMS_KERNEL_STAGED:
            if (block > 256 || chunk != 1 || tile > 4096) return LMS_ERR_ARG;
            break;
        case LMS_KERNEL_SELL:
            if (chunk != 1 && chunk != 4 && chunk != 8) return LMS_ERR_ARG;
            break;
        case LMS_KERNEL_PACKED:
            if (chunk != 2 && chunk != 4 && chunk != 6) return LMS_ERR_ARG;
            if (!b->packed_ok) {
                lms::set_error_detail("packed rows need meshes of fewer than 2^22 id pairs and rows of at most 63");
                return LMS_ERR_ARG;
            }
            break;
        default:
            return LMS_ERR_ARG;
    }
    b->kernel = kernel;
    b->block = block;
    b->chunk = chunk;
    b->tile = tile;
    b->ctas_per_sm = ctas_per_sm;
    b->configured = true;
    b->graphs.clear();
    LMS_TRY(batch_build_items(b, tile));
    if (kernel == LMS_KERNEL_SELL) LMS_TRY(batch_build_sell(b, tile));
    if (batch_occupancy(b) <= 0) {
        lms::set_error_detail("launch configuration does not fit on the device");
        return LMS_ERR_ARG;
    }
    return LMS_OK;
}

}  // extern "C"

namespace {
// Chains of the sweep graph: times 10-sweep graphs of lms_batch_smooth with 1 to 4 chains on the current
// launch configuration and keeps the fastest.  The batch's positions are saved in the scratch buffer
// and put back, so the batch holds the same coordinates afterwards (the sweeps run an even count, so
// the ping-pong index ends where it started; the other buffer's interior values are overwritten by the
// next sweep before anything reads them).
int batch_tune_chains(lms_batch_s* b) {
    if (b->kernel == LMS_KERNEL_SELL || b->k < 2) return LMS_OK;
    cudaStream_t s = b->stream;
    const int cur = b->cur;
    LMS_CUDA(cudaMemcpyAsync(b->d_xy[2], b->d_xy[cur], sizeof(float2) * size_t(b->n_total), cudaMemcpyDeviceToDevice, s));
    cudaEvent_t e0, e1;
    LMS_CUDA(cudaEventCreate(&e0));
    LMS_CUDA(cudaEventCreate(&e1));
    const int iters = 10, reps = 3;
    float best = 1e30f;
    int win = b->chains;
    const bool verbose = std::getenv("LMS_AUTOTUNE_VERBOSE") != nullptr;
    int rc = LMS_OK;
    for (int c = 1; c <= 4 && c <= b->k && rc == LMS_OK; ++c) {
        b->chains = c;
        if ((rc = lms_batch_smooth(b, iters)) != LMS_OK) break;  // capture + warm-up
        float ms = 1e30f;
        for (int round = 0; round < 2 && rc == LMS_OK; ++round) {
            if (cudaEventRecord(e0, s) != cudaSuccess) rc = LMS_ERR_CUDA;
            for (int r = 0; r < reps && rc == LMS_OK; ++r) rc = lms_batch_smooth(b, iters);
            if (rc == LMS_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
                rc = LMS_ERR_CUDA;
            float t = 0.f;
            if (rc == LMS_OK && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms = std::min(ms, t);
        }
        if (verbose) std::fprintf(stderr, "[lms autotune] chains=%d: %.4f ms/sweep\n", c, ms / (reps * iters));
        if (ms < best) {
            best = ms;
            win = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->chains = win;
    if (rc != LMS_OK) return rc;
    LMS_CUDA(cudaMemcpyAsync(b->d_xy[cur], b->d_xy[2], sizeof(float2) * size_t(b->n_total), cudaMemcpyDeviceToDevice, s));
    LMS_CUDA(cudaStreamSynchronize(s));
    b->cur = cur;
    return LMS_OK;
}
}  // namespace

extern "C" {

int lms_batch_autotune(lms_batch b, int32_t* kernel, int32_t* block, int32_t* chunk, int32_t* tile,
                       int32_t* ctas_per_sm) {
    if (!b) return LMS_ERR_ARG;
    const char* cache = std::getenv("LMS_AUTOTUNE_CACHE");
    const std::string key = autotune_key(b);
    if (cache) {
        std::ifstream f(cache);
        std::string line;
        while (std::getline(f, line)) {
            std::istringstream is(line);
            std::string kk;
            int kn, bl, ch, ti, cp, wi, cn;
            if ((is >> kk >> kn >> bl >> ch >> ti >> cp >> wi >> cn) && kk == key && cn >= 1 && cn <= 8 &&
                batch_relayout(b, wi) == LMS_OK && lms_batch_set_config(b, kn, bl, ch, ti, cp) == LMS_OK) {
                b->chains = cn;
                return lms_batch_get_config(b, kernel, block, chunk, tile, ctas_per_sm);
            }
        }
    }
    struct Cand {
        int kernel, block, chunk, tile, window;
    };
    // the storage layout is the ordering itself: windows grouped by row length (lms_batch_set_layout) were
    // 2-7% slower on every configuration of the 512-mesh batch (a warp's gathers spread over more lines)
    std::vector<Cand> cands;
    for (int blk : {128, 256, 512})
        for (int ch : {1, 2, 3, 4, 5, 6, 8})
            for (int ti : {256, 512, 1024}) cands.push_back({LMS_KERNEL_DIRECT, blk, ch, ti, 0});
    for (int blk : {128, 256})
        for (int ti : {128, 256, 512}) cands.push_back({LMS_KERNEL_STAGED, blk, 1, ti, 0});
    for (int ti : {512, 1024, 2048})  // sigma outermost: the SELL tables are rebuilt once per sigma
        for (int blk : {128, 256})
            for (int ch : {4, 8}) cands.push_back({LMS_KERNEL_SELL, blk, ch, ti, 0});
    if (b->packed_ok)
        for (int blk : {128, 256, 512})
            for (int ch : {2, 4, 6})
                for (int ti : {256, 512, 1024}) cands.push_back({LMS_KERNEL_PACKED, blk, ch, ti, 0});
    cudaStream_t s = b->stream;
    cudaEvent_t e0, e1;
    LMS_CUDA(cudaEventCreate(&e0));
    LMS_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    Cand win = cands.front();
    const int reps = 20, rounds = 2;
    const bool verbose = std::getenv("LMS_AUTOTUNE_VERBOSE") != nullptr;
    LMS_TRY(ensure_queue(b, reps + 2));
    for (const Cand& c : cands) {
        if (batch_relayout(b, c.window) != LMS_OK) continue;
        if (lms_batch_set_config(b, c.kernel, c.block, c.chunk, c.tile, 0) != LMS_OK) continue;
        const int grid = batch_grid(b);
        // reads buffer cur, writes the scratch buffer: the batch's positions are untouched
        LMS_CUDA(cudaMemsetAsync(b->d_queue, 0, sizeof(int32_t) * (reps + 1), s));
        LMS_TRY(batch_issue(b, b->cur, 2, reps, grid, s));
        float ms = 1e30f;
        for (int round = 0; round < rounds; ++round) {
            LMS_CUDA(cudaMemsetAsync(b->d_queue, 0, sizeof(int32_t) * reps, s));
            LMS_CUDA(cudaEventRecord(e0, s));
            for (int r = 0; r < reps; ++r) LMS_TRY(batch_issue(b, b->cur, 2, r, grid, s));
            LMS_CUDA(cudaEventRecord(e1, s));
            LMS_CUDA(cudaEventSynchronize(e1));
            float t = 0.f;
            LMS_CUDA(cudaEventElapsedTime(&t, e0, e1));
            ms = std::min(ms, t);
        }
        if (verbose)
            std::fprintf(stderr, "[lms autotune] kernel=%d block=%d chunk=%d tile=%d window=%d grid=%d: %.4f ms/sweep\n",
                         c.kernel, c.block, c.chunk, c.tile, c.window, grid, ms / reps);
        if (ms < best) {
            best = ms;
            win = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    LMS_TRY(batch_relayout(b, win.window));
    LMS_TRY(lms_batch_set_config(b, win.kernel, win.block, win.chunk, win.tile, 0));
    LMS_TRY(batch_tune_chains(b));
    if (cache) {
        std::ofstream f(cache, std::ios::app);
        f << key << " " << win.kernel << " " << win.block << " " << win.chunk << " " << win.tile << " 0 " << win.window
          << " " << b->chains << "\n";
    }
    return lms_batch_get_config(b, kernel, block, chunk, tile, ctas_per_sm);
}

int lms_batch_smooth(lms_batch b, int32_t iters) {
    if (!b || iters < 0) return LMS_ERR_ARG;
    if (iters == 0) return LMS_OK;
    if (!b->configured) LMS_TRY(lms_batch_autotune(b, nullptr, nullptr, nullptr, nullptr, nullptr));
    LMS_TRY(ensure_queue(b, iters));
    const int base = b->cur;
    std::string key = std::to_string(iters) + "/" + std::to_string(base) + "/" + std::to_string(b->chains);
    cudaGraphExec_t exec;
    int64_t kernels = 0;
    auto it = b->graphs.execs.find(key);
    if (it != b->graphs.execs.end()) {
        exec = it->second;
        kernels = b->graphs.kernels[key];
    } else {
        const int grid = batch_grid(b);
        // The batch as parallel chains of sweeps in one graph, one per run of whole meshes with about
        // equal vertex counts: the meshes are independent, so the tail of one chain's sweep overlaps the
        // other chains' work (b->chains, picked by the autotuner; two chains gave 4% faster sweeps than one
        // on the 512-mesh batch).  SELL tiles are not ordered by mesh: one chain.
        const int chains = (b->kernel == LMS_KERNEL_SELL) ? 1 : std::max(1, std::min<int>(b->chains, b->k));
        std::vector<int32_t> cut(chains + 1, b->n_items);  // chain c: tiles [cut[c], cut[c+1])
        {
            const int tile = b->items_tile;
            int32_t tiles = 0, m = 0;
            cut[0] = 0;
            for (int c = 1; c < chains; ++c) {
                const int64_t goal = b->n_total * c / chains;
                do {  // at least one mesh per chain, and leave one for each chain after this one
                    tiles += int32_t((b->voff[m + 1] - b->voff[m] + tile - 1) / tile);
                    ++m;
                } while (m < b->k - (chains - c) && b->voff[m] < goal);
                cut[c] = tiles;
            }
        }
        if (chains > 1 && !b->ev_fork) LMS_CUDA(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
        while (int(b->cap_extra.size()) < chains - 1) {
            cudaStream_t st;
            cudaEvent_t ev;
            LMS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            LMS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            b->cap_extra.push_back(st);
            b->ev_extra.push_back(ev);
        }
        LMS_TRY(ensure_queue(b, chains * iters));
        LMS_TRY(capture(
            b->cap,
            [&](cudaStream_t cs) -> int {
                LMS_CUDA(cudaMemsetAsync(b->d_queue, 0, sizeof(int32_t) * chains * iters, cs));
                if (chains == 1) {
                    for (int32_t i = 0; i < iters; ++i) {
                        const int src = (base + i) & 1;
                        LMS_TRY(batch_issue(b, src, src ^ 1, i, grid, cs));
                    }
                    return LMS_OK;
                }
                LMS_CUDA(cudaEventRecord(b->ev_fork, cs));
                for (int c = 1; c < chains; ++c) LMS_CUDA(cudaStreamWaitEvent(b->cap_extra[c - 1], b->ev_fork, 0));
                for (int32_t i = 0; i < iters; ++i) {
                    const int src = (base + i) & 1;
                    for (int c = 0; c < chains; ++c)
                        LMS_TRY(batch_issue_range(b, src, src ^ 1, c * iters + i, grid,
                                                  c == 0 ? cs : b->cap_extra[c - 1], cut[c], cut[c + 1]));
                }
                for (int c = 1; c < chains; ++c) {
                    LMS_CUDA(cudaEventRecord(b->ev_extra[c - 1], b->cap_extra[c - 1]));
                    LMS_CUDA(cudaStreamWaitEvent(cs, b->ev_extra[c - 1], 0));
                }
                return LMS_OK;
            },
            &exec, &kernels));
        b->graphs.execs[key] = exec;
        b->graphs.kernels[key] = kernels;
    }
    LMS_CUDA(cudaGraphLaunch(exec, b->stream));
    b->last_launches = kernels;
    b->cur = (base + iters) & 1;
    return LMS_OK;
}

int batch_check_err(lms_batch_s* b) {
    int32_t err[2] = {0, 0};
    LMS_CUDA(cudaMemcpyAsync(err, b->d_err, sizeof(err), cudaMemcpyDeviceToHost, b->stream));
    LMS_CUDA(cudaStreamSynchronize(b->stream));
    if (err[0]) {
        lms::set_error_detail("a bounded wait on a tile copy expired");
        return LMS_ERR_TIMEOUT;
    }
    if (err[1]) {
        lms::set_error_detail("the last coordinates passed in contain a value that is not finite");
        return LMS_ERR_ARG;
    }
    return LMS_OK;
}

int lms_batch_get_all_coords(lms_batch b, double* xy) {
    if (!b || !xy) return LMS_ERR_ARG;
    cudaStream_t s = b->stream;
    LMS_TRY(check_launch(lms::launch_batch_store_xy(b->n_items, b->d_items, b->d_item_mesh, b->d_perm, b->d_xy[b->cur],
                                                    b->d_xy64, b->d_cs, b->d_bits, b->d_fixed, s),
                         "batch_store_xy"));
    LMS_CUDA(cudaMemcpyAsync(xy, b->d_xy64, 16 * size_t(b->n_total), cudaMemcpyDeviceToHost, s));
    LMS_CUDA(cudaStreamSynchronize(s));
    return batch_check_err(b);
}

int lms_batch_get_coords(lms_batch b, int32_t mesh, double* xy) {
    if (!b || !xy || mesh < 0 || mesh >= b->k) return LMS_ERR_ARG;
    cudaStream_t s = b->stream;
    LMS_TRY(check_launch(lms::launch_batch_store_xy(b->n_items, b->d_items, b->d_item_mesh, b->d_perm, b->d_xy[b->cur],
                                                    b->d_xy64, b->d_cs, b->d_bits, b->d_fixed, s),
                         "batch_store_xy"));
    const int64_t v0 = b->voff[mesh], nv = b->voff[mesh + 1] - v0;
    LMS_CUDA(cudaMemcpyAsync(xy, b->d_xy64 + 2 * v0, 16 * size_t(nv), cudaMemcpyDeviceToHost, s));
    LMS_CUDA(cudaStreamSynchronize(s));
    return batch_check_err(b);
}

int lms_batch_set_all_coords(lms_batch b, const double* xy) {
    if (!b || !xy) return LMS_ERR_ARG;
    cudaStream_t s = b->stream;
    // the input lands in d_fixed (it also serves the boundary values on output); finiteness is checked
    // by the load kernel and reported by the next call that returns host data
    LMS_CUDA(cudaMemsetAsync(b->d_err + 1, 0, sizeof(int32_t), s));
    LMS_CUDA(cudaMemcpyAsync(b->d_fixed, xy, 16 * size_t(b->n_total), cudaMemcpyHostToDevice, s));
    LMS_TRY(check_launch(lms::launch_batch_load_xy(b->n_items, b->d_items, b->d_item_mesh, b->d_perm, b->d_fixed,
                                                   b->d_xy[0], b->d_xy[1], b->d_cs, b->d_err + 1, s),
                         "batch_load_xy"));
    b->cur = 0;
    return LMS_OK;
}

int lms_batch_run(lms_batch b, const double* xy_in, double* xy_out, int32_t iters, int32_t groups) {
    if (!b || !xy_in || !xy_out || iters < 0 || groups < 1 || groups > b->k) return LMS_ERR_ARG;
    if (!b->configured) LMS_TRY(lms_batch_autotune(b, nullptr, nullptr, nullptr, nullptr, nullptr));
    if (b->kernel == LMS_KERNEL_SELL) groups = 1;  // SELL tiles are not ordered by mesh
    cudaStream_t s = b->stream;
    if (!b->s_in) {
        LMS_CUDA(cudaStreamCreateWithFlags(&b->s_in, cudaStreamNonBlocking));
        LMS_CUDA(cudaStreamCreateWithFlags(&b->s_out, cudaStreamNonBlocking));
        LMS_CUDA(cudaStreamCreateWithFlags(&b->s_c2, cudaStreamNonBlocking));
        LMS_CUDA(cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming));
        LMS_CUDA(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming));
    }
    while (int32_t(b->ev_in.size()) < groups) {
        cudaEvent_t e0, e1;
        LMS_CUDA(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming));
        LMS_CUDA(cudaEventCreateWithFlags(&e1, cudaEventDisableTiming));
        b->ev_in.push_back(e0);
        b->ev_done.push_back(e1);
    }
    // groups of whole meshes with about equal vertex counts, as tile ranges [it[g], it[g+1]) and vertex
    // ranges [vt[g], vt[g+1])
    std::vector<int32_t> it(groups + 1, b->n_items);
    std::vector<int64_t> vt(groups + 1, b->n_total);
    {
        std::vector<int32_t> first_tile(b->k + 1, 0);
        const int tile = b->items_tile;
        for (int32_t m = 0; m < b->k; ++m)
            first_tile[m + 1] = first_tile[m] + int32_t((b->voff[m + 1] - b->voff[m] + tile - 1) / tile);
        // Group sizes ramp up and down by a factor of 4 (1, 4, 16, ..., 16, 4, 1): only the first
        // group's input copy and the last group's output copy are exposed, and every other copy hides
        // behind the sweeps of a neighbouring group at least a quarter of its size (a sweep pass over
        // a vertex takes several times longer than copying it).  Group g starts at the first mesh at or
        // past its share of the vertices, keeping at least one mesh for each group.
        std::vector<double> cum(groups + 1, 0.0);
        for (int32_t g = 0; g < groups; ++g)
            cum[g + 1] = cum[g] + std::pow(4.0, double(std::min(g, groups - 1 - g)));
        int32_t mb = 0;
        for (int32_t g = 0; g < groups; ++g) {
            if (g > 0) {
                const int64_t goal = int64_t(double(b->n_total) * cum[g] / cum[groups]);
                ++mb;
                while (mb < b->k - (groups - g) && b->voff[mb] < goal) ++mb;
            }
            it[g] = first_tile[mb];
            vt[g] = b->voff[mb];
        }
    }
    const int32_t slots = groups * std::max(iters, 1);
    LMS_TRY(ensure_queue(b, slots));
    const int grid = batch_grid(b);
    const int fin = iters & 1;
    // earlier work on the caller's stream (which may read d_fixed) comes first
    LMS_CUDA(cudaMemsetAsync(b->d_err + 1, 0, sizeof(int32_t), s));
    LMS_CUDA(cudaEventRecord(b->ev_start, s));
    LMS_CUDA(cudaStreamWaitEvent(b->s_in, b->ev_start, 0));
    LMS_CUDA(cudaStreamWaitEvent(b->s_c2, b->ev_start, 0));
    for (int32_t g = 0; g < groups; ++g) {
        const int64_t v0 = vt[g], nv = vt[g + 1] - vt[g];
        LMS_CUDA(cudaMemcpyAsync(b->d_fixed + 2 * v0, xy_in + 2 * v0, 16 * size_t(nv), cudaMemcpyHostToDevice, b->s_in));
        LMS_CUDA(cudaEventRecord(b->ev_in[g], b->s_in));
    }
    int64_t kernels_total = 0;
    for (int32_t g = 0; g < groups; ++g) {
        const int32_t i0 = it[g], i1 = it[g + 1];
        const std::string key = "run/" + std::to_string(g) + "/" + std::to_string(groups) + "/" + std::to_string(iters);
        cudaGraphExec_t exec;
        int64_t kernels = 0;
        auto found = b->graphs.execs.find(key);
        if (found != b->graphs.execs.end()) {
            exec = found->second;
            kernels = b->graphs.kernels[key];
        } else {
            LMS_TRY(capture(
                b->cap,
                [&](cudaStream_t cs) -> int {
                    const int32_t q0 = g * std::max(iters, 1);
                    LMS_CUDA(cudaMemsetAsync(b->d_queue + q0, 0, sizeof(int32_t) * std::max(iters, 1), cs));
                    LMS_TRY(check_launch(lms::launch_batch_load_xy(i1 - i0, b->d_items + i0, b->d_item_mesh + i0,
                                                                   b->d_perm, b->d_fixed, b->d_xy[0], b->d_xy[1],
                                                                   b->d_cs, b->d_err + 1, cs),
                                         "batch_load_xy"));
                    for (int32_t k = 0; k < iters; ++k)
                        LMS_TRY(batch_issue_range(b, k & 1, (k & 1) ^ 1, q0 + k, grid, cs, i0, i1));
                    return check_launch(lms::launch_batch_store_xy(i1 - i0, b->d_items + i0, b->d_item_mesh + i0,
                                                                   b->d_perm, b->d_xy[fin], b->d_xy64, b->d_cs,
                                                                   b->d_bits, b->d_fixed, cs),
                                        "batch_store_xy");
                },
                &exec, &kernels));
            b->graphs.execs[key] = exec;
            b->graphs.kernels[key] = kernels;
        }
        // groups alternate between two compute streams, so the tail of one group's sweeps overlaps the
        // next group's (their meshes, tiles and queue counters are disjoint)
        cudaStream_t cs = (g & 1) ? b->s_c2 : s;
        LMS_CUDA(cudaStreamWaitEvent(cs, b->ev_in[g], 0));
        LMS_CUDA(cudaGraphLaunch(exec, cs));
        LMS_CUDA(cudaEventRecord(b->ev_done[g], cs));
        LMS_CUDA(cudaStreamWaitEvent(b->s_out, b->ev_done[g], 0));
        const int64_t v0 = vt[g], nv = vt[g + 1] - vt[g];
        LMS_CUDA(cudaMemcpyAsync(xy_out + 2 * v0, b->d_xy64 + 2 * v0, 16 * size_t(nv), cudaMemcpyDeviceToHost, b->s_out));
        kernels_total += kernels;
    }
    LMS_CUDA(cudaEventRecord(b->ev_join, b->s_out));
    LMS_CUDA(cudaStreamWaitEvent(s, b->ev_join, 0));  // later calls on the caller's stream see every group
    LMS_CUDA(cudaStreamSynchronize(b->s_out));
    b->last_launches = kernels_total;
    b->cur = fin;
    return batch_check_err(b);
}

int lms_batch_info(lms_batch b, int64_t* n_total, int64_t* n_interior, int64_t* nnz_total, int32_t* n_tiles) {
    if (!b) return LMS_ERR_ARG;
    if (n_total) *n_total = b->n_total;
    if (n_interior) *n_interior = b->n_int;
    if (nnz_total) *nnz_total = b->nnz_total;
    if (n_tiles) *n_tiles = b->n_items;
    return LMS_OK;
}

int lms_batch_last_launches(lms_batch b, int64_t* launches) {
    if (!b || !launches) return LMS_ERR_ARG;
    *launches = b->last_launches;
    return LMS_OK;
}

int lms_batch_set_chains(lms_batch b, int32_t chains) {
    if (!b || chains < 1 || chains > 8) return LMS_ERR_ARG;
    b->chains = chains;
    return LMS_OK;
}

int lms_batch_get_chains(lms_batch b, int32_t* chains) {
    if (!b || !chains) return LMS_ERR_ARG;
    *chains = b->chains;
    return LMS_OK;
}

int lms_batch_set_layout(lms_batch b, int32_t window) {
    if (!b || window < 0 || window > 65536 || (window % 32) != 0) return LMS_ERR_ARG;
    return batch_relayout(b, window);
}

int lms_batch_get_layout(lms_batch b, int32_t* window) {
    if (!b || !window) return LMS_ERR_ARG;
    *window = b->window;
    return LMS_OK;
}

int lms_batch_get_permutation(lms_batch b, int32_t mesh, int32_t* new_to_old) {
    if (!b || !new_to_old || mesh < 0 || mesh >= b->k) return LMS_ERR_ARG;
    const int64_t v0 = b->voff[mesh], nv = b->voff[mesh + 1] - v0;
    for (int64_t i = 0; i < nv; ++i) new_to_old[i] = int32_t(b->order_perm[v0 + i] - v0);
    return LMS_OK;
}

void lms_batch_destroy(lms_batch b) { delete b; }

}  // extern "C"
