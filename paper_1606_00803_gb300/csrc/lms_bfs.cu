// lms_bfs.cu - breadth-first vertex ordering on the device, equal to the host
// (sequential) search position for position.
//
// The sequential search (Section 5.2.1's BFS ordering, read as: start at
// vertex 0, append unvisited neighbours in ascending id, restart at the
// smallest unvisited id when the queue runs dry) builds its queue level by
// level.  A vertex u of level L+1 is appended by the first vertex of level L,
// in queue order, that is adjacent to it, and the children of one vertex are
// appended in ascending id.  So level L+1 in queue order is the set of new
// vertices sorted by (queue position of that first neighbour, id), which a
// level-synchronous search computes in three data-parallel phases per level:
//   1. expand - every frontier vertex at position i lowers parent[u] to i for
//      each unvisited neighbour u (atomicMin; the minimum is the first
//      neighbour in queue order);
//   2. count  - frontier position i owns the neighbours u with parent[u] == i;
//      an exclusive scan of the counts over the frontier gives each owner its
//      output range;
//   3. place  - each owner writes its children in ascending id.
//
// One thread-block cluster runs the search of one graph; the CTAs of a
// cluster split every frontier into contiguous blocks, meet at the hardware
// cluster barrier between phases, and read each other's scan totals from
// distributed shared memory.  Several graphs (a batch of meshes) run as
// independent clusters.  Frontier data written by one CTA and read by another
// go through L2 (st.global + ld.global.cg after a release/acquire cluster
// barrier), never through a possibly stale L1 line.
#include <math_constants.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "lms_device.cuh"
#include "lms_internal.h"

namespace lms {

namespace {

constexpr int kBfsThreads = 512;
constexpr int kBfsFastDeg = 16;  // rows up to this length are handled in registers

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_index() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_count() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}

// every thread of every CTA of the cluster; orders prior memory accesses before later ones
__device__ __forceinline__ void cluster_barrier() {
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n\t"
        "barrier.cluster.wait.acquire.aligned;" ::
            : "memory");
}

// the int32 at shared address p of CTA `rank` of this cluster
__device__ __forceinline__ int32_t load_remote(const int32_t* p, uint32_t rank) {
    const uint32_t local = static_cast<uint32_t>(__cvta_generic_to_shared(p));
    uint32_t remote;
    int32_t v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(remote) : "memory");
    return v;
}

// Block-wide exclusive prefix sum of x; *total receives the block's sum.  Uses s_warp[32].
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t x, int32_t* s_warp, int32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int32_t inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < nwarps ? s_warp[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        s_warp[lane] = w;  // inclusive prefix over warps
    }
    __syncthreads();
    const int32_t before_warp = warp > 0 ? s_warp[warp - 1] : 0;
    *total = s_warp[nwarps - 1];
    __syncthreads();  // s_warp may be reused right after
    return before_warp + inc - x;
}

__device__ __forceinline__ int32_t block_min(int32_t x, int32_t* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, d));
    if (lane == 0) s_warp[warp] = x;
    __syncthreads();
    int32_t r = INT_MAX;
    for (int w = 0; w < nwarps; ++w) r = min(r, s_warp[w]);
    __syncthreads();
    return r;
}

// Children of the frontier vertex w at position i (neighbours u with parent[u] == i), for a row of
// at most kBfsFastDeg entries: ids and flags in registers.
struct FastRow {
    int32_t u[kBfsFastDeg];
    uint32_t child;  // bit k: entry k is a child
};

__device__ __forceinline__ void load_fast_row(const BfsArgs& a, int32_t e0, int32_t deg, int32_t i, FastRow& r) {
    r.child = 0u;
#pragma unroll
    for (int k = 0; k < kBfsFastDeg; ++k) {
        r.u[k] = k < deg ? __ldg(a.col_idx + e0 + k) : -1;
        if (r.u[k] >= 0 && !LMS_CHECK(r.u[k] < a.n_total)) r.u[k] = -1;
    }
#pragma unroll
    for (int k = 0; k < kBfsFastDeg; ++k)
        if (r.u[k] >= 0 && __ldcg(a.parent + r.u[k]) == i) r.child |= 1u << k;
}

__global__ void __launch_bounds__(kBfsThreads) k_bfs(BfsArgs a) {
    __shared__ int32_t s_warp[32];
    __shared__ int32_t s_value;  // this CTA's contribution to a cluster-wide sum or minimum
    const uint32_t rank = cluster_rank(), csize = cluster_size();
    const int32_t nthreads = static_cast<int32_t>(csize * blockDim.x);
    const int32_t tid = static_cast<int32_t>(rank * blockDim.x + threadIdx.x);

    for (int32_t g = static_cast<int32_t>(cluster_index()); g < a.k; g += static_cast<int32_t>(cluster_count())) {
        const int32_t v0 = a.voff ? a.voff[g] : 0;
        const int32_t n = a.voff ? a.voff[g + 1] - v0 : a.n_total;
        for (int32_t i = tid; i < n; i += nthreads) {
            a.pos[v0 + i] = -1;
            a.parent[v0 + i] = INT_MAX;
        }
        cluster_barrier();
        int32_t placed = 0, fa = 0, cursor = 0;  // frontier = positions [fa, placed)
        while (placed < n) {
            if (fa == placed) {
                // queue ran dry: the next root is the smallest unplaced id
                int32_t root = INT_MAX;
                while (root == INT_MAX) {
                    const int32_t idx = cursor + tid;
                    const int32_t cand = idx < n && __ldcg(a.pos + v0 + idx) < 0 ? idx : INT_MAX;
                    const int32_t m = block_min(cand, s_warp);
                    if (threadIdx.x == 0) s_value = m;
                    cluster_barrier();
                    for (uint32_t r = 0; r < csize; ++r) root = min(root, load_remote(&s_value, r));
                    cluster_barrier();  // every CTA has read s_value
                    cursor += nthreads;
                }
                if (tid == 0) {
                    a.out[v0 + placed] = v0 + root;
                    a.pos[v0 + root] = placed;
                }
                cursor = root + 1;  // every id below root is placed
                ++placed;
                cluster_barrier();
            }
            const int32_t fb = placed;
            // phase 1: expand
            for (int32_t i = fa + tid; i < fb; i += nthreads) {
                const int32_t w = __ldcg(a.out + v0 + i);
                const int32_t e1 = __ldg(a.row_ptr + w + 1);
                for (int32_t e = __ldg(a.row_ptr + w); e < e1; ++e) {
                    const int32_t u = __ldg(a.col_idx + e);
                    if (!LMS_CHECK(u >= 0 && u < a.n_total)) continue;
                    if (__ldcg(a.pos + u) < 0) atomicMin(a.parent + u, i);
                }
            }
            cluster_barrier();
            // phase 2: count children over a contiguous block of the frontier per thread
            const int32_t F = fb - fa;
            const int32_t per = (F + nthreads - 1) / nthreads;
            const int32_t ia = min(fb, fa + tid * per), ib = min(fb, ia + per);
            int32_t cnt = 0;
            for (int32_t i = ia; i < ib; ++i) {
                const int32_t w = __ldcg(a.out + v0 + i);
                const int32_t e0 = __ldg(a.row_ptr + w), deg = __ldg(a.row_ptr + w + 1) - e0;
                if (deg <= kBfsFastDeg) {
                    FastRow r;
                    load_fast_row(a, e0, deg, i, r);
                    cnt += __popc(r.child);
                } else {
                    for (int32_t e = e0; e < e0 + deg; ++e) {
                        const int32_t u = __ldg(a.col_idx + e);
                        if (LMS_CHECK(u >= 0 && u < a.n_total)) cnt += __ldcg(a.parent + u) == i;
                    }
                }
            }
            int32_t cta_total = 0;
            const int32_t off_in_cta = block_exclusive_scan(cnt, s_warp, &cta_total);
            if (threadIdx.x == 0) s_value = cta_total;
            cluster_barrier();
            int32_t cta_off = 0, total = 0;
            for (uint32_t r = 0; r < csize; ++r) {
                const int32_t t = load_remote(&s_value, r);
                if (r < rank) cta_off += t;
                total += t;
            }
            // phase 3: place the children of each owned position in ascending id
            int32_t o = fb + cta_off + off_in_cta;
            for (int32_t i = ia; i < ib; ++i) {
                const int32_t w = __ldcg(a.out + v0 + i);
                const int32_t e0 = __ldg(a.row_ptr + w), deg = __ldg(a.row_ptr + w + 1) - e0;
                if (deg <= kBfsFastDeg) {
                    FastRow r;
                    load_fast_row(a, e0, deg, i, r);
#pragma unroll
                    for (int k = 0; k < kBfsFastDeg; ++k) {
                        if (!((r.child >> k) & 1u)) continue;
                        int32_t below = 0;
#pragma unroll
                        for (int j = 0; j < kBfsFastDeg; ++j) below += ((r.child >> j) & 1u) && r.u[j] < r.u[k];
                        a.out[v0 + o + below] = r.u[k];
                        a.pos[r.u[k]] = o + below;
                    }
                    o += __popc(r.child);
                } else {
                    int32_t c = 0;
                    for (int32_t e = e0; e < e0 + deg; ++e) {
                        const int32_t u = __ldg(a.col_idx + e);
                        if (!LMS_CHECK(u >= 0 && u < a.n_total) || __ldcg(a.parent + u) != i) continue;
                        int32_t below = 0;
                        for (int32_t f = e0; f < e0 + deg; ++f) {
                            const int32_t x = __ldg(a.col_idx + f);
                            below += x >= 0 && x < a.n_total && x < u && __ldcg(a.parent + x) == i;
                        }
                        a.out[v0 + o + below] = u;
                        a.pos[u] = o + below;
                        ++c;
                    }
                    o += c;
                }
            }
            cluster_barrier();  // placements visible; every CTA has read s_value
            fa = fb;
            placed = fb + total;
        }
    }
}

// ------------------------------------------------------------------ block RDR

constexpr int kBrdrThreads = 512;
constexpr int kBrdrMaxDeg = 64;  // rows of the walk are sorted in a per-thread array of this size

__device__ __forceinline__ bool key_greater(double qa, int32_t ia, double qb, int32_t ib) {
    return qa > qb || (qa == qb && ia > ib);
}

// Ascending sort of `count` (key, id) pairs in shared memory (bitonic network over `cap`, a power of
// two >= count; slots past count hold (+inf, INT_MAX) and stay last).
__device__ void sort_keys(double* kq, int32_t* kid, int32_t count, int32_t cap) {
    for (int32_t i = count + threadIdx.x; i < cap; i += blockDim.x) {
        kq[i] = CUDART_INF;
        kid[i] = INT_MAX;
    }
    __syncthreads();
    for (int32_t k = 2; k <= cap; k <<= 1)
        for (int32_t j = k >> 1; j > 0; j >>= 1) {
            for (int32_t i = threadIdx.x; i < cap; i += blockDim.x) {
                const int32_t p = i ^ j;
                if (p <= i) continue;
                const bool up = (i & k) == 0;
                if (key_greater(kq[i], kid[i], kq[p], kid[p]) == up) {
                    const double tq = kq[i];
                    kq[i] = kq[p];
                    kq[p] = tq;
                    const int32_t ti = kid[i];
                    kid[i] = kid[p];
                    kid[p] = ti;
                }
            }
            __syncthreads();
        }
}

// One CTA per block of BFS positions [start, end) of graph g (vertices from v0): Algorithm 2 on the
// block's own subgraph.  The block's interior vertices are sorted by (quality, id) in shared memory; one
// thread walks (flags in shared memory, indexed by BFS position within the block); the members no walk
// reached are sorted by id and appended.
__global__ void __launch_bounds__(kBrdrThreads) k_block_rdr(BrdrArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    double* kq = reinterpret_cast<double*>(smem);
    int32_t* kid = reinterpret_cast<int32_t*>(kq + a.cap);
    uint8_t* done = reinterpret_cast<uint8_t*>(kid + a.cap);
    uint8_t* placed = done + a.cap;
    __shared__ int32_t s_count, s_placed;
    for (int32_t b = blockIdx.x; b < a.n_blocks; b += gridDim.x) {
        const int4 blk = a.blocks[b];  // (v0, start, end, unused)
        const int32_t v0 = blk.x, start = blk.y, len = blk.z - blk.y;
        const int32_t* members = a.bfs + v0 + start;
        int32_t* out = a.out + v0 + start;
        if (threadIdx.x == 0) s_count = 0;
        for (int32_t i = threadIdx.x; i < len; i += blockDim.x) {
            done[i] = 0;
            placed[i] = 0;
        }
        __syncthreads();
        for (int32_t i = threadIdx.x; i < len; i += blockDim.x) {
            const int32_t v = members[i];
            if (!a.is_boundary[v]) {
                const int32_t k = atomicAdd(&s_count, 1);
                kq[k] = a.q[v];
                kid[k] = v;
            }
        }
        __syncthreads();
        sort_keys(kq, kid, s_count, a.cap);
        if (threadIdx.x == 0) {
            int32_t cnt = 0;
            int32_t l[kBrdrMaxDeg];
            double lq[kBrdrMaxDeg];
            auto local = [&](int32_t u) { return a.bfs_pos[u] - start; };  // position within the block
            auto place = [&](int32_t u, int32_t lu) {
                if (!placed[lu]) {
                    placed[lu] = 1;
                    out[cnt++] = u;
                }
            };
            // l <- unprocessed neighbours of w inside the block, by increasing (quality, id)
            auto gather = [&](int32_t w) {
                int32_t m = 0;
                for (int32_t e = a.row_ptr[w]; e < a.row_ptr[w + 1]; ++e) {
                    const int32_t u = a.col_idx[e];
                    if (!LMS_CHECK(u >= 0 && u < a.n_total)) continue;
                    const int32_t lu = local(u);
                    if (lu < 0 || lu >= len || done[lu]) continue;
                    const double qu = a.q[u];
                    int32_t k = m++;
                    while (k > 0 && key_greater(lq[k - 1], l[k - 1], qu, u)) {
                        l[k] = l[k - 1];
                        lq[k] = lq[k - 1];
                        --k;
                    }
                    l[k] = u;
                    lq[k] = qu;
                }
                return m;
            };
            const int32_t seeds = s_count;
            for (int32_t si = 0; si < seeds; ++si) {
                const int32_t sd = kid[si];
                const int32_t ls = local(sd);
                if (done[ls]) continue;
                place(sd, ls);
                done[ls] = 1;
                int32_t m = gather(sd);
                while (m > 0) {
                    for (int32_t k = 0; k < m; ++k) place(l[k], local(l[k]));
                    const int32_t w = l[0];
                    done[local(w)] = 1;
                    m = gather(w);
                }
            }
            s_placed = cnt;
            s_count = 0;
        }
        __syncthreads();
        // members no walk reached, ascending id
        for (int32_t i = threadIdx.x; i < len; i += blockDim.x)
            if (!placed[i]) {
                const int32_t k = atomicAdd(&s_count, 1);
                kq[k] = 0.0;
                kid[k] = members[i];
            }
        __syncthreads();
        const int32_t rest = s_count;
        sort_keys(kq, kid, rest, a.cap);
        for (int32_t k = threadIdx.x; k < rest; k += blockDim.x) out[s_placed + k] = kid[k];
        __syncthreads();
    }
}

}  // namespace

LMS_CHECK_ACCESSOR(check_violations_orderings)

size_t block_rdr_smem(int32_t cap) { return size_t(cap) * (8 + 4 + 2); }

cudaError_t launch_block_rdr(const BrdrArgs& a, int sms, cudaStream_t stream) {
    if (a.n_blocks <= 0) return cudaSuccess;
    const size_t smem = block_rdr_smem(a.cap);
    cudaError_t e = cudaFuncSetAttribute(k_block_rdr, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_block_rdr, kBrdrThreads, smem);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(a.n_blocks, std::max(1, per_sm) * sms));
    k_block_rdr<<<grid, kBrdrThreads, smem, stream>>>(a);
    return cudaGetLastError();
}

int block_rdr_max_degree() { return kBrdrMaxDeg; }

int bfs_cluster_size(int32_t max_graph_vertices) {
    // one CTA per small graph; a large graph gets a cluster of 8 CTAs
    return max_graph_vertices > (1 << 16) ? 8 : 1;
}

cudaError_t launch_bfs(const BfsArgs& a, int cluster, cudaStream_t stream) {
    if (a.k <= 0) return cudaSuccess;
    if (cluster != 1 && cluster != 2 && cluster != 4 && cluster != 8) return cudaErrorInvalidValue;
    // one cluster per graph: clusters never wait on one another, so they need not be co-resident
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(a.k) * static_cast<unsigned>(cluster));
    cfg.blockDim = dim3(kBfsThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(cluster);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_bfs, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace lms
