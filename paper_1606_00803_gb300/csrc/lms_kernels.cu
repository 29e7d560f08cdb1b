// lms_kernels.cu - sm_103a kernels of liblms.
//
// The hot loop is Eq. 1 of Aupy, Park & Raghavan, "Locality-Aware Laplacian
// Mesh Smoothing": every interior vertex moves to the mean of its mesh
// neighbours.  It is a sparse CSR gather (no dense contraction, so no tensor
// cores): per interior vertex the sweep streams its row offset and its
// neighbour ids, gathers the neighbours' positions (mostly L1/L2 hits when the
// ordering keeps neighbours close in memory - the point of BFS and RDR) and
// writes one position.
//
// Arithmetic contracts (all explicit _rn intrinsics, so no FMA contraction
// changes a result):
//   FP64  sums run left to right over the stored row starting from 0.0, and
//         the mean is the correctly rounded quotient; results equal the
//         sequential FP64 evaluation of Eq. 1 bit for bit.  The quotient by the
//         neighbour count d uses y = RN(1/d) from a table, q = RN(s*y) and one
//         correction RN(q + RN(s - d*q)*y) (Markstein's division refinement,
//         IBM J. Res. Dev. 34(1), 1990); it is checked against IEEE division by
//         the division self-test.  GB300 runs FP64 at ~1/64 of the FP32 rate,
//         and this is ~3 FP64 operations instead of a full division.
//   FP32  coordinates are relative to the bounding-box centre and scaled to
//         unit size; neighbour sums are Kahan-compensated and the mean is the
//         compensated sum divided by the count, correctly rounded (the same
//         refinement of a rounded reciprocal as FP64); quality sums are reduced
//         in FP64.
#include <algorithm>
#include <cfloat>
#include <cstdint>
#include <type_traits>

#include "lms_device.cuh"
#include "lms_fp64_int.cuh"
#include "lms_internal.h"

namespace lms {

namespace {
using namespace dev;



// FP64 sums of Eq. 1: where each add runs (LMS_FP64_ARITH_*).  The first term needs no add: 0.0 + x is x
// with -0 made +0.  The mixed modes send the add of row position j to the integer pipes when j is a
// multiple of 2 (or 3) and to the FP64 unit otherwise, so both run at once; j is the same for every lane
// of a warp at each step, so the choice never diverges.
template <int ARITH>
__device__ __forceinline__ bool int_add_at(int32_t j) {
    if constexpr (ARITH == LMS_FP64_ARITH_FPU) return false;
    else if constexpr (ARITH == LMS_FP64_ARITH_MIXED2) return (j & 1) == 0;
    else if constexpr (ARITH == LMS_FP64_ARITH_MIXED3) return j % 3 == 0;
    else return true;
}

template <int ARITH>
__device__ __forceinline__ void sum_fp64(double& sx, double& sy, double2 p, int32_t j) {
    if (j == 0) {
        sx = plus_zero(p.x);
        sy = plus_zero(p.y);
    } else if (int_add_at<ARITH>(j)) {
        sx = add_rn_int(sx, p.x);
        sy = add_rn_int(sy, p.y);
    } else {
        sx = __dadd_rn(sx, p.x);
        sy = __dadd_rn(sy, p.y);
    }
}

// The FP64 mean s / d: on the integer pipes (LMS_FP64_ARITH_INT and the mixed modes) unless d exceeds the
// table or the sum or
// the quotient is zero or subnormal, else the table-driven FP64 division (itself IEEE division for tiny
// sums).
template <int ARITH>
__device__ __forceinline__ double mean_fp64(double s, int32_t d, const double* recip, const uint32_t* magic) {
    if constexpr (ARITH == LMS_FP64_ARITH_INT || ARITH == LMS_FP64_ARITH_MIXED2 || ARITH == LMS_FP64_ARITH_MIXED3) {
        double q;
        if (d <= kMaxRecipDeg && div_rn_int(s, d, magic, &q)) return q;
    }
    return div_by_count(s, d, recip);
}

// Eq. 1 for one vertex.  FP64 reads the row kChunk entries at a time - all neighbour ids, then all
// position gathers, then the sums in row order - so a thread keeps kChunk loads in flight while its FP64
// adds (1/64 of the FP32 rate on GB300) drain; FP32, issue-bound rather than latency-bound, reads one
// entry at a time.  FP64: sequential sums (sum_fp64) and the correctly rounded division (bit-identical to
// the sequential evaluation); FP32: Kahan sums.  Returns the squared displacement when asked.
template <bool FP64, bool IN_PLACE, int ARITH>
__device__ __forceinline__ double smooth_vertex(const SweepArgs& a, int32_t v, const double* recip,
                                                const uint32_t* magic, bool want_disp) {
    constexpr int kChunk = FP64 ? 4 : 1;
    using V = typename std::conditional<FP64, double2, float2>::type;
    const V* src = static_cast<const V*>(a.src);
    V* dst = static_cast<V*>(a.dst);
    const int32_t e0 = __ldg(a.row_ptr + v), e1 = __ldg(a.row_ptr + v + 1);
    // the old position for the displacement, loaded first so that its latency overlaps the gathers (in an
    // in-place colour pass its line is being written by the pass; loaded last it stalled the warp)
    V o{};
    if (want_disp) o = src[v];
    double dx_ = 0.0, dy_ = 0.0;  // FP64 sums
    float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;  // FP32 Kahan sums
    for (int32_t e = e0; e < e1; e += kChunk) {
        int32_t u[kChunk];
        V p[kChunk];
#pragma unroll
        for (int g = 0; g < kChunk; ++g) {
            u[g] = e + g < e1 ? __ldg(a.col_idx + e + g) : -1;
            if (u[g] >= 0 && !LMS_CHECK(u[g] < a.n_vertices)) u[g] = -1;
        }
#pragma unroll
        for (int g = 0; g < kChunk; ++g)
            if (u[g] >= 0) p[g] = IN_PLACE ? src[u[g]] : __ldg(src + u[g]);
#pragma unroll
        for (int g = 0; g < kChunk; ++g)
            if (u[g] >= 0) {
                if constexpr (FP64) {
                    sum_fp64<ARITH>(dx_, dy_, p[g], e + g - e0);
                } else {
                    kahan_add(sx, cx, p[g].x);
                    kahan_add(sy, cy, p[g].y);
                }
            }
    }
    V r;
    if constexpr (FP64) {
        r.x = mean_fp64<ARITH>(dx_, e1 - e0, recip, magic);
        r.y = mean_fp64<ARITH>(dy_, e1 - e0, recip, magic);
    } else {
        r.x = mean_f32(sx, cx, e1 - e0);
        r.y = mean_f32(sy, cy, e1 - e0);
    }
    double d2 = 0.0;
    if (want_disp) {
        const double ex = static_cast<double>(r.x) - static_cast<double>(o.x);
        const double ey = static_cast<double>(r.y) - static_cast<double>(o.y);
        d2 = __fma_rn(ex, ex, __dmul_rn(ey, ey));
    }
    dst[v] = r;
    return d2;
}

// One thread per vertex over [v_begin, v_end).  Jacobi: src != dst, boundary vertices skipped
// (both ping-pong buffers hold them).  Coloured GS: src == dst, every vertex of the range is
// interior and of one colour, so no two threads touch neighbouring vertices.
template <bool FP64, bool IN_PLACE, int ARITH>
__global__ void __launch_bounds__(256, 6) k_sweep(SweepArgs a) {
    if (a.state != nullptr && *reinterpret_cast<const volatile int32_t*>(&a.state->stop)) return;
    __shared__ double s_recip[kMaxRecipDeg + 1];
    constexpr bool kIntDiv = ARITH == LMS_FP64_ARITH_INT || ARITH == LMS_FP64_ARITH_MIXED2 ||
                             ARITH == LMS_FP64_ARITH_MIXED3;
    __shared__ uint32_t s_magic[kIntDiv ? 2 * (kMaxRecipDeg + 1) : 1];
    if (FP64) {
        const uint32_t* words = reinterpret_cast<const uint32_t*>(a.recip + kMaxRecipDeg + 1);
        for (int i = threadIdx.x; i <= kMaxRecipDeg; i += blockDim.x) {
            s_recip[i] = a.recip[i];
            if (kIntDiv) {
                s_magic[2 * i] = words[2 * i];
                s_magic[2 * i + 1] = words[2 * i + 1];
            }
        }
        __syncthreads();
    }
    // thread -> vertex: the identity, or (a.order) a permutation of [v_begin, v_end) that groups vertices of
    // equal degree into warps, so a warp's lanes run rows of one length
    const int32_t i = a.v_begin + static_cast<int32_t>(blockIdx.x * blockDim.x + threadIdx.x);
    const int32_t v = i < a.v_end && a.order != nullptr ? __ldg(a.order + i) : i;
    const bool want = a.disp2 != nullptr;
    double d2 = 0.0;
    if (i < a.v_end && (a.bnd_bits == nullptr || !boundary_bit(a.bnd_bits, v))) {
        d2 = smooth_vertex<FP64, IN_PLACE, ARITH>(a, v, s_recip, s_magic, want);
    }
    if (want) record_disp(a.disp2, d2);
}

// Block Gauss-Seidel: block b sweeps listed tile a.tile_begin + b, colour group by colour group in place,
// with a block barrier between groups (a group's vertices are never neighbours of one another, and the
// barrier makes the group's writes visible to the next group's reads).  FP64: Eq. 1 with sequential sums
// (first term a copy) and the table-driven division, bit-identical to the oracle's in-place sweep in
// block order; FP32: Kahan sums.
template <bool FP64>
__global__ void __launch_bounds__(256) k_block_gs(BlockGsArgs a) {
    if (a.state != nullptr && *reinterpret_cast<const volatile int32_t*>(&a.state->stop)) return;
    using V = typename std::conditional<FP64, double2, float2>::type;
    __shared__ double s_recip[kMaxRecipDeg + 1];
    if (FP64) {
        for (int i = threadIdx.x; i <= kMaxRecipDeg; i += blockDim.x) s_recip[i] = a.recip[i];
        __syncthreads();
    }
    V* xy = static_cast<V*>(a.xy);
    const int32_t* g = a.group_ofs + static_cast<int64_t>(a.tile_begin + static_cast<int32_t>(blockIdx.x)) *
                                         (a.ncolours + 1);
    const bool want = a.disp2 != nullptr;
    double dmax = 0.0;
    for (int32_t c = 0; c < a.ncolours; ++c) {
        const int32_t b = g[c], end = g[c + 1];
        for (int32_t i = b + static_cast<int32_t>(threadIdx.x); i < end; i += static_cast<int32_t>(blockDim.x)) {
            const int32_t v = a.verts[i];
            const int32_t e0 = __ldg(a.row_ptr + v), e1 = __ldg(a.row_ptr + v + 1);
            const V o = xy[v];
            V r;
            if constexpr (FP64) {
                double sx = 0.0, sy = 0.0;
                for (int32_t e = e0; e < e1; ++e) {
                    const int32_t u = __ldg(a.col_idx + e);
                    if (!LMS_CHECK(u >= 0 && u < a.n_vertices)) continue;
                    const V p = xy[u];
                    if (e == e0) {
                        sx = plus_zero(p.x);
                        sy = plus_zero(p.y);
                    } else {
                        sx = __dadd_rn(sx, p.x);
                        sy = __dadd_rn(sy, p.y);
                    }
                }
                r.x = div_by_count(sx, e1 - e0, s_recip);
                r.y = div_by_count(sy, e1 - e0, s_recip);
            } else {
                float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
                for (int32_t e = e0; e < e1; ++e) {
                    const int32_t u = __ldg(a.col_idx + e);
                    if (!LMS_CHECK(u >= 0 && u < a.n_vertices)) continue;
                    const V p = xy[u];
                    kahan_add(sx, cx, p.x);
                    kahan_add(sy, cy, p.y);
                }
                r.x = mean_f32(sx, cx, e1 - e0);
                r.y = mean_f32(sy, cy, e1 - e0);
            }
            if (want) {
                const double ex = static_cast<double>(r.x) - static_cast<double>(o.x);
                const double ey = static_cast<double>(r.y) - static_cast<double>(o.y);
                dmax = fmax(dmax, __fma_rn(ex, ex, __dmul_rn(ey, ey)));
            }
            xy[v] = r;
        }
        __syncthreads();
    }
    if (want) record_disp(a.disp2, dmax);
}

// Staged block Gauss-Seidel: block b takes listed tile a.tile_begin + b and copies into shared memory the
// tile's positions, its halo (the neighbours of its interior vertices outside the tile), and the tile's
// local rows (neighbours as shared-memory indices) and vertex list; it then sweeps the tile's colour groups
// in turn entirely on chip (a block barrier between groups) and writes back the tile's interior vertices.
// Tiles of one tile colour share no edge between interior vertices, so nothing a CTA reads into its halo
// is written by another CTA of the launch, and the launch equals the in-place sweep over its tiles in
// block order: FP64 bit-identical to the oracle (sums in stored row order, first term a copy, the
// table-driven division), FP32 with Kahan sums.
template <bool FP64>
__global__ void __launch_bounds__(256) k_block_gs_staged(BlockGsStagedArgs a) {
    if (a.state != nullptr && *reinterpret_cast<const volatile int32_t*>(&a.state->stop)) return;
    using V = typename std::conditional<FP64, double2, float2>::type;
    extern __shared__ __align__(16) unsigned char s_raw[];
    // layout: positions [max_slots] | row starts [max_verts + 1] (int32, relative to the tile's first
    // entry) | vertex positions in the tile [max_verts] (uint16) | local neighbour indices [max_entries]
    V* s_pos = reinterpret_cast<V*>(s_raw);
    int32_t* s_row = reinterpret_cast<int32_t*>(s_pos + a.max_slots);
    uint16_t* s_vert = reinterpret_cast<uint16_t*>(s_row + a.max_verts + 1);
    uint16_t* s_col = s_vert + a.max_verts;
    __shared__ double s_recip[kMaxRecipDeg + 1];
    if (FP64)
        for (int i = threadIdx.x; i <= kMaxRecipDeg; i += blockDim.x) s_recip[i] = a.recip[i];
    V* xy = static_cast<V*>(a.xy);
    const int32_t tile = a.tile_begin + static_cast<int32_t>(blockIdx.x);
    const int4 ti = __ldg(a.tile_info + tile);
    const int32_t* g = a.group_ofs + static_cast<int64_t>(tile) * (a.ncolours + 1);
    const int32_t i0 = __ldg(g), i1 = __ldg(g + a.ncolours);
    const int32_t T = ti.y - ti.x, H = ti.w - ti.z, nv = i1 - i0;
    const int32_t r0 = __ldg(a.lrow + i0), ne = __ldg(a.lrow + i1) - r0;
    const bool fits = T + H <= a.max_slots && nv <= a.max_verts && ne <= a.max_entries;
    if (!fits) {  // never by construction (the limits are maxima over the tiles); counted in debug builds
        (void)LMS_CHECK(false);
        return;
    }
    for (int32_t i = threadIdx.x; i < T; i += blockDim.x) s_pos[i] = xy[ti.x + i];
    for (int32_t j = threadIdx.x; j < H; j += blockDim.x) s_pos[T + j] = xy[__ldg(a.halo + ti.z + j)];
    for (int32_t i = threadIdx.x; i <= nv; i += blockDim.x) s_row[i] = __ldg(a.lrow + i0 + i) - r0;
    for (int32_t i = threadIdx.x; i < nv; i += blockDim.x) s_vert[i] = static_cast<uint16_t>(__ldg(a.verts + i0 + i) - ti.x);
    for (int32_t e = threadIdx.x; e < ne; e += blockDim.x) s_col[e] = __ldg(a.lcol + r0 + e);
    __syncthreads();
    const bool want = a.disp2 != nullptr;
    double dmax = 0.0;
    for (int32_t c = 0; c < a.ncolours; ++c) {
        const int32_t b = __ldg(g + c) - i0, end = __ldg(g + c + 1) - i0;
        for (int32_t i = b + static_cast<int32_t>(threadIdx.x); i < end; i += static_cast<int32_t>(blockDim.x)) {
            const int32_t lv = s_vert[i];
            const int32_t e0 = s_row[i], e1 = s_row[i + 1];
            const V o = s_pos[lv];
            V r;
            if constexpr (FP64) {
                double sx = 0.0, sy = 0.0;
                for (int32_t e = e0; e < e1; ++e) {
                    const int32_t l = s_col[e];
                    if (!LMS_CHECK(l < T + H)) continue;
                    const V p = s_pos[l];
                    if (e == e0) {
                        sx = plus_zero(p.x);
                        sy = plus_zero(p.y);
                    } else {
                        sx = __dadd_rn(sx, p.x);
                        sy = __dadd_rn(sy, p.y);
                    }
                }
                r.x = div_by_count(sx, e1 - e0, s_recip);
                r.y = div_by_count(sy, e1 - e0, s_recip);
            } else {
                float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
                for (int32_t e = e0; e < e1; ++e) {
                    const int32_t l = s_col[e];
                    if (!LMS_CHECK(l < T + H)) continue;
                    const V p = s_pos[l];
                    kahan_add(sx, cx, p.x);
                    kahan_add(sy, cy, p.y);
                }
                r.x = mean_f32(sx, cx, e1 - e0);
                r.y = mean_f32(sy, cy, e1 - e0);
            }
            if (want) {
                const double ex = static_cast<double>(r.x) - static_cast<double>(o.x);
                const double ey = static_cast<double>(r.y) - static_cast<double>(o.y);
                dmax = fmax(dmax, __fma_rn(ex, ex, __dmul_rn(ey, ey)));
            }
            s_pos[lv] = r;
        }
        __syncthreads();
    }
    // write back the tile's interior vertices (the only positions the tile changed)
    for (int32_t i = threadIdx.x; i < nv; i += blockDim.x) {
        const int32_t lv = s_vert[i];
        xy[ti.x + lv] = s_pos[lv];
    }
    if (want) record_disp(a.disp2, dmax);
}

// The paper's parallel in-place sweep (Section 5.1: Algorithm 1 under a static schedule that divides the
// vertices evenly between threads): thread t sweeps storage positions [t * per_thread, (t + 1) *
// per_thread) in order, in place, reading each neighbour as it is at that moment - possibly already
// moved by another thread in this sweep.  Neighbour loads and the store go through L2 (ld/st.global.cg)
// so a thread sees other threads' updates as soon as they land there, not a stale L1 copy.  With one
// thread this is the sequential Algorithm 1 in storage order; otherwise the result depends on timing.
template <bool FP64>
__global__ void __launch_bounds__(256) k_inplace_static(SweepArgs a, int32_t per_thread) {
    if (a.state != nullptr && *reinterpret_cast<const volatile int32_t*>(&a.state->stop)) return;
    using V = typename std::conditional<FP64, double2, float2>::type;
    __shared__ double s_recip[kMaxRecipDeg + 1];
    if (FP64) {
        for (int i = threadIdx.x; i <= kMaxRecipDeg; i += blockDim.x) s_recip[i] = a.recip[i];
        __syncthreads();
    }
    V* pos = static_cast<V*>(a.dst);
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t lo = min(t * per_thread, static_cast<int64_t>(a.v_end));
    const int64_t hi = min(lo + per_thread, static_cast<int64_t>(a.v_end));
    const bool want = a.disp2 != nullptr;
    double dmax = 0.0;
    for (int32_t v = static_cast<int32_t>(lo); v < hi; ++v) {
        if (boundary_bit(a.bnd_bits, v)) continue;
        const int32_t e0 = __ldg(a.row_ptr + v), e1 = __ldg(a.row_ptr + v + 1);
        V r;
        if constexpr (FP64) {
            double sx = 0.0, sy = 0.0;
            for (int32_t e = e0; e < e1; ++e) {
                const int32_t u = __ldg(a.col_idx + e);
                if (!LMS_CHECK(u >= 0 && u < a.n_vertices)) continue;
                const V p = __ldcg(pos + u);
                sx = __dadd_rn(sx, p.x);
                sy = __dadd_rn(sy, p.y);
            }
            r.x = div_by_count(sx, e1 - e0, s_recip);
            r.y = div_by_count(sy, e1 - e0, s_recip);
        } else {
            float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
            for (int32_t e = e0; e < e1; ++e) {
                const int32_t u = __ldg(a.col_idx + e);
                if (!LMS_CHECK(u >= 0 && u < a.n_vertices)) continue;
                const V p = __ldcg(pos + u);
                kahan_add(sx, cx, p.x);
                kahan_add(sy, cy, p.y);
            }
            r.x = mean_f32(sx, cx, e1 - e0);
            r.y = mean_f32(sy, cy, e1 - e0);
        }
        if (want) {
            const V o = __ldcg(pos + v);
            const double ex = static_cast<double>(r.x) - static_cast<double>(o.x);
            const double ey = static_cast<double>(r.y) - static_cast<double>(o.y);
            dmax = fmax(dmax, __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)));
        }
        __stcg(pos + v, r);
    }
    if (want) record_disp(a.disp2, dmax);
}

// Batched FP32 Jacobi: a persistent grid pulls vertex tiles (never crossing a mesh) from a device counter;
// the next tile is requested while the current one is processed.  One thread per vertex; a row is read
// CHUNK entries at a time - all neighbour ids, then all position gathers, then the Kahan sums in row
// order - so a thread keeps CHUNK loads in flight.  The batch's row offsets carry the boundary flag in bit
// 31 (row_ptr[v] | boundary(v) << 31), and row_ptr[v + 1] comes from the next lane, so a warp issues one
// offset load per 32 vertices and no separate flag load.
template <int CHUNK, bool EXTRAS>
__global__ void __launch_bounds__(512) k_batch_sweep(SweepArgs a) {
    __shared__ int32_t s_item[2];
    // EXTRAS (single-mesh sweeps): honour the stop flag and record the displacement when asked
    if (EXTRAS && a.state != nullptr && *reinterpret_cast<const volatile int32_t*>(&a.state->stop)) return;
    const float2* __restrict__ src = static_cast<const float2*>(a.src);
    float2* __restrict__ dst = static_cast<float2*>(a.dst);
    const bool want_disp = EXTRAS && a.disp2 != nullptr;
    int buf = 0;
    if (threadIdx.x == 0) s_item[0] = atomicAdd(a.queue, 1);
    __syncthreads();
    for (;;) {
        const int32_t item = s_item[buf];
        if (item >= a.n_items) break;
        if (threadIdx.x == 0) s_item[buf ^ 1] = atomicAdd(a.queue, 1);
        const int2 r = __ldg(a.items + item);
        for (int32_t base = r.x; base < r.y; base += blockDim.x) {  // uniform rounds: every lane shuffles
            const int32_t v = base + threadIdx.x;
            const int32_t f0 = __ldg(a.row_ptr + min(v, r.y));  // rows past the tile end read row_ptr[end]
            int32_t f1 = __shfl_down_sync(0xffffffffu, f0, 1);
            if ((threadIdx.x & 31) == 31) f1 = v < r.y ? __ldg(a.row_ptr + v + 1) : f0;
            if constexpr (!EXTRAS) {
                if (v >= r.y || f0 < 0) continue;  // past the end of the tile, or a boundary vertex
                const int32_t e0 = f0, e1 = f1 & 0x7fffffff;
                float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
                for (int32_t e = e0; e < e1; e += CHUNK) {
                    int32_t u[CHUNK];
                    float2 p[CHUNK];
#pragma unroll
                    for (int g = 0; g < CHUNK; ++g) {
                        u[g] = e + g < e1 ? __ldg(a.col_idx + e + g) : -1;
                        if (u[g] >= 0 && !LMS_CHECK(u[g] < a.n_vertices)) u[g] = -1;
                    }
#pragma unroll
                    for (int g = 0; g < CHUNK; ++g) p[g] = u[g] >= 0 ? __ldg(src + u[g]) : make_float2(0.f, 0.f);
#pragma unroll
                    for (int g = 0; g < CHUNK; ++g)
                        if (u[g] >= 0) {
                            kahan_add(sx, cx, p[g].x);
                            kahan_add(sy, cy, p[g].y);
                        }
                }
                dst[v] = make_float2(mean_f32(sx, cx, e1 - e0), mean_f32(sy, cy, e1 - e0));
                continue;
            }
            double d2 = 0.0;
            if (v < r.y && f0 >= 0) {  // inside the tile and not a boundary vertex
                const int32_t e0 = f0, e1 = f1 & 0x7fffffff;
                // old position for the displacement, loaded before the gathers (see smooth_vertex)
                float2 o = make_float2(0.f, 0.f);
                if (want_disp) o = src[v];
                float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
                for (int32_t e = e0; e < e1; e += CHUNK) {
                    int32_t u[CHUNK];
                    float2 p[CHUNK];
#pragma unroll
                    for (int g = 0; g < CHUNK; ++g) {
                        u[g] = e + g < e1 ? __ldg(a.col_idx + e + g) : -1;
                        if (u[g] >= 0 && !LMS_CHECK(u[g] < a.n_vertices)) u[g] = -1;
                    }
#pragma unroll
                    for (int g = 0; g < CHUNK; ++g) p[g] = u[g] >= 0 ? __ldg(src + u[g]) : make_float2(0.f, 0.f);
#pragma unroll
                    for (int g = 0; g < CHUNK; ++g)
                        if (u[g] >= 0) {
                            kahan_add(sx, cx, p[g].x);
                            kahan_add(sy, cy, p[g].y);
                        }
                }
                const float2 q = make_float2(mean_f32(sx, cx, e1 - e0), mean_f32(sy, cy, e1 - e0));
                if (EXTRAS && want_disp) {
                    const double dx = static_cast<double>(__fsub_rn(q.x, o.x)), dy = static_cast<double>(__fsub_rn(q.y, o.y));
                    d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
                }
                dst[v] = q;
            }
            if (EXTRAS && want_disp) record_disp(a.disp2, d2);
        }
        __syncthreads();
        buf ^= 1;
    }
}

// Batched FP32 Jacobi over packed rows: one 32-bit word per vertex holds its row's first id pair relative
// to its mesh's first pair (bits 0..21), its neighbour count (bits 22..27) and the boundary flag (bit 31),
// so a thread learns its whole row from one coalesced load (no neighbour-lane shuffle, no second load for
// the last lane), issued one round of the tile ahead.  Every row of the id array is padded to an even length with -1, so ids are read as
// aligned pairs: PAIRS 8-byte loads per step, then the gathers, then the Kahan sums in stored row order.
// Tiles come from the work queue as in k_batch_sweep; the mesh's first pair comes with the tile.
template <int PAIRS>
__global__ void __launch_bounds__(512) k_batch_sweep_packed(PackedArgs a) {
    __shared__ int32_t s_item[2];
    const float2* __restrict__ src = static_cast<const float2*>(a.src);
    float2* __restrict__ dst = static_cast<float2*>(a.dst);
    int buf = 0;
    if (threadIdx.x == 0) s_item[0] = atomicAdd(a.queue, 1);
    __syncthreads();
    for (;;) {
        const int32_t item = s_item[buf];
        if (item >= a.n_items) break;
        if (threadIdx.x == 0) s_item[buf ^ 1] = atomicAdd(a.queue, 1);
        const int2 r = __ldg(a.items + item);
        const int32_t pbase = __ldg(a.items_pbase + item);
        // the row word of the thread's next vertex is loaded one round ahead, so a round starts with its
        // id loads instead of waiting for its row word
        int32_t vn = r.x + static_cast<int32_t>(threadIdx.x);
        int32_t wn = vn < r.y ? __ldg(a.row_words + vn) : -1;
        for (int32_t v = vn; v < r.y; v += blockDim.x) {
            const int32_t w = wn;
            vn = v + static_cast<int32_t>(blockDim.x);
            wn = vn < r.y ? __ldg(a.row_words + vn) : -1;
            if (w < 0) continue;  // boundary vertex
            const int32_t d = (w >> kPackedDegreeShift) & kPackedDegreeMask;
            const int32_t q0 = pbase + (w & kPackedOffsetMask), q1 = q0 + ((d + 1) >> 1);
            float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
            for (int32_t q = q0; q < q1; q += PAIRS) {
                int32_t u[2 * PAIRS];
                float2 p[2 * PAIRS];
#pragma unroll
                for (int g = 0; g < PAIRS; ++g) {
                    const int2 x = q + g < q1 ? __ldg(a.id_pairs + q + g) : make_int2(-1, -1);
                    u[2 * g] = x.x;
                    u[2 * g + 1] = x.y;
                }
#pragma unroll
                for (int g = 0; g < 2 * PAIRS; ++g)
                    if (u[g] >= 0 && !LMS_CHECK(u[g] < a.n_vertices)) u[g] = -1;
#pragma unroll
                for (int g = 0; g < 2 * PAIRS; ++g) p[g] = u[g] >= 0 ? __ldg(src + u[g]) : make_float2(0.f, 0.f);
#pragma unroll
                for (int g = 0; g < 2 * PAIRS; ++g)
                    if (u[g] >= 0) {
                        kahan_add(sx, cx, p[g].x);
                        kahan_add(sy, cy, p[g].y);
                    }
            }
            dst[v] = make_float2(mean_f32(sx, cx, d), mean_f32(sy, cy, d));
        }
        __syncthreads();
        buf ^= 1;
    }
}

// Single-mesh FP32 Jacobi sweep over packed rows: as k_batch_sweep_packed, but a row word's offset is
// relative to the first id pair of the vertex's block of 2^kPackedBlockShift storage positions
// (block_pbase), so any mesh size and any tiling fit one table; the rows of the id-pair array are stored
// farthest neighbour first.  Rounds are uniform across the block (every lane takes part in the
// displacement's warp reduction); honours the stop flag; records the largest displacement when asked (old
// position loaded before the gathers).
template <int PAIRS>
__global__ void __launch_bounds__(512) k_sweep_packed_mesh(PackedMeshArgs a) {
    __shared__ int32_t s_item[2];
    if (a.state != nullptr && *reinterpret_cast<const volatile int32_t*>(&a.state->stop)) return;
    const float2* src = static_cast<const float2*>(a.src);
    float2* dst = static_cast<float2*>(a.dst);
    const bool want_disp = a.disp2 != nullptr;
    int buf = 0;
    if (threadIdx.x == 0) s_item[0] = atomicAdd(a.queue, 1);
    __syncthreads();
    for (;;) {
        const int32_t item = s_item[buf];
        if (item >= a.n_items) break;
        if (threadIdx.x == 0) s_item[buf ^ 1] = atomicAdd(a.queue, 1);
        const int2 r = __ldg(a.items + item);
        int32_t vn = r.x + static_cast<int32_t>(threadIdx.x);
        int32_t wn = vn < r.y ? __ldg(a.row_words + vn) : -1;
        int32_t bn = vn < r.y ? __ldg(a.block_pbase + (vn >> kPackedBlockShift)) : 0;
        for (int32_t base = r.x; base < r.y; base += blockDim.x) {  // uniform rounds
            const int32_t v = base + static_cast<int32_t>(threadIdx.x);
            const int32_t w = wn, pb = bn;
            vn = v + static_cast<int32_t>(blockDim.x);
            wn = vn < r.y ? __ldg(a.row_words + vn) : -1;
            bn = vn < r.y ? __ldg(a.block_pbase + (vn >> kPackedBlockShift)) : 0;
            double d2 = 0.0;
            if (w >= 0) {  // inside the tile (w = -1 past its end) and not a boundary vertex
                float2 o = make_float2(0.f, 0.f);
                if (want_disp) o = src[v];
                const int32_t d = (w >> kPackedDegreeShift) & kPackedDegreeMask;
                const int32_t q0 = pb + (w & kPackedOffsetMask), q1 = q0 + ((d + 1) >> 1);
                float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
                for (int32_t q = q0; q < q1; q += PAIRS) {
                    int32_t u[2 * PAIRS];
                    float2 p[2 * PAIRS];
#pragma unroll
                    for (int g = 0; g < PAIRS; ++g) {
                        const int2 x = q + g < q1 ? __ldg(a.id_pairs + q + g) : make_int2(-1, -1);
                        u[2 * g] = x.x;
                        u[2 * g + 1] = x.y;
                    }
#pragma unroll
                    for (int g = 0; g < 2 * PAIRS; ++g)
                        if (u[g] >= 0 && !LMS_CHECK(u[g] < a.n_vertices)) u[g] = -1;
#pragma unroll
                    for (int g = 0; g < 2 * PAIRS; ++g) p[g] = u[g] >= 0 ? __ldg(src + u[g]) : make_float2(0.f, 0.f);
#pragma unroll
                    for (int g = 0; g < 2 * PAIRS; ++g)
                        if (u[g] >= 0) {
                            kahan_add(sx, cx, p[g].x);
                            kahan_add(sy, cy, p[g].y);
                        }
                }
                const float2 m = make_float2(mean_f32(sx, cx, d), mean_f32(sy, cy, d));
                if (want_disp) {
                    const double ex = static_cast<double>(__fsub_rn(m.x, o.x)), ey = static_cast<double>(__fsub_rn(m.y, o.y));
                    d2 = __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey));
                }
                dst[v] = m;
            }
            if (want_disp) record_disp(a.disp2, d2);
        }
        __syncthreads();
        buf ^= 1;
    }
}

// Batched FP32 Jacobi over a SELL-C-sigma work layout (Kreutzer et al., SIAM J. Sci. Comput. 36(5),
// 2014): inside every tile the interior vertices are sorted by degree into slices of 32, and a slice's
// neighbour ids are stored column-major (entry j of slot l at base + 32 j + l, -1 past the slot's row),
// so lane l of a warp handles slot l and each id load of a warp is one coalesced 128-byte access with
// the same trip count for all lanes.  Positions stay in the ordering's storage layout; entries keep
// their row order, so the Kahan sums equal the CSR kernels'.  CTAs pull tiles (slice ranges) from a
// device counter; warps take the tile's slices round-robin.
template <int CHUNK>
__global__ void __launch_bounds__(512) k_batch_sell(SellArgs a) {
    __shared__ int32_t s_item[2];
    const float2* __restrict__ src = static_cast<const float2*>(a.src);
    float2* __restrict__ dst = static_cast<float2*>(a.dst);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int buf = 0;
    if (threadIdx.x == 0) s_item[0] = atomicAdd(a.queue, 1);
    __syncthreads();
    for (;;) {
        const int32_t item = s_item[buf];
        if (item >= a.n_items) break;
        if (threadIdx.x == 0) s_item[buf ^ 1] = atomicAdd(a.queue, 1);
        const int2 r = __ldg(a.items + item);
        for (int32_t sl = r.x + warp; sl < r.y; sl += nwarps) {
            const int2 sd = __ldg(a.slice + sl);  // (first entry, slice degree)
            const int32_t v = __ldg(a.slot + 32 * sl + lane);
            const int32_t* col = a.col + sd.x + lane;
            float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
            int32_t cnt = 0;
            for (int32_t j = 0; j < sd.y; j += CHUNK) {
                int32_t u[CHUNK];
                float2 p[CHUNK];
#pragma unroll
                for (int g = 0; g < CHUNK; ++g) u[g] = j + g < sd.y ? __ldg(col + 32 * (j + g)) : -1;
#pragma unroll
                for (int g = 0; g < CHUNK; ++g)
                    if (u[g] >= 0) p[g] = __ldg(src + u[g]);
#pragma unroll
                for (int g = 0; g < CHUNK; ++g)
                    if (u[g] >= 0) {
                        kahan_add(sx, cx, p[g].x);
                        kahan_add(sy, cy, p[g].y);
                        ++cnt;
                    }
            }
            if (v >= 0) dst[v] = make_float2(mean_f32(sx, cx, cnt), mean_f32(sy, cy, cnt));
        }
        __syncthreads();
        buf ^= 1;
    }
}

// Section 3.2 edge-length ratio, written exactly as the definition: three correctly rounded
// lengths, shortest over longest.
__device__ __forceinline__ double edge_len_exact(double2 p, double2 q) {
    const double dx = __dsub_rn(q.x, p.x), dy = __dsub_rn(q.y, p.y);
    return __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
}

__global__ void k_tri_quality_exact(int32_t ntri, const int32_t* __restrict__ tri, const double2* __restrict__ xy,
                                    double* __restrict__ q_t) {
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntri) return;
    const double2 a = xy[tri[3 * t]], b = xy[tri[3 * t + 1]], c = xy[tri[3 * t + 2]];
    const double l0 = edge_len_exact(a, b), l1 = edge_len_exact(b, c), l2 = edge_len_exact(c, a);
    double lo = l0, hi = l0;
    lo = l1 < lo ? l1 : lo;
    hi = l1 > hi ? l1 : hi;
    lo = l2 < lo ? l2 : lo;
    hi = l2 > hi ? l2 : hi;
    q_t[t] = hi == 0.0 ? 0.0 : __ddiv_rn(lo, hi);
}

// Mean over a vertex's triangles, in ascending triangle id (the incidence rows are ascending).
__global__ void k_vertex_quality_exact(int32_t n, const int32_t* __restrict__ vt_ptr,
                                       const int32_t* __restrict__ vt_idx, const double* __restrict__ q_t,
                                       double* __restrict__ q_v) {
    const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t e0 = vt_ptr[v], e1 = vt_ptr[v + 1];
    double s = 0.0;
    for (int32_t e = e0; e < e1; ++e) s = __dadd_rn(s, q_t[vt_idx[e]]);
    q_v[v] = e1 > e0 ? __ddiv_rn(s, static_cast<double>(e1 - e0)) : 0.0;
}

// Per-sweep quality.  Q = (1/n) sum_v (1/n_t(v)) sum_{t in v} q_t = (1/n) sum_t w_t q_t with
// w_t = sum over t's corners of 1/n_t(corner): one pass over the triangles.  q_t uses the same
// ratio written as sqrt(min l^2 / max l^2) (one root instead of three).
//
// FP64: the squared lengths in FP64; their minimum and maximum by integer compares of the bit patterns
// (non-negative doubles order like their bits); the root of the ratio from an FP32 seed refined by two
// Newton steps q <- q - (q^2 max - min) * c in FP64, with c ~ 1/(2 q max) in FP32.  The seed's relative
// error (under 3e-7) becomes about 1e-13 after one step and a few ulps after two, so the result agrees
// with sqrt(min / max) to a few ulps while the FP64 unit (GB300's narrow pipe) runs 6 instructions for
// the root instead of an IEEE division and square root.  Operands outside the ranges the seed handles
// (a zero or tiny shortest edge, extreme magnitudes) take sqrt(min / max).
__device__ __forceinline__ bool u64_less(uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl) {
    return ah < bh || (ah == bh && al < bl);
}

__device__ __forceinline__ double tri_quality_fast(double2 a, double2 b, double2 c) {
    const double e0 = (b.x - a.x) * (b.x - a.x) + (b.y - a.y) * (b.y - a.y);
    const double e1 = (c.x - b.x) * (c.x - b.x) + (c.y - b.y) * (c.y - b.y);
    const double e2 = (a.x - c.x) * (a.x - c.x) + (a.y - c.y) * (a.y - c.y);
    uint32_t loh = hi32(e0), lol = lo32(e0), hih = loh, hil = lol;
    const uint32_t h1 = hi32(e1), l1 = lo32(e1), h2 = hi32(e2), l2 = lo32(e2);
    if (u64_less(h1, l1, loh, lol)) { loh = h1; lol = l1; }
    if (u64_less(hih, hil, h1, l1)) { hih = h1; hil = l1; }
    if (u64_less(h2, l2, loh, lol)) { loh = h2; lol = l2; }
    if (u64_less(hih, hil, h2, l2)) { hih = h2; hil = l2; }
    return root_of_ratio(from_hilo(loh, lol), from_hilo(hih, hil));
}

__device__ __forceinline__ float tri_quality_fast(float2 a, float2 b, float2 c) {
    const float e0 = (b.x - a.x) * (b.x - a.x) + (b.y - a.y) * (b.y - a.y);
    const float e1 = (c.x - b.x) * (c.x - b.x) + (c.y - b.y) * (c.y - b.y);
    const float e2 = (a.x - c.x) * (a.x - c.x) + (a.y - c.y) * (a.y - c.y);
    const float lo = fminf(e0, fminf(e1, e2)), hi = fmaxf(e0, fmaxf(e1, e2));
    return hi > 0.f ? sqrtf(lo / hi) : 0.f;
}

__device__ __forceinline__ double block_sum(double v, double* smem) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s += smem[w];
    return s;  // valid in thread 0
}

// Per-thread partial sums: FP64 weights and sums for FP64 positions; FP32 weights and Kahan-compensated
// FP32 sums for FP32 positions (no FP64 instruction per triangle).  Blocks reduce in FP64.
__global__ void __launch_bounds__(256) k_quality_partials_f64(int32_t ntri, const int32_t* __restrict__ tri,
                                                              const double2* __restrict__ xy,
                                                              const double* __restrict__ w,
                                                              double* __restrict__ partials, const DevState* state) {
    __shared__ double smem[32];
    if (state != nullptr && *reinterpret_cast<const volatile int32_t*>(&state->stop)) return;
    double acc = 0.0;
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntri; t += gridDim.x * blockDim.x) {
        const double2 a = __ldg(xy + __ldg(tri + 3 * t)), b = __ldg(xy + __ldg(tri + 3 * t + 1)),
                      c = __ldg(xy + __ldg(tri + 3 * t + 2));
        acc = __fma_rn(__ldg(w + t), tri_quality_fast(a, b, c), acc);
    }
    const double s = block_sum(acc, smem);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_quality_partials_f32(int32_t ntri, const int32_t* __restrict__ tri,
                                                              const float2* __restrict__ xy,
                                                              const float* __restrict__ w,
                                                              double* __restrict__ partials, const DevState* state) {
    __shared__ double smem[32];
    if (state != nullptr && *reinterpret_cast<const volatile int32_t*>(&state->stop)) return;
    float acc = 0.f, comp = 0.f;
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntri; t += gridDim.x * blockDim.x) {
        const float2 a = __ldg(xy + __ldg(tri + 3 * t)), b = __ldg(xy + __ldg(tri + 3 * t + 1)),
                     c = __ldg(xy + __ldg(tri + 3 * t + 2));
        kahan_add(acc, comp, __fmul_rn(__ldg(w + t), tri_quality_fast(a, b, c)));
    }
    const double s = block_sum(static_cast<double>(acc) - static_cast<double>(comp), smem);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kQualityBlocks) k_quality_finish(const double* __restrict__ partials,
                                                                   double n, DevState* st, int mode) {
    __shared__ double smem[32];
    const double s = block_sum(partials[threadIdx.x], smem);
    if (threadIdx.x != 0) return;
    const double Q = s / n;
    if (mode == 0) {
        st->q_cur = Q;
    } else if (mode == 1) {
        st->q_first = Q;
        st->q_prev = Q;
        st->q_cur = Q;
    }
}

// Stop check after sweep k (Section 5.1): the rule fires when Q_k - Q_{k-1} < tol (or Q_k >= goal);
// the cap fires at max_iters.  Also clears the displacement slot of sweep k+1.
__global__ void k_stop_check(const double* __restrict__ partials, double n, DevState* st, double tol, double goal,
                             int32_t max_iters) {
    __shared__ double smem[32];
    if (*reinterpret_cast<volatile int32_t*>(&st->stop)) return;
    const double s = block_sum(partials[threadIdx.x], smem);
    if (threadIdx.x != 0) return;
    const double Q = s / n;
    const int32_t k = st->k + 1;
    st->k = k;
    if (Q >= goal || Q - st->q_prev < tol || k >= max_iters) {
        st->stop = 1;
        st->iters_at_stop = k;
    }
    st->q_prev = Q;
    st->q_cur = Q;
    st->disp2[(k + 1) & 1] = 0ull;
}

// Each row's entries ordered by decreasing storage distance |u - v| (stable: equal distances keep their
// order); one thread per row, insertion sort of at most kMaxPackedDegree entries in place.
__global__ void k_sort_rows_far_first(int32_t n, const int32_t* __restrict__ row_ptr, int32_t* __restrict__ col_idx) {
    const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t e0 = row_ptr[v] & 0x7fffffff, e1 = row_ptr[v + 1] & 0x7fffffff;
    for (int32_t i = e0 + 1; i < e1; ++i) {
        const int32_t x = col_idx[i];
        const int32_t dx = abs(x - v);
        int32_t j = i - 1;
        while (j >= e0 && abs(col_idx[j] - v) < dx) {
            col_idx[j + 1] = col_idx[j];
            --j;
        }
        col_idx[j + 1] = x;
    }
}

__global__ void k_gather_rows(int32_t n, const int32_t* __restrict__ new_to_old, const int32_t* __restrict__ rp_src,
                              const int32_t* __restrict__ ci_src, const int32_t* __restrict__ rp_dst,
                              int32_t* __restrict__ ci_dst, const int32_t* __restrict__ map) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t v = new_to_old[k];
    const int32_t s0 = rp_src[v], len = rp_src[v + 1] - s0, d0 = rp_dst[k];
    for (int32_t e = 0; e < len; ++e) {
        const int32_t u = ci_src[s0 + e];
        ci_dst[d0 + e] = map ? map[u] : u;
    }
}

// row_ptr[v] |= boundary(v) << 31 for v < n (row_ptr[n] keeps no flag)
__global__ void k_flag_boundary_rows(int32_t n, const uint32_t* __restrict__ bits, int32_t* __restrict__ row_ptr) {
    const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n && ((bits[v >> 5] >> (v & 31)) & 1u)) row_ptr[v] |= static_cast<int32_t>(0x80000000u);
}

__global__ void k_map_ids(int64_t count, const int32_t* __restrict__ map, const int32_t* __restrict__ src,
                          int32_t* __restrict__ dst) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = map[src[i]];
}

__global__ void k_boundary_bits(int32_t n, const int32_t* __restrict__ new_to_old,
                                const uint8_t* __restrict__ bnd_orig, uint32_t* __restrict__ bits) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;   // blockDim is a multiple of 32
    const bool b = k < n && bnd_orig[new_to_old[k]] != 0;
    const uint32_t word = __ballot_sync(0xffffffffu, b);
    if ((threadIdx.x & 31) == 0 && k < n) bits[k >> 5] = word;
}

template <typename V>
__global__ void k_gather_xy(int32_t n, const int32_t* __restrict__ perm, const V* __restrict__ src,
                            V* __restrict__ dst) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) dst[k] = src[perm[k]];
}

__global__ void k_load_xy_f64(int32_t n, const int32_t* __restrict__ new_to_old, const double2* __restrict__ src,
                              double2* __restrict__ dst) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) dst[k] = src[new_to_old[k]];
}

__device__ __forceinline__ float2 normalise(double2 p, double cx, double cy, double inv_s) {
    return make_float2(__double2float_rn(__dmul_rn(__dsub_rn(p.x, cx), inv_s)),
                       __double2float_rn(__dmul_rn(__dsub_rn(p.y, cy), inv_s)));
}

__device__ __forceinline__ double2 denormalise(float2 p, double cx, double cy, double s) {
    return make_double2(__dadd_rn(cx, __dmul_rn(s, static_cast<double>(p.x))),
                        __dadd_rn(cy, __dmul_rn(s, static_cast<double>(p.y))));
}

__global__ void k_load_xy_f32(int32_t n, const int32_t* __restrict__ new_to_old, const double2* __restrict__ src,
                              float2* __restrict__ dst, double cx, double cy, double inv_s) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) dst[k] = normalise(src[new_to_old[k]], cx, cy, inv_s);
}

__global__ void k_store_xy_f64(int32_t n, const int32_t* __restrict__ new_to_old, const double2* __restrict__ src,
                               double2* __restrict__ dst) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) dst[new_to_old[k]] = src[k];
}

// Boundary vertices never move: they are returned as the FP64 values last stored (fixed_xy, original
// order), not as their FP32 copies mapped back.
__global__ void k_store_xy_f32(int32_t n, const int32_t* __restrict__ new_to_old, const float2* __restrict__ src,
                               double2* __restrict__ dst, double cx, double cy, double s,
                               const uint8_t* __restrict__ bnd_orig, const double2* __restrict__ fixed_xy) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t o = new_to_old[k];
    dst[o] = (fixed_xy != nullptr && bnd_orig[o]) ? fixed_xy[o] : denormalise(src[k], cx, cy, s);
}

// one block per tile; mesh_cs[4m..4m+3] = (cx, cy, inv_s, s).  Writes both ping-pong buffers and raises
// *bad when an input coordinate is not finite.
__global__ void k_batch_load_xy(const int2* __restrict__ items, const int32_t* __restrict__ item_mesh,
                                const int32_t* __restrict__ new_to_old, const double2* __restrict__ src,
                                float2* __restrict__ dst0, float2* __restrict__ dst1,
                                const double* __restrict__ mesh_cs, int32_t* bad) {
    const int2 r = items[blockIdx.x];
    const double* cs = mesh_cs + 4 * item_mesh[blockIdx.x];
    bool finite = true;
    for (int32_t k = r.x + threadIdx.x; k < r.y; k += blockDim.x) {
        const double2 p = src[new_to_old[k]];
        finite = finite && isfinite(p.x) && isfinite(p.y);
        const float2 q = normalise(p, cs[0], cs[1], cs[2]);
        dst0[k] = q;
        dst1[k] = q;
    }
    if (!finite) atomicExch(bad, 1);
}

__global__ void k_batch_store_xy(const int2* __restrict__ items, const int32_t* __restrict__ item_mesh,
                                 const int32_t* __restrict__ new_to_old, const float2* __restrict__ src,
                                 double2* __restrict__ dst, const double* __restrict__ mesh_cs,
                                 const uint32_t* __restrict__ bnd_bits, const double2* __restrict__ fixed_xy) {
    const int2 r = items[blockIdx.x];
    const double* cs = mesh_cs + 4 * item_mesh[blockIdx.x];
    for (int32_t k = r.x + threadIdx.x; k < r.y; k += blockDim.x) {
        const int32_t o = new_to_old[k];
        dst[o] = boundary_bit(bnd_bits, k) ? fixed_xy[o] : denormalise(src[k], cs[0], cs[1], cs[3]);
    }
}

__global__ void k_div_selftest(int32_t count, const double* __restrict__ s, const int32_t* __restrict__ d,
                               const double* __restrict__ recip, double* __restrict__ q) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) q[i] = div_by_count(s[i], d[i], recip);
}

__global__ void k_div32_selftest(int32_t count, const float* __restrict__ s, const int32_t* __restrict__ d,
                                 float* __restrict__ q) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) q[i] = mean_f32(s[i], 0.f, d[i]);
}

__global__ void k_add_selftest(int32_t count, const double* __restrict__ a, const double* __restrict__ b,
                               double* __restrict__ s) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) s[i] = add_rn_int(a[i], b[i]);
}

// q[i] = s[i] / d[i] by the integer-pipe division (FP64 table division where it declines)
__global__ void k_divint_selftest(int32_t count, const double* __restrict__ s, const int32_t* __restrict__ d,
                                  const double* __restrict__ recip, double* __restrict__ q) {
    const uint32_t* words = reinterpret_cast<const uint32_t*>(recip + kMaxRecipDeg + 1);
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) q[i] = mean_fp64<LMS_FP64_ARITH_INT>(s[i], d[i], recip, words);
}

inline unsigned blocks_for(int64_t count, int block) { return static_cast<unsigned>((count + block - 1) / block); }

}  // namespace

cudaError_t launch_sweep(int precision, bool in_place, const SweepArgs& a, int block, int fp64_arith,
                         cudaStream_t stream) {
    const int32_t count = a.v_end - a.v_begin;
    if (count <= 0) return cudaSuccess;
    const unsigned grid = blocks_for(count, block);
    using K = void (*)(SweepArgs);
    K k = nullptr;
    if (precision == LMS_FP64) {
        switch (fp64_arith) {
            case LMS_FP64_ARITH_FPU:
                k = in_place ? k_sweep<true, true, LMS_FP64_ARITH_FPU> : k_sweep<true, false, LMS_FP64_ARITH_FPU>;
                break;
            case LMS_FP64_ARITH_INT_ADDS:
                k = in_place ? k_sweep<true, true, LMS_FP64_ARITH_INT_ADDS> : k_sweep<true, false, LMS_FP64_ARITH_INT_ADDS>;
                break;
            case LMS_FP64_ARITH_INT:
                k = in_place ? k_sweep<true, true, LMS_FP64_ARITH_INT> : k_sweep<true, false, LMS_FP64_ARITH_INT>;
                break;
            case LMS_FP64_ARITH_MIXED2:
                k = in_place ? k_sweep<true, true, LMS_FP64_ARITH_MIXED2> : k_sweep<true, false, LMS_FP64_ARITH_MIXED2>;
                break;
            case LMS_FP64_ARITH_MIXED3:
                k = in_place ? k_sweep<true, true, LMS_FP64_ARITH_MIXED3> : k_sweep<true, false, LMS_FP64_ARITH_MIXED3>;
                break;
            default:
                return cudaErrorInvalidValue;
        }
    } else {
        k = in_place ? k_sweep<false, true, LMS_FP64_ARITH_FPU> : k_sweep<false, false, LMS_FP64_ARITH_FPU>;
    }
    k<<<grid, block, 0, stream>>>(a);
    return cudaGetLastError();
}

using BatchKernel = void (*)(SweepArgs);

BatchKernel batch_kernel(int chunk, bool extras) {
    switch (chunk) {
        case 1: return extras ? k_batch_sweep<1, true> : k_batch_sweep<1, false>;
        case 2: return extras ? k_batch_sweep<2, true> : k_batch_sweep<2, false>;
        case 3: return extras ? k_batch_sweep<3, true> : k_batch_sweep<3, false>;
        case 4: return extras ? k_batch_sweep<4, true> : k_batch_sweep<4, false>;
        case 5: return extras ? k_batch_sweep<5, true> : k_batch_sweep<5, false>;
        case 6: return extras ? k_batch_sweep<6, true> : k_batch_sweep<6, false>;
        case 8: return extras ? k_batch_sweep<8, true> : k_batch_sweep<8, false>;
        default: return nullptr;
    }
}

cudaError_t launch_batch_sweep(const SweepArgs& a, int block, int chunk, int grid, cudaStream_t stream) {
    const BatchKernel k = batch_kernel(chunk, a.state != nullptr || a.disp2 != nullptr);
    if (k == nullptr) return cudaErrorInvalidValue;
    k<<<grid, block, 0, stream>>>(a);
    return cudaGetLastError();
}

int batch_sweep_occupancy(int block, int chunk) {
    const BatchKernel k = batch_kernel(chunk, true);
    int n = 0;
    if (k == nullptr || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, 0) != cudaSuccess) return 0;
    return n;
}

using PackedKernel = void (*)(PackedArgs);

// chunk = ids read per step (pairs of ids: 2, 4 or 6)
PackedKernel packed_kernel(int chunk) {
    switch (chunk) {
        case 2: return k_batch_sweep_packed<1>;
        case 4: return k_batch_sweep_packed<2>;
        case 6: return k_batch_sweep_packed<3>;
        default: return nullptr;
    }
}

cudaError_t launch_batch_sweep_packed(const PackedArgs& a, int block, int chunk, int grid, cudaStream_t stream) {
    const PackedKernel k = packed_kernel(chunk);
    if (k == nullptr) return cudaErrorInvalidValue;
    if (a.n_items <= 0) return cudaSuccess;
    k<<<grid, block, 0, stream>>>(a);
    return cudaGetLastError();
}

int batch_packed_occupancy(int block, int chunk) {
    const PackedKernel k = packed_kernel(chunk);
    int n = 0;
    if (k == nullptr || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, 0) != cudaSuccess) return 0;
    return n;
}

// Row v of the CSR copied to id pairs [pstart[v], pstart[v + 1]) (in ids: 2 * pstart), -1 past its end.
__global__ void k_pad_rows(int32_t n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                           const int32_t* __restrict__ pstart, int32_t* __restrict__ out) {
    const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t e0 = row_ptr[v] & 0x7fffffff, e1 = row_ptr[v + 1] & 0x7fffffff;
    const int64_t o0 = 2 * static_cast<int64_t>(pstart[v]), o1 = 2 * static_cast<int64_t>(pstart[v + 1]);
    for (int64_t k = o0; k < o1; ++k) out[k] = e0 + (k - o0) < e1 ? col_idx[e0 + (k - o0)] : -1;
}

cudaError_t launch_sweep_packed_mesh(const PackedMeshArgs& a, int block, int grid, cudaStream_t stream) {
    if (a.n_items <= 0) return cudaSuccess;
    k_sweep_packed_mesh<2><<<grid, block, 0, stream>>>(a);
    return cudaGetLastError();
}

int sweep_packed_mesh_occupancy(int block) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_packed_mesh<2>, block, 0) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_pad_rows(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const int32_t* pstart,
                            int32_t* out, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    k_pad_rows<<<blocks_for(n, 256), 256, 0, stream>>>(n, row_ptr, col_idx, pstart, out);
    return cudaGetLastError();
}

cudaError_t launch_sort_rows_far_first(int32_t n, const int32_t* row_ptr, int32_t* col_idx, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    k_sort_rows_far_first<<<blocks_for(n, 256), 256, 0, stream>>>(n, row_ptr, col_idx);
    return cudaGetLastError();
}

using SellKernel = void (*)(SellArgs);

SellKernel sell_kernel(int chunk) {
    switch (chunk) {
        case 1: return k_batch_sell<1>;
        case 4: return k_batch_sell<4>;
        case 8: return k_batch_sell<8>;
        default: return nullptr;
    }
}

cudaError_t launch_batch_sell(const SellArgs& a, int block, int chunk, int grid, cudaStream_t stream) {
    const SellKernel k = sell_kernel(chunk);
    if (k == nullptr) return cudaErrorInvalidValue;
    k<<<grid, block, 0, stream>>>(a);
    return cudaGetLastError();
}

int batch_sell_occupancy(int block, int chunk) {
    const SellKernel k = sell_kernel(chunk);
    int n = 0;
    if (k == nullptr || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, 0) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_tri_quality_exact(int32_t ntri, const int32_t* tri, const double* xy64, double* q_t,
                                     cudaStream_t stream) {
    if (ntri <= 0) return cudaSuccess;
    k_tri_quality_exact<<<blocks_for(ntri, 256), 256, 0, stream>>>(ntri, tri, reinterpret_cast<const double2*>(xy64),
                                                                   q_t);
    return cudaGetLastError();
}

cudaError_t launch_vertex_quality_exact(int32_t n, const int32_t* vt_ptr, const int32_t* vt_idx, const double* q_t,
                                        double* q_v, cudaStream_t stream) {
    k_vertex_quality_exact<<<blocks_for(n, 256), 256, 0, stream>>>(n, vt_ptr, vt_idx, q_t, q_v);
    return cudaGetLastError();
}

cudaError_t launch_quality_partials(int precision, int32_t ntri, const int32_t* tri, const void* xy, const void* w,
                                    double* partials, const DevState* state, cudaStream_t stream) {
    if (precision == LMS_FP64)
        k_quality_partials_f64<<<kQualityBlocks, 256, 0, stream>>>(
            ntri, tri, static_cast<const double2*>(xy), static_cast<const double*>(w), partials, state);
    else
        k_quality_partials_f32<<<kQualityBlocks, 256, 0, stream>>>(
            ntri, tri, static_cast<const float2*>(xy), static_cast<const float*>(w), partials, state);
    return cudaGetLastError();
}

cudaError_t launch_quality_finish(const double* partials, double n, DevState* state, int mode, cudaStream_t stream) {
    k_quality_finish<<<1, kQualityBlocks, 0, stream>>>(partials, n, state, mode);
    return cudaGetLastError();
}

cudaError_t launch_stop_check(const double* partials, double n, DevState* state, double tol, double goal,
                              int32_t max_iters, cudaStream_t stream) {
    k_stop_check<<<1, kQualityBlocks, 0, stream>>>(partials, n, state, tol, goal, max_iters);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(int32_t n, const int32_t* new_to_old, const int32_t* rp_src, const int32_t* ci_src,
                               const int32_t* rp_dst, int32_t* ci_dst, const int32_t* map, cudaStream_t stream) {
    k_gather_rows<<<blocks_for(n, 256), 256, 0, stream>>>(n, new_to_old, rp_src, ci_src, rp_dst, ci_dst, map);
    return cudaGetLastError();
}

cudaError_t launch_inplace_static(int precision, const SweepArgs& a, int32_t threads, cudaStream_t stream) {
    if (threads <= 0 || a.v_end <= 0) return cudaErrorInvalidValue;
    const int32_t per = static_cast<int32_t>((static_cast<int64_t>(a.v_end) + threads - 1) / threads);
    const int blocks = static_cast<int>((static_cast<int64_t>(threads) + 255) / 256);
    if (precision == LMS_FP64)
        k_inplace_static<true><<<blocks, 256, 0, stream>>>(a, per);
    else
        k_inplace_static<false><<<blocks, 256, 0, stream>>>(a, per);
    return cudaGetLastError();
}

cudaError_t launch_flag_boundary_rows(int32_t n, const uint32_t* bits, int32_t* row_ptr, cudaStream_t stream) {
    k_flag_boundary_rows<<<blocks_for(n, 256), 256, 0, stream>>>(n, bits, row_ptr);
    return cudaGetLastError();
}

cudaError_t launch_map_ids(int64_t count, const int32_t* map, const int32_t* src, int32_t* dst,
                           cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    k_map_ids<<<blocks_for(count, 256), 256, 0, stream>>>(count, map, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_boundary_bits(int32_t n, const int32_t* new_to_old, const uint8_t* bnd_orig, uint32_t* bits,
                                 cudaStream_t stream) {
    k_boundary_bits<<<blocks_for(n, 256), 256, 0, stream>>>(n, new_to_old, bnd_orig, bits);
    return cudaGetLastError();
}

cudaError_t launch_gather_xy(int precision, int32_t n, const int32_t* perm, const void* src, void* dst,
                             cudaStream_t stream) {
    if (precision == LMS_FP64)
        k_gather_xy<double2><<<blocks_for(n, 256), 256, 0, stream>>>(n, perm, static_cast<const double2*>(src),
                                                                     static_cast<double2*>(dst));
    else
        k_gather_xy<float2><<<blocks_for(n, 256), 256, 0, stream>>>(n, perm, static_cast<const float2*>(src),
                                                                    static_cast<float2*>(dst));
    return cudaGetLastError();
}

cudaError_t launch_load_xy(int precision, int32_t n, const int32_t* new_to_old, const double* src_orig, void* dst,
                           double cx, double cy, double inv_s, cudaStream_t stream) {
    const double2* src = reinterpret_cast<const double2*>(src_orig);
    if (precision == LMS_FP64)
        k_load_xy_f64<<<blocks_for(n, 256), 256, 0, stream>>>(n, new_to_old, src, static_cast<double2*>(dst));
    else
        k_load_xy_f32<<<blocks_for(n, 256), 256, 0, stream>>>(n, new_to_old, src, static_cast<float2*>(dst), cx, cy,
                                                              inv_s);
    return cudaGetLastError();
}

cudaError_t launch_store_xy(int precision, int32_t n, const int32_t* new_to_old, const void* src, double* dst_orig,
                            double cx, double cy, double s, const uint8_t* bnd_orig, const double* fixed_xy,
                            cudaStream_t stream) {
    double2* dst = reinterpret_cast<double2*>(dst_orig);
    if (precision == LMS_FP64)
        k_store_xy_f64<<<blocks_for(n, 256), 256, 0, stream>>>(n, new_to_old, static_cast<const double2*>(src), dst);
    else
        k_store_xy_f32<<<blocks_for(n, 256), 256, 0, stream>>>(n, new_to_old, static_cast<const float2*>(src), dst,
                                                               cx, cy, s, bnd_orig,
                                                               reinterpret_cast<const double2*>(fixed_xy));
    return cudaGetLastError();
}

cudaError_t launch_batch_load_xy(int32_t n_items, const int2* items, const int32_t* item_mesh,
                                 const int32_t* new_to_old, const double* src_orig, float2* dst0, float2* dst1,
                                 const double* mesh_cs, int32_t* bad, cudaStream_t stream) {
    if (n_items <= 0) return cudaSuccess;
    k_batch_load_xy<<<n_items, 256, 0, stream>>>(items, item_mesh, new_to_old,
                                                 reinterpret_cast<const double2*>(src_orig), dst0, dst1, mesh_cs,
                                                 bad);
    return cudaGetLastError();
}

cudaError_t launch_batch_store_xy(int32_t n_items, const int2* items, const int32_t* item_mesh,
                                  const int32_t* new_to_old, const float2* src, double* dst_orig,
                                  const double* mesh_cs, const uint32_t* bnd_bits, const double* fixed_xy,
                                  cudaStream_t stream) {
    if (n_items <= 0) return cudaSuccess;
    k_batch_store_xy<<<n_items, 256, 0, stream>>>(items, item_mesh, new_to_old, src,
                                                  reinterpret_cast<double2*>(dst_orig), mesh_cs, bnd_bits,
                                                  reinterpret_cast<const double2*>(fixed_xy));
    return cudaGetLastError();
}

cudaError_t launch_block_gs(int precision, const BlockGsArgs& a, int32_t n_tiles, cudaStream_t stream) {
    if (n_tiles <= 0) return cudaSuccess;
    if (precision == LMS_FP64)
        k_block_gs<true><<<n_tiles, 256, 0, stream>>>(a);
    else
        k_block_gs<false><<<n_tiles, 256, 0, stream>>>(a);
    return cudaGetLastError();
}

size_t block_gs_staged_smem(int precision, int32_t max_slots, int32_t max_verts, int32_t max_entries) {
    const size_t pos = static_cast<size_t>(std::max(1, max_slots)) * (precision == LMS_FP64 ? sizeof(double2) : sizeof(float2));
    return pos + 4 * (static_cast<size_t>(max_verts) + 1) + 2 * static_cast<size_t>(max_verts) +
           2 * static_cast<size_t>(max_entries) + 16;
}

cudaError_t launch_block_gs_staged(int precision, const BlockGsStagedArgs& a, int32_t n_tiles, cudaStream_t stream) {
    if (n_tiles <= 0) return cudaSuccess;
    const size_t smem = block_gs_staged_smem(precision, a.max_slots, a.max_verts, a.max_entries);
    cudaError_t e;
    if (precision == LMS_FP64) {
        e = cudaFuncSetAttribute(k_block_gs_staged<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e == cudaSuccess) k_block_gs_staged<true><<<n_tiles, 256, smem, stream>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_block_gs_staged<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e == cudaSuccess) k_block_gs_staged<false><<<n_tiles, 256, smem, stream>>>(a);
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_div32_selftest(int32_t count, const float* s, const int32_t* d, float* q, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    k_div32_selftest<<<blocks_for(count, 256), 256, 0, stream>>>(count, s, d, q);
    return cudaGetLastError();
}

cudaError_t launch_add_selftest(int32_t count, const double* a, const double* b, double* s, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    k_add_selftest<<<blocks_for(count, 256), 256, 0, stream>>>(count, a, b, s);
    return cudaGetLastError();
}

cudaError_t launch_divint_selftest(int32_t count, const double* s, const int32_t* d, const double* recip, double* q,
                                   cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    k_divint_selftest<<<blocks_for(count, 256), 256, 0, stream>>>(count, s, d, recip, q);
    return cudaGetLastError();
}

cudaError_t launch_div_selftest(int32_t count, const double* s, const int32_t* d, const double* recip, double* q,
                                cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    k_div_selftest<<<blocks_for(count, 256), 256, 0, stream>>>(count, s, d, recip, q);
    return cudaGetLastError();
}

LMS_CHECK_ACCESSOR(check_violations_kernels)

bool checks_enabled() {
#ifdef LMS_CHECKS
    return true;
#else
    return false;
#endif
}

}  // namespace lms
