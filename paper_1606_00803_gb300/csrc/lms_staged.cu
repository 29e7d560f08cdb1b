// lms_staged.cu - the tile-staged sweep kernel (Eq. 1 over vertex tiles).
//
// A persistent grid pulls vertex tiles from a device counter.  For each tile
// [a, b) one thread issues three TMA bulk copies (cp.async.bulk, completion on
// an mbarrier) that bring the tile's row offsets row_ptr[a..b], its neighbour
// ids col_idx[row_ptr[a] .. row_ptr[b]) and its boundary bits into shared
// memory; the copies for tile i+1 are issued before tile i is processed (two
// buffers).  Then:
//   phase A (edge-parallel): lane k of the block takes entry k of the tile's
//     neighbour list and gathers that neighbour's position into shared memory
//     - every lane of every gather instruction does useful work, and the CSR
//     never passes through the load/store unit;
//   phase B (vertex-parallel): each thread sums its vertex's gathered
//     neighbours from shared memory in row order (FP64: sequential sums and the
//     correctly rounded division, so results equal the oracle's bit for bit;
//     FP32: Kahan sums) and writes the new position.
// Jacobi reads `src` and writes `dst`; the coloured Gauss-Seidel runs one
// launch per colour with src == dst over tiles of that colour's range (no
// vertex of the colour is a neighbour of another, so phase A never reads a
// position phase B writes in the same launch).
//
// Every wait on an mbarrier is bounded (~1 s of clock cycles); on expiry the
// kernel records an error word, drains its own outstanding copies (bounded
// again) and returns, so a fault in the copy path cannot hang the GPU.
#include <cstdint>
#include <type_traits>

#include "lms_device.cuh"
#include "lms_internal.h"

namespace lms {

namespace {
using namespace dev;

constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// bounded wait for the phase with the given parity; false when the bound (in clock cycles) expired
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long bound = kWaitCycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > bound) return false;
    return true;
}

// Self-test of the bounded wait: one thread waits for an mbarrier phase that nothing completes (no
// thread arrives, no copy is issued), gives up after `bound` cycles and records where it gave up in
// *err, as a tile-copy wait of k_sweep_staged would.
__global__ void k_wait_selftest(long long bound, int32_t* err) {
    __shared__ __align__(8) uint64_t bar;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(&bar, 0, bound)) atomicExch(err, 1);
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

struct Layout {
    uint32_t rp_words, ci_words, bit_words;  // per buffer, each a multiple of 4
};

__device__ __forceinline__ Layout layout_of(const StagedArgs& a) {
    Layout L;
    L.rp_words = (static_cast<uint32_t>(a.tile_cap) + 8u + 3u) & ~3u;
    L.ci_words = (static_cast<uint32_t>(a.e_cap) + 8u + 3u) & ~3u;
    L.bit_words = ((static_cast<uint32_t>(a.tile_cap) >> 5) + 8u + 3u) & ~3u;
    return L;
}

// Issue the three copies of tile `item` into buffer `buf`; called by one thread.
__device__ __forceinline__ void issue_tile(const StagedArgs& a, const int4 t, int32_t* rp_s, int32_t* ci_s,
                                           uint32_t* bits_s, uint64_t* bar) {
    const int32_t va = t.x, vb = t.y, e0 = t.z, e1 = t.w;
    const int32_t r0 = va & ~3;
    const uint32_t rp_bytes = static_cast<uint32_t>(((vb + 1 - r0) + 3) & ~3) * 4u;
    const int32_t c0 = e0 & ~3;
    const uint32_t ci_bytes = static_cast<uint32_t>(((e1 - c0) + 3) & ~3) * 4u;
    uint32_t bit_bytes = 0;
    int32_t w0 = 0;
    if (a.bnd_bits != nullptr) {
        w0 = (va >> 5) & ~3;
        const int32_t w1 = (vb - 1) >> 5;
        bit_bytes = static_cast<uint32_t>(((w1 + 1 - w0) + 3) & ~3) * 4u;
    }
    mbar_expect_tx(bar, rp_bytes + ci_bytes + bit_bytes);
    bulk_g2s(rp_s, a.row_ptr + r0, rp_bytes, bar);
    if (ci_bytes) bulk_g2s(ci_s, a.col_idx + c0, ci_bytes, bar);
    if (bit_bytes) bulk_g2s(bits_s, a.bnd_bits + w0, bit_bytes, bar);
}

template <bool FP64, bool IN_PLACE>
__global__ void __launch_bounds__(256) k_sweep_staged(StagedArgs a) {
    using V = typename std::conditional<FP64, double2, float2>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int32_t s_item[3];
    __shared__ double s_recip[kMaxRecipDeg + 1];
    __shared__ int32_t s_abort;

    if (a.state != nullptr && *reinterpret_cast<const volatile int32_t*>(&a.state->stop)) return;
    const Layout L = layout_of(a);
    // buffer b: row offsets, neighbour ids, boundary bits; then the gathered positions
    const uint32_t buf_bytes = 4u * (L.rp_words + L.ci_words + L.bit_words);
    auto rp_buf = [&](int b) { return reinterpret_cast<int32_t*>(smem + b * buf_bytes); };
    auto ci_buf = [&](int b) { return reinterpret_cast<int32_t*>(smem + b * buf_bytes + 4u * L.rp_words); };
    auto bits_buf = [&](int b) {
        return reinterpret_cast<uint32_t*>(smem + b * buf_bytes + 4u * (L.rp_words + L.ci_words));
    };
    V* pos_s = reinterpret_cast<V*>(smem + 2u * buf_bytes);
    const V* src = static_cast<const V*>(a.src);
    V* dst = static_cast<V*>(a.dst);

    if (FP64)
        for (int i = threadIdx.x; i <= kMaxRecipDeg; i += blockDim.x) s_recip[i] = a.recip[i];
    uint32_t issued = 0u;  // bit b: a copy into buffer b is outstanding (thread 0 only)
    uint32_t parity = 0u;  // bit b: parity of buffer b's next phase
    // s_item[i % 3] holds the tile of iteration i; tickets are drawn from the queue two tiles ahead so
    // the atomic's latency overlaps a tile's work
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
        const int32_t first = atomicAdd(a.queue, 1);
        s_item[0] = first;
        s_item[1] = atomicAdd(a.queue, 1);
        if (first < a.n_items) {
            issue_tile(a, __ldg(a.items + first), rp_buf(0), ci_buf(0), bits_buf(0), &bars[0]);
            issued = 1u;
        }
    }
    __syncthreads();

    const bool want_disp = a.disp2 != nullptr;
    int slot = 0;  // it % 3
    for (int it = 0;; ++it) {
        const int buf = it & 1;
        const int32_t item = s_item[slot];
        if (item >= a.n_items) break;
        int32_t ticket = 0;
        if (threadIdx.x == 0) {
            // prefetch the next tile into the other buffer (all threads finished reading it)
            const int32_t next = s_item[slot == 2 ? 0 : slot + 1];
            if (next < a.n_items) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue_tile(a, __ldg(a.items + next), rp_buf(buf ^ 1), ci_buf(buf ^ 1), bits_buf(buf ^ 1),
                           &bars[buf ^ 1]);
                issued |= 2u >> buf;
            }
            ticket = atomicAdd(a.queue, 1);  // tile of iteration it + 2, stored at the end of this one
            if (mbar_wait(&bars[buf], (parity >> buf) & 1u))
                issued &= ~(1u << buf);
            else
                s_abort = 1;
        }
        __syncthreads();
        if (s_abort) break;
        parity ^= 1u << buf;

        const int4 t = __ldg(a.items + item);
        const int32_t va = t.x, vb = t.y, e0 = t.z, e1 = t.w;
        const int32_t* ci = ci_buf(buf) + (e0 & 3);
        const int32_t* rp = rp_buf(buf) + (va & 3);
        const uint32_t* bits = bits_buf(buf);
        // phase A: gather every neighbour position of the tile into shared memory; each thread keeps
        // kGather independent loads in flight
        {
            constexpr int kGather = 8;
            const int32_t E = e1 - e0;
            for (int32_t k0 = threadIdx.x; k0 < E; k0 += kGather * blockDim.x) {
                int32_t u[kGather];
                V p[kGather];
#pragma unroll
                for (int g = 0; g < kGather; ++g) {
                    const int32_t k = k0 + g * static_cast<int32_t>(blockDim.x);
                    u[g] = k < E ? ci[k] : -1;
                    if (u[g] >= 0 && !LMS_CHECK(u[g] < a.n_vertices)) u[g] = -1;
                }
#pragma unroll
                for (int g = 0; g < kGather; ++g)
                    if (u[g] >= 0) p[g] = IN_PLACE ? src[u[g]] : __ldg(src + u[g]);
#pragma unroll
                for (int g = 0; g < kGather; ++g) {
                    const int32_t k = k0 + g * static_cast<int32_t>(blockDim.x);
                    if (k < E) pos_s[k] = p[g];
                }
            }
        }
        __syncthreads();
        // phase B: Eq. 1 per vertex, summing in row order (rounds are uniform across the block, so the
        // warp-wide displacement reduction sees every lane)
        const int32_t w0 = (va >> 5) & ~3;
        for (int32_t base = 0; base < vb - va; base += blockDim.x) {
            const int32_t j = base + threadIdx.x;
            const int32_t v = va + j;
            double d2 = 0.0;
            const bool active =
                j < vb - va && !(a.bnd_bits != nullptr && ((bits[(v >> 5) - w0] >> (v & 31)) & 1u));
            if (active) {
                // (a batch's offsets carry a boundary flag in bit 31)
                const int32_t r0 = (rp[j] & 0x7fffffff) - e0, r1 = (rp[j + 1] & 0x7fffffff) - e0;
                V r;
                if constexpr (FP64) {
                    double sx = 0.0, sy = 0.0;
                    for (int32_t e = r0; e < r1; ++e) {
                        const V p = pos_s[e];
                        sx = __dadd_rn(sx, p.x);
                        sy = __dadd_rn(sy, p.y);
                    }
                    r.x = div_by_count(sx, r1 - r0, s_recip);
                    r.y = div_by_count(sy, r1 - r0, s_recip);
                } else {
                    float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
                    for (int32_t e = r0; e < r1; ++e) {
                        const V p = pos_s[e];
                        kahan_add(sx, cx, p.x);
                        kahan_add(sy, cy, p.y);
                    }
                    r.x = mean_f32(sx, cx, r1 - r0);
                    r.y = mean_f32(sy, cy, r1 - r0);
                }
                if (want_disp) {
                    const V o = src[v];
                    const double dx = static_cast<double>(r.x) - static_cast<double>(o.x);
                    const double dy = static_cast<double>(r.y) - static_cast<double>(o.y);
                    d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
                }
                dst[v] = r;
            }
            if (want_disp) record_disp(a.disp2, d2);
        }
        if (threadIdx.x == 0) s_item[slot == 0 ? 2 : slot - 1] = ticket;  // slot of iteration it + 2
        slot = slot == 2 ? 0 : slot + 1;
        __syncthreads();
    }
    if (threadIdx.x == 0 && s_abort) {
        atomicExch(a.err, 1);
        // drain this CTA's own outstanding copies (bounded) before its shared memory goes away
        for (int i = 0; i < 2; ++i)
            if ((issued >> i) & 1u) (void)mbar_wait(&bars[i], (parity >> i) & 1u);
    }
}

template <bool FP64, bool IN_PLACE>
cudaError_t launch_t(const StagedArgs& a, int grid, int block, size_t smem, cudaStream_t stream) {
    auto kern = k_sweep_staged<FP64, IN_PLACE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<grid, block, smem, stream>>>(a);
    return cudaGetLastError();
}

template <bool FP64, bool IN_PLACE>
int occupancy_t(int block, size_t smem) {
    auto kern = k_sweep_staged<FP64, IN_PLACE>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
        cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, block, smem) != cudaSuccess) return 0;
    return n;
}

}  // namespace

cudaError_t launch_wait_selftest(long long bound_cycles, int32_t* err, cudaStream_t stream) {
    k_wait_selftest<<<1, 1, 0, stream>>>(bound_cycles, err);
    return cudaGetLastError();
}

size_t staged_smem_bytes(int precision, int32_t tile_cap, int32_t e_cap) {
    const size_t rp = ((size_t(tile_cap) + 8 + 3) & ~size_t(3)) * 4;
    const size_t ci = ((size_t(e_cap) + 8 + 3) & ~size_t(3)) * 4;
    const size_t bits = (((size_t(tile_cap) >> 5) + 8 + 3) & ~size_t(3)) * 4;
    const size_t pos = size_t(e_cap + 8) * (precision == LMS_FP64 ? 16 : 8);
    return 2 * (rp + ci + bits) + 16 + pos;
}

cudaError_t launch_sweep_staged(int precision, bool in_place, const StagedArgs& a, int grid, int block,
                                cudaStream_t stream) {
    if (a.n_items <= 0) return cudaSuccess;
    const size_t smem = staged_smem_bytes(precision, a.tile_cap, a.e_cap);
    if (precision == LMS_FP64)
        return in_place ? launch_t<true, true>(a, grid, block, smem, stream)
                        : launch_t<true, false>(a, grid, block, smem, stream);
    return in_place ? launch_t<false, true>(a, grid, block, smem, stream)
                    : launch_t<false, false>(a, grid, block, smem, stream);
}

LMS_CHECK_ACCESSOR(check_violations_staged)

int staged_occupancy(int precision, bool in_place, int block, int32_t tile_cap, int32_t e_cap) {
    const size_t smem = staged_smem_bytes(precision, tile_cap, e_cap);
    if (precision == LMS_FP64) return in_place ? occupancy_t<true, true>(block, smem) : occupancy_t<true, false>(block, smem);
    return in_place ? occupancy_t<false, true>(block, smem) : occupancy_t<false, false>(block, smem);
}

}  // namespace lms
