// lms_noalloc.cu - FP64 Jacobi sweeps that allocate no device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or under a fixed device-memory budget, services
// that forbid allocations on their steady-state path, or code recorded into a
// CUDA graph by a caller that manages every buffer itself.  This entry point
// takes all inputs and outputs from the caller; the only scratch the sweeps
// need - one work-queue counter per sweep - lives in a fixed file-scope
// device array, so each GPU that loads the library holds it (4 KB) until the
// process exits.
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "lms_device.cuh"
#include "lms_internal.h"

namespace {

constexpr int kNoAllocMaxSweeps = 1024;  // sweeps one call can run (one counter each)
constexpr int kNoAllocTile = 256;        // vertices per work item (= threads per CTA)
constexpr int kMaxDevices = 64;

// Work-queue counters, one per sweep of a call.  Shared by every call on a device.
__device__ __align__(256) int32_t g_noalloc_queue[kNoAllocMaxSweeps];

std::mutex g_setup_mu;
int32_t* g_queue_addr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

// Every interior vertex moves to the mean of its neighbours' positions (FP64 sums in stored row order,
// then one IEEE division by the neighbour count); boundary vertices are copied.  CTAs pull tiles of
// kNoAllocTile vertices from *queue.
__global__ void __launch_bounds__(kNoAllocTile) k_jacobi_noalloc(int32_t n, const int32_t* __restrict__ row_ptr,
                                                                 const int32_t* __restrict__ col_idx,
                                                                 const uint8_t* __restrict__ is_boundary,
                                                                 const double2* __restrict__ src,
                                                                 double2* __restrict__ dst, int32_t* queue) {
    __shared__ int32_t s_tile;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(queue, 1);
        __syncthreads();
        const int64_t first = static_cast<int64_t>(s_tile) * kNoAllocTile;
        __syncthreads();
        if (first >= n) break;
        const int64_t v = first + threadIdx.x;
        if (v < n) {
            double2 r = src[v];
            if (!is_boundary[v]) {
                const int32_t e0 = row_ptr[v], e1 = row_ptr[v + 1];
                double sx = 0.0, sy = 0.0;
                for (int32_t e = e0; e < e1; ++e) {
                    const int32_t u = col_idx[e];
                    if (!LMS_CHECK(u >= 0 && u < n)) continue;
                    const double2 p = src[u];
                    sx = __dadd_rn(sx, p.x);
                    sy = __dadd_rn(sy, p.y);
                }
                r.x = __ddiv_rn(sx, static_cast<double>(e1 - e0));
                r.y = __ddiv_rn(sy, static_cast<double>(e1 - e0));
            }
            dst[v] = r;
        }
    }
}

// Address of the counters on the current device.  The first call on a device looks it up and caches it;
// a cudaDeviceReset of that device ends the context the array lived in, so the cached address is stale
// afterwards (the header tells callers not to use this entry point on a device after a reset).
int noalloc_setup(int32_t** queue, int* sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        lms::set_error_detail(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return LMS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        lms::set_error_detail("device index beyond the 64 devices lms_jacobi_noalloc supports");
        return LMS_ERR_ARG;
    }
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (g_queue_addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_queue);
        if (e != cudaSuccess) {
            lms::set_error_detail(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return LMS_ERR_CUDA;
        }
        int count = 0;
        e = cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) {
            lms::set_error_detail(std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
            return LMS_ERR_CUDA;
        }
        g_sm_count[dev] = count;
        g_queue_addr[dev] = static_cast<int32_t*>(p);
    }
    *queue = g_queue_addr[dev];
    *sms = g_sm_count[dev];
    return LMS_OK;
}

}  // namespace

namespace lms {
LMS_CHECK_ACCESSOR(check_violations_noalloc)
}  // namespace lms

extern "C" int lms_jacobi_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                  const uint8_t* is_boundary, double* xy, double* xy_tmp, int32_t iters,
                                  void* cuda_stream) {
    if (n <= 0 || !row_ptr || !col_idx || !is_boundary || !xy || !xy_tmp || iters < 0) return LMS_ERR_ARG;
    {  // the two position buffers must not share a byte: [xy, xy + 2n) and [xy_tmp, xy_tmp + 2n)
        const uintptr_t a0 = reinterpret_cast<uintptr_t>(xy), b0 = reinterpret_cast<uintptr_t>(xy_tmp);
        const uintptr_t len = sizeof(double) * 2 * uintptr_t(n);
        if (a0 < b0 + len && b0 < a0 + len) {
            lms::set_error_detail("lms_jacobi_noalloc: xy and xy_tmp overlap");
            return LMS_ERR_ARG;
        }
    }
    if (iters > kNoAllocMaxSweeps) {
        lms::set_error_detail("lms_jacobi_noalloc runs at most 1024 sweeps per call");
        return LMS_ERR_ARG;
    }
    int32_t* queue = nullptr;
    int sms = 0;
    const int rc = noalloc_setup(&queue, &sms);
    if (rc != LMS_OK) return rc;
    if (iters == 0) return LMS_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the counters keep the previous call's values: clear the ones this call uses
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int32_t) * size_t(iters), s);
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>(8 * int64_t(sms), (int64_t(n) + kNoAllocTile - 1) /
                                                                                    kNoAllocTile)));
    double2* a = reinterpret_cast<double2*>(xy);
    double2* b = reinterpret_cast<double2*>(xy_tmp);
    for (int32_t k = 0; k < iters && e == cudaSuccess; ++k) {
        const bool even = (k & 1) == 0;
        k_jacobi_noalloc<<<grid, kNoAllocTile, 0, s>>>(n, row_ptr, col_idx, is_boundary, even ? a : b, even ? b : a,
                                                       queue + k);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && (iters & 1))
        e = cudaMemcpyAsync(xy, xy_tmp, sizeof(double2) * size_t(n), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        lms::set_error_detail(std::string("lms_jacobi_noalloc: ") + cudaGetErrorString(e));
        return LMS_ERR_CUDA;
    }
    return LMS_OK;
}
