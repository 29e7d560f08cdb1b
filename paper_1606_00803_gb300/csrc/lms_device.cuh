// lms_device.cuh - device helpers shared by the sweep kernels (lms_kernels.cu, lms_staged.cu).
#pragma once

#include <cstdint>

#include "lms_internal.h"

// Bounds checks of debug builds (nvcc -DLMS_CHECKS): LMS_CHECK(cond) counts a failed check in this
// translation unit's g_check_violations and yields false, so the caller skips the access; in release
// builds it is the constant true and compiles away.  Each kernel source defines a host accessor with
// LMS_CHECK_ACCESSOR(name).
namespace lms {
namespace dev {
#ifdef LMS_CHECKS
static __device__ unsigned long long g_check_violations;
__device__ __forceinline__ bool check_ok(bool c) {
    if (!c) atomicAdd(&g_check_violations, 1ull);
    return c;
}
#define LMS_CHECK(cond) (::lms::dev::check_ok(cond))
#define LMS_CHECK_ACCESSOR(name)                                                                  \
    unsigned long long name(bool reset) {                                                         \
        unsigned long long v = 0;                                                                 \
        cudaMemcpyFromSymbol(&v, ::lms::dev::g_check_violations, sizeof(v));                      \
        if (reset) {                                                                              \
            const unsigned long long zero = 0;                                                    \
            cudaMemcpyToSymbol(::lms::dev::g_check_violations, &zero, sizeof(zero));              \
        }                                                                                         \
        return v;                                                                                 \
    }
#else
#define LMS_CHECK(cond) true
#define LMS_CHECK_ACCESSOR(name) \
    unsigned long long name(bool) { return 0; }
#endif

__device__ __forceinline__ bool boundary_bit(const uint32_t* __restrict__ bits, int32_t v) {
    return (__ldg(bits + (v >> 5)) >> (v & 31)) & 1u;
}

// s / d for a positive integer d, correctly rounded: y = RN(1/d) from the table, q = RN(s*y), then one
// correction q + RN(s - d*q)*y with fused operations (Markstein's division refinement, IBM J. Res. Dev.
// 34(1), 1990).  About three FP64 operations instead of a full IEEE division; lms_selftest_div64 checks it
// against IEEE division.  The refinement can miss by an ulp when the quotient is subnormal, so sums below
// 2^-959 (biased exponent under 64; an integer test on the high word) take the IEEE division.
__device__ __forceinline__ double div_by_count(double s, int32_t d, const double* recip) {
    if (d <= kMaxRecipDeg && ((__double2hiint(s) >> 20) & 0x7ff) >= 64) {
        const double y = recip[d];
        const double q = __dmul_rn(s, y);
        const double r = __fma_rn(-q, static_cast<double>(d), s);
        return __fma_rn(r, y, q);
    }
    return __ddiv_rn(s, static_cast<double>(d));
}

// FP32 mean of a compensated sum: a = s - c divided by the neighbour count d.  y = RN(1/d), q = RN(a*y),
// then one fused correction q + RN(a - d*q)*y (Markstein's division refinement, as for the FP64 sweep):
// the correctly rounded quotient for every |a| >= 2^-100 - every sum of a mesh normalised to unit size -
// and zero for a zero sum (the select keeps the sign of a negative zero); within one ulp below 2^-100
// (subnormal quotients).  The single rounding, against 1.5 ulp for a multiply by the rounded reciprocal,
// is most of the error an FP32 sweep adds to the stored positions.  Two FMAs and no branch: an IEEE
// division, or a branch to one for special values, costs 1-4% of a batched sweep.  lms_selftest_div32
// checks it against IEEE division.
__device__ __forceinline__ float mean_f32(float s, float c, int32_t d) {
    const float a = __fsub_rn(s, c);
    const float df = static_cast<float>(d);
    const float y = __frcp_rn(df);
    const float q = __fmul_rn(a, y);
    const float r = __fmaf_rn(-q, df, a);
    const float m = __fmaf_rn(r, y, q);
    return a == 0.f ? a : m;
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// The largest squared displacement of a warp into *disp2 (bits of a non-negative double, which order like
// the values); warp maxima by 32-bit shuffles.  Every warp of a sweep reports to the same word, so the atomic is issued only when the
// warp's maximum exceeds the value already there: a plain read first, which turns hundreds of thousands
// of same-address atomics per sweep (serialised at one L2 slice) into a handful.
__device__ __forceinline__ void max_to(unsigned long long* disp2, unsigned long long m) {
    if (m != 0ull && m > *reinterpret_cast<volatile unsigned long long*>(disp2)) atomicMax(disp2, m);
}

__device__ __forceinline__ void record_disp(unsigned long long* disp2, double d2) {
    uint32_t hi = static_cast<uint32_t>(__double2hiint(d2)), lo = static_cast<uint32_t>(__double2loint(d2));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint32_t h = __shfl_xor_sync(0xffffffffu, hi, o), l = __shfl_xor_sync(0xffffffffu, lo, o);
        if (h > hi || (h == hi && l > lo)) {
            hi = h;
            lo = l;
        }
    }
    if ((threadIdx.x & 31) == 0) max_to(disp2, (static_cast<unsigned long long>(hi) << 32) | lo);
}


}  // namespace dev
}  // namespace lms
