// lms_fp64_int.cuh - the FP64 arithmetic of the sweep's Eq. 1 on the integer pipes.
//
// GB300 executes FP64 instructions at about 1/64 of its FP32 rate (a little over one lane-operation per
// clock per SM in the sweep), so the sequential FP64 adds and the division of one vertex update bind the
// FP64 sweep.  The routines here compute the same correctly rounded results (IEEE 754 binary64, round to
// nearest, ties to even) from the bit patterns with integer instructions:
//
//   add_rn_int(a, b)          RN(a + b).  Both operands normal with exponents at most 9 apart: the
//                             larger significand is shifted left by the exponent difference so that the
//                             sum or difference of the two integers is exact (at most 63 bits), and it is
//                             rounded once.  Otherwise (zero or subnormal operands, the top binade, a wider
//                             exponent gap, a subnormal result) the FP64 unit adds.
//   root_of_ratio(lo, hi)     sqrt(lo / hi) within a few ulps for the per-sweep quality: an FP32 seed and
//                             two FP64 Newton steps (6 FP64 instructions instead of a division and a root).
//   div_rn_int(s, d, magic)   RN(s / d) for an integer 1 <= d <= 64: N = significand * 2^11 is divided by d
//                             with a multiply-high by floor((2^64 - 1) / d) (words magic[2d], magic[2d+1])
//                             and at most one correction (division by invariant integers, Granlund & Montgomery, PLDI 1994),
//                             giving the exact quotient and remainder, then rounded once.  Zero and
//                             subnormal sums, and subnormal results, are reported by returning false.
//
// Host builds (for CPU tests of this arithmetic) use the same integer code and the host FP unit for the
// excluded cases.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define LMS_HD __host__ __device__ __forceinline__
#else
#define LMS_HD inline
#endif

namespace lms {
namespace dev {

// Everything below works on 32-bit words: with a first form of these routines written on 64-bit
// integers, ncu counted the FP64 pipe as busy as with the FP64 adds they replaced - 64-bit integer
// instructions appear to share that narrow pipe on GB300.

LMS_HD uint32_t hi32(double x) {
#ifdef __CUDA_ARCH__
    return static_cast<uint32_t>(__double2hiint(x));
#else
    uint64_t u;
    std::memcpy(&u, &x, sizeof u);
    return static_cast<uint32_t>(u >> 32);
#endif
}

LMS_HD uint32_t lo32(double x) {
#ifdef __CUDA_ARCH__
    return static_cast<uint32_t>(__double2loint(x));
#else
    uint64_t u;
    std::memcpy(&u, &x, sizeof u);
    return static_cast<uint32_t>(u);
#endif
}

LMS_HD double from_hilo(uint32_t hi, uint32_t lo) {
#ifdef __CUDA_ARCH__
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
#else
    const uint64_t u = (static_cast<uint64_t>(hi) << 32) | lo;
    double x;
    std::memcpy(&x, &u, sizeof x);
    return x;
#endif
}

LMS_HD int clz32(uint32_t x) {  // x != 0
#ifdef __CUDA_ARCH__
    return __clz(static_cast<int>(x));
#else
    return __builtin_clz(x);
#endif
}

LMS_HD uint32_t umulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return static_cast<uint32_t>((static_cast<uint64_t>(a) * b) >> 32);
#endif
}

// upper word of (hi:lo) << k and lower word of (hi:lo) >> k, 0 <= k < 32
LMS_HD uint32_t shl_hi(uint32_t hi, uint32_t lo, int k) { return k ? (hi << k) | (lo >> (32 - k)) : hi; }
LMS_HD uint32_t shr_lo(uint32_t hi, uint32_t lo, int k) { return k ? (lo >> k) | (hi << (32 - k)) : lo; }

LMS_HD double add_rn_fpu(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dadd_rn(a, b);
#else
    volatile double s = a + b;  // one IEEE addition, never contracted
    return s;
#endif
}

// 0.0 + x for finite x: x itself, except that -0 becomes +0 (round to nearest).  The first term of a
// sum that starts at 0.0, with no FP64 instruction.
LMS_HD double plus_zero(double x) {
    const uint32_t h = hi32(x), l = lo32(x);
    return (h == 0x80000000u && l == 0u) ? 0.0 : x;
}

// Round the positive integer (sh:sl), whose leading bit is at position p (52 <= p <= 63), to its top 53
// bits (nearest, ties to even) and pack them under biased exponent e (the exponent of that leading bit)
// and `sign`.  `above` marks an exact value strictly greater than (sh:sl) (a nonzero remainder below bit
// 0).  Requires e >= 1.
LMS_HD double round_pack(uint32_t sh, uint32_t sl, int p, int e, bool above, uint32_t sign) {
    const int k = p - 52;  // bits dropped, 0..11
    const uint32_t rest = sl & ((1u << k) - 1u), half = k > 0 ? 1u << (k - 1) : 1u;
    uint32_t ql = shr_lo(sh, sl, k), qh = sh >> k;
    // k == 0: nothing dropped (rest == 0 < half)
    const uint32_t up = k > 0 && (rest > half || (rest == half && (above || (ql & 1u)))) ? 1u : 0u;
    ql += up;
    qh += (up && ql == 0u) ? 1u : 0u;
    // adding the significand (implicit bit 20 of the high word) to the biased exponent minus one carries
    // a rounded-up 2^53 into the exponent (and exponent 2047 is infinity, the round-to-nearest overflow)
    return from_hilo(((static_cast<uint32_t>(e - 1) << 20) + qh) | sign, ql);
}

// RN(a + b), bit for bit the IEEE 754 binary64 sum.
LMS_HD double add_rn_int(double a, double b) {
    const uint32_t ah = hi32(a), al = lo32(a), bh = hi32(b), bl = lo32(b);
    const uint32_t mah = ah & 0x7fffffffu, mbh = bh & 0x7fffffffu;
    const bool swap = mbh > mah || (mbh == mah && bl > al);
    const uint32_t xh = swap ? mbh : mah, xl = swap ? bl : al;  // |x| >= |y|
    const uint32_t yh = swap ? mah : mbh, yl = swap ? al : bl;
    const uint32_t sign = (swap ? bh : ah) & 0x80000000u;
    const int ex = static_cast<int>(xh >> 20), ey = static_cast<int>(yh >> 20);
    const int d = ex - ey;
    if (ey == 0 || ex >= 2046 || d > 9) return add_rn_fpu(a, b);
    // exact: x's significand shifted by d (<= 62 bits), in units of y's last bit
    const uint32_t fxh0 = (xh & 0xfffffu) | 0x100000u;
    const uint32_t fxh = shl_hi(fxh0, xl, d), fxl = xl << d;
    const uint32_t fyh = (yh & 0xfffffu) | 0x100000u, fyl = yl;
    uint32_t sh, sl;
    if ((ah ^ bh) & 0x80000000u) {  // |x| - |y| >= 0
        sl = fxl - fyl;
        sh = fxh - fyh - (fxl < fyl ? 1u : 0u);
    } else {
        sl = fxl + fyl;
        sh = fxh + fyh + (sl < fxl ? 1u : 0u);
    }
    if ((sh | sl) == 0u) return 0.0;  // exact cancellation gives +0 under round to nearest
    const int p = sh != 0u ? 63 - clz32(sh) : 31 - clz32(sl);
    const int e = ey + p - 52;  // biased exponent of the result
    if (p < 52) {  // cancellation: exact, shifted up to 53 bits
        if (e <= 0) return add_rn_fpu(a, b);  // subnormal result
        const int k = 52 - p;
        const uint32_t qh = k >= 32 ? sl << (k - 32) : shl_hi(sh, sl, k), ql = k >= 32 ? 0u : sl << k;
        return from_hilo(((static_cast<uint32_t>(e - 1) << 20) + qh) | sign, ql);
    }
    return round_pack(sh, sl, p, e, false, sign);
}

// magic[2d], magic[2d + 1] = high and low words of floor((2^64 - 1) / d), for the division below
LMS_HD void div_magic(int d, uint32_t* hi, uint32_t* lo) {
    const uint64_t m = ~0ull / static_cast<uint64_t>(d);
    *hi = static_cast<uint32_t>(m >> 32);
    *lo = static_cast<uint32_t>(m);
}

// RN(s / d) into *q for 1 <= d <= 64, bit for bit the IEEE quotient; false (and *q untouched) when s is
// zero or subnormal or the quotient would be subnormal - the caller divides on the FP64 unit then.
LMS_HD bool div_rn_int(double s, int d, const uint32_t* magic, double* q) {
    const uint32_t h = hi32(s), l = lo32(s);
    const int es = static_cast<int>((h >> 20) & 0x7ffu);
    if (es == 0) return false;
    // n = significand * 2^11, leading bit at 63
    const uint32_t nh = (((h & 0xfffffu) | 0x100000u) << 11) | (l >> 21), nl = l << 11;
    const uint32_t mh = magic[2 * d], ml = magic[2 * d + 1];
    // high 64 bits of n * magic (32 x 32 partial products, carries counted in 32 bits); n * magic / 2^64
    // lies within n / 2^64 < 1 below n / d (2^64 - d * magic <= d), so this is floor(n / d) or one less
    const uint32_t t0 = umulhi32(nl, ml);
    const uint32_t a1 = nl * mh, b1 = umulhi32(nl, mh);
    const uint32_t a2 = nh * ml, b2 = umulhi32(nh, ml);
    const uint32_t a3 = nh * mh, b3 = umulhi32(nh, mh);
    uint32_t mid = t0 + a1;
    uint32_t c = mid < a1 ? 1u : 0u;
    mid += a2;
    c += mid < a2 ? 1u : 0u;
    uint32_t ql = b1 + c;
    uint32_t c2 = ql < c ? 1u : 0u;
    ql += b2;
    c2 += ql < b2 ? 1u : 0u;
    ql += a3;
    c2 += ql < a3 ? 1u : 0u;
    uint32_t qh = b3 + c2;
    // remainder n - q*d < 2d <= 128: its low word is exact
    const uint32_t dd = static_cast<uint32_t>(d);
    uint32_t r = nl - ql * dd;
    if (r >= dd) {
        r -= dd;
        ++ql;
        qh += ql == 0u ? 1u : 0u;
    }
    const int p = 63 - clz32(qh);  // 57..63: n / d >= 2^63 / 64
    const int e = es + p - 63;     // s / d = q * 2^(es - 1086), leading bit p
    if (e <= 0) return false;
    *q = round_pack(qh, ql, p, e, r != 0u, h & 0x80000000u);
    return true;
}

// ---- sqrt(lo / hi) for the per-sweep quality: an FP32 seed refined by two FP64 Newton steps

LMS_HD float f32_from_bits(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __int_as_float(static_cast<int>(u));
#else
    float x;
    std::memcpy(&x, &u, sizeof x);
    return x;
#endif
}

LMS_HD uint32_t f32_bits(float x) {
#ifdef __CUDA_ARCH__
    return static_cast<uint32_t>(__float_as_int(x));
#else
    uint32_t u;
    std::memcpy(&u, &x, sizeof u);
    return u;
#endif
}

// one IEEE operation each, rounded to nearest
LMS_HD float f32_sqrt_of_ratio(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsqrt_rn(__fdiv_rn(a, b));
#else
    volatile float q = a / b;
    return std::sqrt(static_cast<float>(q));
#endif
}

LMS_HD float f32_rcp_twice_product(float y, float h) {
#ifdef __CUDA_ARCH__
    return __frcp_rn(__fmul_rn(2.f, __fmul_rn(y, h)));
#else
    volatile float p = y * h;
    volatile float p2 = 2.f * p;
    return 1.f / static_cast<float>(p2);
#endif
}

LMS_HD double f64_newton_step(double q, double lo, double hi, double c) {  // q - (q*q*hi - lo) * c
#ifdef __CUDA_ARCH__
    return __fma_rn(-__fma_rn(__dmul_rn(q, q), hi, -lo), c, q);
#else
    volatile double qq = q * q;
    return std::fma(-std::fma(static_cast<double>(qq), hi, -lo), c, q);
#endif
}

LMS_HD double root_of_ratio_fpu(double lo, double hi) {
    if (!(hi > 0.0)) return 0.0;
#ifdef __CUDA_ARCH__
    return sqrt(lo / hi);
#else
    volatile double r = lo / hi;
    return std::sqrt(static_cast<double>(r));
#endif
}

// sqrt(lo / hi) for 0 <= lo <= hi (the shortest and longest squared edge of a triangle), within a few
// ulps.  The seed: FP32 images of lo and hi scaled by 2^-(ehi - 1023) so that hi lies in [1, 2)
// (mantissas truncated to 23 bits), y0 = sqrt(lo' / hi') and c = 1 / (2 y0 hi') in FP32 (relative error
// under 3e-7), both widened exactly to FP64 through their bit patterns (c rescaled by 2^-(ehi - 1023)).
// Two Newton steps q <- q - (q^2 hi - lo) c square that error (about 1e-13 after one step, a few ulps
// after two).  lo zero or subnormal, hi outside [2^-959, 2^959], or lo/hi below 2^-126 take the FPU.
LMS_HD double root_of_ratio(double lo, double hi) {
    const uint32_t hih = hi32(hi), hil = lo32(hi), loh = hi32(lo), lol = lo32(lo);
    const int ehi = static_cast<int>(hih >> 20), elo = static_cast<int>(loh >> 20);
    if (ehi < 64 || ehi > 1982 || ehi - elo > 126 || elo == 0) return root_of_ratio_fpu(lo, hi);
    const float hf = f32_from_bits((127u << 23) | ((hih & 0xfffffu) << 3) | (hil >> 29));
    const float lf = f32_from_bits((static_cast<uint32_t>(elo - ehi + 127) << 23) | ((loh & 0xfffffu) << 3) |
                                   (lol >> 29));
    const float y0 = f32_sqrt_of_ratio(lf, hf);   // in [2^-64, 1]
    const float cf = f32_rcp_twice_product(y0, hf);  // in (1/4, 2^63]
    const uint32_t yb = f32_bits(y0), cb = f32_bits(cf);
    const double q0 = from_hilo((((yb >> 23) + 896u) << 20) | ((yb & 0x7fffffu) >> 3), yb << 29);
    const double c = from_hilo((static_cast<uint32_t>(static_cast<int>(cb >> 23) + 1919 - ehi) << 20) |
                                   ((cb & 0x7fffffu) >> 3),
                               cb << 29);
    return f64_newton_step(f64_newton_step(q0, lo, hi, c), lo, hi, c);
}

}  // namespace dev
}  // namespace lms
