// fp64_math.cuh -- table-driven FP64 exponential and logarithm for the 1-D rate
// lookups of the FP64 evolution.  GB300's FP64 pipe bounds that kernel, so its
// speed is its FP64 instruction count, and these two functions are a quarter
// of it.  Both take P. T. P. Tang's table-driven reductions (ACM TOMS 15 (1989)
// 144 for the exponential, 16 (1990) 378 for the logarithm) with Taylor
// polynomials of the reduced argument; the tables hold correctly rounded values
// (fp64_tables.h, written by gen_fp64_tables.py).  Every table index and the
// power-of-two scaling come from integer operations on the bits.  Errors, over
// the whole double range (checked against the CUDA library and the host's
// libm): the exponential within 2 ulp; the logarithm within 2 ulp plus 2^-57
// absolute (near x = 1, where ln x is small, the roundings of ln c_j, 1/c_j
// and r, each of order 2^-61, no longer shrink with the result; the rate
// lookups use ln chi as an interpolation coordinate, where only the absolute
// error counts).
#pragma once

#include "fp64_tables.h"

namespace qed {

// x = n ln2/64 + r with n = 64 k + j and |r| <= ln2/128; e^r - 1 by its Taylor
// polynomial of degree 5 (the remainder r^6/720 is below 2^-54, a third of an
// ulp of e^r), and e^x = 2^k 2^(j/64) e^r.  No range check.
__device__ __forceinline__ double exp_tang_core(double x, int &k)
{
    const double kShift = 0x1.8p52;  // adding it rounds to an integer, held in the low word
    const double t = fma(x, kExpInvL, kShift);
    const double n = t - kShift;
    const int ni = __double2loint(t);  // n = 64 k + j, |n| < 2^31
    double r = fma(-n, kExpLHi, x);    // exact (the high part has 32 bits, |n| < 2^17)
    r = fma(-n, kExpLLo, r);
    double q = fma(r, 1.0 / 120, 1.0 / 24);
    q = fma(r, q, 1.0 / 6);
    q = fma(r, q, 0.5);
    q = fma(r, q, 1.0);
    const double tj = __ldg(&kExp2J64[ni & 63]);
    k = ni >> 6;  // floor(n / 64)
    return fma(tj, r * q, tj);  // 2^(j/64) e^r, in [0.994, 2.02)
}

static __device__ __noinline__ double exp_tang_edge(double x)
{
    if (x != x) return x;
    if (x > 710.0) return __longlong_as_double(0x7ff0000000000000ll);
    if (x < -746.0) return 0.0;
    // 708 < |x| <= 746: 2^k in two halves; m 2^k1 is exact, the second product
    // rounds once (to a subnormal, to infinity, or to the nearest double)
    int k;
    const double m = exp_tang_core(x, k);
    const int k1 = k / 2, k2 = k - k1;
    const double s1 = __hiloint2double((k1 + 1023) << 20, 0), s2 = __hiloint2double((k2 + 1023) << 20, 0);
    return (m * s1) * s2;
}

// e^x (Tang): for |x| <= 708 the scaling by 2^k is an add to the exponent field
// (the result stays normal); beyond it, and for NaN, exp_tang_edge.
__device__ __forceinline__ double exp_tang(double x)
{
    if (!(fabs(x) <= 708.0)) return exp_tang_edge(x);
    int k;
    const double m = exp_tang_core(x, k);
    return __hiloint2double(__double2hiint(m) + (int)((unsigned)k << 20), __double2loint(m));
}

// ln x for a positive normal x = 2^e m, m in [1, 2), taken as 2^e' m' with m'
// in [0.75, 1.5) (m' = m / 2 and e' = e + 1 when m >= 1.5), so that x near 1,
// on either side, has e' = 0 and no e' ln 2 term to cancel against.  c_j, the
// centre of m''s interval (width 1/128 below 1.5, 1/256 above 0.75 .. 1), has
// ln c_j in the table; r = (m' - c_j)/c_j with m' - c_j exact and |r| < 2^-8,
// and ln x = e' ln 2 + ln c_j + log1p(r), log1p by its Taylor polynomial of
// degree 6 (remainder below r^7/7 < 2^-58).
__device__ __forceinline__ double log_tang_core(double x, int extra_e)
{
    const int hi = __double2hiint(x);
    const int lo = __double2loint(x);
    const int j = (hi >> 13) & 127;  // top 7 of the 52 fraction bits
    const int half = j >> 6;         // m >= 1.5
    const int e = (hi >> 20) - 1023 + extra_e + half;
    const int ex = (0x3ff - half) << 20;
    const double m = __hiloint2double((hi & 0x000fffff) | ex, lo);      // m'
    const double c = __hiloint2double(((2 * j + 1) << 12) | ex, 0);     // (1 + (2j + 1)/256) / 2^half
    const double inv_c = __ldg(&kLogC128[2 * j]);
    const double ln_c = __ldg(&kLogC128[2 * j + 1]);
    const double r = (m - c) * inv_c;
    double q = fma(r, -1.0 / 6, 0.2);
    q = fma(r, q, -0.25);
    q = fma(r, q, 1.0 / 3);
    q = fma(r, q, -0.5);
    const double l = fma(r * r, q, r);  // log1p(r)
    const double ed = (double)e;
    return fma(ed, kLn2Hi, ln_c) + fma(ed, kLn2Lo, l);  // e kLn2Hi is exact
}

static __device__ __noinline__ double log_tang_edge(double x)
{
    if (x != x || x < 0.0) return __longlong_as_double(0x7ff8000000000000ll);
    if (x == 0.0) return __longlong_as_double(0xfff0000000000000ll);
    if (x > 0x1.fffffffffffffp1023) return x;  // +inf
    return log_tang_core(x * 0x1p54, -54);     // subnormal
}

__device__ __forceinline__ double log_tang(double x)
{
    if (!(x >= 0x1p-1022 && x <= 0x1.fffffffffffffp1023)) return log_tang_edge(x);
    return log_tang_core(x, 0);
}

}  // namespace qed
