// physics.cuh -- per-particle device functions of the QED substep (templated on
// float / double): quantum parameters (§2), 1-D rate lookups (§3.1, §3.2),
// 2-D inverse-CDF sampling (§3.1, §3.2) and the optical-depth reset.
#pragma once

#include "common.cuh"
#include "fp64_math.cuh"

namespace qed {

__device__ __forceinline__ float d_log(float x) { return logf(x); }
__device__ __forceinline__ double d_log(double x) { return log(x); }
__device__ __forceinline__ float d_exp(float x) { return expf(x); }
__device__ __forceinline__ double d_exp(double x) { return exp(x); }
__device__ __forceinline__ float d_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double d_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float d_fma(float a, float b, float c) { return fmaf(a, b, c); }
// logarithm and exponential of the 1-D rate lookups: in FP32 the hardware's
// approximate forms (__logf: absolute error ~2^-21 near 1; __expf: ~2 + 1.2 |x|
// ulp), whose ~1e-6 relative effect on a rate is far below the tables'
// interpolation error; in FP64 Tang's table-driven forms (fp64_math.cuh, within
// 2 ulp), which take fewer FP64 instructions than the library functions
__device__ __forceinline__ float r_log(float x) { return __logf(x); }
__device__ __forceinline__ double r_log(double x) { return log_tang(x); }
__device__ __forceinline__ float r_exp(float x) { return __expf(x); }
__device__ __forceinline__ double r_exp(double x) { return exp_tang(x); }
__device__ __forceinline__ double d_fma(double a, double b, double c) { return fma(a, b, c); }
// logarithm and exponential of the 2-D inverse-CDF sampling: FP32 the library
// forms; FP64 Tang's (ln chi and ln r are interpolation coordinates, where the
// logarithm's 2^-57 absolute error near 1 is far below the tables' spacing)
__device__ __forceinline__ float s_log(float x) { return logf(x); }
__device__ __forceinline__ double s_log(double x) { return log_tang(x); }
__device__ __forceinline__ float s_exp(float x) { return expf(x); }
__device__ __forceinline__ double s_exp(double x) { return exp_tang(x); }

// leading asymptotes of T outside the table (Eq. (t_func), read in the paper's
// chi_gamma convention): T ~ 3 sqrt(3) / (16 sqrt(2)) exp(-8 / (3 chi)) for
// small chi, T ~ C chi^{-1/3} with C = 15 3^{2/3} Gamma(2/3)^3 / (14 pi sqrt(3)
// Gamma(1/3)) for large chi.
constexpr double kTSmall = 0.22963966338592293;
constexpr double kTLarge = 0.37961230854357125;
constexpr double kLnTSmall = -1.4712438795175893;  // ln kTSmall
constexpr double kLnTLarge = -0.9686047877362934;  // ln kTLarge

// chi of a lepton, §2: chi^2 = (gamma E + p x B)^2 - (p.E)^2 in these units.
// FP32: with n = p/|p| and E_perp = E - (n.E) n the same quantity is the sum of
// squares |gamma E_perp + p x B|^2 + (n.E)^2 (expand gamma^2 = 1 + p^2 and use
// p x B perpendicular to n), which avoids the cancellation of the difference
// form when chi is small against gamma |E| + |p| |B|; a particle at rest has
// chi = |E|.  FP64 keeps the difference form: its cancellation error, 1e-16
// (S/chi)^2 relative, is below the FP64 tolerance, and it saves the FP64
// square root and division of n, FP64 being GB300's scarce unit.
// The rate multiplies by 1/gamma.  FP64 takes gamma and 1/gamma from one
// reciprocal square root (within 1 ulp); FP32 keeps IEEE square roots and
// divisions here (with reciprocal square roots the HBM-bound evolution kernel
// measured ~1.5 % slower; photons, below, take them).
// Returns chi, gamma and 1/gamma; NaN inputs give NaN.
__device__ __forceinline__ float chi_lepton(float px, float py, float pz, float ex, float ey, float ez, float bx,
                                            float by, float bz, float &gamma, float &inv_gamma)
{
    const float p2 = px * px + py * py + pz * pz;
    gamma = sqrtf(1.0f + p2);
    inv_gamma = 1.0f / gamma;
    const float pm = sqrtf(p2);
    const float inv = pm > 0.0f ? 1.0f / pm : 0.0f;
    const float nx = px * inv, ny = py * inv, nz = pz * inv;
    const float ne = nx * ex + ny * ey + nz * ez;
    const float fx = gamma * (ex - ne * nx) + (py * bz - pz * by);
    const float fy = gamma * (ey - ne * ny) + (pz * bx - px * bz);
    const float fz = gamma * (ez - ne * nz) + (px * by - py * bx);
    const float s = fx * fx + fy * fy + fz * fz + (p2 > 0.0f ? ne * ne : ex * ex + ey * ey + ez * ez);
    return sqrtf(s);
}

__device__ __forceinline__ double chi_lepton(double px, double py, double pz, double ex, double ey, double ez,
                                             double bx, double by, double bz, double &gamma, double &inv_gamma)
{
    const double g2 = 1.0 + (px * px + py * py + pz * pz);
    inv_gamma = rsqrt(g2);
    gamma = g2 * inv_gamma;
    const double fx = gamma * ex + (py * bz - pz * by);
    const double fy = gamma * ey + (pz * bx - px * bz);
    const double fz = gamma * ez + (px * by - py * bx);
    const double pe = px * ex + py * ey + pz * ez;
    const double s = fx * fx + fy * fy + fz * fz - pe * pe;
    return sqrt(s < 0.0 ? 0.0 : s);  // (NaN stays NaN)
}

// chi_gamma of a photon, §2 (gamma -> |p|, v -> c n).  FP32: | |p| E_perp + p x B |,
// the perpendicular part of |p| E + p x B; FP64: the difference form.  Returns
// chi, |p| and 1/|p| (0 for p = 0), from a reciprocal square root (rsqrtf within
// 2 ulp, FP64 rsqrt within 1 ulp).
__device__ __forceinline__ float chi_photon(float px, float py, float pz, float ex, float ey, float ez, float bx,
                                            float by, float bz, float &pm, float &inv_pm)
{
    const float p2 = px * px + py * py + pz * pz;
    inv_pm = p2 > 0.0f ? rsqrtf(p2) : 0.0f;
    pm = p2 * inv_pm;
    const float nx = px * inv_pm, ny = py * inv_pm, nz = pz * inv_pm;
    const float ne = nx * ex + ny * ey + nz * ez;
    const float fx = pm * (ex - ne * nx) + (py * bz - pz * by);
    const float fy = pm * (ey - ne * ny) + (pz * bx - px * bz);
    const float fz = pm * (ez - ne * nz) + (px * by - py * bx);
    return sqrtf(fx * fx + fy * fy + fz * fz);
}

__device__ __forceinline__ double chi_photon(double px, double py, double pz, double ex, double ey, double ez,
                                             double bx, double by, double bz, double &pm, double &inv_pm)
{
    const double p2 = px * px + py * py + pz * pz;
    inv_pm = p2 > 0.0 ? rsqrt(p2) : 0.0;
    pm = p2 * inv_pm;
    const double fx = pm * ex + (py * bz - pz * by);
    const double fy = pm * ey + (pz * bx - px * bz);
    const double fz = pm * ez + (px * by - py * bx);
    const double pe = px * ex + py * ey + pz * ez;
    const double s = fx * fx + fy * fy + fz * fz - pe * pe;
    return sqrt(s < 0.0 ? 0.0 : s);
}

// log-log interpolation of a 1-D table held in `tab` (shared or global):
// ln f(chi) = ln f_n + (ln chi - ln chi_n) (ln f_{n+1} - ln f_n) / (ln chi_{n+1} - ln chi_n),
// n = clamp(floor((ln chi - ln chi_min) / d), 0, N - 2); chi clamped into the table.
template <typename T>
__device__ __forceinline__ T interp_ln(const T *tab, T lc, T ln_min, T inv_d, int n)
{
    T t = (lc - ln_min) * inv_d;
    t = t < T(0) ? T(0) : (t > T(n - 1) ? T(n - 1) : t);
    int i = (int)t;
    i = i > n - 2 ? n - 2 : i;
    const T f = t - T(i);
    const T a = tab[i], b = tab[i + 1];
    return d_fma(f, b - a, a);
}

// QS rate (Eq. (qs_total_cross)): (2/3) alpha G(chi) / gamma; G clamped to the
// end values outside [chi_min, chi_max] (§3.2); chi == 0 gives 0.
template <typename T>
__device__ __forceinline__ T qs_rate(const T *tab, const Table1D<T> &v, T chi, T, T inv_gamma)
{
    if (!(chi > T(0))) return T(0);
    const T lnG = interp_ln(tab, r_log(chi), v.ln_min, v.inv_d, v.n);
    return T(2.0 / 3.0 * kAlpha) * r_exp(lnG) * inv_gamma;
}

// BW rate (Eq. (bw_cross_tot)): alpha chi T(chi) / gamma_g; the asymptotes of
// Eq. (t_func) outside [chi_min, chi_max] (§3.1).  All three branches give
// ln T, so a warp whose photons straddle the table's ends runs one exponential:
// ln T = ln(kTSmall) - 8 / (3 chi) below, ln(kTLarge) - (ln chi) / 3 above.
template <typename T>
__device__ __forceinline__ T bw_rate(const T *tab, const Table1D<T> &v, T chi, T pm, T inv_pm)
{
    if (!(chi > T(0)) || !(pm > T(0))) return T(0);
    const T lc = r_log(chi);
    T lnT;
    if (chi < v.chi_min)
        lnT = T(kLnTSmall) - T(8.0 / 3.0) / chi;
    else if (chi > v.chi_max)
        lnT = d_fma(lc, T(-1.0 / 3.0), T(kLnTLarge));
    else
        lnT = interp_ln(tab, lc, v.ln_min, v.inv_d, v.n);
    return T(kAlpha) * chi * r_exp(lnT) * inv_pm;
}

// uniform for sampling in the working precision: FP64 as drawn; FP32 rounded
// toward zero so that it stays in (0, 1)
template <typename T>
__device__ __forceinline__ T sample_uniform(double u);
template <>
__device__ __forceinline__ double sample_uniform<double>(double u) { return u; }
// FP32: u rounded toward zero, from the bits (u >= 2^-54 is a normal float;
// the same value as __double2float_rz without an FP64 instruction)
template <>
__device__ __forceinline__ float sample_uniform<float>(double u)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(u);
    return __uint_as_float((unsigned int)((((b >> 52) & 0x7ffu) - 1023u + 127u) << 23) |
                           (unsigned int)((b >> 29) & 0x7fffffu));
}

// 1 - u rounded toward zero to FP32 for a draw u in [1/2, 1] (the BW fold):
// 1 - u = (2^53 - M) 2^-53 exactly, M the 53-bit significand of u, then the
// top 24 bits of that integer
__device__ __forceinline__ float one_minus_rz(double u)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(u);
    if (b >= 0x3ff0000000000000ull) return 0.0f;                        // u = 1
    const unsigned long long n = (1ull << 53) - ((b & 0xfffffffffffffull) | (1ull << 52));  // u in [1/2, 1)
    const int len = 64 - __clzll((long long)n);                          // 1 .. 52
    const unsigned int mant = (unsigned int)(len > 24 ? n >> (len - 24) : n << (24 - len)) & 0x7fffffu;
    return __uint_as_float(((unsigned int)(len - 1 - 53 + 127) << 23) | mant);
}

// interpolated row value of a 2-D table at column m: v_n,m + w (v_{n+1},m - v_n,m)
template <typename T>
__device__ __forceinline__ T row_val(const T *r0, const T *r1, T w, int m)
{
    const T a = __ldg(r0 + m), b = __ldg(r1 + m);
    return d_fma(w, b - a, a);
}

// locate the chi interval of a 2-D table (chi clamped into the table, §3.1/§3.2);
// r0, r1 are the two rows, off their offset (for the difference table)
template <typename T>
__device__ __forceinline__ void locate_2d(const Table2D<T> &tb, T chi, const T *&r0, const T *&r1, T &w,
                                          size_t &off, int &row)
{
    T c = chi < tb.chi_min ? tb.chi_min : (chi > tb.chi_max ? tb.chi_max : chi);
    T t = (s_log(c) - tb.ln_min) * tb.inv_d;
    t = t < T(0) ? T(0) : (t > T(tb.n_chi - 1) ? T(tb.n_chi - 1) : t);
    int n = (int)t;
    n = n > tb.n_chi - 2 ? tb.n_chi - 2 : n;
    w = t - T(n);
    row = n;
    off = (size_t)n * tb.n_xi;
    r0 = tb.v + off;
    r1 = r0 + tb.n_xi;
}

// largest m in [0, M-1] with P_m <= x on the interpolated row (binary search;
// the row is non-decreasing), then clamped to [0, M-2]; m = 0 when x < P_0.
// The search starts from the bracket that the guide tables of the two rows give
// for bin b of the draw (both rows' answers, hence the interpolated row's, lie
// between their guides at b and b + 1), widened by one entry on each side
// against rounding at the edges.
template <typename T>
__device__ __forceinline__ int search_row(const T *r0, const T *r1, T w, int M, T x, const int32_t *g0,
                                          const int32_t *g1, int b)
{
    const int a0 = __ldg(g0 + b), a1 = __ldg(g1 + b), c0 = __ldg(g0 + b + 1), c1 = __ldg(g1 + b + 1);
    int lo = (a0 < a1 ? a0 : a1) - 1, hi = (c0 > c1 ? c0 : c1) + 2;
    lo = lo < 0 ? 0 : lo;
    hi = hi > M ? M : hi;  // invariant: P_lo <= x (or lo == 0), P_hi > x (hi == M: sentinel)
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (row_val(r0, r1, w, mid) <= x)
            lo = mid;
        else
            hi = mid;
    }
    return lo > M - 2 ? M - 2 : lo;
}

// QS inverse CDF (§3.2): ln P interpolated in ln chi, binary search on ln r, then
// ln xi = ln xi_m + (ln r - ln P_m)(ln xi_{m+1} - ln xi_m)/(ln P_{m+1} - ln P_m).
// The denominator is interpolated from the FP64-formed column differences, so
// that it keeps its relative accuracy in the FP32 tables (where two neighbouring
// entries share most of their digits); the same holds below xi_min, where the
// first segment is extrapolated.
template <typename T>
__device__ __forceinline__ T qs_sample_xi(const Table2D<T> &tb, T chi, T r)
{
    const T *r0, *r1;
    T w;
    size_t off;
    int row;
    locate_2d(tb, chi, r0, r1, w, off, row);
    const T lr = s_log(r);
    const int *g0 = tb.guide + (size_t)row * (kGuideBins + 1);
    int b = (int)(r * T(kGuideBins));
    b = b > kGuideBins - 1 ? kGuideBins - 1 : (b < 0 ? 0 : b);
    const int m = search_row(r0, r1, w, tb.n_xi, lr, g0, g0 + kGuideBins + 1, b);
    const T p0 = row_val(r0, r1, w, m);
    const T dp = row_val(tb.dv + off, tb.dv + off + tb.n_xi, w, m);  // P_{m+1} - P_m
    const T x0 = tb.x0 + T(m) * tb.dx;
    const T x1 = (m + 1 == tb.n_xi - 1) ? T(0) : tb.x0 + T(m + 1) * tb.dx;
    if (!(dp > T(0))) return s_exp(x0);
    T lx = x0 + (lr - p0) * (x1 - x0) / dp;
    lx = lx > T(0) ? T(0) : lx;
    return s_exp(lx);
}

// BW inverse CDF (§3.1): r <= 1/2 samples the electron, otherwise the positron
// with r -> 1 - r; P interpolated in ln chi_g, binary search on r, linear in xi
// (denominator from the column differences, as for QS).
template <typename T>
__device__ __forceinline__ T bw_sample_xi(const Table2D<T> &tb, T chi, double u, bool &electron)
{
    // split on the FP64 draw, then round the folded value (keeps 1 - u accurate)
    electron = __double_as_longlong(u) <= __double_as_longlong(0.5);  // u <= 1/2 (u > 0: the bits order as the values)
    T r;
    if constexpr (sizeof(T) == 4)
        r = electron ? sample_uniform<T>(u) : one_minus_rz(u);
    else
        r = electron ? u : 1.0 - u;
    const T *r0, *r1;
    T w;
    size_t off;
    int row;
    locate_2d(tb, chi, r0, r1, w, off, row);
    const int *g0 = tb.guide + (size_t)row * (kGuideBins + 1);
    int b = (int)(r * T(2 * kGuideBins));
    b = b > kGuideBins - 1 ? kGuideBins - 1 : (b < 0 ? 0 : b);
    const int m = search_row(r0, r1, w, tb.n_xi, r, g0, g0 + kGuideBins + 1, b);
    const T p0 = row_val(r0, r1, w, m);
    const T dp = row_val(tb.dv + off, tb.dv + off + tb.n_xi, w, m);
    const T x0 = T(m) * tb.dx;
    const T x1 = (m + 1 == tb.n_xi - 1) ? T(0.5) : T(m + 1) * tb.dx;
    if (!(dp > T(0))) return x0;
    T x = x0 + (r - p0) * (x1 - x0) / dp;
    return x > T(0.5) ? T(0.5) : (x < T(0) ? T(0) : x);
}


// store an FP64 optical depth: FP64 as is; FP32 as (tau, tau_c) with tau_c the
// rounding residual (the optical depth is tau - tau_c)
template <typename T>
__device__ __forceinline__ void store_tau(T *tau, T *tau_c, int64_t i, double x);
template <>
__device__ __forceinline__ void store_tau<double>(double *tau, double *, int64_t i, double x) { tau[i] = x; }
// (h, c) = (fl32(x), fl32(h - x)), both rounded to nearest even.  Where both are
// normal floats (2^-74 <= |x| < 2^127) from the bits of x with integer
// operations, without an FP64 instruction (GB300's FP64 pipe bounds the event
// kernels when many particles fire): h keeps the top 24 of x's 53 significant
// bits, rounded; h - x is the rounding residual, an integer of at most 29 bits
// times 2^(e - 52), exact in FP64, rounded once by the integer-to-float
// conversion and scaled exactly.  Elsewhere (0, tiny, huge, infinite, NaN) by
// FP64 conversions, with the same results.
__device__ __forceinline__ void split_f32_pair(double x, float &h, float &c)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ffu) - 1023;
    if (e < -74 || e > 126) {
        h = __double2float_rn(x);
        c = __double2float_rn((double)h - x);
        return;
    }
    const unsigned long long m = (b & 0xfffffffffffffull) | 0x10000000000000ull;  // 53 significant bits
    unsigned int keep = (unsigned int)(m >> 29);                                  // the top 24
    const unsigned int rem = (unsigned int)(m & 0x1fffffffu);                     // the other 29
    const bool up = rem > 0x10000000u || (rem == 0x10000000u && (keep & 1u));
    int diff = up ? (int)(0x20000000u - rem) : -(int)rem;  // (|h| - |x|) / 2^(e - 52)
    keep += up ? 1u : 0u;
    int eh = e;
    if (keep == 0x1000000u) {  // rounded up into the next binade
        keep >>= 1;
        ++eh;
    }
    const bool neg = (b >> 63) != 0;
    h = __uint_as_float((neg ? 0x80000000u : 0u) | ((unsigned int)(eh + 127) << 23) | (keep & 0x7fffffu));
    if (neg) diff = -diff;
    c = __int2float_rn(diff) * __uint_as_float((unsigned int)(e - 52 + 127) << 23);  // exact scaling by 2^(e - 52)
}

template <>
__device__ __forceinline__ void store_tau<float>(float *tau, float *tau_c, int64_t i, double x)
{
    float h, c;
    split_f32_pair(x, h, c);
    tau[i] = h;
    tau_c[i] = c;
}

// -ln U in FP64 for U in [2^-54, 1]: Tang's logarithm (within 2 ulp); above
// 1 - 2^-8, where ln U is small and that logarithm's error no longer shrinks
// with it, the Taylor series of log1p(d) with d = U - 1 (exact: U >= 1/2), whose
// remainder d^8/8 is below 2^-59 of the result.  The optical-depth resets are
// the event kernels' largest FP64 cost, and GB300's FP64 pipe their bound when
// many particles fire.
static __device__ __noinline__ double neg_log1p_series(double u)
{
    const double d = u - 1.0;
    double q = fma(d, -1.0 / 7, 1.0 / 6);
    q = fma(d, q, -0.2);
    q = fma(d, q, 0.25);
    q = fma(d, q, -1.0 / 3);
    q = fma(d, q, 0.5);
    return fma(d * d, q, -d);  // -(d - d^2/2 + d^3/3 - ... - d^7/7)
}

__device__ __forceinline__ double neg_log_u(double u)
{
    // (positive doubles order as their bit patterns: the test costs no FP64
    // instruction; the series is out of line, so that the other 99.6 % of the
    // draws do not issue it predicated off; U >= 2^-54 is normal, so Tang's core
    // needs no range check)
    if (__double_as_longlong(u) > __double_as_longlong(1.0 - 0x1p-8)) return neg_log1p_series(u);
    return -log_tang_core(u, 0);
}

// tau = -ln U, U the 53-bit uniform of (seed, (id, step, purpose)), in FP64 (§3)
__device__ __forceinline__ double tau_draw(uint64_t seed, uint64_t id, int64_t step, uint32_t purpose)
{
    const U4 w = draw(seed, id, step, purpose);
    return neg_log_u(uniform53(w.x, w.y));
}

}  // namespace qed
