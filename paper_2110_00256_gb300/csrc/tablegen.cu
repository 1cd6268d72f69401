// tablegen.cu -- FP64 generation of the four lookup tables on the GPU (§3 says
// the paper's generator needed CPU-only special functions and quadrature; here
// both run on the device).
//
//   Bessel functions: e^x K_nu(x) and e^x int_x^inf K_nu(s) ds from the integral
//   representation K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt (and the same
//   integrand over cosh t for the tail integral), by the trapezoid rule in t,
//   which converges exponentially for this analytic, even integrand (Trefethen &
//   Weideman, SIAM Review 56 (2014) 385).  Step h = min(1/4, 0.6/sqrt(x)) keeps
//   the discretisation error near exp(-40); both integrals share one pass.
//   Outer integrals over xi: tanh-sinh (double-exponential) quadrature on every
//   table interval (Takahasi & Mori 1974; Bailey, Jeyabalan & Li, Exp. Math. 14
//   (2005) 317), which absorbs the steep endpoint behaviour at xi -> 0 and 1.
//   QS (Eq. (qs_g_func)) integrates S(chi, xi) d(ln xi); BW (Eq. (t_func_0))
//   integrates the bracket in xi = chi_- / chi_gamma over [0, 1/2].
//
// One CTA per table row; one warp per xi interval; the interval sums are
// reduced by shuffles in a fixed order, so the tables are bit-reproducible.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace qed {

qed_status check_params(const qed_table_params *p);
qed_status alloc_tables(const qed_table_params *p, qed_tables **out);
qed_status finish_tables(qed_tables *t, cudaStream_t st);

constexpr double kPi = 3.14159265358979323846;
constexpr double kTsStep = 1.0 / 16.0;  // tanh-sinh step
constexpr int kTsHalf = 52;             // nodes k = -52..52 (|k h| <= 3.25)
constexpr double kQsBelow = 100.0;  // the QS integral below xi_min starts at xi_min e^{-100}

// e^x int_x^inf K_a and e^x K_b, trapezoid rule in t
__device__ void bessel_scaled(double x, double nu_a, double nu_b, double &ia, double &kb)
{
    const double h = fmin(0.25, 0.6 / sqrt(x));
    const double nmax = fmax(nu_a, nu_b);
    double sa = 0.5, sb = 0.5;  // t = 0 terms, weight 1/2
    const double ra = exp(nu_a * h), rb = exp(nu_b * h), r1 = exp(h);
    double pa = 1.0, pb = 1.0, p1 = 1.0;
    for (int k = 1; k < 4000; ++k) {
        const double t = k * h;
        if ((k & 15) == 0) {
            pa = exp(nu_a * t), pb = exp(nu_b * t), p1 = exp(t);
        } else {
            pa *= ra, pb *= rb, p1 *= r1;
        }
        const double s = sinh(0.5 * t);
        const double arg = 2.0 * x * s * s;  // x (cosh t - 1)
        if (arg - nmax * t > 40.0 && arg > 40.0) break;
        const double e = exp(-arg);
        const double cha = 0.5 * (pa + 1.0 / pa), chb = 0.5 * (pb + 1.0 / pb), ch1 = 0.5 * (p1 + 1.0 / p1);
        sa += e * cha / ch1;
        sb += e * chb;
    }
    ia = h * sa;
    kb = h * sb;
}

// QS integrand in u = ln xi: S(chi, xi) = sqrt(3)/(2 pi) xi [int_Y K_{5/3} + xi^2/(1-xi) K_{2/3}(Y)]
__device__ double qs_integrand(double chi, double u)
{
    const double xi = exp(u);
    const double om = -expm1(u);  // 1 - xi
    if (!(om > 0.0)) return 0.0;
    const double Y = (2.0 / 3.0) * xi / (chi * om);
    if (Y > 745.0) return 0.0;
    double ia, kb;
    bessel_scaled(Y, 5.0 / 3.0, 2.0 / 3.0, ia, kb);
    return (0.27566444771089600 /* sqrt(3) / (2 pi) */) * xi * exp(-Y) * (ia + xi * xi / om * kb);
}

// BW bracket in xi: int_z K_{1/3} + (xi/(1-xi) + (1-xi)/xi) K_{2/3}(z), z = 2/(3 chi xi (1-xi))
__device__ double bw_integrand(double chi, double xi)
{
    if (!(xi > 0.0) || !(xi < 1.0)) return 0.0;
    const double om = 1.0 - xi;
    const double z = 2.0 / (3.0 * chi * xi * om);
    if (z > 745.0) return 0.0;
    double ia, kb;
    bessel_scaled(z, 1.0 / 3.0, 2.0 / 3.0, ia, kb);
    return exp(-z) * (ia + (xi / om + om / xi) * kb);
}

// node k of tanh-sinh on [a, b]: abscissa (taken as an offset from the nearer
// end so that it stays exact near the ends) and weight
__device__ __forceinline__ void ts_node(double a, double b, int k, double &x, double &w)
{
    const double r = 0.5 * (b - a);
    const double tk = k * kTsStep;
    const double s = 0.5 * kPi * sinh(tk);
    const double e = exp(2.0 * fabs(s));
    const double d = 2.0 * r / (1.0 + e);  // distance to the nearer end
    x = (k < 0) ? a + d : (k > 0 ? b - d : 0.5 * (a + b));
    const double ch = cosh(s);
    w = r * kTsStep * 0.5 * kPi * cosh(tk) / (ch * ch);
}

struct GenArgs {
    double *qs_lnG, *qs_lnP, *bw_lnT, *bw_P;
    double qs_l0, qs_l1, qs_xi_min, bw_l0, bw_l1;
    int qs_n_chi, qs_n_xi, bw_n_chi, bw_n_xi;
};

__global__ void __launch_bounds__(256) table_rows_kernel(const __grid_constant__ GenArgs a)
{
    __shared__ double acc[QED_MAX_TABLE_N];
    const bool qs = blockIdx.x < (unsigned)a.qs_n_chi;
    const int row = qs ? blockIdx.x : blockIdx.x - a.qs_n_chi;
    const int N = qs ? a.qs_n_chi : a.bw_n_chi;
    const int M = qs ? a.qs_n_xi : a.bw_n_xi;
    const double l0 = qs ? a.qs_l0 : a.bw_l0, l1 = qs ? a.qs_l1 : a.bw_l1;
    const double chi = exp(row == N - 1 ? l1 : l0 + row * (l1 - l0) / (N - 1));
    const double lxm = log(a.qs_xi_min);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;

    // interval j of the row: QS j = 0 is [xi_min e^-100, xi_min] in ln xi, j >= 1 is
    // [xi_{j-1}, xi_j]; BW j >= 1 is [xi_{j-1}, xi_j] on the linear grid, j = 0 empty
    for (int j = warp; j < M; j += nw) {
        double lo, hi;
        if (qs) {
            if (j == 0) {
                lo = lxm - kQsBelow, hi = lxm;
            } else {
                lo = lxm + (j - 1) * (-lxm) / (M - 1);
                hi = (j == M - 1) ? 0.0 : lxm + j * (-lxm) / (M - 1);
            }
        } else {
            lo = 0.5 * (j - 1) / (M - 1);
            hi = (j == M - 1) ? 0.5 : 0.5 * j / (M - 1);
        }
        double part = 0.0;
        if (qs || j > 0) {
            for (int k = lane - kTsHalf; k <= kTsHalf; k += 32) {
                double x, w;
                ts_node(lo, hi, k, x, w);
                part += w * (qs ? qs_integrand(chi, x) : bw_integrand(chi, x));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) acc[j] = part;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int j = 0; j < M; ++j) tot += acc[j];
        if (qs) {
            double *out = a.qs_lnP + (size_t)row * M;
            double C = 0.0;
            for (int m = 0; m < M; ++m) {
                C += acc[m];
                out[m] = C / tot;  // P_m
            }
            // ln P = ln(C/G), except near P = 1 where log1p(-tail/G) keeps the
            // relative accuracy; tail = sum of the intervals right of m
            double tr = 0.0;
            for (int m = M - 1; m >= 0; --m) {
                const double q = tr / tot;
                out[m] = (q < 0.5) ? log1p(-q) : log(out[m]);
                tr += acc[m];
            }
            out[M - 1] = 0.0;
            a.qs_lnG[row] = log(tot);
        } else {
            double *out = a.bw_P + (size_t)row * M;
            double C = 0.0;
            for (int m = 0; m < M; ++m) {
                C += acc[m];
                out[m] = tot > 0.0 ? C / (2.0 * tot) : 0.0;
            }
            out[0] = 0.0;
            if (tot > 0.0) out[M - 1] = 0.5;
            // T = int_0^1 bracket / (pi sqrt(3) chi) = 2 tot / (pi sqrt(3) chi)
            a.bw_lnT[row] = log(2.0 * tot / (kPi * 1.7320508075688772 * chi));
        }
    }
}

// ---------------------------------------------------------------------------
// Exact inverse CDF, no table (the learned sampler's training targets).  Per chi
// row, the cumulative integral of the spectrum on a fine grid and its density
// at the nodes; per draw, the bracketing interval by binary search, a first
// guess from the cubic Hermite interpolant of the cumulative integral on that
// interval (value and slope at both nodes), then Newton steps on the partial
// integral from the interval's left node (Gauss-Legendre, 8 points).
// Grid variables (both smooth in them over the whole range):
//   QS: v = ln(xi / (1 - xi)) on [ln 1e-12, -ln 1e-12] in kExactIntervals - 1
//       equal intervals, plus [ln 1e-12 - 100, ln 1e-12] below (where P follows
//       its xi^(1/3) law; tanh-sinh there); the density is S(chi, xi) (1 - xi),
//       which resolves both the soft end and the cut-off at 1 - xi ~ 1/chi;
//   BW: v = ln xi on [ln 1e-12, ln 1/2] in kExactIntervals equal intervals,
//       density xi times the bracket of Eq. (t_func_0), normalised to P(1/2) = 1.
// ---------------------------------------------------------------------------
constexpr int kExactIntervals = 1024;
constexpr double kExactLo = -27.631021115928547;  // ln 1e-12

struct GaussLegendre8 {
    double x[8], w[8];  // nodes and weights on [-1, 1]
};

// density in v of the QS photon number spectrum: S(chi, xi) (1 - xi)
__device__ double qs_density_v(double chi, double v)
{
    const double e = exp(-fabs(v));
    const double xi = v >= 0.0 ? 1.0 / (1.0 + e) : e / (1.0 + e);
    const double om = v >= 0.0 ? e / (1.0 + e) : 1.0 / (1.0 + e);  // 1 - xi without cancellation
    if (!(om > 0.0) || !(xi > 0.0)) return 0.0;
    const double Y = (2.0 / 3.0) * xi / (chi * om);
    if (Y > 745.0) return 0.0;
    double ia, kb;
    bessel_scaled(Y, 5.0 / 3.0, 2.0 / 3.0, ia, kb);
    return (0.27566444771089600 /* sqrt(3) / (2 pi) */) * xi * om * exp(-Y) * (ia + xi * xi / om * kb);
}

// density in v = ln xi of the BW split: xi times the bracket
__device__ double bw_density_v(double chi, double v)
{
    const double xi = exp(v);
    return xi * bw_integrand(chi, xi);
}

__device__ __forceinline__ double exact_density(bool qs, double chi, double v)
{
    return qs ? qs_density_v(chi, v) : bw_density_v(chi, v);
}

// node j of the grid (j = 0 .. kExactIntervals)
__device__ __forceinline__ double exact_node(bool qs, int j)
{
    if (qs) {
        if (j == 0) return kExactLo - kQsBelow;
        return kExactLo + (j - 1) * (-2.0 * kExactLo) / (kExactIntervals - 1);
    }
    return kExactLo + j * (-0.6931471805599453 - kExactLo) / kExactIntervals;
}

__device__ double gl8(const GaussLegendre8 &g, bool qs, double chi, double a, double b)
{
    const double c = 0.5 * (a + b), h = 0.5 * (b - a);
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += g.w[i] * exact_density(qs, chi, fma(h, g.x[i], c));
    return h * s;
}

// The QS interval below the grid (v from ln 1e-12 - 100 to ln 1e-12): there the
// density grows like e^{v/3} (the xi^(1/3) law of P), so it is integrated in
// w = e^{v/3}, where the integrand 3 density / w is nearly constant (8-point
// Gauss-Legendre on [w(a), w(v)]).
__device__ double gl8_below(const GaussLegendre8 &g, double chi, double a, double v)
{
    const double wa = exp(a / 3.0), wb = exp(v / 3.0);
    const double c = 0.5 * (wa + wb), h = 0.5 * (wb - wa);
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const double w = fma(h, g.x[i], c);
        s += g.w[i] * 3.0 * qs_density_v(chi, 3.0 * log(w)) / w;
    }
    return h * s;
}

constexpr int kExactRowStride = 2 * (kExactIntervals + 1) + 1;  // P[0..M], p[0..M], total

// one CTA per chi row: P at the nodes (P_0 = 0 .. P_M = 1), the density p at
// the nodes divided by the total, then the total
__global__ void __launch_bounds__(256) exact_rows_kernel(int qs, const double *__restrict__ chi_rows,
                                                          double *__restrict__ work, GaussLegendre8 g)
{
    __shared__ double acc[kExactIntervals];
    const double chi = chi_rows[blockIdx.x];
    double *out = work + (size_t)blockIdx.x * kExactRowStride;
    if (qs && threadIdx.x == 0) acc[0] = gl8_below(g, chi, exact_node(true, 0), exact_node(true, 1));
    for (int j = threadIdx.x + (qs ? 1 : 0); j < kExactIntervals; j += blockDim.x)
        acc[j] = gl8(g, qs, chi, exact_node(qs, j), exact_node(qs, j + 1));
    for (int j = threadIdx.x; j <= kExactIntervals; j += blockDim.x)
        out[kExactIntervals + 1 + j] = exact_density(qs, chi, exact_node(qs, j));
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int j = 0; j < kExactIntervals; ++j) tot += acc[j];
        double c = 0.0;
        out[0] = 0.0;
        for (int j = 0; j < kExactIntervals; ++j) {
            c += acc[j];
            out[j + 1] = tot > 0.0 ? c / tot : 0.0;
        }
        out[kExactIntervals] = 1.0;
        out[2 * (kExactIntervals + 1)] = tot;
    }
    __syncthreads();
    const double tot = out[2 * (kExactIntervals + 1)];
    for (int j = threadIdx.x; j <= kExactIntervals; j += blockDim.x)
        out[kExactIntervals + 1 + j] = tot > 0.0 ? out[kExactIntervals + 1 + j] / tot : 0.0;
}

__global__ void __launch_bounds__(128) exact_draw_kernel(int qs, const double *__restrict__ chi_rows,
                                                          const double *__restrict__ work, int64_t m, int64_t k,
                                                          const double *__restrict__ uu, double *__restrict__ xi,
                                                          GaussLegendre8 g)
{
    const int64_t n = m * k;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / k;
        const double chi = chi_rows[row];
        const double *P = work + (size_t)row * kExactRowStride;
        const double *D = P + kExactIntervals + 1;
        const double tot = P[2 * (kExactIntervals + 1)];
        double u = uu[i];
        u = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
        const double r = qs ? u : 2.0 * (u < 1.0 - u ? u : 1.0 - u);
        double v;
        if (!(tot > 0.0) || r >= 1.0) {
            v = qs ? 1e300 : -0.6931471805599453;
        } else if (r <= 0.0) {
            v = -1e300;
        } else {
            int lo = 0, hi = kExactIntervals;  // j: P_j <= r < P_{j+1}
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (P[mid] <= r) lo = mid; else hi = mid;
            }
            const int j = lo;
            const double a = exact_node(qs, j), b = exact_node(qs, j + 1), L = b - a;
            const double P0 = P[j], P1 = P[j + 1];
            if (qs && j == 0) {
                // below the grid: the xi^(1/3) law as the first guess, Newton on ln P
                v = b + 3.0 * (log(r) - log(P1));
                v = v < a ? a : (v > b ? b : v);
                for (int it = 0; it < 8; ++it) {
                    const double F = P0 + gl8_below(g, chi, a, v) / tot;
                    const double f = exact_density(true, chi, v) / tot;
                    if (!(F > 0.0) || !(f > 0.0)) break;
                    double vn = v - (log(F) - log(r)) * F / f;
                    vn = vn < a ? a : (vn > b ? b : vn);
                    const double dv = fabs(vn - v);
                    v = vn;
                    if (dv < 1e-13) break;
                }
            } else {
                // cubic Hermite of P on t in [0, 1]: P(t) = P0 + ... with slopes L p_j, L p_{j+1};
                // its inverse by Newton from the linear guess
                const double m0 = L * D[j], m1 = L * D[j + 1], dP = P1 - P0;
                double t = dP > 0.0 ? (r - P0) / dP : 0.5;
                for (int it = 0; it < 6; ++it) {
                    const double t2 = t * t, t3 = t2 * t;
                    const double h = P0 * (2 * t3 - 3 * t2 + 1) + m0 * (t3 - 2 * t2 + t) + P1 * (-2 * t3 + 3 * t2) +
                                     m1 * (t3 - t2);
                    const double dh = P0 * (6 * t2 - 6 * t) + m0 * (3 * t2 - 4 * t + 1) + P1 * (-6 * t2 + 6 * t) +
                                      m1 * (3 * t2 - 2 * t);
                    if (!(dh > 0.0)) break;
                    double tn = t - (h - r) / dh;
                    tn = tn < 0.0 ? 0.0 : (tn > 1.0 ? 1.0 : tn);
                    t = tn;
                }
                v = a + L * t;
                // Newton on the partial integral (the cumulative integral itself)
                for (int it = 0; it < 4; ++it) {
                    const double F = P0 + gl8(g, qs, chi, a, v) / tot;
                    const double f = exact_density(qs, chi, v) / tot;
                    if (!(f > 0.0)) break;
                    double vn = v - (F - r) / f;
                    vn = vn < a ? a : (vn > b ? b : vn);
                    const double dv = fabs(vn - v);
                    v = vn;
                    if (dv < 1e-7 * L) break;  // the next correction is ~(dv / L)^2 of this one
                }
            }
        }
        double out;
        if (qs) {
            const double e = exp(-fabs(v));
            out = v >= 0.0 ? 1.0 / (1.0 + e) : e / (1.0 + e);
        } else {
            out = exp(v);
            out = out > 0.5 ? 0.5 : out;
            out = (u <= 0.5) ? out : 1.0 - out;
        }
        xi[i] = out;
    }
}

// Gauss-Legendre nodes and weights (Newton's method on the three-term recurrence)
static GaussLegendre8 gauss_legendre8()
{
    GaussLegendre8 g;
    const int n = 8;
    for (int i = 0; i < n; ++i) {
        double x = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1, p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        g.x[i] = x;
        g.w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    return g;
}

}  // namespace qed

using namespace qed;

extern "C" qed_status qed_exact_sample(qed_process proc, const double *d_chi, int64_t m, const double *d_u,
                                       int64_t k, double *d_xi, double *d_work, int64_t work_capacity, void *stream)
{
    clear_error();
    if (proc != QED_PROC_QS && proc != QED_PROC_BW) QED_FAIL(QED_ERR_INVALID_ARG, "bad process %d", (int)proc);
    if (m < 0 || k < 0) QED_FAIL(QED_ERR_INVALID_ARG, "negative sizes");
    if (m == 0 || k == 0) return QED_OK;
    if (!d_chi || !d_u || !d_xi || !d_work) QED_FAIL(QED_ERR_INVALID_ARG, "a device array is NULL");
    if (m >= (int64_t)1 << 31 || k > ((int64_t)1 << 40) / m) QED_FAIL(QED_ERR_INVALID_ARG, "too many draws");
    if (work_capacity < QED_EXACT_WORK(m))
        QED_FAIL(QED_ERR_INVALID_ARG, "d_work holds %lld doubles, %lld needed", (long long)work_capacity,
                 (long long)QED_EXACT_WORK(m));
    static_assert(QED_EXACT_WORK(1) == kExactRowStride, "work layout");
    static const GaussLegendre8 gl = gauss_legendre8();
    cudaStream_t st = as_stream(stream);
    const int qs = proc == QED_PROC_QS;
    exact_rows_kernel<<<(unsigned)m, 256, 0, st>>>(qs, d_chi, d_work, gl);
    QED_LAUNCH_CHECK();
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t blocks = (m * k + 127) / 128;
    const int g = (int)(blocks < (int64_t)sms * 8 ? blocks : (int64_t)sms * 8);
    exact_draw_kernel<<<g, 128, 0, st>>>(qs, d_chi, d_work, m, k, d_u, d_xi, gl);
    QED_LAUNCH_CHECK();
    return QED_OK;
}

extern "C" qed_status qed_tables_generate(const qed_table_params *params, qed_tables **out, void *stream)
{
    clear_error();
    if (!out) QED_FAIL(QED_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    qed_status s = check_params(params);
    if (s) return s;
    qed_tables *t = nullptr;
    if ((s = alloc_tables(params, &t))) return s;
    cudaStream_t st = as_stream(stream);
    GenArgs a;
    a.qs_lnG = t->d_qs_lnG, a.qs_lnP = t->d_qs_lnP, a.bw_lnT = t->d_bw_lnT, a.bw_P = t->d_bw_P;
    a.qs_l0 = std::log(params->qs.chi_min), a.qs_l1 = std::log(params->qs.chi_max);
    a.qs_xi_min = params->qs.xi_min;
    a.bw_l0 = std::log(params->bw.chi_min), a.bw_l1 = std::log(params->bw.chi_max);
    a.qs_n_chi = params->qs.n_chi, a.qs_n_xi = params->qs.n_xi;
    a.bw_n_chi = params->bw.n_chi, a.bw_n_xi = params->bw.n_xi;
    table_rows_kernel<<<params->qs.n_chi + params->bw.n_chi, 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        qed_tables_destroy(t);
        QED_FAIL(QED_ERR_CUDA, "table generation failed: %s", cudaGetErrorString(e));
    }
    // every entry must be finite (a chi range whose rates underflow FP64 is rejected)
    std::vector<double> g(params->qs.n_chi), tt(params->bw.n_chi);
    if ((s = qed_tables_copy_to_host(t, g.data(), nullptr, tt.data(), nullptr))) {
        qed_tables_destroy(t);
        return s;
    }
    for (double v : g)
        if (!std::isfinite(v)) {
            qed_tables_destroy(t);
            QED_FAIL(QED_ERR_NUMERIC, "ln G is not finite over the requested chi range");
        }
    for (double v : tt)
        if (!std::isfinite(v)) {
            qed_tables_destroy(t);
            QED_FAIL(QED_ERR_NUMERIC, "ln T is not finite over the requested chi_gamma range");
        }
    if ((s = finish_tables(t, st))) {
        qed_tables_destroy(t);
        return s;
    }
    *out = t;
    return QED_OK;
}
