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

}  // namespace qed

using namespace qed;

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
