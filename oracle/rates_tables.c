/*
 * rates_tables.c -- quantum parameters, differential/total rates, cumulative
 * distributions and the four lookup tables of the QED substep (§2, §3.1, §3.2).
 *
 * TEST INFRASTRUCTURE ONLY (see qed_oracle.h).  Plain FP64 code, the paper's
 * formulas written out and integrated by the adaptive quadrature of
 * quad_bessel.c.  Readings where the paper is ambiguous:
 *   - QS cumulative distribution, Eq. (qs_prob_dist): number spectrum,
 *     P(chi, xi) = int_0^xi S(chi,u)/u du / G(chi) (the same S/xi integrand whose
 *     total is G in Eq. (qs_g_func)).
 *   - BW inner integral of Eq. (t_func_0): int_X^inf sqrt(s) K_{1/3}(2/3 s^{3/2}) ds
 *     = int_z^inf K_{1/3}(w) dw with w = (2/3) s^{3/2}, z = (2/3) X^{3/2}; and
 *     chi_g X^{3/2} - 2 = xi/(1-xi) + (1-xi)/xi with xi = chi_-/chi_g.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include "qed_oracle.h"

typedef double (*oracle_fn)(double x, void *ctx);
double oracle_integrate(oracle_fn f, void *ctx, double a, double b, double rel, int coarse);
double oracle_bessel_k(double nu, double x);
double oracle_bessel_kint(double nu, double x);

static const double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------- */
/* §2: quantum parameters chi (lepton) and chi_gamma (photon), normalised units */
/* chi = gamma sqrt((E + v x B)^2 - (v.E)^2) with v = p/gamma                  */
/* ------------------------------------------------------------------------- */
double oracle_chi_lepton(double px, double py, double pz, double ex, double ey,
                         double ez, double bx, double by, double bz)
{
    double gamma = sqrt(1.0 + px * px + py * py + pz * pz);
    double vx = px / gamma, vy = py / gamma, vz = pz / gamma;
    double fx = ex + (vy * bz - vz * by);
    double fy = ey + (vz * bx - vx * bz);
    double fz = ez + (vx * by - vy * bx);
    double ve = vx * ex + vy * ey + vz * ez;
    double s = fx * fx + fy * fy + fz * fz - ve * ve;
    return gamma * sqrt(s > 0.0 ? s : 0.0);
}

/* photon: v -> c n (unit vector along p), gamma -> gamma_gamma = |p| */
double oracle_chi_photon(double px, double py, double pz, double ex, double ey,
                         double ez, double bx, double by, double bz)
{
    double gg = sqrt(px * px + py * py + pz * pz);
    if (gg == 0.0) return 0.0;
    double nx = px / gg, ny = py / gg, nz = pz / gg;
    double fx = ex + (ny * bz - nz * by);
    double fy = ey + (nz * bx - nx * bz);
    double fz = ez + (nx * by - ny * bx);
    double ne = nx * ex + ny * ey + nz * ez;
    double s = fx * fx + fy * fy + fz * fz - ne * ne;
    return gg * sqrt(s > 0.0 ? s : 0.0);
}

/* ------------------------------------------------------------------------- */
/* §2.2 quantum synchrotron: S(chi, xi) of Eq. (qs_diff_cross)-(qs_g_func)    */
/*   S = sqrt(3)/(2 pi) xi [ int_Y^inf K_{5/3} + xi^2/(1-xi) K_{2/3}(Y) ]     */
/*   Y = (2/3) xi / (chi (1 - xi))                                            */
/* one_minus_xi is passed separately to keep 1-xi accurate near xi = 1.       */
/* ------------------------------------------------------------------------- */
static double qs_S_om(double chi, double xi, double one_minus_xi)
{
    if (xi <= 0.0 || one_minus_xi <= 0.0) return 0.0;
    double Y = (2.0 / 3.0) * xi / (chi * one_minus_xi);
    double br = oracle_bessel_kint(5.0 / 3.0, Y) +
                xi * xi / one_minus_xi * oracle_bessel_k(2.0 / 3.0, Y);
    return sqrt(3.0) / (2.0 * PI) * xi * br;
}

double oracle_qs_S(double chi, double xi) { return qs_S_om(chi, xi, 1.0 - xi); }

/* ------------------------------------------------------------------------- */
/* §2.1 Breit-Wheeler: the bracket of Eq. (t_func_0) in xi = chi_-/chi_gamma  */
/*   br(chi_g, xi) = int_z^inf K_{1/3} + (xi/(1-xi) + (1-xi)/xi) K_{2/3}(z)    */
/*   z = (2/3) X^{3/2} = 2 / (3 chi_g xi (1 - xi))                            */
/* so that F(chi_g, chi_-) = br / (pi sqrt(3) chi_g^2)  (Eq. (bw_cross_diff))  */
/* and T(chi_g) = int_0^chi_g F du = 1/(pi sqrt(3) chi_g) int_0^1 br dxi.     */
/* ------------------------------------------------------------------------- */
double oracle_bw_bracket(double chig, double xi)
{
    if (xi <= 0.0 || xi >= 1.0) return 0.0;
    double q = xi * (1.0 - xi);
    double z = 2.0 / (3.0 * chig * q);
    return oracle_bessel_kint(1.0 / 3.0, z) +
           (xi / (1.0 - xi) + (1.0 - xi) / xi) * oracle_bessel_k(2.0 / 3.0, z);
}

/* F(chi_g, chi_-) of Eq. (bw_cross_diff), chi_- in (0, chi_g) */
double oracle_bw_F(double chig, double chim)
{
    return oracle_bw_bracket(chig, chim / chig) / (PI * sqrt(3.0) * chig * chig);
}

/* ------------------------------------------------------------------------- */
/* integrands for the cumulative integrals                                    */
/* ------------------------------------------------------------------------- */
typedef struct { double chi; } qs_ctx;

/* QS in u = ln xi: (S/xi) dxi = S du */
static double qs_integrand_lnxi(double u, void *c)
{
    double chi = ((qs_ctx *)c)->chi;
    double xi = exp(u);
    return qs_S_om(chi, xi, -expm1(u));
}

typedef struct { double chig; } bw_ctx;
static double bw_integrand_xi(double xi, void *c)
{
    return oracle_bw_bracket(((bw_ctx *)c)->chig, xi);
}

#define OUTER_REL 1e-13

/* Row of the QS 2-D table (§3.2): xi_m log-spaced on [xi_min, 1], m = 0..n_xi-1.
 * Writes ln P(chi, xi_m) and returns G(chi) (Eq. (qs_g_func)).
 * The cumulative integral is accumulated interval by interval; the integral
 * below xi_min is taken down to xi_min * exp(-150) (S ~ xi^{1/3} there). */
double oracle_qs_row(double chi, int n_xi, double xi_min, double *lnP_row)
{
    qs_ctx c = {chi};
    double lmin = log(xi_min);
    double *dC = (double *)malloc(sizeof(double) * (size_t)n_xi);
    dC[0] = oracle_integrate(qs_integrand_lnxi, &c, lmin - 150.0, lmin, OUTER_REL, 16);
    for (int m = 1; m < n_xi; ++m) {
        double u0 = lmin + (m - 1) * (0.0 - lmin) / (n_xi - 1);
        double u1 = (m == n_xi - 1) ? 0.0 : lmin + m * (0.0 - lmin) / (n_xi - 1);
        dC[m] = oracle_integrate(qs_integrand_lnxi, &c, u0, u1, OUTER_REL, 1);
    }
    double G = 0.0;
    for (int m = 0; m < n_xi; ++m) G += dC[m];
    if (lnP_row) {
        /* P_m = C_m / G.  Near P = 1 use the complementary tail sum so that
         * ln P = log1p(-tail/G) keeps its relative accuracy. */
        double C = 0.0;
        for (int m = 0; m < n_xi; ++m) {
            C += dC[m];
            double tail = 0.0;
            for (int k = m + 1; k < n_xi; ++k) tail += dC[k];
            double q = tail / G;
            lnP_row[m] = (q < 0.5) ? log1p(-q) : log(C / G);
        }
        lnP_row[n_xi - 1] = 0.0;
    }
    free(dC);
    return G;
}

/* Row of the BW 2-D table (§3.1): xi_m = 0.5 m / (n_xi - 1).  Writes
 * P(chi_g, xi_m) = int_0^xi_m br / int_0^1 br, using the symmetry of br under
 * xi -> 1 - xi for the denominator (int_0^1 = 2 int_0^{1/2}); returns T(chi_g)
 * of Eq. (t_func_0). */
double oracle_bw_row(double chig, int n_xi, double *P_row)
{
    bw_ctx c = {chig};
    double *dC = (double *)malloc(sizeof(double) * (size_t)n_xi);
    dC[0] = 0.0;
    for (int m = 1; m < n_xi; ++m) {
        double a = 0.5 * (m - 1) / (n_xi - 1);
        double b = (m == n_xi - 1) ? 0.5 : 0.5 * m / (n_xi - 1);
        dC[m] = oracle_integrate(bw_integrand_xi, &c, a, b, OUTER_REL, 1);
    }
    double half = 0.0;
    for (int m = 0; m < n_xi; ++m) half += dC[m];
    if (P_row) {
        double C = 0.0;
        for (int m = 0; m < n_xi; ++m) {
            C += dC[m];
            P_row[m] = (half > 0.0) ? C / (2.0 * half) : 0.0;
        }
        P_row[0] = 0.0;
        if (half > 0.0) P_row[n_xi - 1] = 0.5;
    }
    free(dC);
    return 2.0 * half / (PI * sqrt(3.0) * chig);
}

/* ------------------------------------------------------------------------- */
/* stand-alone functions (same quadrature on a fine default grid)             */
/* ------------------------------------------------------------------------- */
double oracle_qs_G(double chi) { return oracle_qs_row(chi, 65, 1e-12, NULL); }
double oracle_bw_T(double chig) { return oracle_bw_row(chig, 65, NULL); }

/* upper half of the BW bracket integral, int_{1/2}^{1} br dxi, integrated
 * directly (used to check the symmetry the table relies on) */
double oracle_bw_upper_half(double chig)
{
    bw_ctx c = {chig};
    double s = 0.0;
    for (int k = 0; k < 64; ++k)
        s += oracle_integrate(bw_integrand_xi, &c, 0.5 + 0.5 * k / 64.0,
                              (k == 63) ? 1.0 : 0.5 + 0.5 * (k + 1) / 64.0, OUTER_REL, 1);
    return s;
}

/* exact cumulative distributions by direct quadrature, used to test sampling:
 * QS P(chi, xi), xi in (0, 1]; BW P(chi_g, xi), xi in [0, 1] */
double oracle_qs_cdf(double chi, double xi)
{
    if (xi <= 0.0) return 0.0;
    if (xi >= 1.0) return 1.0;
    qs_ctx c = {chi};
    double G = oracle_qs_G(chi);
    double lx = log(xi);
    /* int_0^xi: below 1e-12 as in the table, then up to xi on a grid of 64 */
    double lo = log(1e-12) < lx ? log(1e-12) : lx;
    double s = oracle_integrate(qs_integrand_lnxi, &c, lo - 150.0, lo, OUTER_REL, 16);
    for (int k = 0; k < 64; ++k)
        s += oracle_integrate(qs_integrand_lnxi, &c, lo + (lx - lo) * k / 64.0,
                              (k == 63) ? lx : lo + (lx - lo) * (k + 1) / 64.0, OUTER_REL, 1);
    return s / G;
}

double oracle_bw_cdf(double chig, double xi)
{
    if (xi <= 0.0) return 0.0;
    if (xi >= 1.0) return 1.0;
    bw_ctx c = {chig};
    double half = 0.0;
    for (int k = 0; k < 64; ++k)
        half += oracle_integrate(bw_integrand_xi, &c, 0.5 * k / 64.0,
                                 (k == 63) ? 0.5 : 0.5 * (k + 1) / 64.0, OUTER_REL, 1);
    double s = 0.0;
    for (int k = 0; k < 64; ++k)
        s += oracle_integrate(bw_integrand_xi, &c, xi * k / 64.0,
                              (k == 63) ? xi : xi * (k + 1) / 64.0, OUTER_REL, 1);
    return s / (2.0 * half);
}

/* ------------------------------------------------------------------------- */
/* full table build, rows in parallel                                         */
/* chi_n = exp(ln chi_min + n (ln chi_max - ln chi_min)/(N-1)), both ends in. */
/* ------------------------------------------------------------------------- */
void oracle_build_qs_tables(double chi_min, double chi_max, int n_chi, int n_xi,
                            double xi_min, double *lnG, double *lnP)
{
    double l0 = log(chi_min), l1 = log(chi_max);
#pragma omp parallel for schedule(dynamic, 1)
    for (int n = 0; n < n_chi; ++n) {
        double lc = (n == n_chi - 1) ? l1 : l0 + n * (l1 - l0) / (n_chi - 1);
        double G = oracle_qs_row(exp(lc), n_xi, xi_min, lnP + (size_t)n * n_xi);
        lnG[n] = log(G);
    }
}

void oracle_build_bw_tables(double chi_min, double chi_max, int n_chi, int n_xi,
                            double *lnT, double *P)
{
    double l0 = log(chi_min), l1 = log(chi_max);
#pragma omp parallel for schedule(dynamic, 1)
    for (int n = 0; n < n_chi; ++n) {
        double lc = (n == n_chi - 1) ? l1 : l0 + n * (l1 - l0) / (n_chi - 1);
        double T = oracle_bw_row(exp(lc), n_xi, P + (size_t)n * n_xi);
        lnT[n] = log(T);
    }
}

/* exact cumulative distributions at n ascending points xs[] (0 < xs < 1), the
 * integral accumulated between consecutive points; used for KS distances */
void oracle_qs_cdf_sorted(double chi, int64_t n, const double *xs, double *out)
{
    qs_ctx c = {chi};
    double G = oracle_qs_G(chi);
    double lo = log(1e-12);
    if (n > 0 && log(xs[0]) < lo) lo = log(xs[0]);
    double acc = oracle_integrate(qs_integrand_lnxi, &c, lo - 150.0, lo, OUTER_REL, 16);
    double prev = lo;
    for (int64_t i = 0; i < n; ++i) {
        double lx = log(xs[i]);
        if (lx > prev) {
            for (int k = 0; k < 4; ++k)
                acc += oracle_integrate(qs_integrand_lnxi, &c, prev + (lx - prev) * k / 4.0,
                                        (k == 3) ? lx : prev + (lx - prev) * (k + 1) / 4.0, OUTER_REL, 1);
            prev = lx;
        }
        out[i] = acc / G;
    }
}

void oracle_bw_cdf_sorted(double chig, int64_t n, const double *xs, double *out)
{
    bw_ctx c = {chig};
    double half = 0.0;
    for (int k = 0; k < 64; ++k)
        half += oracle_integrate(bw_integrand_xi, &c, 0.5 * k / 64.0,
                                 (k == 63) ? 0.5 : 0.5 * (k + 1) / 64.0, OUTER_REL, 1);
    double acc = 0.0, prev = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double x = xs[i];
        if (x > prev) {
            for (int k = 0; k < 4; ++k)
                acc += oracle_integrate(bw_integrand_xi, &c, prev + (x - prev) * k / 4.0,
                                        (k == 3) ? x : prev + (x - prev) * (k + 1) / 4.0, OUTER_REL, 1);
            prev = x;
        }
        out[i] = acc / (2.0 * half);
    }
}

/* ------------------------------------------------------------------------- */
/* pointwise spectra on many points (the kinetic-equation reference)          */
/* ------------------------------------------------------------------------- */
void oracle_qs_S_array(double chi, int64_t n, const double *xi, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_qs_S(chi, xi[i]);
}

void oracle_bw_bracket_array(double chig, int64_t n, const double *xi, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_bw_bracket(chig, xi[i]);
}
