/*
 * quad_bessel.c -- adaptive Gauss-Legendre quadrature and the modified Bessel
 * functions of the second kind used by the QED rates (§2.1, §2.2).
 *
 * TEST INFRASTRUCTURE ONLY (see qed_oracle.h).  Plain, slow FP64 reference code:
 * every quantity is the textbook definition, integrated numerically.
 *
 *   K_nu(x)            = int_0^inf exp(-x cosh t) cosh(nu t) dt
 *   Kint_nu(x)         = int_x^inf K_nu(s) ds
 *                      = int_0^inf exp(-x cosh t) cosh(nu t) / cosh t dt
 * (the second line swaps the order of integration; int_x^inf exp(-s cosh t) ds
 * = exp(-x cosh t)/cosh t).  These are the K_{1/3}, K_{2/3}, K_{5/3} and
 * int K_{5/3}, int K_{1/3} terms of Eq. (bw_cross_diff)-(t_func_0) and
 * Eq. (qs_diff_cross_exp)-(qs_g_func).
 */
#include <math.h>
#include <stddef.h>
#include "qed_oracle.h"

/* ------------------------------------------------------------------------- */
/* Gauss-Legendre nodes on [-1, 1], computed at load time by Newton iteration  */
/* on the three-term Legendre recurrence (no stored constants).               */
/* ------------------------------------------------------------------------- */
#define GL_N 12
static double gl_x[GL_N], gl_w[GL_N];

__attribute__((constructor)) static void gl_init(void)
{
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < GL_N; ++i) {
        double z = cos(pi * (i + 0.75) / (GL_N + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= GL_N; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            /* p1 = P_n(z), p0 = P_{n-1}(z) */
            dp = GL_N * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        /* recompute derivative at the converged node */
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= GL_N; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = GL_N * (z * p1 - p0) / (z * z - 1.0);
        }
        gl_x[i] = z;
        gl_w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

typedef double (*oracle_fn)(double x, void *ctx);

static double gl_panel(oracle_fn f, void *ctx, double a, double b)
{
    double h = 0.5 * (b - a), c = 0.5 * (a + b), s = 0.0;
    for (int i = 0; i < GL_N; ++i) s += gl_w[i] * f(c + h * gl_x[i], ctx);
    return h * s;
}

/* Recursive bisection: accept [a,b] once the two-half estimate agrees with the
 * whole-panel estimate to tol_abs (a pessimistic bound for the error of the
 * two-half sum, since the 12-point rule is exact to degree 23). */
static double adapt(oracle_fn f, void *ctx, double a, double b, double whole,
                    double tol_abs, int depth)
{
    double m = 0.5 * (a + b);
    double l = gl_panel(f, ctx, a, m), r = gl_panel(f, ctx, m, b);
    if (depth >= 60 || fabs(l + r - whole) <= tol_abs) return l + r;
    return adapt(f, ctx, a, m, l, tol_abs, depth + 1) +
           adapt(f, ctx, m, b, r, tol_abs, depth + 1);
}

/* int_a^b f to a relative tolerance rel (relative to a coarse estimate of the
 * whole integral, so that negligible tails are not over-resolved). */
double oracle_integrate(oracle_fn f, void *ctx, double a, double b, double rel,
                        int coarse_panels)
{
    if (!(b > a)) return 0.0;
    if (coarse_panels < 1) coarse_panels = 1;
    if (coarse_panels > 64) coarse_panels = 64;
    double part[64];
    double h = (b - a) / coarse_panels, total = 0.0;
    for (int k = 0; k < coarse_panels; ++k) {
        double lo = a + k * h, hi = (k == coarse_panels - 1) ? b : a + (k + 1) * h;
        part[k] = gl_panel(f, ctx, lo, hi);
        total += fabs(part[k]);
    }
    if (total == 0.0) return 0.0;
    double tol = rel * total;
    double s = 0.0;
    for (int k = 0; k < coarse_panels; ++k) {
        double lo = a + k * h, hi = (k == coarse_panels - 1) ? b : a + (k + 1) * h;
        s += adapt(f, ctx, lo, hi, part[k], tol, 0);
    }
    return s;
}

/* ------------------------------------------------------------------------- */
/* Bessel K_nu and its tail integral, exponentially scaled by exp(x).         */
/* ------------------------------------------------------------------------- */
typedef struct {
    double nu, x;
    int over_cosh; /* 1: integrand divided by cosh t (tail integral) */
} kctx;

static double k_integrand(double t, void *c)
{
    const kctx *k = (const kctx *)c;
    double s = sinh(0.5 * t);
    /* exp(-x cosh t) * exp(x) = exp(-x (cosh t - 1)) = exp(-2 x sinh^2(t/2)) */
    double v = exp(-2.0 * k->x * s * s) * cosh(k->nu * t);
    if (k->over_cosh) v /= cosh(t);
    return v;
}

/* upper limit where the scaled integrand has fallen below exp(-60) of its
 * value anywhere before */
static double k_tmax(double nu, double x)
{
    double t = 0.5;
    for (int it = 0; it < 2000; ++it) {
        double s = sinh(0.5 * t);
        if (2.0 * x * s * s - nu * t > 60.0 && 2.0 * x * s * s > 60.0) break;
        t += 0.25 + 0.1 * t;
    }
    return t;
}

static double k_scaled(double nu, double x, int over_cosh)
{
    kctx c = {nu, x, over_cosh};
    return oracle_integrate(k_integrand, &c, 0.0, k_tmax(nu, x), 1e-15, 6);
}

/* exp(x) K_nu(x), x > 0 */
double oracle_bessel_k_scaled(double nu, double x) { return k_scaled(nu, x, 0); }

/* exp(x) int_x^inf K_nu(s) ds, x > 0 */
double oracle_bessel_kint_scaled(double nu, double x) { return k_scaled(nu, x, 1); }

/* K_nu(x); 0 where exp(-x) underflows */
double oracle_bessel_k(double nu, double x)
{
    if (x > 745.0) return 0.0;
    return exp(-x) * k_scaled(nu, x, 0);
}

/* int_x^inf K_nu(s) ds */
double oracle_bessel_kint(double nu, double x)
{
    if (x > 745.0) return 0.0;
    return exp(-x) * k_scaled(nu, x, 1);
}
