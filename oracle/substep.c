/*
 * substep.c -- table lookups, optical-depth evolution, inverse-CDF sampling,
 * product kinematics and the Philox4x32-10 counter-based generator: the
 * per-particle QED substep (§2, §3, §5), FP64.
 *
 * TEST INFRASTRUCTURE ONLY (see qed_oracle.h).  Plain loops over particles in
 * the order given; no blocking, no fusion.  Readings of the paper taken here
 * (where it is silent or ambiguous):
 *   - interval index n with chi_n <= chi* < chi_{n+1}, clamped to [0, N-2]
 *     (so chi* = chi_max uses the last interval);
 *   - QS rate outside [chi_min, chi_max]: ln G clamped to the first/last table
 *     value (§3.2), except chi == 0 exactly, which has rate 0;
 *   - BW rate outside the table: leading asymptotes of T (Eq. (t_func)) in the
 *     paper's chi_gamma convention, T ~ 3 sqrt(3)/(16 sqrt(2)) exp(-8/(3 chi_g))
 *     for small chi_g and T ~ C_inf chi_g^{-1/3} for large chi_g, with
 *     C_inf = 15 3^{2/3} Gamma(2/3)^3 / (14 pi sqrt(3) Gamma(1/3));
 *   - search: m* = the last m with P_m <= r, clamped to [0, N_xi - 2]; a flat
 *     segment (P_{m*+1} == P_{m*}) returns xi_{m*}; for QS, ln r below the
 *     first tabulated value extrapolates the first segment (log-log);
 *   - BW: r <= 1/2 samples the electron, r > 1/2 the positron with r -> 1 - r;
 *     photon energy gamma_g <= 2 produces no pair (the event is counted and the
 *     optical depth reset);
 *   - an event fires iff the decremented optical depth is < 0; at most one
 *     event per particle per step; the optical depth is then reset to -ln U.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include "qed_oracle.h"

double oracle_chi_lepton(double, double, double, double, double, double, double, double, double);
double oracle_chi_photon(double, double, double, double, double, double, double, double, double);

/* CODATA 2018 fine-structure constant (the paper prints no value) */
#define ALPHA_F 7.2973525693e-3

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random numbers: */
/* as easy as 1, 2, 3"): ten rounds of two 32x32->64 multiplies with a Weyl    */
/* key schedule.                                                               */
/* ------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * c[0];
        uint64_t p1 = (uint64_t)PHILOX_M1 * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    memcpy(out, c, sizeof(c));
}

/* purposes of a draw, the fourth counter word */
enum { PURPOSE_SAMPLE = 0, PURPOSE_TAU_RESET = 1, PURPOSE_TAU_INIT = 2, PURPOSE_CHILD_ID = 3 };

static void draw(uint64_t seed, uint64_t id, int64_t step, uint32_t purpose, uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), (uint32_t)(uint64_t)step, purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    oracle_philox4x32_10(ctr, key, out);
}

/* 53-bit uniform in (0, 1) from two words: ((w_lo | w_hi << 32) >> 11 + 1/2) 2^-53 */
static double u53(uint32_t lo, uint32_t hi)
{
    uint64_t v = ((uint64_t)lo | ((uint64_t)hi << 32)) >> 11;
    return ((double)v + 0.5) * 0x1.0p-53;
}

double oracle_uniform(uint64_t seed, uint64_t id, int64_t step, uint32_t purpose, int which)
{
    uint32_t w[4];
    draw(seed, id, step, purpose, w);
    return which ? u53(w[2], w[3]) : u53(w[0], w[1]);
}

/* optical depth drawn from p(x) = exp(-x) (§3): tau = -ln U, U in (0,1) */
double oracle_tau_draw(uint64_t seed, uint64_t id, int64_t step, uint32_t purpose)
{
    return -log(oracle_uniform(seed, id, step, purpose, 0));
}

void oracle_child_ids(uint64_t seed, uint64_t parent, int64_t step, uint64_t out[2])
{
    uint32_t w[4];
    draw(seed, parent, step, PURPOSE_CHILD_ID, w);
    out[0] = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
    out[1] = (uint64_t)w[2] | ((uint64_t)w[3] << 32);
}

/* ------------------------------------------------------------------------- */
/* 1-D table lookups (§3.1 interpolation formula for T; §3.2 formula for G)   */
/* ln f(chi*) = ln f_n + (ln chi* - ln chi_n)(ln f_{n+1} - ln f_n)/(ln chi_{n+1} - ln chi_n) */
/* ------------------------------------------------------------------------- */
static double grid_ln(double lmin, double lmax, int N, int n)
{
    return (n == N - 1) ? lmax : lmin + n * (lmax - lmin) / (N - 1);
}

static int find_interval(double lmin, double lmax, int N, double lc)
{
    /* n with ln chi_n <= lc < ln chi_{n+1}, clamped to [0, N-2] */
    int n = 0;
    while (n < N - 2 && grid_ln(lmin, lmax, N, n + 1) <= lc) ++n;
    return n;
}

static double interp_1d(const double *lnf, double lmin, double lmax, int N, double lc)
{
    int n = find_interval(lmin, lmax, N, lc);
    double l0 = grid_ln(lmin, lmax, N, n), l1 = grid_ln(lmin, lmax, N, n + 1);
    return lnf[n] + (lc - l0) * (lnf[n + 1] - lnf[n]) / (l1 - l0);
}

/* G(chi) from the table (§3.2): clamped outside [chi_min, chi_max] */
double oracle_qs_G_table(const oracle_tables *t, double chi)
{
    if (chi == 0.0) return 0.0;
    double lmin = log(t->qs_chi_min), lmax = log(t->qs_chi_max);
    if (chi <= t->qs_chi_min) return exp(t->qs_lnG[0]);
    if (chi >= t->qs_chi_max) return exp(t->qs_lnG[t->qs_n_chi - 1]);
    return exp(interp_1d(t->qs_lnG, lmin, lmax, t->qs_n_chi, log(chi)));
}


static double t_large_coef(void)
{
    const double pi = 3.14159265358979323846;
    double g23 = tgamma(2.0 / 3.0), g13 = tgamma(1.0 / 3.0);
    return 15.0 * cbrt(9.0) * g23 * g23 * g23 / (14.0 * pi * sqrt(3.0) * g13);
}

double oracle_bw_T_small(double chig)
{
    return (3.0 * sqrt(3.0) / (16.0 * sqrt(2.0))) * exp(-8.0 / (3.0 * chig));
}
double oracle_bw_T_large(double chig) { return t_large_coef() / cbrt(chig); }

/* T(chi_g) from the table (§3.1), asymptotes (Eq. (t_func)) outside */
double oracle_bw_T_table(const oracle_tables *t, double chig)
{
    if (chig == 0.0) return 0.0;
    if (chig < t->bw_chi_min) return oracle_bw_T_small(chig);
    if (chig > t->bw_chi_max) return oracle_bw_T_large(chig);
    double lmin = log(t->bw_chi_min), lmax = log(t->bw_chi_max);
    return exp(interp_1d(t->bw_lnT, lmin, lmax, t->bw_n_chi, log(chig)));
}

/* dN/dt in units of m_e c^2/hbar:
 *   QS, Eq. (qs_total_cross): (2/3) alpha G(chi) / gamma
 *   BW, Eq. (bw_cross_tot):   alpha chi_g T(chi_g) / gamma_g */
double oracle_qs_rate(const oracle_tables *t, double chi, double gamma)
{
    return (2.0 / 3.0) * ALPHA_F * oracle_qs_G_table(t, chi) / gamma;
}
double oracle_bw_rate(const oracle_tables *t, double chig, double gg)
{
    if (gg == 0.0) return 0.0;
    return ALPHA_F * chig * oracle_bw_T_table(t, chig) / gg;
}

/* ------------------------------------------------------------------------- */
/* 2-D inverse-CDF sampling                                                   */
/* ------------------------------------------------------------------------- */
/* QS (§3.2): r in (0,1) -> xi = chi_gamma / chi */
double oracle_qs_sample_xi(const oracle_tables *t, double chi, double r)
{
    int N = t->qs_n_chi, M = t->qs_n_xi;
    double lmin = log(t->qs_chi_min), lmax = log(t->qs_chi_max);
    double c = chi < t->qs_chi_min ? t->qs_chi_min : (chi > t->qs_chi_max ? t->qs_chi_max : chi);
    double lc = log(c);
    int n = find_interval(lmin, lmax, N, lc);
    double l0 = grid_ln(lmin, lmax, N, n), l1 = grid_ln(lmin, lmax, N, n + 1);
    const double *a = t->qs_lnP + (size_t)n * M, *b = a + M;
    double lr = log(r);
    /* ln P_m on the interpolated row, then m* = last m with ln P_m <= ln r */
    int ms = 0;
    for (int m = 0; m < M; ++m) {
        double lp = a[m] + (lc - l0) * (b[m] - a[m]) / (l1 - l0);
        if (lp <= lr) ms = m;
    }
    if (ms > M - 2) ms = M - 2;
    double lp0 = a[ms] + (lc - l0) * (b[ms] - a[ms]) / (l1 - l0);
    double lp1 = a[ms + 1] + (lc - l0) * (b[ms + 1] - a[ms + 1]) / (l1 - l0);
    double lx_min = log(t->qs_xi_min);
    double lx0 = grid_ln(lx_min, 0.0, M, ms), lx1 = grid_ln(lx_min, 0.0, M, ms + 1);
    if (lp1 == lp0) return exp(lx0);
    double lxi = lx0 + (lr - lp0) * (lx1 - lx0) / (lp1 - lp0);
    if (lxi > 0.0) lxi = 0.0;
    return exp(lxi);
}

/* BW (§3.1): r in (0,1) -> xi of the sampled lepton in [0, 1/2], and whether
 * that lepton is the electron (r <= 1/2) or the positron (r > 1/2) */
double oracle_bw_sample_xi(const oracle_tables *t, double chig, double r, int *is_electron)
{
    int N = t->bw_n_chi, M = t->bw_n_xi;
    double lmin = log(t->bw_chi_min), lmax = log(t->bw_chi_max);
    *is_electron = (r <= 0.5);
    if (r > 0.5) r = 1.0 - r;
    double c = chig < t->bw_chi_min ? t->bw_chi_min : (chig > t->bw_chi_max ? t->bw_chi_max : chig);
    double lc = log(c);
    int n = find_interval(lmin, lmax, N, lc);
    double l0 = grid_ln(lmin, lmax, N, n), l1 = grid_ln(lmin, lmax, N, n + 1);
    const double *a = t->bw_P + (size_t)n * M, *b = a + M;
    int ms = 0;
    for (int m = 0; m < M; ++m) {
        double p = a[m] + (lc - l0) * (b[m] - a[m]) / (l1 - l0);
        if (p <= r) ms = m;
    }
    if (ms > M - 2) ms = M - 2;
    double p0 = a[ms] + (lc - l0) * (b[ms] - a[ms]) / (l1 - l0);
    double p1 = a[ms + 1] + (lc - l0) * (b[ms + 1] - a[ms + 1]) / (l1 - l0);
    double x0 = 0.5 * ms / (M - 1), x1 = 0.5 * (ms + 1) / (M - 1);
    if (p1 == p0) return x0;
    double xi = x0 + (r - p0) * (x1 - x0) / (p1 - p0);
    if (xi > 0.5) xi = 0.5;
    if (xi < 0.0) xi = 0.0;
    return xi;
}

/* ------------------------------------------------------------------------- */
/* optical-depth evolution (§3): tau_{n+1} = tau_n - dN/dt dt, for n particles */
/* proc 0 = QS (leptons), 1 = BW (photons).  Outputs chi, rate, new tau, and   */
/* fire[i] = (tau_new < 0).                                                    */
/* ------------------------------------------------------------------------- */
void oracle_evolve(int proc, const oracle_tables *t, int64_t n, const oracle_fields *f,
                   const double *tau, double dt, double *tau_out, double *chi_out,
                   double *rate_out, uint8_t *fire)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double px = f->px[i], py = f->py[i], pz = f->pz[i];
        double chi, rate;
        if (proc == 0) {
            chi = oracle_chi_lepton(px, py, pz, f->ex[i], f->ey[i], f->ez[i], f->bx[i], f->by[i], f->bz[i]);
            double gamma = sqrt(1.0 + px * px + py * py + pz * pz);
            rate = oracle_qs_rate(t, chi, gamma);
        } else {
            chi = oracle_chi_photon(px, py, pz, f->ex[i], f->ey[i], f->ez[i], f->bx[i], f->by[i], f->bz[i]);
            double gg = sqrt(px * px + py * py + pz * pz);
            rate = oracle_bw_rate(t, chi, gg);
        }
        double tn = tau[i] - rate * dt;
        if (chi_out) chi_out[i] = chi;
        if (rate_out) rate_out[i] = rate;
        tau_out[i] = tn;
        fire[i] = (tn < 0.0);
    }
}

/* ------------------------------------------------------------------------- */
/* events for m firing particles (already gathered, FP64)                     */
/* ------------------------------------------------------------------------- */
/* QS photon emission (§2.2 end): gamma_g = (gamma - 1) xi, photon along p,
 * lepton kinetic energy reduced by gamma_g (energy conserved: gamma' + gamma_g
 * = gamma), direction unchanged.  keep[k] = photon kept (gamma_g >= threshold,
 * §5).  Parent tau reset -log U(purpose 1); photon id from purpose 3, its
 * tau from purpose 2 with its own id. */
void oracle_qs_events(const oracle_tables *t, int64_t m, const double *px, const double *py,
                      const double *pz, const double *chi, const uint64_t *id, uint64_t seed,
                      int64_t step, double threshold, double *xi_out, double *lep_px,
                      double *lep_py, double *lep_pz, double *lep_tau, double *ph_px,
                      double *ph_py, double *ph_pz, double *ph_tau, uint64_t *ph_id,
                      uint8_t *keep)
{
    for (int64_t k = 0; k < m; ++k) {
        double r = oracle_uniform(seed, id[k], step, PURPOSE_SAMPLE, 0);
        double xi = oracle_qs_sample_xi(t, chi[k], r);
        double p2 = px[k] * px[k] + py[k] * py[k] + pz[k] * pz[k];
        double pm = sqrt(p2);
        double gamma = sqrt(1.0 + p2);
        double gg = (gamma - 1.0) * xi;
        double nx = px[k] / pm, ny = py[k] / pm, nz = pz[k] / pm;
        double g1 = gamma - gg;
        double q = (g1 - 1.0) * (g1 + 1.0);
        double pn = sqrt(q > 0.0 ? q : 0.0);
        xi_out[k] = xi;
        lep_px[k] = pn * nx;
        lep_py[k] = pn * ny;
        lep_pz[k] = pn * nz;
        lep_tau[k] = oracle_tau_draw(seed, id[k], step, PURPOSE_TAU_RESET);
        ph_px[k] = gg * nx;
        ph_py[k] = gg * ny;
        ph_pz[k] = gg * nz;
        uint64_t cid[2];
        oracle_child_ids(seed, id[k], step, cid);
        ph_id[k] = cid[0];
        ph_tau[k] = oracle_tau_draw(seed, cid[0], step, PURPOSE_TAU_INIT);
        keep[k] = (gg >= threshold);
    }
}

/* BW pair production (§2.1 end): K_pm = (gamma_g - 2) chi_pm / chi_g, products
 * along the photon momentum; gamma_+ + gamma_- = gamma_g.  made[k] = 0 when
 * gamma_g <= 2 (no pair).  The photon is removed in either case. */
void oracle_bw_events(const oracle_tables *t, int64_t m, const double *px, const double *py,
                      const double *pz, const double *chi, const uint64_t *id, uint64_t seed,
                      int64_t step, double *xi_minus, double *el_px, double *el_py,
                      double *el_pz, double *el_tau, uint64_t *el_id, double *po_px,
                      double *po_py, double *po_pz, double *po_tau, uint64_t *po_id,
                      uint8_t *made)
{
    for (int64_t k = 0; k < m; ++k) {
        double r = oracle_uniform(seed, id[k], step, PURPOSE_SAMPLE, 0);
        int is_el;
        double xs = oracle_bw_sample_xi(t, chi[k], r, &is_el);
        double xm = is_el ? xs : 1.0 - xs;
        double xp = is_el ? 1.0 - xs : xs;
        double gg = sqrt(px[k] * px[k] + py[k] * py[k] + pz[k] * pz[k]);
        xi_minus[k] = xm;
        uint64_t cid[2];
        oracle_child_ids(seed, id[k], step, cid);
        el_id[k] = cid[0];
        po_id[k] = cid[1];
        el_tau[k] = oracle_tau_draw(seed, cid[0], step, PURPOSE_TAU_INIT);
        po_tau[k] = oracle_tau_draw(seed, cid[1], step, PURPOSE_TAU_INIT);
        if (!(gg > 2.0)) {
            made[k] = 0;
            el_px[k] = el_py[k] = el_pz[k] = 0.0;
            po_px[k] = po_py[k] = po_pz[k] = 0.0;
            continue;
        }
        made[k] = 1;
        double nx = px[k] / gg, ny = py[k] / gg, nz = pz[k] / gg;
        double km = (gg - 2.0) * xm, kp = (gg - 2.0) * xp;
        double pmm = sqrt(km * (km + 2.0)), pmp = sqrt(kp * (kp + 2.0));
        el_px[k] = pmm * nx;
        el_py[k] = pmm * ny;
        el_pz[k] = pmm * nz;
        po_px[k] = pmp * nx;
        po_py[k] = pmp * ny;
        po_pz[k] = pmp * nz;
    }
}

/* initial optical depth for n particles with ids, purpose 2 (§3) */
void oracle_init_tau(int64_t n, const uint64_t *id, uint64_t seed, int64_t step, double *tau)
{
    for (int64_t i = 0; i < n; ++i) tau[i] = oracle_tau_draw(seed, id[i], step, PURPOSE_TAU_INIT);
}

/* rate lookups for n given (chi, energy) pairs: QS energy = gamma, BW energy = |p| */
void oracle_rates(int proc, const oracle_tables *t, int64_t n, const double *chi, const double *energy,
                  double *out)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = proc == 0 ? oracle_qs_rate(t, chi[i], energy[i]) : oracle_bw_rate(t, chi[i], energy[i]);
}

/* Forward maps of the table sampling: the r that the inverse-CDF lookup of
 * §3.2 / §3.1 maps to xi (the interpolated row evaluated at xi on the same
 * piecewise log-log (QS) or linear (BW) interpolant).  Used to measure the
 * backward error of a sampled xi. */
double oracle_qs_table_cdf(const oracle_tables *t, double chi, double xi)
{
    int N = t->qs_n_chi, M = t->qs_n_xi;
    double lmin = log(t->qs_chi_min), lmax = log(t->qs_chi_max);
    double c = chi < t->qs_chi_min ? t->qs_chi_min : (chi > t->qs_chi_max ? t->qs_chi_max : chi);
    double lc = log(c);
    int n = find_interval(lmin, lmax, N, lc);
    double l0 = grid_ln(lmin, lmax, N, n), l1 = grid_ln(lmin, lmax, N, n + 1);
    const double *a = t->qs_lnP + (size_t)n * M, *b = a + M;
    double lx_min = log(t->qs_xi_min), lx = log(xi);
    int m = find_interval(lx_min, 0.0, M, lx);
    double lx0 = grid_ln(lx_min, 0.0, M, m), lx1 = grid_ln(lx_min, 0.0, M, m + 1);
    double lp0 = a[m] + (lc - l0) * (b[m] - a[m]) / (l1 - l0);
    double lp1 = a[m + 1] + (lc - l0) * (b[m + 1] - a[m + 1]) / (l1 - l0);
    return exp(lp0 + (lx - lx0) * (lp1 - lp0) / (lx1 - lx0));
}

/* BW: xi of the sampled lepton in [0, 1/2] -> r in [0, 1/2] */
double oracle_bw_table_cdf(const oracle_tables *t, double chig, double xi)
{
    int N = t->bw_n_chi, M = t->bw_n_xi;
    double lmin = log(t->bw_chi_min), lmax = log(t->bw_chi_max);
    double c = chig < t->bw_chi_min ? t->bw_chi_min : (chig > t->bw_chi_max ? t->bw_chi_max : chig);
    double lc = log(c);
    int n = find_interval(lmin, lmax, N, lc);
    double l0 = grid_ln(lmin, lmax, N, n), l1 = grid_ln(lmin, lmax, N, n + 1);
    const double *a = t->bw_P + (size_t)n * M, *b = a + M;
    int m = (int)floor(xi * 2.0 * (M - 1));
    if (m < 0) m = 0;
    if (m > M - 2) m = M - 2;
    double x0 = 0.5 * m / (M - 1), x1 = 0.5 * (m + 1) / (M - 1);
    double p0 = a[m] + (lc - l0) * (b[m] - a[m]) / (l1 - l0);
    double p1 = a[m + 1] + (lc - l0) * (b[m + 1] - a[m + 1]) / (l1 - l0);
    return p0 + (xi - x0) * (p1 - p0) / (x1 - x0);
}

/* the forward maps above at n points (the kinetic-equation reference of the tabulated method) */
void oracle_qs_table_cdf_array(const oracle_tables *t, double chi, int64_t n, const double *xi, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_qs_table_cdf(t, chi, xi[i]);
}

void oracle_bw_table_cdf_array(const oracle_tables *t, double chig, int64_t n, const double *xi, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_bw_table_cdf(t, chig, xi[i]);
}
