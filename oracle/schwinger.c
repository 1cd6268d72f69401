/*
 * schwinger.c -- FP64 oracle of Schwinger pair production per cell (§2.3,
 * Eq. (shw)).  TEST INFRASTRUCTURE ONLY (see qed_oracle.h).
 *
 * Normalised units (c = 1, fields in E_s): F = (E^2 - B^2)/2, G = E.B,
 * eps = sqrt(sqrt(F^2 + G^2) + F), eta = sqrt(sqrt(F^2 + G^2) - F), and the
 * prefactor q_e^2 E_s^2 / (4 pi^2 hbar^2 c) of Eq. (shw) is 1/(4 pi^2) in units
 * of 1/(lambda_C^3 t_C) (lambda_C = hbar/(m_e c), t_C = hbar/(m_e c^2)):
 *     d2N/dt dV = eps eta coth(pi eta / eps) exp(-pi / eps) / (4 pi^2).
 * The number of pairs a cell of volume dV makes in dt is Poisson distributed
 * with mean lambda = rate dV dt / w, for pairs of weight w, drawn from the
 * Philox counter (cell, step, 4): inversion of the cumulative distribution
 * (k = first k with U <= P(K <= k), probabilities by the recurrence
 * p_k = p_{k-1} lambda / k) for lambda <= 100; above, k = max(0, floor(lambda +
 * sqrt(lambda) z + 1/2)) with z = sqrt(-2 ln U1) cos(2 pi U2) (Box-Muller).
 * Pair j of a cell takes the ids of Philox (cell, step, 5 + 256 j): words 0-1
 * the electron's, words 2-3 the positron's; both start at rest.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "qed_oracle.h"

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]);

static const double PI = 3.14159265358979323846;

double oracle_schwinger_rate(double ex, double ey, double ez, double bx, double by, double bz)
{
    double F = 0.5 * ((ex * ex + ey * ey + ez * ez) - (bx * bx + by * by + bz * bz));
    double G = ex * bx + ey * by + ez * bz;
    double r = sqrt(F * F + G * G);
    double eps = sqrt(r + F);
    double eta = sqrt(r - F > 0.0 ? r - F : 0.0);
    if (!(eps > 0.0)) return 0.0;
    /* eta coth(pi eta / eps) = (eps / pi) x coth x, x = pi eta / eps; x coth x -> 1 as x -> 0 */
    double x = PI * eta / eps;
    double xcothx = x < 1e-8 ? 1.0 : x / tanh(x);
    return eps * (eps / PI) * xcothx * exp(-PI / eps) / (4.0 * PI * PI);
}

static void draw(uint64_t seed, uint64_t cell, int64_t step, uint32_t purpose, uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)cell, (uint32_t)(cell >> 32), (uint32_t)(uint64_t)step, purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    oracle_philox4x32_10(ctr, key, out);
}

static double u53(uint32_t lo, uint32_t hi)
{
    uint64_t v = ((uint64_t)lo | ((uint64_t)hi << 32)) >> 11;
    return ((double)v + 0.5) * 0x1.0p-53;
}

int64_t oracle_poisson(double lambda, uint64_t seed, uint64_t cell, int64_t step)
{
    if (!(lambda > 0.0)) return 0;
    uint32_t w[4];
    draw(seed, cell, step, 4u, w);
    double u = u53(w[0], w[1]);
    if (lambda <= 100.0) {
        double p = exp(-lambda), cdf = p;
        int64_t k = 0;
        while (u > cdf && k < 1000) {
            ++k;
            p *= lambda / (double)k;
            cdf += p;
        }
        return k;
    }
    double z = sqrt(-2.0 * log(u)) * cos(2.0 * PI * u53(w[2], w[3]));
    double k = floor(lambda + sqrt(lambda) * z + 0.5);
    return k > 0.0 ? (int64_t)k : 0;
}

void oracle_schwinger_pair_ids(uint64_t seed, uint64_t cell, int64_t step, int64_t j, uint64_t out[2])
{
    uint32_t w[4];
    draw(seed, cell, step, 5u + 256u * (uint32_t)j, w);
    out[0] = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
    out[1] = (uint64_t)w[2] | ((uint64_t)w[3] << 32);
}

/* per cell: expected pairs lambda and the drawn count k */
void oracle_schwinger_cells(int64_t n, const double *ex, const double *ey, const double *ez, const double *bx,
                            const double *by, const double *bz, double dv, double dt, double weight, uint64_t seed,
                            int64_t step, double *lambda, int64_t *count)
{
    for (int64_t c = 0; c < n; ++c) {
        double l = oracle_schwinger_rate(ex[c], ey[c], ez[c], bx[c], by[c], bz[c]) * dv * dt / weight;
        lambda[c] = l;
        count[c] = oracle_poisson(l, seed, (uint64_t)c, step);
    }
}
