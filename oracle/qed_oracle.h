/*
 * qed_oracle.h -- declarations of the FP64 CPU oracle for the strong-field QED
 * Monte Carlo substep (Fedeli et al., "PICSAR-QED", arXiv 2110.00256).
 *
 * TEST INFRASTRUCTURE ONLY.  This header belongs to oracle/ and is included by
 * oracle/*.c alone.  Only tests/, __graft_entry__.smoke() and the cpu_baseline
 * leg of bench.py may load the oracle library.  Nothing of the GPU path includes
 * or links this file, and the oracle includes nothing of the GPU path.
 *
 * Units (normalised, single system): momentum in m_e c, E in E_s = m_e^2 c^3/(q_e hbar)
 * (§2, definition of the Schwinger field), B in E_s/c, time in hbar/(m_e c^2).
 */
#ifndef QED_ORACLE_H
#define QED_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Read-only view of the four lookup tables (§3.1, §3.2).  Row-major 2-D arrays:
 * element (n, m) at [n * n_xi + m], n = chi index, m = xi index. */
typedef struct {
    double qs_chi_min, qs_chi_max, qs_xi_min;
    int32_t qs_n_chi, qs_n_xi;
    double bw_chi_min, bw_chi_max;
    int32_t bw_n_chi, bw_n_xi;
    const double *qs_lnG;   /* [qs_n_chi]            ln G(chi_n)                */
    const double *qs_lnP;   /* [qs_n_chi * qs_n_xi]  ln P(chi_n, xi_m)          */
    const double *bw_lnT;   /* [bw_n_chi]            ln T(chi_n)                */
    const double *bw_P;     /* [bw_n_chi * bw_n_xi]  P(chi_n, xi_m), xi <= 1/2  */
} oracle_tables;

/* one species, structure of arrays, FP64 */
typedef struct {
    const double *px, *py, *pz, *ex, *ey, *ez, *bx, *by, *bz;
} oracle_fields;

#ifdef __cplusplus
}
#endif
#endif
