"""Pins of the oracle's rate functions G (QS) and T (BW), the cumulative
distributions and the tables against closed-form asymptotes, the classical
(Larmor) limit, the Breit-Wheeler symmetry and scipy quadrature.

Closed forms used (derived from the definitions in §2.1-§2.2; the paper prints
only the garbled Eq. (t_func)):
  G(chi -> 0)   = (5 sqrt(3) / 4) chi                 [int_0^inf s K_{5/3}(s) ds = 5 pi / 3]
  G(chi -> inf) = (7/9) 3^{2/3} Gamma(2/3) chi^{2/3}
  T(chi -> 0)   = 3 sqrt(3) / (16 sqrt(2)) exp(-8 / (3 chi))     (Laplace at xi = 1/2)
  T(chi -> inf) = 15 3^{2/3} Gamma(2/3)^3 / (14 pi sqrt(3) Gamma(1/3)) chi^{-1/3}
  int_0^1 S(chi, xi) dxi -> chi^2  (classical synchrotron power, chi -> 0)
The corrections to each limit vanish at a known rate; the tests check both the
limit and that rate, so a wrong constant or a dropped term cannot hide.
"""
import math

import numpy as np
import pytest

import oracle

G23 = math.gamma(2.0 / 3.0)
G13 = math.gamma(1.0 / 3.0)
C_G_SMALL = 5.0 * math.sqrt(3.0) / 4.0
C_G_LARGE = 7.0 / 9.0 * 3.0 ** (2.0 / 3.0) * G23
C_T_SMALL = 3.0 * math.sqrt(3.0) / (16.0 * math.sqrt(2.0))
C_T_LARGE = 15.0 * 3.0 ** (2.0 / 3.0) * G23 ** 3 / (14.0 * math.pi * math.sqrt(3.0) * G13)


def _rate(dev_a, dev_b, ratio):
    return math.log(abs(dev_a / dev_b)) / math.log(ratio)


def test_G_small_chi():
    dev = [oracle.qs_G(c) / (C_G_SMALL * c) - 1.0 for c in (1e-5, 1e-4)]
    assert abs(dev[0]) < 2e-5
    assert _rate(dev[1], dev[0], 10.0) == pytest.approx(1.0, abs=0.02)  # correction ~ chi


def test_G_large_chi():
    dev = [oracle.qs_G(c) / (C_G_LARGE * c ** (2 / 3)) - 1.0 for c in (1e6, 1e8)]
    assert abs(dev[1]) < 1e-5
    assert _rate(dev[0], dev[1], 100.0) == pytest.approx(2.0 / 3.0, abs=0.03)  # ~ chi^{-2/3}


def test_T_small_chi():
    dev = [oracle.bw_T(c) / (C_T_SMALL * math.exp(-8.0 / (3.0 * c))) - 1.0 for c in (0.005, 0.01)]
    assert abs(dev[0]) < 2e-3
    assert _rate(dev[1], dev[0], 2.0) == pytest.approx(1.0, abs=0.05)  # correction ~ chi


def test_T_large_chi():
    dev = [oracle.bw_T(c) * c ** (1 / 3) / C_T_LARGE - 1.0 for c in (1e7, 1e9)]
    assert abs(dev[1]) < 1e-5
    assert _rate(dev[0], dev[1], 100.0) == pytest.approx(2.0 / 3.0, abs=0.03)


def test_asymptote_helpers_match_closed_forms():
    assert oracle.bw_T_small(0.01) == pytest.approx(C_T_SMALL * math.exp(-800.0 / 3.0), rel=1e-14)
    assert oracle.bw_T_large(1e4) == pytest.approx(C_T_LARGE * 1e4 ** (-1 / 3), rel=1e-14)


def test_classical_synchrotron_power():
    integrate = pytest.importorskip("scipy.integrate")
    for chi in (1e-4, 1e-3):
        # int_0^1 S dxi, split in ln xi where S ~ xi^{1/3}
        f = lambda u: oracle.qs_S(chi, math.exp(u)) * math.exp(u)
        lo = math.log(chi) - 60
        pts = np.linspace(lo, 0.0, 41)
        val = sum(integrate.quad(f, a, b, epsrel=1e-12, epsabs=0)[0] for a, b in zip(pts[:-1], pts[1:]))
        # correction to the classical limit is O(chi)
        assert val / chi ** 2 == pytest.approx(1.0, abs=60 * chi)


@pytest.mark.parametrize("chig", (0.05, 1.0, 30.0, 800.0))
def test_bw_symmetry(chig):
    # F(chi_g, chi_-) = F(chi_g, chi_g - chi_-): the halves of the xi integral agree
    lower = oracle.bw_T(chig) * math.pi * math.sqrt(3.0) * chig / 2.0
    assert oracle.bw_upper_half(chig) == pytest.approx(lower, rel=1e-11)


@pytest.mark.parametrize("chig,xi", ((0.3, 0.2), (3.0, 0.05), (30.0, 0.37)))
def test_bw_F_definition_symmetry_and_scale(chig, xi):
    # F(chi_g, chi_-) = F(chi_g, chi_+); T = int_0^chi_g F du
    a = oracle.bw_F(chig, xi * chig)
    b = oracle.bw_F(chig, (1 - xi) * chig)
    assert a == pytest.approx(b, rel=1e-12)


def _scipy_kint(special, integrate, nu, y):
    """int_y^inf K_nu by scipy: in w = ln s up to s = 60 (smooth for small y), then s."""
    if y >= 60.0:
        return integrate.quad(lambda s: special.kv(nu, s), y, np.inf, epsrel=1e-13, limit=400)[0]
    a = integrate.quad(lambda w: special.kv(nu, math.exp(w)) * math.exp(w), math.log(y),
                       math.log(60.0), epsrel=1e-13, limit=400)[0]
    return a + integrate.quad(lambda s: special.kv(nu, s), 60.0, np.inf, epsrel=1e-13, limit=400)[0]


def test_G_against_scipy_quadrature():
    special = pytest.importorskip("scipy.special")
    integrate = pytest.importorskip("scipy.integrate")
    chi = 1.0

    def s_du(u):  # S(chi, xi) with xi = e^u: (S/xi) dxi = S du
        xi = math.exp(u)
        om = -math.expm1(u)
        y = 2.0 * xi / (3.0 * chi * om)
        kint = _scipy_kint(special, integrate, 5 / 3, y)
        return math.sqrt(3) / (2 * math.pi) * xi * (kint + xi * xi / om * special.kv(2 / 3, y))

    pts = np.concatenate([np.linspace(-150.0, -5.0, 30), np.log(1 - np.geomspace(0.993, 1e-4, 20))])
    val = sum(integrate.quad(s_du, a, b, epsrel=1e-11, limit=400)[0] for a, b in zip(pts[:-1], pts[1:]))
    val += integrate.quad(s_du, pts[-1], 0.0, epsrel=1e-11, limit=400)[0]
    assert oracle.qs_G(chi) == pytest.approx(val, rel=1e-8)


def test_T_against_scipy_quadrature():
    special = pytest.importorskip("scipy.special")
    integrate = pytest.importorskip("scipy.integrate")
    chig = 2.0

    def bracket(xi):
        z = 2.0 / (3.0 * chig * xi * (1.0 - xi))
        kint = _scipy_kint(special, integrate, 1 / 3, z)
        return kint + (xi / (1 - xi) + (1 - xi) / xi) * special.kv(2 / 3, z)

    pts = np.linspace(0.0, 1.0, 21)
    val = sum(integrate.quad(bracket, a, b, epsrel=1e-11, limit=400)[0] for a, b in zip(pts[:-1], pts[1:]))
    assert oracle.bw_T(chig) == pytest.approx(val / (math.pi * math.sqrt(3) * chig), rel=1e-8)


# ---------------------------------------------------------------------------------------
# cumulative distributions and tables
# ---------------------------------------------------------------------------------------
def test_tables_shape_monotone_ends(oracle_tables_small):
    t = oracle_tables_small
    assert np.all(np.diff(t.qs_lnP, axis=1) >= 0)
    assert np.all(t.qs_lnP <= 0) and np.all(t.qs_lnP[:, -1] == 0.0)
    assert np.all(np.diff(t.bw_P, axis=1) >= 0)
    assert np.all(t.bw_P[:, 0] == 0.0) and np.all(t.bw_P[:, -1] == 0.5)
    assert np.all(np.isfinite(t.qs_lnG)) and np.all(np.isfinite(t.bw_lnT))
    # G increasing in chi; chi T(chi)/... T itself rises then falls (max near chi ~ 10-20)
    assert np.all(np.diff(t.qs_lnG) > 0)


def test_table_rows_consistent_with_totals(oracle_tables_small):
    # row totals of the 2-D computation equal the stand-alone G / T at the grid chi
    t = oracle_tables_small
    p = t.params
    for n in (0, 17, 40, 63):
        chi = math.exp(math.log(p["qs_chi_min"]) + n * (math.log(p["qs_chi_max"]) - math.log(p["qs_chi_min"])) / 63)
        assert math.exp(t.qs_lnG[n]) == pytest.approx(oracle.qs_G(chi), rel=1e-11)
        chg = math.exp(math.log(p["bw_chi_min"]) + n * (math.log(p["bw_chi_max"]) - math.log(p["bw_chi_min"])) / 63)
        assert math.exp(t.bw_lnT[n]) == pytest.approx(oracle.bw_T(chg), rel=1e-11)


@pytest.mark.parametrize("chi,xi", ((0.3, 1e-3), (3.0, 0.2), (30.0, 0.7)))
def test_qs_cdf_matches_table_row(chi, xi):
    # P(chi, xi) by direct quadrature equals the table-row cumulative value at a grid xi
    n_xi = 33
    G, row = oracle.qs_row(chi, n_xi, 1e-12)
    lx = np.linspace(math.log(1e-12), 0.0, n_xi)
    m = int(np.argmin(abs(lx - math.log(xi))))
    assert oracle.qs_cdf(chi, math.exp(lx[m])) == pytest.approx(math.exp(row[m]), rel=1e-10)


def test_qs_cdf_number_spectrum_small_xi_power_law():
    # the number spectrum dN/dxi ~ xi^{-2/3} at small xi, so P ~ xi^{1/3}
    chi = 1.0
    a, b = oracle.qs_cdf(chi, 1e-10), oracle.qs_cdf(chi, 1e-7)
    assert math.log(b / a) / math.log(1e3) == pytest.approx(1.0 / 3.0, abs=2e-3)


@pytest.mark.parametrize("chig", (0.3, 3.0, 30.0))
def test_bw_cdf_symmetry(chig):
    for xi in (0.1, 0.25, 0.4):
        assert oracle.bw_cdf(chig, xi) + oracle.bw_cdf(chig, 1 - xi) == pytest.approx(1.0, rel=1e-10)
    assert oracle.bw_cdf(chig, 0.5) == pytest.approx(0.5, rel=1e-11)
