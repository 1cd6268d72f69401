"""Pins of the oracle's special functions and quantum parameters against closed
forms, recurrences, an independent library (scipy) and Lorentz invariance.

The oracle (oracle/) is checked here against facts outside itself, before any
GPU result is compared with it.
"""
import math

import numpy as np
import pytest

import oracle

NUS = (1.0 / 3.0, 2.0 / 3.0, 5.0 / 3.0)
XS = (1e-8, 1e-4, 0.05, 0.7, 3.0, 25.0, 180.0, 650.0)


@pytest.mark.parametrize("x", XS)
def test_k_half_closed_form(x):
    # K_{1/2}(x) = sqrt(pi / (2x)) exp(-x): pins the quadrature machinery
    want = math.sqrt(math.pi / (2 * x)) * math.exp(-x)
    assert oracle.bessel_k(0.5, x) == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("x", XS)
def test_k_recurrence(x):
    # K_{nu+1} = K_{nu-1} + (2 nu / x) K_nu at nu = 2/3, with K_{-1/3} = K_{1/3}
    k13, k23, k53 = (oracle.bessel_k(n, x) for n in NUS)
    assert k53 == pytest.approx(k13 + 4.0 / (3.0 * x) * k23, rel=1e-12)


@pytest.mark.parametrize("x", (1e-6, 1e-3, 0.3, 2.0, 40.0))
@pytest.mark.parametrize("nu", NUS)
def test_k_against_scipy(nu, x):
    special = pytest.importorskip("scipy.special")
    assert oracle.bessel_k(nu, x) == pytest.approx(float(special.kv(nu, x)), rel=1e-12)


def test_kint_at_zero_limit():
    # int_0^inf K_nu = pi / (2 cos(nu pi / 2)); for nu = 1/3 that is pi / sqrt(3)
    want = math.pi / (2 * math.cos(math.pi / 6))
    assert oracle.bessel_kint(1.0 / 3.0, 1e-14) == pytest.approx(want, rel=1e-8)
    # nu = 2/3 with the leading small-x correction int_0^x K_{2/3} ~ (3/2) Gamma(2/3) (4x)^{1/3}
    x = 1e-14
    want23 = math.pi / (2 * math.cos(math.pi / 3)) - 1.5 * math.gamma(2 / 3) * (4 * x) ** (1 / 3)
    assert oracle.bessel_kint(2.0 / 3.0, x) == pytest.approx(want23, rel=1e-8)


@pytest.mark.parametrize("x", (1e-3, 0.2, 1.5, 12.0))
@pytest.mark.parametrize("nu", (1.0 / 3.0, 5.0 / 3.0))
def test_kint_derivative_is_minus_k(nu, x):
    h = 1e-5 * x
    d = (oracle.bessel_kint(nu, x + h) - oracle.bessel_kint(nu, x - h)) / (2 * h)
    assert d == pytest.approx(-oracle.bessel_k(nu, x), rel=1e-8)


@pytest.mark.parametrize("x", (1e-3, 0.2, 1.5, 12.0))
def test_kint_against_scipy_quad(x):
    special = pytest.importorskip("scipy.special")
    integrate = pytest.importorskip("scipy.integrate")
    val, _ = integrate.quad(lambda s: special.kv(5.0 / 3.0, s), x, np.inf, epsabs=0,
                            epsrel=1e-12, limit=500)
    assert oracle.bessel_kint(5.0 / 3.0, x) == pytest.approx(val, rel=1e-9)


def test_large_argument_underflow():
    assert oracle.bessel_k(2.0 / 3.0, 800.0) == 0.0
    assert oracle.bessel_kint(5.0 / 3.0, 800.0) == 0.0


# ---------------------------------------------------------------------------------------
# chi (§2, the Lorentz-invariant quantum parameters)
# ---------------------------------------------------------------------------------------
def _boost(beta, p, energy, E, B):
    """Fields and momentum in a frame moving with velocity beta (c = 1)."""
    beta = np.asarray(beta, float)
    b2 = beta @ beta
    g = 1.0 / math.sqrt(1.0 - b2)
    n = beta / math.sqrt(b2)
    E, B, p = (np.asarray(v, float) for v in (E, B, p))
    Ep = g * (E + np.cross(beta, B)) - g * g / (g + 1.0) * (beta @ E) * beta
    Bp = g * (B - np.cross(beta, E)) - g * g / (g + 1.0) * (beta @ B) * beta
    ppar = p @ n
    pp = p + ((g - 1.0) * ppar - g * math.sqrt(b2) * energy) * n
    return pp, Ep, Bp


def test_chi_lorentz_invariant():
    rng = np.random.default_rng(11)
    for _ in range(200):
        p = rng.normal(size=3) * 50
        E = rng.normal(size=3) * 1e-3
        B = rng.normal(size=3) * 1e-3
        beta = rng.normal(size=3)
        beta *= rng.uniform(0.05, 0.9) / np.linalg.norm(beta)
        gam = math.sqrt(1 + p @ p)
        c0 = oracle.chi_lepton(p, E, B)
        pp, Ep, Bp = _boost(beta, p, gam, E, B)
        assert oracle.chi_lepton(pp, Ep, Bp) == pytest.approx(c0, rel=1e-9)
        g0 = oracle.chi_photon(p, E, B)
        pp, Ep, Bp = _boost(beta, p, math.sqrt(p @ p), E, B)
        assert oracle.chi_photon(pp, Ep, Bp) == pytest.approx(g0, rel=1e-9)


def test_chi_special_cases():
    # magnetic field perpendicular to the momentum, no E: chi = |p| |B|
    assert oracle.chi_lepton((0, 0, 1000.0), (0, 0, 0), (0.01, 0, 0)) == pytest.approx(10.0, rel=1e-14)
    assert oracle.chi_photon((0, 300.0, 0), (0, 0, 0), (0, 0, 0.02)) == pytest.approx(6.0, rel=1e-14)
    # momentum along B, no E: chi = 0
    assert oracle.chi_lepton((0, 0, 5.0), (0, 0, 0), (0, 0, 0.3)) == 0.0
    # photon co-propagating with a plane wave (E perp B, |E| = |B|, p along E x B): chi = 0
    assert oracle.chi_photon((0, 0, 7.0), (0.01, 0, 0), (0, 0.01, 0)) == pytest.approx(0.0, abs=1e-15)
    # counter-propagating photon: chi = 2 |p| |E|
    assert oracle.chi_photon((0, 0, -7.0), (0.01, 0, 0), (0, 0.01, 0)) == pytest.approx(0.14, rel=1e-13)
    # a lepton at rest in a pure E field: chi = |E|
    assert oracle.chi_lepton((0, 0, 0), (0, 0.2, 0), (0, 0, 0)) == pytest.approx(0.2, rel=1e-15)
