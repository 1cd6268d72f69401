"""Pins of the oracle's Schwinger pair production (§2.3, Eq. (shw)): the pure
electric field reduces to Schwinger's leading term eps^2 exp(-pi/eps)/(4 pi^3);
parallel fields give eps = |E|, eta = |B|; the rate depends on the fields only
through their invariants (random Lorentz boosts leave it unchanged); null and
purely magnetic fields make nothing; the per-cell Poisson draw has the Poisson
distribution (against scipy) and the right mean and variance in its
normal-approximation branch."""
import math

import numpy as np
import pytest

import oracle


def boost(E, B, v):
    """fields in a frame moving with velocity v (c = 1)"""
    E, B, v = map(np.asarray, (E, B, v))
    g = 1.0 / math.sqrt(1.0 - v @ v)
    n = v / np.linalg.norm(v)
    Epar, Bpar = (E @ n) * n, (B @ n) * n
    Ep = Epar + g * (E - Epar + np.cross(v, B))
    Bp = Bpar + g * (B - Bpar - np.cross(v, E))
    return Ep, Bp


def test_pure_electric_field_is_schwinger_leading_term():
    r = np.random.default_rng(1)
    for eps in (0.05, 0.1, 0.3, 1.0, 3.0):
        d = r.normal(size=3)
        E = eps * d / np.linalg.norm(d)
        expected = eps * eps / (4 * math.pi ** 3) * math.exp(-math.pi / eps)
        assert oracle.schwinger_rate(E, (0, 0, 0)) == pytest.approx(expected, rel=1e-13)


def test_parallel_fields():
    for e, b in ((0.2, 0.1), (0.5, 2.0), (1.0, 1e-6)):
        got = oracle.schwinger_rate((0, 0, e), (0, 0, b))
        x = math.pi * b / e
        expected = e * b / math.tanh(x) * math.exp(-math.pi / e) / (4 * math.pi ** 2)
        assert got == pytest.approx(expected, rel=1e-12)


def test_lorentz_invariance():
    r = np.random.default_rng(2)
    for _ in range(50):
        E, B = r.normal(0, 0.2, 3), r.normal(0, 0.2, 3)
        v = r.normal(size=3)
        v = 0.9 * r.uniform() * v / np.linalg.norm(v)
        Ep, Bp = boost(E, B, v)
        a, b = oracle.schwinger_rate(E, B), oracle.schwinger_rate(Ep, Bp)
        assert b == pytest.approx(a, rel=1e-10, abs=1e-300)


def test_fields_that_make_nothing():
    assert oracle.schwinger_rate((0.3, 0, 0), (0, 0.3, 0)) == 0.0   # null field: F = G = 0
    assert oracle.schwinger_rate((0, 0, 0), (0.5, 0.1, 0)) == 0.0   # magnetic only
    assert oracle.schwinger_rate((0, 0, 0), (0, 0, 0)) == 0.0
    assert oracle.schwinger_rate((1e-3, 0, 0), (0, 0, 0)) == 0.0    # exp(-pi/eps) underflows


@pytest.mark.parametrize("lam", [0.02, 0.7, 4.0, 40.0])
def test_poisson_draw_distribution(lam):
    from scipy import stats
    n = 40000
    k = np.array([oracle.poisson(lam, 9, c, 3) for c in range(n)])
    kmax = int(lam + 8 * math.sqrt(lam) + 6)
    obs = np.bincount(np.minimum(k, kmax), minlength=kmax + 1)
    pmf = stats.poisson.pmf(np.arange(kmax + 1), lam)
    pmf[-1] += stats.poisson.sf(kmax, lam)
    exp = n * pmf
    m = exp >= 5
    chi2 = float(np.sum((obs[m] - exp[m]) ** 2 / exp[m]) + (obs[~m].sum() - exp[~m].sum()) ** 2 / max(exp[~m].sum(), 1e-9))
    assert stats.chi2.sf(chi2, m.sum()) > 1e-4, (lam, chi2)
    assert oracle.poisson(0.0, 9, 1, 3) == 0


def test_poisson_normal_branch():
    lam = 400.0
    k = np.array([oracle.poisson(lam, 5, c, 1) for c in range(40000)], dtype=np.float64)
    assert k.mean() == pytest.approx(lam, abs=4 * math.sqrt(lam / 40000) + 0.5)
    assert k.var() == pytest.approx(lam, rel=0.05)


def test_cells_and_pair_ids():
    r = np.random.default_rng(3)
    n = 500
    f = {k: r.normal(0, 0.15, n) for k in ("ex", "ey", "ez", "bx", "by", "bz")}
    out = oracle.schwinger(f, dv=1e6, dt=10.0, weight=1.0, seed=4, step=2)
    lam = out["lambda"]
    for c in range(0, n, 50):
        rate = oracle.schwinger_rate((f["ex"][c], f["ey"][c], f["ez"][c]), (f["bx"][c], f["by"][c], f["bz"][c]))
        assert lam[c] == pytest.approx(rate * 1e6 * 10.0, rel=1e-15)
    assert out["count"].sum() == len(out["e_id"]) > 0
    ids = np.concatenate([out["e_id"], out["p_id"]])
    assert len(np.unique(ids)) == len(ids)
    assert np.all(out["e_tau"] > 0) and np.all(np.isfinite(out["p_tau"]))
