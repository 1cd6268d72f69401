"""Pins of the kinetic-equation reference (oracle/kinetic.py): its fine-grid
spectra against the oracle's exact G, T and distributions; the generator's
conservation laws (one lepton stays one lepton; a decay turns one photon into
two leptons); the initial energy-loss rate against the emitted power computed
by independent quadrature; energy conservation of the solution; and the stored
reference spectra reproduced."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import kinetic

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("chi", [0.01, 0.3, 1.0, 9.0])
def test_qs_spectrum_matches_exact(chi):
    xi, cdf, G = kinetic.qs_spectrum(chi)
    assert G == pytest.approx(oracle.qs_G(chi), rel=1e-5)
    pts = np.array([1e-6, 1e-3, 0.1, 0.5, 0.9])
    got = np.interp(np.log(pts) - np.log1p(-pts), np.log(xi) - np.log1p(-xi), cdf)
    exact = [oracle.qs_cdf(chi, p) for p in pts]
    assert np.max(np.abs(got - exact)) < 2e-5
    assert np.all(np.diff(cdf) >= 0) and cdf[-1] == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("chig", [0.1, 1.0, 9.0, 50.0])
def test_bw_spectrum_matches_exact(chig):
    xi, cdf, T = kinetic.bw_spectrum(chig)
    assert T == pytest.approx(oracle.bw_T(chig), rel=5e-5)
    pts = np.array([0.01, 0.1, 0.3, 0.5, 0.8])
    got = np.interp(np.log(pts) - np.log1p(-pts), np.log(xi) - np.log1p(-xi), cdf)
    exact = [oracle.bw_cdf(chig, p) for p in pts]
    assert np.max(np.abs(got - exact)) < 5e-5
    assert np.allclose(cdf + cdf[::-1], 1.0, atol=1e-12)  # symmetry about xi = 1/2


@pytest.fixture(scope="module")
def small_generator():
    b0 = 1e-2
    lep = kinetic.LogBins(999.0, 1e-2, 120)
    pho = kinetic.LogBins(999.0, 1e-3, 120)
    A = kinetic.build_generator(lambda g: math.sqrt(g * g - 1) * b0, lambda g: g * b0, lep, pho)
    return A, lep, pho, b0


def test_generator_conservation(small_generator):
    A, lep, pho, _ = small_generator
    n, m = lep.n, pho.n
    P, G, S = slice(0, n + 1), slice(n + 1, n + 1 + m + 1), slice(n + 1 + m + 1, None)
    scale = np.abs(A).max()
    # emission moves a lepton within its population: lepton columns sum to zero there
    assert np.max(np.abs(A[P, P].sum(0))) < 1e-13 * scale
    assert np.max(np.abs(A[S, S].sum(0))) < 1e-13 * scale
    # a decay removes one photon and adds two leptons
    rate = -np.diag(A[G, G])
    assert np.allclose(A[S, G].sum(0), 2.0 * rate, rtol=1e-12, atol=1e-13 * scale)
    # photons are only made, never moved: off-diagonal photon-photon entries vanish
    off = A[G, G] - np.diag(np.diag(A[G, G]))
    assert not off.any()
    assert np.all(A[G, P] >= 0) and np.all(A[S, G] >= 0)


def test_initial_energy_loss_equals_emitted_power(small_generator):
    """d<gamma>/dt at t = 0 from the generator against the emitted power
    (2/3) alpha (K / gamma) int_0^1 S(chi, xi) dxi, by scipy quadrature."""
    from scipy.integrate import quad
    A, lep, pho, b0 = small_generator
    n = lep.n
    j = n - 1
    K = lep.centres[j]
    gamma = 1.0 + K
    chi = math.sqrt(gamma * gamma - 1) * b0
    integral = quad(lambda x: oracle.qs_S(chi, x), 0.0, 1.0, limit=400, epsabs=0, epsrel=1e-10)[0]
    power = (2.0 / 3.0) * oracle.ALPHA_F * K / gamma * integral
    loss = -float(np.dot(lep.centres, A[:n, j]))
    assert loss == pytest.approx(power, rel=1e-4)
    photon_power = float(np.dot(pho.centres, A[n + 1:n + 1 + pho.n, j]))
    assert photon_power == pytest.approx(power, rel=1e-4)


def test_stored_reference_reproduced_and_energy_conserved():
    with open(os.path.join(HERE, "golden", "ridgers_kinetic.json")) as f:
        ref = json.load(f)
    from golden.make_ridgers_reference import chi_functions, coarse, FINE
    c = ref["cases"]["3"]
    chi_l, chi_g = chi_functions(3)
    r = kinetic.spectra(chi_l, chi_g, c["gamma0"], c["t"], n_lepton=FINE, n_photon=FINE)
    for k in ("primary", "photons", "secondary"):
        assert np.allclose(coarse(r[k]), c["exact"][k], rtol=1e-9, atol=1e-15), k
    e = (np.sum(r["primary"][:FINE] * (1 + r["lepton_centres"])) + np.sum(r["photons"][:FINE] * r["photon_centres"])
         + np.sum(r["secondary"][:FINE] * (1 + r["lepton_centres"])))
    assert e == pytest.approx(c["gamma0"], rel=1e-4)


def test_tabulated_method_against_exact_spectra():
    """What the 256 / 256x256 tables sample against the exact spectra (stored
    references): the primary electron spectra agree above a fifth of gamma0 in
    every case; at chi = 9 (case 3) the table's last xi interval [0.897, 1],
    inside which the log-log interpolant spreads the hardest photons almost
    uniformly in ln xi, over-populates the lowest electron energies."""
    with open(os.path.join(HERE, "golden", "ridgers_kinetic.json")) as f:
        ref = json.load(f)
    for case, c in ref["cases"].items():
        edges = np.asarray(c["lepton_edges"])
        ex, tb = np.asarray(c["exact"]["primary"][:-1]), np.asarray(c["tables_256"]["primary"][:-1])
        bulk = (edges[:-1] >= 0.2 * c["gamma0"]) & (ex > 1e-3)
        assert np.max(np.abs(tb[bulk] / ex[bulk] - 1)) < 0.01, case
        assert c["tables_256"]["mean_gamma_primary"] == pytest.approx(c["exact"]["mean_gamma_primary"], rel=2e-3)
    c = ref["cases"]["3"]
    edges = np.asarray(c["lepton_edges"])
    ex, tb = np.asarray(c["exact"]["primary"][:-1]), np.asarray(c["tables_256"]["primary"][:-1])
    low = (edges[:-1] < 0.02 * c["gamma0"]) & (ex * 1e5 > 100)
    assert np.all(tb[low] > 1.3 * ex[low])
