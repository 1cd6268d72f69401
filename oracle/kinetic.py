"""Deterministic reference for many-step runs: the kinetic (master) equation of
the energy distributions of leptons and photons under photon emission (§2.2)
and pair production (§2.1), for fields in which a particle's chi is a function
of its energy alone (a uniform magnetic field perpendicular to the motion; a
circularly polarised plane wave met head-on).  This is the kind of solution the
paper's §5 benchmarks compare the Monte Carlo spectra against.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The substep's Monte Carlo (an optical depth per particle, an event when it runs
out, §3) samples a Markov jump process:
  * a lepton of kinetic energy K = gamma - 1 emits at the rate
    W_e = (2/3) alpha G(chi)/gamma (Eq. (qs_total_cross)) a photon of energy
    K xi, xi from the number spectrum S(chi, xi)/xi / G(chi) (reading R1), and
    keeps K (1 - xi) (§2.2, energy bookkeeping of the recoil);
  * a photon of energy g decays at W_g = alpha chi_g T(chi_g) / g
    (Eq. (bw_cross_tot)) into two leptons of kinetic energies (g - 2) xi and
    (g - 2)(1 - xi), xi from dP/dxi of Eq. (bw_prob_dist) on [0, 1]
    (symmetric); g <= 2 makes no pair.
The number densities f then obey d f / dt = A f with A built from these rates
and spectra; f(t) = exp(A t) f(0).

Discretisation: log-spaced energy bins; a particle sits at its bin's centre and
the landing point of a jump is shared between the two bins whose centres
bracket it, with weights linear in energy (this keeps the energy of every jump
exact, so that many small emissions drift the lepton correctly).  The
spectra are integrated on fine grids from the oracle's pointwise S and the
bracket of Eq. (t_func_0), so the rates are the oracle's exact G and T (not the
tables).  Three populations: the primary leptons, the photons, and the
secondary leptons (electrons and positrons of the pairs, together), each with an
underflow bin below the lowest energy.
"""
from __future__ import annotations

import math

import numpy as np

from . import ALPHA_F, bw_bracket_array, qs_S_array


# ----------------------------------------------------------------------------
# spectra on fine grids
# ----------------------------------------------------------------------------
def qs_spectrum(chi: float, n_low: int = 2400, n_high: int = 2400, xi_floor: float = 1e-12):
    """Number spectrum of photon emission at chi: returns (xi, cdf, G) with xi
    ascending in (0, 1), cdf(xi) = int_0^xi S/u du / G and G = int_0^1 S/u du.
    Below xi = 1/2 the integral runs in ln xi (integrand S), above it in
    -ln(1 - xi) (integrand S (1 - xi)/xi); below xi_floor S ~ c xi^(1/3), whose
    integral is 3 S(xi_floor)."""
    lo = np.geomspace(xi_floor, 0.5, n_low)
    eta = np.geomspace(0.5, 1e-12, n_high)[1:]
    hi = 1.0 - eta
    s_lo = qs_S_array(chi, lo)
    s_hi = qs_S_array(chi, hi)
    c_lo = np.concatenate([[0.0], np.cumsum(0.5 * (s_lo[1:] + s_lo[:-1]) * np.diff(np.log(lo)))])
    w = -np.log(eta)
    g_hi = s_hi * eta / hi
    g_mid = s_lo[-1] * 0.5 / 0.5  # S (1 - xi)/xi at xi = 1/2
    gw = np.concatenate([[g_mid], g_hi])
    ww = np.concatenate([[math.log(2.0)], w])
    c_hi = c_lo[-1] + np.cumsum(0.5 * (gw[1:] + gw[:-1]) * np.diff(ww))
    tail = 3.0 * s_lo[0]
    xi = np.concatenate([lo, hi])
    cum = tail + np.concatenate([c_lo, c_hi])
    G = cum[-1]
    return xi, cum / G, G


def bw_spectrum(chig: float, n_half: int = 4000, xi_floor: float = 1e-9):
    """Pair-energy distribution at chi_gamma: returns (xi, cdf, T) with xi
    ascending in (0, 1), cdf(xi) the fraction with chi_-/chi_gamma < xi
    (symmetric about 1/2) and T = (1 / (pi sqrt(3) chi_g)) int_0^1 bracket."""
    lo = np.geomspace(xi_floor, 0.5, n_half)
    b = bw_bracket_array(chig, lo)
    c = np.concatenate([[0.0], np.cumsum(0.5 * (b[1:] * lo[1:] + b[:-1] * lo[:-1]) * np.diff(np.log(lo)))])
    half = c[-1]
    if not half > 0.0:  # the rate underflows FP64 (chi_gamma of a few 1e-3)
        return None, None, 0.0
    xi = np.concatenate([lo, 1.0 - lo[-2::-1]])
    cdf = np.concatenate([c / (2 * half), 1.0 - c[-2::-1] / (2 * half)])
    T = 2.0 * half / (math.pi * math.sqrt(3.0) * chig)
    return xi, cdf, T


# ----------------------------------------------------------------------------
# bins and the linear sharing of a landing point between two bin centres
# ----------------------------------------------------------------------------
class LogBins:
    """n bins of equal width d in ln E whose top centre is `top`."""

    def __init__(self, top: float, bottom: float, n: int):
        self.n = n
        self.d = math.log(top / bottom) / (n - 1)
        self.ln_top = math.log(top)
        self.centres = np.exp(self.ln_top - self.d * np.arange(n)[::-1])  # ascending
        self.edges = np.exp(np.log(self.centres[0]) - 0.5 * self.d + self.d * np.arange(n + 1))

    def share(self, ln_e: np.ndarray, mass: np.ndarray) -> np.ndarray:
        """Distribute `mass` landing at ln energies `ln_e` over the n bins and an
        underflow bin (index n): returns an array of n + 1.  A landing point
        between two centres is shared linearly in energy, which keeps the
        energy of every jump."""
        pos = (ln_e - math.log(self.centres[0])) / self.d
        out = np.zeros(self.n + 1)
        under = pos < 0.0
        out[self.n] += mass[under].sum()
        top = pos >= self.n - 1
        out[self.n - 1] += mass[top & ~under].sum()
        keep = ~under & ~top
        pos, m, e = pos[keep], mass[keep], np.exp(ln_e[keep])
        i0 = np.floor(pos).astype(np.int64)
        lo, hi = self.centres[i0], self.centres[i0 + 1]
        fr = (e - lo) / (hi - lo)
        np.add.at(out, i0, m * (1.0 - fr))
        np.add.at(out, i0 + 1, m * fr)
        return out


def _masses(cdf):
    """probability masses of the grid intervals, placed at the interval's
    geometric middle in the logit of xi"""
    return np.diff(cdf)


def _mid(xi):
    lg = np.log(xi) - np.log1p(-xi)
    m = 0.5 * (lg[1:] + lg[:-1])
    return 1.0 / (1.0 + np.exp(-m))


# ----------------------------------------------------------------------------
# the two models: the exact spectra, or the tabulated method (§3.1, §3.2)
# ----------------------------------------------------------------------------
class ExactModel:
    """Rates and spectra of §2 from the oracle's quadrature."""

    def qs(self, chi: float, gamma: float):
        xi, cdf, G = qs_spectrum(chi)
        return xi, cdf, (2.0 / 3.0) * ALPHA_F * G / gamma

    def bw(self, chig: float, g: float):
        xi, cdf, T = bw_spectrum(chig)
        return xi, cdf, (ALPHA_F * chig * T / g if T > 0.0 else 0.0)


class TableModel:
    """What the substep samples with tables `t` (an OracleTables): the rates
    from the 1-D tables (with their out-of-table rules) and, as the spectra,
    the forward maps of the inverse-CDF lookups on the 2-D tables."""

    def __init__(self, t):
        self.t = t

    def qs(self, chi: float, gamma: float):
        n_low, n_high, floor = qs_spectrum.__defaults__
        xi = np.concatenate([np.geomspace(floor, 0.5, n_low), 1.0 - np.geomspace(0.5, 1e-12, n_high)[1:]])
        cdf = np.minimum(self.t.qs_table_cdf_array(chi, xi), 1.0)
        cdf = np.maximum.accumulate(cdf)
        return xi, cdf, float(self.t.rates(0, np.array([chi]), np.array([gamma]))[0])

    def bw(self, chig: float, g: float):
        n_half, floor = bw_spectrum.__defaults__
        lo = np.geomspace(floor, 0.5, n_half)
        c = self.t.bw_table_cdf_array(chig, lo)
        xi = np.concatenate([lo, 1.0 - lo[-2::-1]])
        cdf = np.concatenate([c, 1.0 - c[-2::-1]])
        return xi, cdf, float(self.t.rates(1, np.array([chig]), np.array([g]))[0])


# ----------------------------------------------------------------------------
# the generator
# ----------------------------------------------------------------------------
def build_generator(chi_lepton, chi_photon, leptons: LogBins, photons: LogBins, model=None):
    """A for the state [primary leptons (n+1), photons (m+1), secondary leptons
    (n+1)], the +1 being each population's underflow bin (absorbing).
    chi_lepton(gamma), chi_photon(g): the fields' chi as a function of energy;
    model: ExactModel() (default) or TableModel(tables)."""
    model = model or ExactModel()
    n, m = leptons.n, photons.n
    P0, G0, S0 = 0, n + 1, n + 1 + m + 1
    N = S0 + n + 1
    A = np.zeros((N, N))
    for j in range(n):
        K = leptons.centres[j]
        gamma = 1.0 + K
        chi = chi_lepton(gamma)
        if not chi > 0.0:
            continue
        xi, cdf, W = model.qs(chi, gamma)
        if not W > 0.0:
            continue
        xm, dm = _mid(xi), _masses(cdf)
        # below the first grid point (the xi^(1/3) tail): no visible change;
        # above the last (xi -> 1): the lepton keeps nothing, the photon all
        lead, top = cdf[0], 1.0 - cdf[-1]
        lep = leptons.share(math.log(K) + np.log1p(-xm), dm)
        lep[j] += lead
        lep[n] += top
        pho = photons.share(math.log(K) + np.log(xm), dm)
        pho[m] += lead
        pho += photons.share(np.array([math.log(K)]), np.array([top]))
        for base in (P0, S0):
            col = base + j
            A[base:base + n + 1, col] += W * lep
            A[col, col] -= W
            A[G0:G0 + m + 1, col] += W * pho
    for k in range(m):
        g = photons.centres[k]
        if g <= 2.0:
            continue
        chig = chi_photon(g)
        if not chig > 0.0:
            continue
        xi, cdf, W = model.bw(chig, g)
        if not W > 0.0:
            continue
        xm, dm = _mid(xi), _masses(cdf)
        lep = leptons.share(math.log(g - 2.0) + np.log(xm), dm)
        lep[n] += cdf[0]
        lep += leptons.share(np.array([math.log(g - 2.0)]), np.array([1.0 - cdf[-1]]))
        col = G0 + k
        A[col, col] -= W
        A[S0:S0 + n + 1, col] += 2.0 * W * lep
    return A


def solve(A: np.ndarray, f0: np.ndarray, t: float) -> np.ndarray:
    """f(t) = exp(A t) f0."""
    from scipy.sparse.linalg import expm_multiply
    return expm_multiply(A * t, f0)


def spectra(chi_lepton, chi_photon, gamma0: float, t: float, n_lepton: int = 500, n_photon: int = 500,
            lepton_floor: float = 1e-2, photon_floor: float = 1e-3, model=None):
    """Energy distributions at time t of one primary lepton started at gamma0,
    of the photons it and its descendants made (alive, i.e. not decayed), and
    of the secondary leptons; per primary.  Returns a dict of bin centres,
    edges (kinetic energy for leptons, energy for photons) and densities, the
    last entry of each density being its underflow bin."""
    lep = LogBins(gamma0 - 1.0, lepton_floor, n_lepton)
    pho = LogBins(gamma0 - 1.0, photon_floor, n_photon)
    A = build_generator(chi_lepton, chi_photon, lep, pho, model)
    f0 = np.zeros(A.shape[0])
    f0[n_lepton - 1] = 1.0  # the top lepton bin's centre is gamma0 - 1
    f = solve(A, f0, t)
    n, m = n_lepton, n_photon
    return {"lepton_centres": lep.centres, "lepton_edges": lep.edges, "photon_centres": pho.centres,
            "photon_edges": pho.edges, "primary": f[:n + 1], "photons": f[n + 1:n + 1 + m + 1],
            "secondary": f[n + 1 + m + 1:], "generator": A}
