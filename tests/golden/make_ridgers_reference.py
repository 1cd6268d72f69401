"""Writes tests/golden/ridgers_kinetic.json: the kinetic-equation spectra
(oracle/kinetic.py) of the three test cases of Ridgers et al. (2014) that §5
of the paper reproduces, coarse-grained to 50 log bins per population, for the
exact rates and spectra ("exact") and for what the method samples with the
paper's 256 / 256x256 tables ("tables_256", the oracle's tables).  Calls only
the oracle; run from the repository root:

    python tests/golden/make_ridgers_reference.py

The cases (energies in m_e c^2, fields in E_s and E_s/c, time in
hbar/(m_e c^2)) and the chi of a particle of energy gamma (lepton) or g
(photon) in each field, both moving across it (a particle moving
perpendicular to a static B keeps doing so) or head-on (a circularly polarised
plane wave: chi = E0 (gamma - n.p), n.p = -|p|):
  1: gamma0 = 1000, B0 = 1e-3, 1 fs;   chi_e = |p| B0,        chi_g = g B0
  2: gamma0 = 4120, E0 = 1.22e-4, 3 fs; chi_e = (gamma + |p|) E0, chi_g = 2 g E0
  3: gamma0 = 1000, B0 = 9e-3, 0.1 fs; as case 1
"""
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from oracle import kinetic  # noqa: E402

T_C = 1.28808866712e-21  # hbar / (m_e c^2) in s (CODATA 2018)
FINE = 500
GROUP = 10


def chi_functions(case):
    if case in (1, 3):
        b0 = 1e-3 if case == 1 else 9e-3
        return (lambda g: math.sqrt(g * g - 1.0) * b0), (lambda g: g * b0)
    e0 = 1.22e-4
    return (lambda g: (g + math.sqrt(g * g - 1.0)) * e0), (lambda g: 2.0 * g * e0)


CASES = {1: (1000.0, 1.0), 2: (4120.0, 3.0), 3: (1000.0, 0.1)}


def coarse(dens):
    """fine densities (FINE bins + underflow) -> GROUP-bin sums + underflow"""
    d = np.asarray(dens[:FINE])
    return [float(v) for v in d.reshape(-1, GROUP).sum(1)] + [float(dens[FINE])]


def main():
    out = {"source": "oracle/kinetic.py (kinetic equation of emission and pair production, exact G and T); "
                     "the three cases of Ridgers et al., J. Comput. Phys. 260, 273 (2014), as listed in §5 of "
                     "arXiv 2110.00256",
           "units": "lepton bins: kinetic energy gamma - 1; photon bins: energy; densities per primary electron; "
                    "last entry of each density: everything below the lowest edge",
           "fine_bins": FINE, "group": GROUP, "cases": {}}
    models = {"exact": kinetic.ExactModel(), "tables_256": kinetic.TableModel(oracle.tables())}
    for case, (g0, fs) in CASES.items():
        chi_l, chi_g = chi_functions(case)
        t = fs * 1e-15 / T_C
        entry = {"gamma0": g0, "fs": fs, "t": t}
        for name, model in models.items():
            r = kinetic.spectra(chi_l, chi_g, g0, t, n_lepton=FINE, n_photon=FINE, model=model)
            entry["lepton_edges"] = [float(v) for v in r["lepton_edges"][::GROUP]]
            entry["photon_edges"] = [float(v) for v in r["photon_edges"][::GROUP]]
            entry[name] = {"primary": coarse(r["primary"]), "photons": coarse(r["photons"]),
                           "secondary": coarse(r["secondary"]),
                           "mean_gamma_primary": float(np.sum(r["primary"][:FINE] * (1.0 + r["lepton_centres"])))}
        out["cases"][str(case)] = entry
        print(case, "done", flush=True)
    with open(os.path.join(HERE, "ridgers_kinetic.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
