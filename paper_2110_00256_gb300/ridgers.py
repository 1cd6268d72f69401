"""The three test cases of Ridgers et al. (J. Comput. Phys. 260, 273, 2014) that
§5 of the paper runs to validate the Monte Carlo against the kinetic equations:
a population of electrons, all with the same initial Lorentz factor,
  case 1: gamma0 = 1000 across a static uniform magnetic field B0 = 1e-3 E_s/c
          (chi = 1), for 1 fs;
  case 2: gamma0 = 4120 head-on into a circularly polarised plane wave of
          amplitude E0 = 1.22e-4 E_s (chi = 1), for 3 fs;
  case 3: gamma0 = 1000 across B0 = 9e-3 E_s/c (chi = 9), for 0.1 fs;
and the energy spectra of the electrons, photons and pairs at the end.  The
run uses the library's pushers (stored uniform field / analytic plane wave)
and its full substep (emission, pair production, secondaries) every step.

The paper gives no wavelength for case 2; 1 um is taken.  With circular
polarisation the field strength seen by a head-on electron is constant, so
chi, and with it the spectra, do not depend on that choice.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import api

HBAR_OVER_MC2_S = 1.28808866712e-21  # hbar / (m_e c^2) in s (CODATA 2018)
HBAR_OMEGA_1UM = 1.239841984 / 0.51099895e6  # photon energy at 1 um in m_e c^2

CASES = {
    1: {"gamma0": 1000.0, "b0": 1e-3, "fs": 1.0},
    2: {"gamma0": 4120.0, "e0": 1.22e-4, "fs": 3.0},
    3: {"gamma0": 1000.0, "b0": 9e-3, "fs": 0.1},
}


def duration(case: int) -> float:
    """Run time in hbar / (m_e c^2)."""
    return CASES[case]["fs"] * 1e-15 / HBAR_OVER_MC2_S


def run(tables: api.Tables, case: int, n: int, prec: int, steps: int = 1000, seed: int = 2014,
        photons_per_electron: float = 10.0, stream=None) -> dict:
    """n electrons through `steps` steps of case `case`.  Returns kinetic
    energies (gamma - 1) of the primary electrons (ids 0 .. n-1) and of the
    secondary leptons (pair electrons and positrons), the energies of the
    photons still alive, and the substep statistics."""
    c = CASES[case]
    g0 = c["gamma0"]
    dt = duration(case) / steps
    r = np.random.default_rng(seed)
    e = api.SpeciesBuffers(int(1.5 * n) + 1024, prec, positions=True)
    q = api.SpeciesBuffers(n // 2 + 1024, prec, positions=True)
    g = api.SpeciesBuffers(int(photons_per_electron * n) + 1024, prec, positions=True)
    pm = math.sqrt(g0 * g0 - 1.0)
    zeros = np.zeros(n)
    init = {"py": zeros, "pz": zeros, "y": zeros, "z": zeros, "ex": zeros, "ey": zeros, "ez": zeros,
            "bx": zeros, "by": zeros, "weight": np.ones(n), "id": np.arange(n, dtype=np.uint64), "tau": zeros}
    if "b0" in c:  # across B = B0 z-hat
        init.update(px=np.full(n, pm), x=zeros, bz=np.full(n, c["b0"]))
        wave = None
    else:  # head-on: the wave travels along +x, the electrons along -x
        omega = HBAR_OMEGA_1UM
        init.update(px=np.full(n, -pm), x=r.uniform(0.0, 2.0 * math.pi / omega, n), bz=zeros)
        wave = api.plane_wave(c["e0"], omega, 0.0, circular=True, direction=1)
    e.set(init)
    api.qed_init_optical_depth(e, seed, 0, stream=stream)
    fire = [api.FireBuffers(b.capacity) for b in (e, q, g)]
    stats = api.Stats()
    call = api.SubstepCall(tables, e, q, g, fire, dt, seed, stats=stats)
    for k in range(steps):
        t = k * dt
        for sp, charge in ((e, -1.0), (q, 1.0), (g, 0.0)):
            if wave is None:
                api.qed_push_stored_fields(sp, charge, dt, stream=stream)
            else:
                api.qed_push_plane_wave(sp, charge, wave, t, dt, stream=stream)
        call(k, stream)
    torch.cuda.synchronize()
    he, hq, hg = e.to_host(), q.to_host(), g.to_host()

    def kinetic(h):
        p2 = h["px"].astype(np.float64) ** 2 + h["py"].astype(np.float64) ** 2 + h["pz"].astype(np.float64) ** 2
        return p2 / (np.sqrt(1.0 + p2) + 1.0)  # gamma - 1 without cancellation

    live_e = he["weight"] > 0
    prim = live_e & (he["id"] < n)
    sec_e = live_e & (he["id"] >= n)
    live_q = hq["weight"] > 0
    alive = hg["weight"] > 0
    gp = np.sqrt(hg["px"].astype(np.float64) ** 2 + hg["py"].astype(np.float64) ** 2
                 + hg["pz"].astype(np.float64) ** 2)
    return {"primary": kinetic({k: v[prim] for k, v in he.items()}),
            "secondary": np.concatenate([kinetic({k: v[sec_e] for k, v in he.items()}),
                                         kinetic({k: v[live_q] for k, v in hq.items()})]),
            "photons": gp[alive], "stats": stats.as_dict(), "n": n, "dt": dt, "steps": steps}
