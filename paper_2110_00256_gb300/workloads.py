"""Seeded synthetic inputs with the shapes and distributions of the paper's
workloads.  This module holds no arithmetic of the QED method: it only draws
particle states (momenta, fields, optical depths, ids); both the GPU path and
the oracle consume what it produces.

Units: momentum in m_e c, E in the Schwinger field E_s, B in E_s / c.

* ``paper_benchmark`` -- §4 benchmark particles: every component of E uniform
  in [-E_s/100, E_s/100], of B in [-E_s/(100c), E_s/(100c)], of p in
  [-1, 1] GeV/c; optical depth exponential (mean 1); weight 1.
* ``isotropic_beam`` -- electrons with gamma log-uniform in [1e2, 1e4], isotropic
  directions, in a static B = 0.01 E_s/c along z (the 10^4-electron FP64 case).
* ``gaussian_fields`` -- p as in the benchmark, E and B components N(0, 1) and a
  log-uniform target chi per particle; the caller rescales E and B (chi is
  homogeneous of degree one in the fields).
"""
from __future__ import annotations

import numpy as np

# 1 GeV/c in units of m_e c (m_e c^2 = 0.51099895000 MeV, CODATA 2018)
GEV_IN_MEC = 1.0e3 / 0.51099895000


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def paper_benchmark(n: int, seed: int, id_offset: int = 0, dtype=np.float64) -> dict:
    """§4 benchmark distribution (numpy, host)."""
    r = _rng(seed)
    d = {}
    for k in ("px", "py", "pz"):
        d[k] = r.uniform(-GEV_IN_MEC, GEV_IN_MEC, n).astype(dtype)
    for k in ("ex", "ey", "ez", "bx", "by", "bz"):
        d[k] = r.uniform(-0.01, 0.01, n).astype(dtype)
    d["tau"] = r.exponential(1.0, n).astype(dtype)
    d["tau_c"] = np.zeros(n, dtype=dtype)
    d["weight"] = np.ones(n, dtype=dtype)
    d["id"] = np.arange(id_offset, id_offset + n, dtype=np.uint64)
    return d


def paper_benchmark_torch(n: int, seed: int, id_offset: int = 0, dtype=None, device="cuda") -> dict:
    """Same distribution drawn on the device with a seeded torch generator
    (for the 10^8-particle workloads)."""
    import torch
    dtype = dtype or torch.float32
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    d = {}
    for k, s in (("px", GEV_IN_MEC), ("py", GEV_IN_MEC), ("pz", GEV_IN_MEC), ("ex", 0.01), ("ey", 0.01),
                 ("ez", 0.01), ("bx", 0.01), ("by", 0.01), ("bz", 0.01)):
        d[k] = (torch.rand(n, generator=g, device=device, dtype=torch.float64) * 2.0 - 1.0).mul_(s).to(dtype)
    d["tau"] = torch.empty(n, device=device, dtype=torch.float64).exponential_(1.0, generator=g).to(dtype)
    d["tau_c"] = torch.zeros(n, device=device, dtype=dtype)
    d["weight"] = torch.ones(n, device=device, dtype=dtype)
    d["id"] = torch.arange(id_offset, id_offset + n, device=device, dtype=torch.int64)
    return d


def isotropic_beam(n: int, seed: int, b_z: float = 0.01, id_offset: int = 0) -> dict:
    """Electrons, gamma = 10^(2 + 2U), isotropic direction, E = 0, B = (0, 0, b_z)."""
    r = _rng(seed)
    gamma = 10.0 ** (2.0 + 2.0 * r.uniform(0.0, 1.0, n))
    cth = 2.0 * r.uniform(0.0, 1.0, n) - 1.0
    phi = 2.0 * np.pi * r.uniform(0.0, 1.0, n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    pm = np.sqrt(gamma * gamma - 1.0)
    z = np.zeros(n)
    return dict(px=pm * sth * np.cos(phi), py=pm * sth * np.sin(phi), pz=pm * cth, ex=z.copy(),
                ey=z.copy(), ez=z.copy(), bx=z.copy(), by=z.copy(), bz=np.full(n, b_z),
                tau=r.exponential(1.0, n), tau_c=z.copy(), weight=np.ones(n),
                id=np.arange(id_offset, id_offset + n, dtype=np.uint64))


def gaussian_fields(n: int, seed: int, chi_lo: float = 1e-3, chi_hi: float = 1e2, id_offset: int = 0) -> dict:
    """Benchmark momenta, N(0,1) field components, and a log-uniform target chi."""
    r = _rng(seed)
    d = {k: r.uniform(-GEV_IN_MEC, GEV_IN_MEC, n) for k in ("px", "py", "pz")}
    for k in ("ex", "ey", "ez", "bx", "by", "bz"):
        d[k] = r.normal(0.0, 1.0, n)
    d["chi_target"] = 10.0 ** r.uniform(np.log10(chi_lo), np.log10(chi_hi), n)
    d["tau"] = r.exponential(1.0, n)
    d["tau_c"] = np.zeros(n)
    d["weight"] = np.ones(n)
    d["id"] = np.arange(id_offset, id_offset + n, dtype=np.uint64)
    return d


def rescale_fields(d: dict, chi_now: np.ndarray) -> dict:
    """Scale E and B by chi_target / chi_now (chi is linear in the fields)."""
    s = np.where(chi_now > 0, d["chi_target"] / np.where(chi_now > 0, chi_now, 1.0), 0.0)
    out = dict(d)
    for k in ("ex", "ey", "ez", "bx", "by", "bz"):
        out[k] = d[k] * s
    return out


def patch_counts(n_patches: int = 64, seed: int = 7, lo_exp: float = 3.0, hi_exp: float = 7.0) -> np.ndarray:
    """Patch sizes round(10^(3 + 4U)) for the batched-launch workload."""
    r = _rng(seed)
    return np.round(10.0 ** (lo_exp + (hi_exp - lo_exp) * r.uniform(0.0, 1.0, n_patches))).astype(np.int64)


def subsample_ids(n: int, m: int, seed: int) -> np.ndarray:
    """m distinct sorted indices in [0, n)."""
    r = _rng(seed)
    return np.sort(r.choice(n, size=min(m, n), replace=False))
