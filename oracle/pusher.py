"""FP64 reference of the particle push used to drive the cascade workload:
analytic plane-wave fields and the relativistic Boris rotation.  The paper's
substep runs inside a PIC code; this minimal pusher (not from the paper) stands
in for it.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Units: c = m_e = 1, momentum in m_e c, fields in E_s and E_s/c, time in
hbar/(m_e c^2), lengths in hbar/(m_e c).  Then dp/dt = q (E + v x B), q = -1
(electron), +1 (positron); photons move along p at speed 1.

Plane wave travelling along direction d x-hat (d = -1 or +1), phase
phi = omega (t - d x) + phase0:
  linear:   E = E0 (0, cos phi, 0)
  circular: E = E0 (0, cos phi, sin phi)
and B = d x-hat cross E.

Step (time-centred, positions at t_n, momenta at t_{n+1/2}): fields at (x_n, t_n);
p <- Boris(p, E, B, q, dt); x_{n+1} = x_n + v dt with v = p / gamma (leptons)
or p / |p| (photons).  Boris (J. P. Boris, 1970): half electric kick, magnetic
rotation with t = q B dt / (2 gamma), s = 2 t / (1 + t.t), half electric kick.
"""
from __future__ import annotations

import numpy as np


def plane_wave(x, t, e0, omega, phase0=0.0, circular=False, direction=-1):
    x = np.asarray(x, dtype=np.float64)
    phi = omega * (t - direction * x) + phase0
    z = np.zeros_like(phi)
    E = np.stack([z, e0 * np.cos(phi), e0 * np.sin(phi) if circular else z], axis=-1)
    d = np.array([float(direction), 0.0, 0.0])
    B = np.cross(np.broadcast_to(d, E.shape), E)
    return E, B


def boris(p, E, B, q, dt):
    p = np.asarray(p, dtype=np.float64)
    pm = p + 0.5 * q * dt * E
    g = np.sqrt(1.0 + np.sum(pm * pm, axis=-1, keepdims=True))
    tv = 0.5 * q * dt * B / g
    s = 2.0 * tv / (1.0 + np.sum(tv * tv, axis=-1, keepdims=True))
    pp = pm + np.cross(pm, tv)
    return pm + np.cross(pp, s) + 0.5 * q * dt * E


def push(pos, p, q, t, dt, e0, omega, phase0=0.0, circular=False, direction=-1):
    """One step for particles at positions pos (n, 3) with momenta p (n, 3).
    Returns (E, B) used, the new momentum and the new position."""
    E, B = plane_wave(pos[:, 0], t, e0, omega, phase0, circular, direction)
    if q == 0:
        pn = np.asarray(p, dtype=np.float64).copy()
        v = pn / np.linalg.norm(pn, axis=-1, keepdims=True)
    else:
        pn = boris(p, E, B, q, dt)
        v = pn / np.sqrt(1.0 + np.sum(pn * pn, axis=-1, keepdims=True))
    return E, B, pn, pos + v * dt
