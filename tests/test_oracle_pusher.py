"""Pins of the reference particle push (oracle/pusher.py) against exact
solutions: uniform E (momentum grows as q E t), uniform B (|p| conserved, the
gyration period 2 pi gamma / (|q| B)), and a plane wave (the light-front
momentum gamma - d p_x and the transverse canonical momentum p_y + q A_y are
conserved)."""
import math

import numpy as np
import pytest

from oracle import pusher


def test_uniform_electric_field_exact():
    p = np.zeros((1, 3))
    E = np.array([[0.0, 0.3, 0.0]])
    B = np.zeros((1, 3))
    for _ in range(100):
        p = pusher.boris(p, E, B, -1.0, 0.01)
    assert p[0, 1] == pytest.approx(-0.3 * 1.0, rel=1e-13)


def test_uniform_magnetic_field_rotation():
    p0 = np.array([[3.0, 0.0, 0.5]])
    B = np.array([[0.0, 0.0, 0.2]])
    E = np.zeros((1, 3))
    gamma = math.sqrt(1 + np.sum(p0 ** 2))
    period = 2 * math.pi * gamma / 0.2
    n = 2000
    dt = period / n
    p = p0.copy()
    for _ in range(n):
        p = pusher.boris(p, E, B, 1.0, dt)
        assert np.linalg.norm(p) == pytest.approx(np.linalg.norm(p0), rel=1e-13)
    # back where it started after one period, up to the O(dt^2) phase error
    assert np.allclose(p, p0, atol=3e-4 * np.linalg.norm(p0))


@pytest.mark.parametrize("circular", [False, True])
def test_plane_wave_invariants(circular):
    e0, omega = 3e-4, 3.0e-6
    period = 2 * math.pi / omega
    n = 400
    dt = period / n
    pos = np.array([[0.0, 0.0, 0.0]])
    p = np.array([[2000.0, 0.0, 0.0]])  # counter-propagating with the wave along -x
    q = -1.0
    g0 = math.sqrt(1 + np.sum(p ** 2))
    lf0 = g0 + p[0, 0]  # gamma - d p_x with d = -1
    t = 0.0
    for _ in range(n):
        E, B, p, pos = pusher.push(pos, p, q, t, dt, e0, omega, circular=circular)
        t += dt
    g = math.sqrt(1 + np.sum(p ** 2))
    assert (g + p[0, 0]) == pytest.approx(lf0, rel=1e-4)
    # transverse canonical momentum: p_y + q A_y with E_y = -dA_y/dt, A_y = -(E0/omega) sin(phi)
    phi = omega * (t - dt / 2 + pos[0, 0])  # momentum is at the half step
    assert abs(p[0, 1] + q * (-(e0 / omega) * math.sin(phi))) < 2e-2 * (e0 / omega)
