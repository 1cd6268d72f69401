"""Unit systems of the boundary (§3.3), no GPU needed: the library's field
unit is the Schwinger field the paper prints (§2, ~1.32e18 V/m); a reference-
frequency normalisation gives the familiar a0 = 1 field at 0.8 um and the
identity E0/E_s = a0 hbar omega / (m_e c^2) that the cascade workload uses;
Heaviside-Lorentz with 1 MeV gives E_s = m_e^2 / q_e in MeV^2; conversions
compose."""
import math

import pytest


@pytest.fixture(scope="module")
def units():
    from paper_2110_00256_gb300 import build, units as u
    build.build()
    return u


def test_library_units_are_the_schwinger_system(units):
    lib = units.library()
    assert lib["e_field"] == pytest.approx(1.32e18, rel=5e-3)          # §2 prints E_s ~ 1.32e18 V/m
    assert lib["e_field"] == pytest.approx(1.32328e18, rel=1e-5)
    assert lib["b_field"] == pytest.approx(lib["e_field"] / 299792458.0, rel=1e-15)
    assert lib["time"] == pytest.approx(1.28808866712e-21, rel=1e-9)    # hbar / (m_e c^2)
    assert lib["length"] == pytest.approx(3.8615926796e-13, rel=1e-9)   # reduced Compton wavelength
    assert lib["energy"] == pytest.approx(0.51099895e6 * 1.602176634e-19, rel=1e-9)
    assert lib["length"] / lib["time"] == pytest.approx(299792458.0, rel=1e-15)


def test_reference_frequency_normalisation(units):
    lam = 0.8e-6
    ref = units.reference_length(lam)
    omega = 2 * math.pi * 299792458.0 / lam
    assert ref == units.reference_frequency(omega)
    assert ref["e_field"] == pytest.approx(4.013e12, rel=1e-3)          # a0 = 1 at 0.8 um
    lib = units.library()
    hbar_omega = units.factor("energy", {"energy": 1.054571817e-34 * omega}, lib)
    # a field of amplitude a0 in PIC units is a0 hbar omega / (m_e c^2) in units of E_s
    assert units.factor("e_field", ref, lib) == pytest.approx(hbar_omega, rel=1e-12)
    assert hbar_omega == pytest.approx(3.0328877982211224e-6, rel=1e-6)  # the cascade workload's omega at 0.8 um
    assert units.factor("time", ref, lib) * units.factor("time", lib, ref) == pytest.approx(1.0, rel=1e-15)


def test_heaviside_lorentz_mev(units):
    hl, lib = units.heaviside_lorentz_mev(), units.library()
    me = 0.51099895  # MeV
    q = math.sqrt(4 * math.pi * 7.2973525693e-3)
    assert units.factor("e_field", lib, hl) == pytest.approx(me * me / q, rel=1e-8)   # E_s = m_e^2 / q_e
    assert units.factor("energy", lib, hl) == pytest.approx(me, rel=1e-9)
    assert hl["length"] == pytest.approx(197.3269804e-15, rel=1e-9)                   # hbar c / MeV
    assert units.factor("momentum", lib, hl) == pytest.approx(me, rel=1e-9)


def test_invalid_arguments(units):
    from paper_2110_00256_gb300._lib import QedError
    with pytest.raises(QedError):
        units.reference_frequency(0.0)
    with pytest.raises(QedError):
        units.reference_length(-1.0)
