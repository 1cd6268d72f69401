"""Unit systems at the boundary (§3.3): the library computes in one normalised
system; a caller working in SI, in a PIC code's reference-frequency or
reference-length normalisation, or in Heaviside-Lorentz natural units with
1 MeV converts with the scales libqed returns (include/qed.h)."""
from __future__ import annotations

import ctypes as C

from ._lib import UnitScales, check, lib

QUANTITIES = ("length", "time", "momentum", "energy", "e_field", "b_field")


def _get(fn, *args) -> dict:
    out = UnitScales()
    check(fn(*args, C.byref(out)))
    return {k: getattr(out, k) for k in QUANTITIES}


def library() -> dict:
    """SI value of one library unit of each quantity."""
    return _get(lib().qed_units_library)


def reference_frequency(omega_r: float) -> dict:
    return _get(lib().qed_units_reference_frequency, float(omega_r))


def reference_length(lambda_r: float) -> dict:
    return _get(lib().qed_units_reference_length, float(lambda_r))


def heaviside_lorentz_mev() -> dict:
    return _get(lib().qed_units_heaviside_lorentz_mev)


def factor(quantity: str, frm: dict, to: dict) -> float:
    """Multiply a value of `quantity` in system `frm` by this to express it in `to`."""
    return frm[quantity] / to[quantity]
