"""FP64 CPU oracle of the strong-field QED Monte Carlo substep (PICSAR-QED,
Fedeli et al., arXiv 2110.00256, §2-§3, §5).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the GPU path (``paper_2110_00256_gb300``) and
imports nothing from it; the GPU path never imports it.

The numerics live in plain C (``oracle/*.c``), compiled with gcc into
``oracle/_build/liboracle.so``; this module only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["quad_bessel.c", "rates_tables.c", "substep.c", "schwinger.c"]
_lock = threading.Lock()
_lib = None

ALPHA_F = 7.2973525693e-3  # CODATA 2018; the paper prints no value


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no fast-math, OpenMP over rows/particles)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    hdr = os.path.join(_HERE, "qed_oracle.h")
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr])
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-ffp-contract=off", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Tables(C.Structure):
    _fields_ = [
        ("qs_chi_min", C.c_double), ("qs_chi_max", C.c_double), ("qs_xi_min", C.c_double),
        ("qs_n_chi", C.c_int32), ("qs_n_xi", C.c_int32),
        ("bw_chi_min", C.c_double), ("bw_chi_max", C.c_double),
        ("bw_n_chi", C.c_int32), ("bw_n_xi", C.c_int32),
        ("qs_lnG", C.c_void_p), ("qs_lnP", C.c_void_p),
        ("bw_lnT", C.c_void_p), ("bw_P", C.c_void_p),
    ]


class Fields(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("px", "py", "pz", "ex", "ey", "ez", "bx", "by", "bz")]


_D = C.c_double
_P = C.c_void_p
_I64 = C.c_int64
_U64 = C.c_uint64


def lib():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        L = C.CDLL(build())
        sig = {
            "oracle_bessel_k": (_D, [_D, _D]),
            "oracle_bessel_kint": (_D, [_D, _D]),
            "oracle_bessel_k_scaled": (_D, [_D, _D]),
            "oracle_bessel_kint_scaled": (_D, [_D, _D]),
            "oracle_chi_lepton": (_D, [_D] * 9),
            "oracle_chi_photon": (_D, [_D] * 9),
            "oracle_qs_S": (_D, [_D, _D]),
            "oracle_bw_bracket": (_D, [_D, _D]),
            "oracle_bw_F": (_D, [_D, _D]),
            "oracle_qs_row": (_D, [_D, C.c_int, _D, _P]),
            "oracle_bw_row": (_D, [_D, C.c_int, _P]),
            "oracle_qs_G": (_D, [_D]),
            "oracle_bw_T": (_D, [_D]),
            "oracle_bw_upper_half": (_D, [_D]),
            "oracle_qs_cdf": (_D, [_D, _D]),
            "oracle_bw_cdf": (_D, [_D, _D]),
            "oracle_qs_cdf_sorted": (None, [_D, _I64, _P, _P]),
            "oracle_qs_S_array": (None, [_D, _I64, _P, _P]),
            "oracle_schwinger_rate": (_D, [_D, _D, _D, _D, _D, _D]),
            "oracle_poisson": (_I64, [_D, _U64, _U64, _I64]),
            "oracle_schwinger_pair_ids": (None, [_U64, _U64, _I64, _I64, _P]),
            "oracle_schwinger_cells": (None, [_I64, _P, _P, _P, _P, _P, _P, _D, _D, _D, _U64, _I64, _P, _P]),
            "oracle_bw_bracket_array": (None, [_D, _I64, _P, _P]),
            "oracle_bw_cdf_sorted": (None, [_D, _I64, _P, _P]),
            "oracle_build_qs_tables": (None, [_D, _D, C.c_int, C.c_int, _D, _P, _P]),
            "oracle_build_bw_tables": (None, [_D, _D, C.c_int, C.c_int, _P, _P]),
            "oracle_philox4x32_10": (None, [_P, _P, _P]),
            "oracle_uniform": (_D, [_U64, _U64, _I64, C.c_uint32, C.c_int]),
            "oracle_tau_draw": (_D, [_U64, _U64, _I64, C.c_uint32]),
            "oracle_child_ids": (None, [_U64, _U64, _I64, _P]),
            "oracle_qs_G_table": (_D, [C.POINTER(Tables), _D]),
            "oracle_bw_T_table": (_D, [C.POINTER(Tables), _D]),
            "oracle_bw_T_small": (_D, [_D]),
            "oracle_bw_T_large": (_D, [_D]),
            "oracle_qs_rate": (_D, [C.POINTER(Tables), _D, _D]),
            "oracle_bw_rate": (_D, [C.POINTER(Tables), _D, _D]),
            "oracle_qs_sample_xi": (_D, [C.POINTER(Tables), _D, _D]),
            "oracle_bw_sample_xi": (_D, [C.POINTER(Tables), _D, _D, C.POINTER(C.c_int)]),
            "oracle_evolve": (None, [C.c_int, C.POINTER(Tables), _I64, C.POINTER(Fields), _P, _D,
                                     _P, _P, _P, _P]),
            "oracle_qs_events": (None, [C.POINTER(Tables), _I64] + [_P] * 5 + [_U64, _I64, _D]
                                 + [_P] * 10),
            "oracle_bw_events": (None, [C.POINTER(Tables), _I64] + [_P] * 5 + [_U64, _I64]
                                 + [_P] * 11),
            "oracle_init_tau": (None, [_I64, _P, _U64, _I64, _P]),
            "oracle_rates": (None, [C.c_int, C.POINTER(Tables), _I64, _P, _P, _P]),
            "oracle_qs_table_cdf": (_D, [C.POINTER(Tables), _D, _D]),
            "oracle_bw_table_cdf": (_D, [C.POINTER(Tables), _D, _D]),
            "oracle_qs_table_cdf_array": (None, [C.POINTER(Tables), _D, _I64, _P, _P]),
            "oracle_bw_table_cdf_array": (None, [C.POINTER(Tables), _D, _I64, _P, _P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ----------------------------------------------------------------------------------------
# special functions and rates (§2)
# ----------------------------------------------------------------------------------------
def bessel_k(nu: float, x: float) -> float:
    """K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt."""
    return lib().oracle_bessel_k(nu, x)


def bessel_kint(nu: float, x: float) -> float:
    """int_x^inf K_nu(s) ds."""
    return lib().oracle_bessel_kint(nu, x)


def chi_lepton(p, E, B) -> float:
    """Quantum parameter of a lepton (§2, definition of chi)."""
    return lib().oracle_chi_lepton(*map(float, (*p, *E, *B)))


def chi_photon(p, E, B) -> float:
    """Quantum parameter of a photon (§2, definition of chi_gamma)."""
    return lib().oracle_chi_photon(*map(float, (*p, *E, *B)))


def qs_S(chi: float, xi: float) -> float:
    """S(chi, xi) of Eq. (qs_diff_cross)."""
    return lib().oracle_qs_S(chi, xi)


def bw_F(chig: float, chim: float) -> float:
    """F(chi_gamma, chi_-) of Eq. (bw_cross_diff)."""
    return lib().oracle_bw_F(chig, chim)


def bw_bracket(chig: float, xi: float) -> float:
    return lib().oracle_bw_bracket(chig, xi)


def qs_G(chi: float) -> float:
    """G(chi) of Eq. (qs_g_func) by quadrature."""
    return lib().oracle_qs_G(chi)


def bw_T(chig: float) -> float:
    """T(chi_gamma) of Eq. (t_func_0) by quadrature."""
    return lib().oracle_bw_T(chig)


def bw_upper_half(chig: float) -> float:
    return lib().oracle_bw_upper_half(chig)


def qs_row(chi: float, n_xi: int, xi_min: float):
    row = np.zeros(n_xi)
    G = lib().oracle_qs_row(chi, n_xi, xi_min, _ptr(row))
    return G, row


def bw_row(chig: float, n_xi: int):
    row = np.zeros(n_xi)
    T = lib().oracle_bw_row(chig, n_xi, _ptr(row))
    return T, row


def qs_cdf(chi: float, xi: float) -> float:
    """Exact QS cumulative distribution (number spectrum reading of Eq. (qs_prob_dist))."""
    return lib().oracle_qs_cdf(chi, xi)


def bw_cdf(chig: float, xi: float) -> float:
    """Exact BW cumulative distribution of Eq. (bw_prob_dist), xi = chi_-/chi_gamma."""
    return lib().oracle_bw_cdf(chig, xi)


def qs_cdf_sorted(chi: float, xs) -> np.ndarray:
    """Exact QS cumulative distribution at ascending points xs (one pass)."""
    xs = _f64(xs)
    assert np.all(np.diff(xs) >= 0)
    out = np.zeros(xs.shape[0])
    lib().oracle_qs_cdf_sorted(chi, xs.shape[0], _ptr(xs), _ptr(out))
    return out


def bw_cdf_sorted(chig: float, xs) -> np.ndarray:
    """Exact BW cumulative distribution at ascending points xs in [0, 1] (one pass)."""
    xs = _f64(xs)
    assert np.all(np.diff(xs) >= 0)
    out = np.zeros(xs.shape[0])
    lib().oracle_bw_cdf_sorted(chig, xs.shape[0], _ptr(xs), _ptr(out))
    return out


def qs_S_array(chi: float, xs) -> np.ndarray:
    """S(chi, xi) of Eq. (qs_diff_cross) at every point of xs."""
    xs = _f64(xs)
    out = np.zeros(xs.shape[0])
    lib().oracle_qs_S_array(chi, xs.shape[0], _ptr(xs), _ptr(out))
    return out


def bw_bracket_array(chig: float, xs) -> np.ndarray:
    """The bracket of Eq. (t_func_0) at every point of xs (xi = chi_-/chi_gamma)."""
    xs = _f64(xs)
    out = np.zeros(xs.shape[0])
    lib().oracle_bw_bracket_array(chig, xs.shape[0], _ptr(xs), _ptr(out))
    return out


def bw_T_small(chig: float) -> float:
    return lib().oracle_bw_T_small(chig)


def bw_T_large(chig: float) -> float:
    return lib().oracle_bw_T_large(chig)


# ----------------------------------------------------------------------------------------
# tables (§3.1, §3.2)
# ----------------------------------------------------------------------------------------
class OracleTables:
    """The four lookup tables, FP64, built by the oracle's quadrature."""

    def __init__(self, qs_chi_min, qs_chi_max, qs_n_chi, qs_n_xi, qs_xi_min,
                 bw_chi_min, bw_chi_max, bw_n_chi, bw_n_xi):
        self.params = dict(qs_chi_min=float(qs_chi_min), qs_chi_max=float(qs_chi_max),
                           qs_n_chi=int(qs_n_chi), qs_n_xi=int(qs_n_xi), qs_xi_min=float(qs_xi_min),
                           bw_chi_min=float(bw_chi_min), bw_chi_max=float(bw_chi_max),
                           bw_n_chi=int(bw_n_chi), bw_n_xi=int(bw_n_xi))
        self.qs_lnG = np.zeros(qs_n_chi)
        self.qs_lnP = np.zeros((qs_n_chi, qs_n_xi))
        self.bw_lnT = np.zeros(bw_n_chi)
        self.bw_P = np.zeros((bw_n_chi, bw_n_xi))
        self._struct = None

    def build(self):
        p = self.params
        L = lib()
        L.oracle_build_qs_tables(p["qs_chi_min"], p["qs_chi_max"], p["qs_n_chi"], p["qs_n_xi"],
                                 p["qs_xi_min"], _ptr(self.qs_lnG), _ptr(self.qs_lnP))
        L.oracle_build_bw_tables(p["bw_chi_min"], p["bw_chi_max"], p["bw_n_chi"], p["bw_n_xi"],
                                 _ptr(self.bw_lnT), _ptr(self.bw_P))
        return self

    @property
    def struct(self) -> Tables:
        if self._struct is None:
            p = self.params
            self._struct = Tables(p["qs_chi_min"], p["qs_chi_max"], p["qs_xi_min"], p["qs_n_chi"],
                                  p["qs_n_xi"], p["bw_chi_min"], p["bw_chi_max"], p["bw_n_chi"],
                                  p["bw_n_xi"], _ptr(self.qs_lnG).value, _ptr(self.qs_lnP).value,
                                  _ptr(self.bw_lnT).value, _ptr(self.bw_P).value)
        return self._struct

    def save(self, path):
        np.savez(path, **{k: np.asarray(v) for k, v in self.params.items()}, qs_lnG=self.qs_lnG,
                 qs_lnP=self.qs_lnP, bw_lnT=self.bw_lnT, bw_P=self.bw_P)

    @classmethod
    def load(cls, path):
        z = np.load(path)
        t = cls(**{k: z[k].item() for k in ("qs_chi_min", "qs_chi_max", "qs_n_chi", "qs_n_xi",
                                            "qs_xi_min", "bw_chi_min", "bw_chi_max", "bw_n_chi",
                                            "bw_n_xi")})
        t.qs_lnG[:] = z["qs_lnG"]
        t.qs_lnP[:] = z["qs_lnP"]
        t.bw_lnT[:] = z["bw_lnT"]
        t.bw_P[:] = z["bw_P"]
        return t

    # lookups -----------------------------------------------------------------
    def qs_G(self, chi):
        return lib().oracle_qs_G_table(C.byref(self.struct), chi)

    def bw_T(self, chig):
        return lib().oracle_bw_T_table(C.byref(self.struct), chig)

    def rates(self, proc, chi, energy):
        """Vectorised rate lookup; energy is gamma (QS) or |p| (BW)."""
        chi = np.ascontiguousarray(chi, dtype=np.float64)
        energy = np.ascontiguousarray(energy, dtype=np.float64)
        out = np.zeros(chi.shape[0])
        lib().oracle_rates(proc, C.byref(self.struct), chi.shape[0], _ptr(chi), _ptr(energy), _ptr(out))
        return out

    def qs_table_cdf(self, chi, xi):
        """r that the QS table lookup maps to xi (forward map of the sampling)."""
        return lib().oracle_qs_table_cdf(C.byref(self.struct), chi, xi)

    def bw_table_cdf(self, chig, xi):
        """r in [0, 1/2] that the BW table lookup maps to xi in [0, 1/2]."""
        return lib().oracle_bw_table_cdf(C.byref(self.struct), chig, xi)

    def qs_table_cdf_array(self, chi, xs):
        xs = _f64(xs)
        out = np.zeros(xs.shape[0])
        lib().oracle_qs_table_cdf_array(C.byref(self.struct), chi, xs.shape[0], _ptr(xs), _ptr(out))
        return out

    def bw_table_cdf_array(self, chig, xs):
        xs = _f64(xs)
        out = np.zeros(xs.shape[0])
        lib().oracle_bw_table_cdf_array(C.byref(self.struct), chig, xs.shape[0], _ptr(xs), _ptr(out))
        return out

    def qs_sample_xi(self, chi, r):
        return lib().oracle_qs_sample_xi(C.byref(self.struct), chi, r)

    def bw_sample_xi(self, chig, r):
        e = C.c_int(0)
        xi = lib().oracle_bw_sample_xi(C.byref(self.struct), chig, r, C.byref(e))
        return xi, bool(e.value)


_CACHE_DIR = os.path.join(_BUILD, "tables")


def tables(qs_chi_min=1e-3, qs_chi_max=1e3, qs_n_chi=256, qs_n_xi=256, qs_xi_min=1e-12,
           bw_chi_min=2e-2, bw_chi_max=1e3, bw_n_chi=256, bw_n_xi=256, cache=True) -> OracleTables:
    """Oracle tables for the given axes; cached on disk (git-ignored) by parameters,
    since the FP64 quadrature of a 256x256 pair takes tens of seconds."""
    t = OracleTables(qs_chi_min, qs_chi_max, qs_n_chi, qs_n_xi, qs_xi_min,
                     bw_chi_min, bw_chi_max, bw_n_chi, bw_n_xi)
    key = "_".join(f"{t.params[k]!r}" for k in sorted(t.params))
    # (a digest of the parameters: Python's hash() of a string differs from process to process)
    path = os.path.join(_CACHE_DIR, f"t_{hashlib.sha1(key.encode()).hexdigest()[:16]}_{qs_n_chi}x{qs_n_xi}.npz")
    if cache and os.path.exists(path):
        loaded = OracleTables.load(path)
        if loaded.params == t.params:
            return loaded
    t.build()
    if cache:
        os.makedirs(_CACHE_DIR, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}.npz"
        t.save(tmp)
        os.replace(tmp, path)
    return t


# ----------------------------------------------------------------------------------------
# random numbers: Philox4x32-10 (Salmon et al., SC'11)
# ----------------------------------------------------------------------------------------
PURPOSE_SAMPLE, PURPOSE_TAU_RESET, PURPOSE_TAU_INIT, PURPOSE_CHILD_ID = 0, 1, 2, 3


def philox(counter, key):
    ctr = np.asarray(counter, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(ctr), _ptr(k), _ptr(out))
    return out


def uniform(seed, pid, step, purpose, which=0) -> float:
    return lib().oracle_uniform(seed, pid, step, purpose, which)


def tau_draw(seed, pid, step, purpose) -> float:
    return lib().oracle_tau_draw(seed, pid, step, purpose)


def child_ids(seed, parent, step):
    out = np.zeros(2, dtype=np.uint64)
    lib().oracle_child_ids(seed, parent, step, _ptr(out))
    return int(out[0]), int(out[1])


def init_tau(ids: np.ndarray, seed: int, step: int) -> np.ndarray:
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    out = np.zeros(ids.shape[0])
    lib().oracle_init_tau(ids.shape[0], _ptr(ids), seed, step, _ptr(out))
    return out


# ----------------------------------------------------------------------------------------
# the substep (§3, §5)
# ----------------------------------------------------------------------------------------
QS, BW = 0, 1
_FIELD_NAMES = ("px", "py", "pz", "ex", "ey", "ez", "bx", "by", "bz")


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def evolve(proc: int, t: OracleTables, state: dict, dt: float, chi_cut: float = 0.0):
    """Optical-depth evolution of every particle in ``state`` (dict of arrays).
    Particles with chi < chi_cut (a cut-off applied by PIC codes, §5) take no
    part: rate zero, optical depth unchanged, no event.  Returns (tau_new, chi,
    rate, fire)."""
    arrs = {k: _f64(state[k]) for k in _FIELD_NAMES}
    tau = _f64(state["tau"])
    n = tau.shape[0]
    f = Fields(*[_ptr(arrs[k]).value for k in _FIELD_NAMES])
    tau_out, chi, rate = np.zeros(n), np.zeros(n), np.zeros(n)
    fire = np.zeros(n, dtype=np.uint8)
    lib().oracle_evolve(proc, C.byref(t.struct), n, C.byref(f), _ptr(tau), dt, _ptr(tau_out),
                        _ptr(chi), _ptr(rate), _ptr(fire))
    fire = fire.astype(bool)
    below = chi < chi_cut
    tau_out[below], rate[below], fire[below] = tau[below], 0.0, False
    return tau_out, chi, rate, fire


def qs_events(t: OracleTables, p: np.ndarray, chi: np.ndarray, ids: np.ndarray, seed: int,
              step: int, threshold: float = 0.0) -> dict:
    """Photon emission for the firing leptons; p is (m, 3)."""
    m = chi.shape[0]
    px, py, pz = (_f64(p[:, i]) for i in range(3))
    chi = _f64(chi)
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    out = {k: np.zeros(m) for k in ("xi", "lep_px", "lep_py", "lep_pz", "lep_tau", "ph_px",
                                    "ph_py", "ph_pz", "ph_tau")}
    out["ph_id"] = np.zeros(m, dtype=np.uint64)
    out["keep"] = np.zeros(m, dtype=np.uint8)
    lib().oracle_qs_events(C.byref(t.struct), m, _ptr(px), _ptr(py), _ptr(pz), _ptr(chi),
                           _ptr(ids), seed, step, threshold,
                           *[_ptr(out[k]) for k in ("xi", "lep_px", "lep_py", "lep_pz", "lep_tau",
                                                    "ph_px", "ph_py", "ph_pz", "ph_tau", "ph_id",
                                                    "keep")])
    out["keep"] = out["keep"].astype(bool)
    return out


def bw_events(t: OracleTables, p: np.ndarray, chi: np.ndarray, ids: np.ndarray, seed: int,
              step: int) -> dict:
    """Pair production for the firing photons; p is (m, 3)."""
    m = chi.shape[0]
    px, py, pz = (_f64(p[:, i]) for i in range(3))
    chi = _f64(chi)
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    names = ("xi_minus", "el_px", "el_py", "el_pz", "el_tau", "el_id", "po_px", "po_py", "po_pz",
             "po_tau", "po_id", "made")
    out = {k: np.zeros(m) for k in names}
    out["el_id"] = np.zeros(m, dtype=np.uint64)
    out["po_id"] = np.zeros(m, dtype=np.uint64)
    out["made"] = np.zeros(m, dtype=np.uint8)
    lib().oracle_bw_events(C.byref(t.struct), m, _ptr(px), _ptr(py), _ptr(pz), _ptr(chi),
                           _ptr(ids), seed, step, *[_ptr(out[k]) for k in names])
    out["made"] = out["made"].astype(bool)
    return out


def substep(t: OracleTables, species: dict, dt: float, seed: int, step: int,
            photon_threshold: float = 0.0, qs_chi_cut: float = 0.0, bw_chi_cut: float = 0.0) -> dict:
    """One QED substep over the three species (§3, §5).

    ``species`` maps "electrons", "positrons", "photons" to dicts of FP64 arrays
    (px..bz, tau, weight, id).  Every particle is evolved; particles whose optical
    depth went negative fire once: leptons emit a photon (recoil, tau reset),
    photons decay into a pair (photon removed: weight 0, tau = +inf).  Newborn
    particles are appended with tau from their own id and are first evolved on the
    next step.  Returns new species dicts plus per-species firing masks and chi.
    """
    out = {}
    fire = {}
    chis = {}
    for name, proc in (("electrons", QS), ("positrons", QS), ("photons", BW)):
        s = species[name]
        tau_new, chi, _, f = evolve(proc, t, s, dt, qs_chi_cut if proc == QS else bw_chi_cut)
        ns = {k: np.array(v, copy=True) for k, v in s.items()}
        ns["tau"] = tau_new
        out[name], fire[name], chis[name] = ns, f, chi
    new = {"electrons": [], "positrons": [], "photons": []}
    # photons: pair production
    ph = out["photons"]
    idx = np.nonzero(fire["photons"])[0]
    if idx.size:
        p = np.stack([ph["px"][idx], ph["py"][idx], ph["pz"][idx]], axis=1)
        ev = bw_events(t, p, chis["photons"][idx], ph["id"][idx], seed, step)
        for j, i in enumerate(idx):
            if ev["made"][j]:
                for sp, pre in (("electrons", "el"), ("positrons", "po")):
                    new[sp].append(dict(px=ev[pre + "_px"][j], py=ev[pre + "_py"][j],
                                        pz=ev[pre + "_pz"][j], ex=ph["ex"][i], ey=ph["ey"][i],
                                        ez=ph["ez"][i], bx=ph["bx"][i], by=ph["by"][i],
                                        bz=ph["bz"][i], tau=ev[pre + "_tau"][j],
                                        weight=ph["weight"][i], id=ev[pre + "_id"][j]))
                ph["weight"][i] = 0.0
                ph["tau"][i] = np.inf
            else:  # gamma_g <= 2: no pair, the photon survives with a fresh optical depth
                ph["tau"][i] = tau_draw(seed, int(ph["id"][i]), step, PURPOSE_TAU_RESET)
    # leptons: photon emission
    for name in ("electrons", "positrons"):
        s = out[name]
        idx = np.nonzero(fire[name])[0]
        if not idx.size:
            continue
        p = np.stack([s["px"][idx], s["py"][idx], s["pz"][idx]], axis=1)
        ev = qs_events(t, p, chis[name][idx], s["id"][idx], seed, step, photon_threshold)
        for j, i in enumerate(idx):
            s["px"][i], s["py"][i], s["pz"][i] = ev["lep_px"][j], ev["lep_py"][j], ev["lep_pz"][j]
            s["tau"][i] = ev["lep_tau"][j]
            if ev["keep"][j]:
                new["photons"].append(dict(px=ev["ph_px"][j], py=ev["ph_py"][j],
                                           pz=ev["ph_pz"][j], ex=s["ex"][i], ey=s["ey"][i],
                                           ez=s["ez"][i], bx=s["bx"][i], by=s["by"][i],
                                           bz=s["bz"][i], tau=ev["ph_tau"][j],
                                           weight=s["weight"][i], id=ev["ph_id"][j]))
    result = {}
    for name in ("electrons", "positrons", "photons"):
        s = out[name]
        if new[name]:
            keys = list(s.keys())
            add = {k: np.array([d.get(k, 0) for d in new[name]], dtype=s[k].dtype) for k in keys}
            s = {k: np.concatenate([s[k], add[k]]) for k in keys}
        result[name] = s
    result["fire"] = fire
    result["chi"] = chis
    result["n_new"] = {k: len(v) for k, v in new.items()}
    return result


# ----------------------------------------------------------------------------------------
# Schwinger pair production per cell (§2.3, Eq. (shw)); see schwinger.c
# ----------------------------------------------------------------------------------------
def schwinger_rate(E, B) -> float:
    """Pairs per unit volume per unit time (units 1/(lambda_C^3 t_C)) in fields E, B (units of E_s)."""
    return lib().oracle_schwinger_rate(*map(float, (*E, *B)))


def poisson(lam: float, seed: int, cell: int, step: int) -> int:
    return int(lib().oracle_poisson(float(lam), seed, cell, step))


def schwinger_pair_ids(seed: int, cell: int, step: int, j: int):
    out = np.zeros(2, dtype=np.uint64)
    lib().oracle_schwinger_pair_ids(seed, cell, step, j, _ptr(out))
    return int(out[0]), int(out[1])


def schwinger_cells(fields: dict, dv: float, dt: float, weight: float, seed: int, step: int):
    """Per cell: the expected number of pairs of weight `weight` and the drawn count."""
    arrs = [_f64(fields[k]) for k in ("ex", "ey", "ez", "bx", "by", "bz")]
    n = arrs[0].shape[0]
    lam = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int64)
    lib().oracle_schwinger_cells(n, *[_ptr(a) for a in arrs], dv, dt, weight, seed, step, _ptr(lam), _ptr(cnt))
    return lam, cnt


def schwinger(fields: dict, dv: float, dt: float, weight: float, seed: int, step: int) -> dict:
    """The pairs cells make in one step: per pair its cell, electron and
    positron ids and optical depths (both at rest, with the cell's fields)."""
    lam, cnt = schwinger_cells(fields, dv, dt, weight, seed, step)
    cells, ide, idp = [], [], []
    for c in np.nonzero(cnt)[0]:
        for j in range(int(cnt[c])):
            a, b = schwinger_pair_ids(seed, int(c), step, j)
            cells.append(int(c)), ide.append(a), idp.append(b)
    ide = np.array(ide, dtype=np.uint64)
    idp = np.array(idp, dtype=np.uint64)
    return {"lambda": lam, "count": cnt, "cell": np.array(cells, dtype=np.int64), "e_id": ide, "p_id": idp,
            "e_tau": init_tau(ide, seed, step), "p_tau": init_tau(idp, seed, step)}
