"""ctypes declarations of the C ABI in include/qed.h (argument marshalling only).

The shared library is ``paper_2110_00256_gb300/_build/libqed.so``, built by
``paper_2110_00256_gb300.build.build()``.  There is no fallback: if the library
is missing or fails to load, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libqed.so")

QED_OK = 0
STATUS_NAMES = {0: "QED_OK", 1: "QED_ERR_INVALID_ARG", 2: "QED_ERR_CUDA", 3: "QED_ERR_CAPACITY",
                4: "QED_ERR_NUMERIC", 5: "QED_ERR_TIMEOUT", 6: "QED_ERR_IO", 7: "QED_ERR_UNSUPPORTED"}
QED_F32, QED_F64 = 0, 1
QED_PROC_QS, QED_PROC_BW = 0, 1
QED_EVOLVE_DEFAULT, QED_EVOLVE_DIRECT, QED_EVOLVE_BULK = 0, 1, 2
QED_MAX_TABLE_N = 1024
(QED_STAT_QS_EVENTS, QED_STAT_BW_EVENTS, QED_STAT_PHOTONS_KEPT, QED_STAT_PHOTONS_DISCARDED,
 QED_STAT_PAIRS, QED_STAT_BW_NO_PAIR, QED_STAT_DROPPED_CAPACITY, QED_STAT_NONFINITE,
 QED_STAT_FIRE_OVERFLOW, QED_STAT_WAIT_TIMEOUT, QED_STAT_SCHWINGER_PAIRS, QED_STAT_EVOLVED,
 QED_STAT_COMPACTED, QED_STAT_COUNT) = range(14)
QED_EW_WAIT_TIMEOUT, QED_EW_NONFINITE, QED_EW_CAPACITY, QED_EW_FIRE_OVERFLOW = 1, 2, 4, 8


def QED_EXACT_WORK(m: int) -> int:
    return int(m) * 2051


def QED_COMPACT_WORK(cap: int) -> int:
    return 2 * int(cap) + (int(cap) + 2047) // 2048 + 8


class QedError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class TableAxis(C.Structure):
    _fields_ = [("chi_min", C.c_double), ("chi_max", C.c_double), ("n_chi", C.c_int32),
                ("n_xi", C.c_int32), ("xi_min", C.c_double)]


class TableParams(C.Structure):
    _fields_ = [("qs", TableAxis), ("bw", TableAxis)]


class Species(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("px", "py", "pz", "ex", "ey", "ez", "bx", "by", "bz",
                                          "tau", "tau_c", "weight", "id")] + \
               [("capacity", C.c_int64), ("d_count", C.c_void_p), ("x", C.c_void_p), ("y", C.c_void_p),
                ("z", C.c_void_p)]


class FireList(C.Structure):
    _fields_ = [("idx", C.c_void_p), ("chi", C.c_void_p), ("d_count", C.c_void_p),
                ("capacity", C.c_int64)]


class PlaneWave(C.Structure):
    _fields_ = [("e0", C.c_double), ("omega", C.c_double), ("phase0", C.c_double), ("polarization", C.c_int32),
                ("direction", C.c_int32)]


class Patch(C.Structure):
    _fields_ = [("electrons", Species), ("positrons", Species), ("photons", Species), ("fire", FireList * 3)]


class Cells(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("ex", "ey", "ez", "bx", "by", "bz", "x", "y", "z")] + [("n", C.c_int64)]


class UnitScales(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("length", "time", "momentum", "energy", "e_field", "b_field")]


class SubstepOpts(C.Structure):
    _fields_ = [("photon_threshold", C.c_double), ("sampler", C.c_int32), ("mlp", C.c_void_p),
                ("d_stats", C.c_void_p), ("evolve_begin", C.c_void_p), ("evolve_end", C.c_void_p),
                ("d_step", C.c_void_p), ("evolve_threads", C.c_int32), ("evolve_ctas_per_sm", C.c_int32),
                ("evolve_pipeline", C.c_int32), ("qs_chi_cut", C.c_double), ("bw_chi_cut", C.c_double),
                ("wait_limit_cycles", C.c_int64)]


_P = C.c_void_p
_S = C.c_int32
_U64 = C.c_uint64
_I64 = C.c_int64
_D = C.c_double

SIGNATURES = {
    "qed_last_error_message": (C.c_char_p, []),
    "qed_version": (C.c_char_p, []),
    "qed_tables_generate": (_S, [C.POINTER(TableParams), C.POINTER(_P), _P]),
    "qed_tables_create": (_S, [C.POINTER(TableParams), _P, _P, _P, _P, C.POINTER(_P), _P]),
    "qed_tables_copy_to_host": (_S, [_P, _P, _P, _P, _P]),
    "qed_tables_get_params": (_S, [_P, C.POINTER(TableParams)]),
    "qed_tables_save": (_S, [_P, C.c_char_p]),
    "qed_tables_load": (_S, [C.c_char_p, C.POINTER(_P), _P]),
    "qed_tables_destroy": (_S, [_P]),
    "qed_init_optical_depth": (_S, [C.POINTER(Species), _S, _U64, _I64, _P]),
    "qed_evolve_optical_depth": (_S, [_P, _S, C.POINTER(Species), _D, _S, C.POINTER(FireList), _P, _P]),
    "qed_generate_photons": (_S, [_P, C.POINTER(Species), C.POINTER(Species), C.POINTER(FireList), _U64,
                                  _I64, C.POINTER(SubstepOpts), _S, _P]),
    "qed_generate_pairs": (_S, [_P, C.POINTER(Species), C.POINTER(Species), C.POINTER(Species),
                                C.POINTER(FireList), _U64, _I64, C.POINTER(SubstepOpts), _S, _P]),
    "qed_substep": (_S, [_P, C.POINTER(Species), C.POINTER(Species), C.POINTER(Species), _D, _U64, _I64,
                         C.POINTER(SubstepOpts), _S, C.POINTER(FireList), _P]),
    "qed_substep_noalloc": (_S, [_P, C.POINTER(Species), C.POINTER(Species), C.POINTER(Species), _D, _U64,
                                 _I64, C.POINTER(SubstepOpts), _S, _P]),
    "qed_batch_create": (_S, [C.POINTER(Patch), C.c_int32, _S, C.POINTER(_P), _P]),
    "qed_batch_destroy": (_S, [_P]),
    "qed_substep_batched": (_S, [_P, _P, _D, _U64, _I64, C.POINTER(SubstepOpts), _P]),
    "qed_tune_evolve": (_S, [_P, _P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_float), _P]),
    "qed_push_plane_wave": (_S, [C.POINTER(Species), _D, C.POINTER(PlaneWave), _D, _D, _S, _P]),
    "qed_push_stored_fields": (_S, [C.POINTER(Species), _D, _D, _S, _P]),
    "qed_units_library": (_S, [C.POINTER(UnitScales)]),
    "qed_schwinger_pairs": (_S, [C.POINTER(Cells), _D, _D, _D, _U64, _I64, C.POINTER(Species), C.POINTER(Species),
                                 _S, _P, _P]),
    "qed_units_reference_frequency": (_S, [_D, C.POINTER(UnitScales)]),
    "qed_units_reference_length": (_S, [_D, C.POINTER(UnitScales)]),
    "qed_units_heaviside_lorentz_mev": (_S, [C.POINTER(UnitScales)]),
    "qed_push_substep_batched": (_S, [_P, _P, C.POINTER(PlaneWave), _D, _D, _U64, _I64, C.POINTER(SubstepOpts), _S,
                                      _P]),
    "qed_push_batched": (_S, [_P, C.POINTER(PlaneWave), _D, _D, _I64, _P, _P]),
    "qed_mlp_create": (_S, [_P, _U64, C.POINTER(_P), _P]),
    "qed_mlp_destroy": (_S, [_P]),
    "qed_mlp_save": (_S, [_P, C.c_char_p]),
    "qed_mlp_load": (_S, [C.c_char_p, C.POINTER(_P), _P]),
    "qed_mlp_get_params": (_S, [_P, _S, _P]),
    "qed_mlp_set_params": (_S, [_P, _S, _P, _P]),
    "qed_mlp_train_step": (_S, [_P, _S, _P, _P, _P, _I64, C.c_float, _P, _P]),
    "qed_mlp_gradients": (_S, [_P, _S, _P, _P, _P, _I64, _P, _P, _P]),
    "qed_mlp_sample": (_S, [_P, _S, _P, _P, _I64, _P, _P]),
    "qed_table_sample": (_S, [_P, _S, _S, _P, _P, _I64, _P, _P]),
    "qed_device_status": (_S, [_P, C.POINTER(C.c_uint32), C.c_int32]),
    "qed_species_energy": (_S, [C.POINTER(Species), _S, C.c_int32, _P, _P]),
    "qed_compact_species": (_S, [C.POINTER(Species), _S, _P, _I64, _P, _P]),
    "qed_exact_sample": (_S, [_S, _P, _I64, _P, _I64, _P, _P, _I64, _P]),
    "qed_probe_fp64_fma": (_S, [_I64, C.c_int32, _P, C.POINTER(C.c_double), C.POINTER(C.c_float), _P]),
    "qed_probe_tanh": (_S, [_I64, C.c_int32, _P, C.POINTER(C.c_double), C.POINTER(C.c_float), _P]),
    "qed_probe_fp64_logexp": (_S, [_P, _I64, _P, _P]),
}
QED_MLP_PARAMS = 4417
QED_MAX_PATCHES = 1024
QED_NOALLOC_MAX_PARTICLES = 1 << 20

_lock = threading.Lock()
_lib = None


def lib():
    """Load libqed.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2110_00256_gb300.build.build() "
                               "(or __graft_entry__.build()); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def check(status: int):
    if status != QED_OK:
        msg = lib().qed_last_error_message()
        raise QedError(status, msg.decode() if msg else "")
