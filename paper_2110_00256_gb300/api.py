"""Python binding of libqed with the names of the C ABI (include/qed.h).

Argument marshalling only: device memory comes from torch tensors, streams from
torch.cuda; every step of the substep runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib
from ._lib import (QED_EVOLVE_BULK, QED_EVOLVE_DEFAULT, QED_EVOLVE_DIRECT, QED_F32, QED_F64, QED_PROC_BW,
                   QED_PROC_QS, QED_STAT_COUNT, FireList, QedError, SubstepOpts, TableAxis, TableParams, check,
                   lib)

__all__ = [
    "QED_F32", "QED_F64", "QED_PROC_QS", "QED_PROC_BW", "QED_EVOLVE_DEFAULT", "QED_EVOLVE_DIRECT",
    "QED_EVOLVE_BULK", "QedError", "table_params", "Tables",
    "SpeciesBuffers", "FireBuffers", "Stats", "qed_tables_generate", "qed_tables_create",
    "qed_tables_copy_to_host", "qed_tables_save", "qed_tables_load", "qed_init_optical_depth",
    "qed_evolve_optical_depth", "qed_generate_photons", "qed_generate_pairs", "qed_substep",
    "qed_substep_noalloc", "qed_version", "Mlp", "qed_table_sample", "substep_opts_mlp", "SubstepCall",
    "Batch", "qed_substep_batched", "qed_tune_evolve", "make_opts", "plane_wave", "qed_push_plane_wave", "qed_push_stored_fields", "qed_push_substep_batched",
    "qed_schwinger_pairs",
    "qed_push_batched", "qed_exact_sample", "qed_probe_fp64_fma", "qed_probe_tanh", "qed_device_status", "qed_species_energy", "qed_compact_species", "CompactWork",
]

FIELDS = ("px", "py", "pz", "ex", "ey", "ez", "bx", "by", "bz")


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dtype(prec: int):
    return torch.float32 if prec == QED_F32 else torch.float64


def table_params(qs_chi_min=1e-3, qs_chi_max=1e3, qs_n_chi=256, qs_n_xi=256, qs_xi_min=1e-12,
                 bw_chi_min=2e-2, bw_chi_max=1e3, bw_n_chi=256, bw_n_xi=256) -> TableParams:
    """Table axes; defaults are the paper's benchmark tables (§4)."""
    return TableParams(TableAxis(qs_chi_min, qs_chi_max, qs_n_chi, qs_n_xi, qs_xi_min),
                       TableAxis(bw_chi_min, bw_chi_max, bw_n_chi, bw_n_xi, 0.0))


class Tables:
    """Owning wrapper of a qed_tables* handle."""

    def __init__(self, handle: int):
        self.handle = C.c_void_p(handle)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                lib().qed_tables_destroy(h)
            except Exception:
                pass
            self.handle = None

    @property
    def params(self) -> TableParams:
        p = TableParams()
        check(lib().qed_tables_get_params(self.handle, C.byref(p)))
        return p


def qed_version() -> str:
    return lib().qed_version().decode()


def qed_tables_generate(params: TableParams, stream=None) -> Tables:
    out = C.c_void_p()
    check(lib().qed_tables_generate(C.byref(params), C.byref(out), _stream(stream)))
    return Tables(out.value)


def qed_tables_create(params: TableParams, qs_lnG, qs_lnP, bw_lnT, bw_P, stream=None) -> Tables:
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (qs_lnG, qs_lnP, bw_lnT, bw_P)]
    exp = [params.qs.n_chi, params.qs.n_chi * params.qs.n_xi, params.bw.n_chi, params.bw.n_chi * params.bw.n_xi]
    for a, n in zip(arrs, exp):
        if a.size != n:
            raise ValueError(f"table array has {a.size} entries, expected {n}")
    out = C.c_void_p()
    check(lib().qed_tables_create(C.byref(params), *[a.ctypes.data_as(C.c_void_p) for a in arrs],
                                  C.byref(out), _stream(stream)))
    return Tables(out.value)


def qed_tables_copy_to_host(t: Tables) -> dict:
    p = t.params
    out = dict(qs_lnG=np.zeros(p.qs.n_chi), qs_lnP=np.zeros((p.qs.n_chi, p.qs.n_xi)),
               bw_lnT=np.zeros(p.bw.n_chi), bw_P=np.zeros((p.bw.n_chi, p.bw.n_xi)))
    check(lib().qed_tables_copy_to_host(t.handle, *[out[k].ctypes.data_as(C.c_void_p)
                                                    for k in ("qs_lnG", "qs_lnP", "bw_lnT", "bw_P")]))
    return out


def qed_tables_save(t: Tables, path: str):
    check(lib().qed_tables_save(t.handle, str(path).encode()))


def qed_tables_load(path: str, stream=None) -> Tables:
    out = C.c_void_p()
    check(lib().qed_tables_load(str(path).encode(), C.byref(out), _stream(stream)))
    return Tables(out.value)


# ---------------------------------------------------------------------------------------
# particle buffers (caller-owned device memory)
# ---------------------------------------------------------------------------------------
@dataclass
class SpeciesBuffers:
    """Structure-of-arrays species on the GPU with a fixed capacity."""
    capacity: int
    prec: int = QED_F32
    device: str = "cuda"
    positions: bool = False
    arrays: dict = field(default_factory=dict)

    def __post_init__(self):
        dt = _dtype(self.prec)
        cap = max(int(self.capacity), 1)
        names = FIELDS + ("tau", "tau_c", "weight") + (("x", "y", "z") if self.positions else ())
        for k in names:
            self.arrays[k] = torch.zeros(cap, dtype=dt, device=self.device)
        self.arrays["id"] = torch.zeros(cap, dtype=torch.int64, device=self.device)
        self.count = torch.zeros(1, dtype=torch.int64, device=self.device)

    def __getitem__(self, k):
        return self.arrays[k]

    def set(self, data: dict, n: int | None = None):
        """Copy host/device arrays into [0, n) and set the live count."""
        n = int(n if n is not None else len(data["px"]))
        if n > self.capacity:
            raise ValueError("more particles than capacity")
        for k, v in data.items():
            if k == "count":
                continue
            t = torch.as_tensor(v)
            if k == "id":
                t = t.to(torch.int64) if t.dtype != torch.uint64 else t.view(torch.int64)
                self.arrays["id"][:n].copy_(t[:n].to(self.device))
            else:
                self.arrays[k][:n].copy_(t[:n].to(device=self.device, dtype=self.arrays[k].dtype))
        self.count.fill_(n)
        return self

    def n(self) -> int:
        return int(self.count.item())

    def struct(self) -> _lib.Species:
        a = self.arrays
        pos = [a[k].data_ptr() for k in ("x", "y", "z")] if self.positions else [None, None, None]
        return _lib.Species(*[a[k].data_ptr() for k in FIELDS + ("tau", "tau_c", "weight", "id")],
                            int(self.capacity), self.count.data_ptr(), *pos)

    def to_host(self) -> dict:
        n = self.n()
        out = {k: v[:n].cpu().numpy() for k, v in self.arrays.items()}
        out["id"] = out["id"].view(np.uint64)
        return out


@dataclass
class FireBuffers:
    capacity: int
    device: str = "cuda"

    def __post_init__(self):
        cap = max(int(self.capacity), 1)
        self.idx = torch.zeros(cap, dtype=torch.int64, device=self.device)
        self.chi = torch.zeros(cap, dtype=torch.float64, device=self.device)
        self.count = torch.zeros(1, dtype=torch.int64, device=self.device)

    def struct(self) -> FireList:
        return FireList(self.idx.data_ptr(), self.chi.data_ptr(), self.count.data_ptr(), int(self.capacity))

    def n(self) -> int:
        return int(self.count.item())


class Stats:
    """Device counters (QED_STAT_*)."""

    NAMES = ("qs_events", "bw_events", "photons_kept", "photons_discarded", "pairs", "bw_no_pair",
             "dropped_capacity", "nonfinite", "fire_overflow", "wait_timeout", "schwinger_pairs", "evolved",
             "compacted")

    def __init__(self, device="cuda"):
        self.t = torch.zeros(QED_STAT_COUNT, dtype=torch.int64, device=device)

    def as_dict(self) -> dict:
        return dict(zip(self.NAMES, self.t.cpu().tolist()))


def _opts(photon_threshold=0.0, stats: Stats | None = None, qs_chi_cut=0.0, bw_chi_cut=0.0) -> SubstepOpts:
    o = SubstepOpts(float(photon_threshold), 0, None, stats.t.data_ptr() if stats is not None else None)
    o.qs_chi_cut = float(qs_chi_cut)
    o.bw_chi_cut = float(bw_chi_cut)
    return o


def qed_init_optical_depth(sp: SpeciesBuffers, seed: int, step: int = 0, stream=None):
    s = sp.struct()
    check(lib().qed_init_optical_depth(C.byref(s), sp.prec, seed, step, _stream(stream)))


def qed_evolve_optical_depth(t: Tables, proc: int, sp: SpeciesBuffers, dt: float, fire: FireBuffers,
                             stats: Stats | None = None, stream=None):
    s, f = sp.struct(), fire.struct()
    check(lib().qed_evolve_optical_depth(t.handle, proc, C.byref(s), float(dt), sp.prec, C.byref(f),
                                         stats.t.data_ptr() if stats is not None else None,
                                         _stream(stream)))


def qed_generate_photons(t: Tables, leptons: SpeciesBuffers, photons: SpeciesBuffers, fire: FireBuffers,
                         seed: int, step: int, photon_threshold=0.0, stats: Stats | None = None, stream=None):
    a, b, f, o = leptons.struct(), photons.struct(), fire.struct(), _opts(photon_threshold, stats)
    check(lib().qed_generate_photons(t.handle, C.byref(a), C.byref(b), C.byref(f), seed, step, C.byref(o),
                                     leptons.prec, _stream(stream)))


def qed_generate_pairs(t: Tables, photons: SpeciesBuffers, electrons: SpeciesBuffers,
                       positrons: SpeciesBuffers, fire: FireBuffers, seed: int, step: int,
                       stats: Stats | None = None, stream=None):
    a, b, c, f, o = photons.struct(), electrons.struct(), positrons.struct(), fire.struct(), _opts(0.0, stats)
    check(lib().qed_generate_pairs(t.handle, C.byref(a), C.byref(b), C.byref(c), C.byref(f), seed, step,
                                   C.byref(o), photons.prec, _stream(stream)))


class SubstepCall:
    """Pre-marshalled arguments of qed_substep, so that repeated calls (a timed
    loop, a graph capture) pay no Python-side struct building."""

    def __init__(self, t: Tables, electrons: SpeciesBuffers, positrons: SpeciesBuffers,
                 photons: SpeciesBuffers, fire: list, dt: float, seed: int, photon_threshold=0.0,
                 stats: Stats | None = None, mlp: "Mlp | None" = None, pipeline: int = 0, threads: int = 0,
                 ctas_per_sm: int = 0, qs_chi_cut: float = 0.0, bw_chi_cut: float = 0.0):
        self.t = t
        self.keep = (electrons, positrons, photons, fire, stats, mlp)
        self.e, self.p, self.g = electrons.struct(), positrons.struct(), photons.struct()
        self.fire = (FireList * 3)(*[f.struct() for f in fire])
        self.opts = _opts(photon_threshold, stats, qs_chi_cut, bw_chi_cut)
        if mlp is not None:
            self.opts.sampler = 1
            self.opts.mlp = mlp.handle.value
        self.opts.evolve_pipeline = int(pipeline)
        self.opts.evolve_threads = int(threads)
        self.opts.evolve_ctas_per_sm = int(ctas_per_sm)
        self.dt = float(dt)
        self.seed = int(seed)
        self.prec = electrons.prec
        self.fn = lib().qed_substep

    def __call__(self, step: int, stream=None):
        check(self.fn(self.t.handle, C.byref(self.e), C.byref(self.p), C.byref(self.g), self.dt, self.seed,
                      int(step), C.byref(self.opts), self.prec, self.fire, _stream(stream)))


def qed_substep(t: Tables, electrons: SpeciesBuffers, positrons: SpeciesBuffers, photons: SpeciesBuffers,
                dt: float, seed: int, step: int, fire: list, photon_threshold=0.0, stats: Stats | None = None,
                stream=None, mlp: "Mlp | None" = None, pipeline: int = 0, threads: int = 0, ctas_per_sm: int = 0,
                qs_chi_cut: float = 0.0, bw_chi_cut: float = 0.0):
    """One substep (include/qed.h).  pipeline / threads / ctas_per_sm choose the
    evolution kernel's variant and shape (QED_EVOLVE_*; 0 = library default);
    qs_chi_cut / bw_chi_cut are the processes' chi cut-offs (0 = off)."""
    SubstepCall(t, electrons, positrons, photons, fire, dt, seed, photon_threshold, stats, mlp, pipeline, threads,
                ctas_per_sm, qs_chi_cut, bw_chi_cut)(step, stream)


def qed_substep_noalloc(t: Tables, electrons: SpeciesBuffers, positrons: SpeciesBuffers,
                        photons: SpeciesBuffers, dt: float, seed: int, step: int, photon_threshold=0.0,
                        stats: Stats | None = None, stream=None):
    """qed_substep without caller-provided firing lists, for callers that cannot
    allocate device memory: the lists live in a fixed array inside libqed, so the
    three capacities together are limited to QED_NOALLOC_MAX_PARTICLES and calls
    that overlap on the GPU race (see include/qed.h)."""
    e, p, g, o = electrons.struct(), positrons.struct(), photons.struct(), _opts(photon_threshold, stats)
    check(lib().qed_substep_noalloc(t.handle, C.byref(e), C.byref(p), C.byref(g), float(dt), int(seed),
                                    int(step), C.byref(o), electrons.prec, _stream(stream)))


# ---------------------------------------------------------------------------------------
# learned sampler
# ---------------------------------------------------------------------------------------
class Mlp:
    """Owning wrapper of a qed_mlp* (the two networks, QS and BW)."""

    NPARAM = _lib.QED_MLP_PARAMS

    def __init__(self, tables: Tables | None, seed: int = 0, stream=None, _handle=None):
        out = C.c_void_p()
        if _handle is None:
            check(lib().qed_mlp_create(tables.handle, int(seed), C.byref(out), _stream(stream)))
        else:
            out = _handle
        self.handle = out
        self.tables = tables

    def save(self, path: str):
        """Both networks (chi ranges and FP32 parameters) to a file (qed_mlp_save)."""
        check(lib().qed_mlp_save(self.handle, str(path).encode()))

    @classmethod
    def load(cls, path: str, stream=None) -> "Mlp":
        """Networks that save() wrote (qed_mlp_load); the chi ranges come from the file."""
        out = C.c_void_p()
        check(lib().qed_mlp_load(str(path).encode(), C.byref(out), _stream(stream)))
        return cls(None, _handle=out)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                lib().qed_mlp_destroy(h)
            except Exception:
                pass
            self.handle = None

    def get_params(self, proc: int) -> np.ndarray:
        out = np.zeros(self.NPARAM, dtype=np.float32)
        check(lib().qed_mlp_get_params(self.handle, proc, out.ctypes.data_as(C.c_void_p)))
        return out

    def set_params(self, proc: int, params, stream=None):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.NPARAM
        check(lib().qed_mlp_set_params(self.handle, proc, p.ctypes.data_as(C.c_void_p), _stream(stream)))

    def train_step(self, proc: int, chi: torch.Tensor, u: torch.Tensor, xi: torch.Tensor, lr: float,
                   loss: torch.Tensor | None = None, stream=None):
        check(lib().qed_mlp_train_step(self.handle, proc, chi.data_ptr(), u.data_ptr(), xi.data_ptr(),
                                       int(chi.numel()), float(lr),
                                       loss.data_ptr() if loss is not None else None, _stream(stream)))

    def gradients(self, proc: int, chi: torch.Tensor, u: torch.Tensor, xi: torch.Tensor, stream=None):
        g = torch.zeros(self.NPARAM, dtype=torch.float32, device=chi.device)
        loss = torch.zeros(1, dtype=torch.float32, device=chi.device)
        check(lib().qed_mlp_gradients(self.handle, proc, chi.data_ptr(), u.data_ptr(), xi.data_ptr(),
                                      int(chi.numel()), g.data_ptr(), loss.data_ptr(), _stream(stream)))
        return g, loss

    def sample(self, proc: int, chi: torch.Tensor, u: torch.Tensor, out: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
        out = torch.empty_like(chi) if out is None else out
        check(lib().qed_mlp_sample(self.handle, proc, chi.data_ptr(), u.data_ptr(), int(chi.numel()),
                                   out.data_ptr(), _stream(stream)))
        return out


def qed_table_sample(t: Tables, proc: int, prec: int, chi: torch.Tensor, u: torch.Tensor,
                     out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Inverse-CDF samples through the 2-D tables (QS: xi; BW: the electron's fraction)."""
    out = torch.empty_like(chi) if out is None else out
    check(lib().qed_table_sample(t.handle, proc, prec, chi.data_ptr(), u.data_ptr(), int(chi.numel()),
                                 out.data_ptr(), _stream(stream)))
    return out


def substep_opts_mlp(mlp: Mlp, photon_threshold=0.0, stats: Stats | None = None) -> SubstepOpts:
    o = _opts(photon_threshold, stats)
    o.sampler = 1
    o.mlp = mlp.handle.value
    return o


# ---------------------------------------------------------------------------------------
# many patches per launch
# ---------------------------------------------------------------------------------------
class Batch:
    """Owning wrapper of a qed_batch* over a list of patches (dicts with
    "electrons", "positrons", "photons" SpeciesBuffers and "fire", three FireBuffers)."""

    def __init__(self, patches: list, prec: int, stream=None):
        arr = (_lib.Patch * len(patches))()
        for i, p in enumerate(patches):
            arr[i].electrons = p["electrons"].struct()
            arr[i].positrons = p["positrons"].struct()
            arr[i].photons = p["photons"].struct()
            for k in range(3):
                arr[i].fire[k] = p["fire"][k].struct()
        out = C.c_void_p()
        check(lib().qed_batch_create(arr, len(patches), prec, C.byref(out), _stream(stream)))
        self.handle = out
        self.patches = patches  # keeps the buffers alive
        self.prec = prec

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                lib().qed_batch_destroy(h)
            except Exception:
                pass
            self.handle = None


def qed_substep_batched(t: Tables, b: Batch, dt: float, seed: int, step: int, opts: SubstepOpts | None = None,
                        stream=None):
    check(lib().qed_substep_batched(t.handle, b.handle, float(dt), int(seed), int(step),
                                    C.byref(opts) if opts is not None else None, _stream(stream)))


def qed_push_substep_batched(t: Tables, b: Batch, wave, t0: float, dt: float, seed: int, step: int,
                             opts: SubstepOpts | None = None, store_fields: bool = False, stream=None):
    """Push in `wave` fused with the batched substep (include/qed.h)."""
    check(lib().qed_push_substep_batched(t.handle, b.handle, C.byref(wave), float(t0), float(dt), int(seed), int(step),
                                         C.byref(opts) if opts is not None else None, 1 if store_fields else 0,
                                         _stream(stream)))


def qed_schwinger_pairs(fields: dict, dv: float, dt: float, weight: float, seed: int, step: int,
                        electrons: SpeciesBuffers, positrons: SpeciesBuffers, stats: Stats | None = None,
                        positions: dict | None = None, stream=None):
    """Schwinger pairs made in the cells whose fields (device tensors ex .. bz,
    one entry per cell, the species' precision) are given (include/qed.h)."""
    n = int(fields["ex"].numel())
    ptr = lambda d, k: d[k].data_ptr() if d is not None else None  # noqa: E731
    cells = _lib.Cells(*[fields[k].data_ptr() for k in ("ex", "ey", "ez", "bx", "by", "bz")],
                       ptr(positions, "x"), ptr(positions, "y"), ptr(positions, "z"), n)
    e, p = electrons.struct(), positrons.struct()
    check(lib().qed_schwinger_pairs(C.byref(cells), float(dv), float(dt), float(weight), int(seed), int(step),
                                    C.byref(e), C.byref(p), electrons.prec,
                                    stats.t.data_ptr() if stats is not None else None, _stream(stream)))


def qed_tune_evolve(t: Tables, b: Batch, stream=None) -> dict:
    th, ct, ms = C.c_int32(), C.c_int32(), C.c_float()
    check(lib().qed_tune_evolve(t.handle, b.handle, C.byref(th), C.byref(ct), C.byref(ms), _stream(stream)))
    return {"threads": th.value, "ctas_per_sm": ct.value, "ms": ms.value}


def make_opts(photon_threshold=0.0, stats: Stats | None = None, mlp: "Mlp | None" = None,
              d_step: torch.Tensor | None = None, evolve_threads: int = 0, evolve_ctas_per_sm: int = 0,
              evolve_pipeline: int = 0, qs_chi_cut: float = 0.0, bw_chi_cut: float = 0.0,
              wait_limit_cycles: int = 0) -> SubstepOpts:
    o = _opts(photon_threshold, stats, qs_chi_cut, bw_chi_cut)
    o.wait_limit_cycles = int(wait_limit_cycles)
    if mlp is not None:
        o.sampler = 1
        o.mlp = mlp.handle.value
    if d_step is not None:
        o.d_step = d_step.data_ptr()
    o.evolve_threads = int(evolve_threads)
    o.evolve_ctas_per_sm = int(evolve_ctas_per_sm)
    o.evolve_pipeline = int(evolve_pipeline)
    return o


# ---------------------------------------------------------------------------------------
# plane-wave push (drives the cascade workload)
# ---------------------------------------------------------------------------------------
def plane_wave(e0: float, omega: float, phase0: float = 0.0, circular: bool = False, direction: int = -1):
    return _lib.PlaneWave(float(e0), float(omega), float(phase0), 1 if circular else 0, int(direction))


def qed_push_plane_wave(sp: SpeciesBuffers, charge: float, wave, t: float, dt: float, stream=None):
    s = sp.struct()
    check(lib().qed_push_plane_wave(C.byref(s), float(charge), C.byref(wave), float(t), float(dt), sp.prec,
                                    _stream(stream)))


def qed_push_stored_fields(sp: SpeciesBuffers, charge: float, dt: float, stream=None):
    s = sp.struct()
    check(lib().qed_push_stored_fields(C.byref(s), float(charge), float(dt), sp.prec, _stream(stream)))


def qed_push_batched(b: Batch, wave, t0: float, dt: float, step: int = 0, d_step: torch.Tensor | None = None,
                     stream=None):
    check(lib().qed_push_batched(b.handle, C.byref(wave), float(t0), float(dt), int(step),
                                 d_step.data_ptr() if d_step is not None else None, _stream(stream)))


# ---------------------------------------------------------------------------------------
# device error word, species diagnostics and upkeep
# ---------------------------------------------------------------------------------------
def qed_device_status(stream=None, clear: bool = True) -> tuple:
    """Synchronise the stream and read (and by default clear) the device error
    word; returns (status, word) without raising (include/qed.h)."""
    w = C.c_uint32(0)
    st = lib().qed_device_status(_stream(stream), C.byref(w), 1 if clear else 0)
    return st, w.value


def qed_species_energy(sp: SpeciesBuffers, photon: bool, out: torch.Tensor | None = None, stream=None):
    """Adds (sum of weight x energy, number with nonzero weight) of the species
    to the device FP64 pair `out` (zeros if None) and returns it."""
    if out is None:
        out = torch.zeros(2, dtype=torch.float64, device=sp.device)
    s = sp.struct()
    check(lib().qed_species_energy(C.byref(s), sp.prec, 1 if photon else 0, out.data_ptr(), _stream(stream)))
    return out


class CompactWork:
    """Device scratch of qed_compact_species for species of up to `capacity` particles."""

    def __init__(self, capacity: int, device="cuda"):
        self.capacity = int(capacity)
        self.t = torch.empty(_lib.QED_COMPACT_WORK(capacity), dtype=torch.int64, device=device)


def qed_compact_species(sp: SpeciesBuffers, work: CompactWork, stats: Stats | None = None, stream=None):
    s = sp.struct()
    check(lib().qed_compact_species(C.byref(s), sp.prec, work.t.data_ptr(), int(work.t.numel()),
                                    stats.t.data_ptr() if stats is not None else None, _stream(stream)))


def qed_exact_sample(proc: int, chi_rows: torch.Tensor, u: torch.Tensor, out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
    """The exact inverse CDF (include/qed.h) for m chi values and k draws each:
    u and the result have shape (m, k), FP64 on the device."""
    m = int(chi_rows.numel())
    k = int(u.numel()) // max(m, 1)
    if u.numel() != m * k:
        raise ValueError("u must hold k draws for each of the m chi values")
    if out is None:
        out = torch.empty_like(u)
    work = torch.empty(_lib.QED_EXACT_WORK(m), dtype=torch.float64, device=chi_rows.device)
    check(lib().qed_exact_sample(int(proc), chi_rows.data_ptr(), m, u.data_ptr(), k, out.data_ptr(), work.data_ptr(),
                                 int(work.numel()), _stream(stream)))
    return out


def qed_probe_fp64_fma(iters: int = 200_000, ctas_per_sm: int = 4, stream=None) -> dict:
    """FP64 FMA instructions per second of this GPU (include/qed.h)."""
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    r, ms = C.c_double(), C.c_float()
    check(lib().qed_probe_fp64_fma(int(iters), int(ctas_per_sm), sink.data_ptr(), C.byref(r), C.byref(ms),
                                   _stream(stream)))
    return {"fma_per_s": r.value, "ms": ms.value}


def qed_probe_tanh(iters: int = 200_000, ctas_per_sm: int = 8, stream=None) -> dict:
    """tanh.approx.f32 evaluations per second of this GPU (include/qed.h)."""
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    r, ms = C.c_double(), C.c_float()
    check(lib().qed_probe_tanh(int(iters), int(ctas_per_sm), sink.data_ptr(), C.byref(r), C.byref(ms),
                               _stream(stream)))
    return {"tanh_per_s": r.value, "ms": ms.value}


def qed_probe_fp64_logexp(x: torch.Tensor, stream=None) -> dict:
    """The rate lookups' FP64 logarithm and exponential and the CUDA library's
    on the device doubles x (include/qed.h)."""
    x = x.contiguous()
    out = torch.empty(4 * x.numel(), dtype=torch.float64, device=x.device)
    check(lib().qed_probe_fp64_logexp(x.data_ptr(), int(x.numel()), out.data_ptr(), _stream(stream)))
    o = out.view(4, -1)
    return {"log": o[0], "exp": o[1], "log_lib": o[2], "exp_lib": o[3]}
