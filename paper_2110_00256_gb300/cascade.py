"""The batched cascade workload: many patches of uneven size, an electron beam
counter-propagating a linearly polarised plane wave whose fields are evaluated
analytically at each particle, the substep (photon emission, pair production)
after every push, all steps captured in one CUDA graph with a device step
counter.  By default the push is fused into the evolution
(qed_push_substep_batched: one pass per particle, 4 launches per step);
fused=False runs the separate push and substep (5 launches per step) with the
evolution launch shape chosen by qed_tune_evolve.  Every 50 steps the photons
that pair production removed are compacted out of the arrays.

Parameters: 64 patches with round(10^(3 + 4U)) electrons each (seed 7), gamma =
2000 (1 + 0.05 (2U - 1)) along +x, positions uniform over one wavelength;
a0 = 100 at 0.8 um (omega = 3.0329e-6 m_e c^2/hbar, E0 = a0 omega E_s), the wave
travelling along -x; dt = T_L / 200; tables 256 / 256x256.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import api, workloads

OMEGA_08UM = 3.0328877982211224e-6
A0 = 100.0


def make_patches(scale: float = 1.0, photon_factor: float = 40.0, prec: int = api.QED_F32, seed: int = 7,
                 fire_fraction: float = 1.0):
    """The patches; photon buffers hold photon_factor photons per electron, and
    the photons' firing lists fire_fraction of that (a photon beyond a full list
    keeps its negative optical depth and fires in the next step)."""
    counts = workloads.patch_counts(64, seed)
    counts = np.maximum((counts * scale).astype(np.int64), 1)
    r = np.random.default_rng(seed + 1)
    dt = torch.float32 if prec == api.QED_F32 else torch.float64
    g = torch.Generator(device="cuda")
    g.manual_seed(seed + 2)
    lam = 2 * math.pi / OMEGA_08UM
    patches = []
    offset = 0
    for n in counts:
        n = int(n)
        e = api.SpeciesBuffers(n + max(256, n // 10), prec, positions=True)
        u = torch.rand(n, generator=g, device="cuda", dtype=torch.float64)
        gam = 2000.0 * (1.0 + 0.05 * (2.0 * u - 1.0))
        e.arrays["px"][:n].copy_(torch.sqrt(gam * gam - 1.0).to(dt))
        e.arrays["x"][:n].copy_((lam * torch.rand(n, generator=g, device="cuda", dtype=torch.float64)).to(dt))
        e.arrays["tau"][:n].copy_(torch.empty(n, device="cuda", dtype=torch.float64).exponential_(1.0, generator=g)
                                  .to(dt))
        e.arrays["weight"][:n].fill_(1.0)
        e.arrays["id"][:n].copy_(torch.arange(offset, offset + n, device="cuda", dtype=torch.int64))
        e.count.fill_(n)
        offset += n
        pos = api.SpeciesBuffers(max(256, n // 10), prec, positions=True)
        ph = api.SpeciesBuffers(int(photon_factor * n) + 64, prec, positions=True)
        patches.append({"electrons": e, "positrons": pos, "photons": ph,
                        "fire": [api.FireBuffers(e.capacity), api.FireBuffers(pos.capacity),
                                 api.FireBuffers(max(64, int(fire_fraction * ph.capacity)))]})
    return patches, counts


def run(tables: api.Tables, steps: int = 2000, scale: float = 1.0, photon_factor: float = 40.0,
        prec: int = api.QED_F32, tune: bool = True, photon_threshold: float = 2.0, fused: bool = True,
        compact_every: int = 50, fire_fraction: float = 1.0) -> dict:
    """The cascade; every compact_every steps (0: never) the photons that pair
    production removed are dropped from every patch (qed_compact_species, inside
    the graph, one scratch buffer shared by the patches)."""
    patches, counts = make_patches(scale, photon_factor, prec, fire_fraction=fire_fraction)
    b = api.Batch(patches, prec)
    work = api.CompactWork(max(p["photons"].capacity for p in patches)) if compact_every else None
    tuned = api.qed_tune_evolve(tables, b) if tune and not fused else None
    wave = api.plane_wave(A0 * OMEGA_08UM, OMEGA_08UM)
    dt = 2 * math.pi / OMEGA_08UM / 200
    d_step = torch.zeros(1, dtype=torch.int64, device="cuda")
    stats = api.Stats()
    opts = api.make_opts(photon_threshold=photon_threshold, stats=stats, d_step=d_step)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):  # first calls outside the capture (dt = 0: nothing moves or fires)
        if fused:
            api.qed_push_substep_batched(tables, b, wave, 0.0, 0.0, 1, 0, api.make_opts(), stream=stream)
        else:
            api.qed_push_batched(b, wave, 0.0, 0.0, 0, stream=stream)
            api.qed_substep_batched(tables, b, 0.0, 1, 0, api.make_opts(), stream=stream)
        if work is not None:
            api.qed_compact_species(patches[0]["photons"], work, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(graph, stream=stream):
            for k in range(steps):
                if fused:
                    api.qed_push_substep_batched(tables, b, wave, 0.0, dt, 1, 0, opts, stream=stream)
                else:
                    api.qed_push_batched(b, wave, 0.0, dt, 0, d_step, stream=stream)
                    api.qed_substep_batched(tables, b, dt, 1, 0, opts, stream=stream)
                if work is not None and (k + 1) % compact_every == 0:
                    for p in patches:
                        api.qed_compact_species(p["photons"], work, stats, stream=stream)
    capture_s = time.perf_counter() - t0

    def live():
        return sum(int(p[k].count.item()) for p in patches for k in ("electrons", "positrons", "photons"))

    n0 = live()
    d_step.zero_()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):  # replay on the stream the events are recorded on
        ev0.record(stream)
        graph.replay()
        ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    n1 = live()
    s = stats.as_dict()
    # particle-steps: each step adds the live count of every species of every
    # patch, as the evolution reads it, to the 'evolved' counter
    particle_steps = s["evolved"]
    per_step = 4 if fused else 5
    extra = (4 * len(patches) / compact_every) if compact_every else 0.0
    return {"patches": int(len(counts)), "electrons": int(counts.sum()), "steps": steps, "ms": ms,
            "particle_steps": particle_steps, "value": particle_steps / (ms * 1e-3), "n_start": n0, "n_end": n1,
            "graph_nodes_per_step": per_step + extra, "capture_s": capture_s, "tuned": tuned, "stats": s,
            "launches_per_step": per_step + extra, "fused": fused, "compact_every": compact_every,
            "memory_gb": round(torch.cuda.max_memory_allocated() / 1e9, 1)}
