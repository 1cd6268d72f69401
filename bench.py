#!/usr/bin/env python3
"""Throughput of the strong-field QED Monte Carlo substep on GB300.

Workload (the precision-study case): 10^8 particles, 5e7 electrons and 5e7
photons drawn from the paper's §4 benchmark distribution (E, B components
uniform in +-E_s/100, p components uniform in +-1 GeV/c, optical depth
exponential), FP32 structure of arrays with a Kahan word for the optical depth,
tables of 256 points and 256x256 generated in FP64 on the GPU, dt = 10 hbar/(m_e c^2).
One step = one qed_substep call: evolution of all three species in one batched
launch, pair production, photon emission, secondaries appended.

Further legs (each with its own key in the same line): the evolution kernel's
variants, the end-to-end leg from host buffers, the FP64 table path, the learned
sampler, the paper's per-kernel table (each of its four kernels on all 1e8
particles, FP64 and FP32), the cascade, the batched substep, Schwinger pairs,
the 1000-step QS + BW workload, and the oracle timed on the host cores.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the host cores on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QED substep particle-steps/s on 1 GB300 (FP32 table & MLP vs FP64 table), % HBM peak"
UNIT = "particle-steps/s"
WORKLOAD = "precision study: 1e8 mixed particles (5e7 e-, 5e7 photons), FP32 SoA + Kahan tau, 256/256x256 tables"
N_PER_SPECIES = 50_000_000
DT = 10.0
SEED = 20211001
BYTES_F32 = 52  # algorithmic bytes per evolved particle: p, E, B, tau, tau_c read (44) + tau, tau_c written (8)
BYTES_F64 = 88  # p, E, B, tau read (80) + tau written (8)
FALLBACK_HBM_GBS = 6800.0
TANH_PER_SAMPLE = 128  # the learned sampler's GELUs: two hidden layers of 64
TC_FLOP_PER_SAMPLE = 2 * 64 * (16 + 80)  # its tensor-core MMAs: layer 1 (K = 16) and layer 2 (K = 80)


def headline_config(n: int, ws: int) -> dict:
    """The headline workload's description (the same in both arms)."""
    return {"workload": WORKLOAD, "particles": 2 * n, "electrons": n, "photons": n, "dt": DT,
            "tables": "256 / 256x256, FP64 generated, FP32 copies", "seed": SEED,
            "l2": "inputs (%.1f GB) larger than L2, no flush" % (2 * n * 48 / 1e9),
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--n", type=int, default=N_PER_SPECIES, help="particles per species (electrons, photons)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-mlp", action="store_true")
    ap.add_argument("--no-cascade", action="store_true")
    ap.add_argument("--no-schwinger", action="store_true")
    ap.add_argument("--no-longrun", action="store_true")
    ap.add_argument("--no-paper-table", action="store_true")
    ap.add_argument("--paper-table-n", type=int, default=100_000_000,
                    help="particles of the per-kernel table leg (the paper's tables use 1e8)")
    ap.add_argument("--cascade-scale", type=float, default=1.0,
                    help="fraction of the 64 patch counts round(10^(3+4U)) to run in the cascade leg")
    ap.add_argument("--cascade-steps", type=int, default=2000)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


KERNEL_SOURCES = ("evolve.cu", "evolve.cuh", "evolve_core.cuh", "physics.cuh", "common.cuh", "pipeline.cuh",
                  "fp64_math.cuh", "fp64_tables.h")


def kernel_hash() -> str:
    """Hash of the sources the evolution kernel is compiled from."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2110_00256_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profile_record(name: str, key: str):
    """A per-particle figure of the evolution kernel from a committed ncu
    summary (profiles/<name>), valid only while the kernel's sources are
    unchanged."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        rec = {}
        for line in open(path):
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                rec[k.strip()] = v.strip()
        if rec.get("kernel_sources_sha256_16") != kernel_hash():
            return None
        return float(rec[key])
    except Exception:
        return None


def traffic_record():
    """DRAM bytes per particle of the FP32 evolution kernel (the bulk-copy pipeline)."""
    return profile_record("evolve_bulk_kernel_fp32_traffic.txt", "dram_bytes_per_particle")


class Clocks:
    """nvidia-smi sampling of SM clock, power and throttle reasons every 20 ms,
    started ahead of the timed region; stop() keeps the samples whose
    timestamps fall inside [t0, t1] (host clock), the timed region."""

    def __init__(self, index: int):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"qed_bench_clocks_{os.getpid()}_rank{index}.csv")
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader",
                                          "-lms", "20"], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(2.0)  # nvidia-smi takes a moment before its first sample
        except Exception:
            self.proc = None

    def stop(self, t0: float | None = None, t1: float | None = None):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        import datetime
        rows = []
        with open(self.path) as fh:
            lines = fh.readlines()
        try:
            os.remove(self.path)
        except OSError:
            pass
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2].split()[0]), float(parts[3].split()[0]), parts[6:10]))
            except ValueError:
                continue
        inside = [r for r in rows if t0 is None or (t0 - 0.025 <= r[0] <= t1 + 0.025)]
        where = "timed region"
        if not inside:  # the region was shorter than the sampling interval: the nearest sample
            inside = sorted(rows, key=lambda r: abs(r[0] - 0.5 * (t0 + t1)))[:1] if rows else []
            where = "nearest sample to the timed region"
        if not inside:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in inside for n, v in zip(names, r[3]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside), "window": where}


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x: float, op) -> float:
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"  # (gloo: the host-side tests)
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.MAX)


def sum_over_ranks(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.SUM)


# ----------------------------------------------------------------------------------------
# GPU leg
# ----------------------------------------------------------------------------------------
def make_species(api, workloads, prec, n, extra, seed, rank):
    import torch
    dt = torch.float32 if prec == api.QED_F32 else torch.float64
    bufs = {}
    for k, s, off in (("electrons", 1, 0), ("photons", 2, 2 * 10 ** 12)):
        b = api.SpeciesBuffers(n + extra, prec)
        d = workloads.paper_benchmark_torch(n, seed + 7919 * rank + s, off + rank * 10 ** 10, dtype=dt)
        for c, v in d.items():
            b.arrays[c][:n].copy_(v)
        del d
        b.count.fill_(n)
        bufs[k] = b
    bufs["positrons"] = api.SpeciesBuffers(extra, prec)
    fire = [api.FireBuffers(bufs[k].capacity) for k in ("electrons", "positrons", "photons")]
    return bufs, fire


def counts(bufs):
    return sum(int(bufs[k].count.item()) for k in ("electrons", "positrons", "photons"))


def time_substep(api, t, bufs, fire, steps, warmup, ws, step0=0, evolve_events=True, mlp=None, shape=(0, 0, 0)):
    import torch
    stats = api.Stats()
    call = api.SubstepCall(t, bufs["electrons"], bufs["positrons"], bufs["photons"], fire, DT, SEED, stats=stats,
                           mlp=mlp, pipeline=shape[0], threads=shape[1], ctas_per_sm=shape[2])
    for s in range(warmup):
        call(step0 + s)
    # the photons that pair production removed so far are dropped before the timed
    # steps (outside them), so that the particle-steps counted below (the live count
    # at the start, times the steps) include no removed particle; the timed steps
    # append more particles than they remove, so the count stays a lower bound
    work = api.CompactWork(bufs["photons"].capacity)
    api.qed_compact_species(bufs["photons"], work, stats)
    del work
    torch.cuda.synchronize()
    n_before = counts(bufs)
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in evs:  # materialise the events
        a.record(stream), b.record(stream)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    t0_host = time.time()
    t0.record(stream)
    for s in range(steps):
        if evolve_events:
            call.opts.evolve_begin = evs[s][0].cuda_event
            call.opts.evolve_end = evs[s][1].cuda_event
        call(step0 + warmup + s)
    t1.record(stream)
    torch.cuda.synchronize()
    t1_host = time.time()
    barrier(ws)
    ms = t0.elapsed_time(t1)
    ev_ms = [a.elapsed_time(b) for a, b in evs] if evolve_events else []
    n_after = counts(bufs)
    return dict(ms=ms, n_before=n_before, n_after=n_after, evolve_ms=ev_ms, stats=stats.as_dict(), t0_host=t0_host,
                t1_host=t1_host)


def mlp_leg(api, tabs, bufs, fire, args, ws):
    """The learned sampler: both networks trained on 1e7 exact samples each (the
    GPU's exact inverse CDF, no table) by the library's kernels; the substep
    with the network in place of the 2-D tables; the two samplers alone on 1e8
    (chi, U) pairs; their KS distance to the exact inverse CDF in 5 chi bins;
    and the hard-photon tail P(xi > 0.99) at chi = 9."""
    import math

    import numpy as np
    import torch

    from paper_2110_00256_gb300 import surrogate
    mlp = api.Mlp(tabs, seed=3)
    t0 = time.perf_counter()
    train = {p: surrogate.train(mlp, tabs, p, n_samples=10_000_000) for p in (0, 1)}
    train_s = time.perf_counter() - t0
    k = max(3, args.steps // 4)
    r = time_substep(api, tabs, bufs, fire, k, 2, ws, step0=1000, mlp=mlp)
    ms = max_over_ranks(ws, r["ms"])
    out = {"value": sum_over_ranks(ws, r["n_before"] * k) / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / k,
           "train_s": round(train_s, 2), "train_samples_per_process": 10_000_000, "train_epochs": {"0": 48, "1": 96},
           "train_batch": 4096, "exact_targets_s": {p: round(train[p]["data_seconds"], 2) for p in train},
           "train_final_loss": {p: round(train[p]["final_loss"], 6) for p in train}}
    n = 100_000_000
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    for p, name in ((0, "qs"), (1, "bw")):
        lo, hi = (math.log(v) for v in surrogate.chi_range(tabs, p))
        chi = torch.exp(lo + (hi - lo) * torch.rand(n, generator=g, device="cuda", dtype=torch.float64))
        u = torch.rand(n, generator=g, device="cuda", dtype=torch.float64).clamp_(1e-15, 1 - 1e-15)
        o = torch.empty_like(chi)
        for label, fn in (("mlp", lambda: mlp.sample(p, chi, u, o)),
                          ("table_f32", lambda: api.qed_table_sample(tabs, p, api.QED_F32, chi, u, o))):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                fn()
            e1.record()
            torch.cuda.synchronize()
            out[f"{name}_{label}_samples_per_s"] = 3 * n / (e0.elapsed_time(e1) * 1e-3)
        del chi, u, o
        torch.cuda.empty_cache()
        kn = surrogate.compare(lambda c, uu: mlp.sample(p, c, uu), tabs, p, n=2_000_000)
        kt = surrogate.compare(lambda c, uu: api.qed_table_sample(tabs, p, api.QED_F32, c, uu), tabs, p,
                               n=2_000_000)
        out[f"{name}_ks_vs_exact"] = {"mlp_overall": round(kn["overall"], 5),
                                      "mlp_bins": [round(v, 5) for v in kn["bins"]],
                                      "table256_f32_overall": round(kt["overall"], 5),
                                      "table256_f32_bins": [round(v, 5) for v in kt["bins"]]}
    # P(xi > 0.99 | chi = 9): the smallest U mapped above 0.99, on a grid dense near U = 1
    uu = np.concatenate([np.linspace(0.5, 1 - 1e-3, 20000), 1 - np.logspace(-3, -12, 20000)])
    ut = torch.tensor(uu, dtype=torch.float64, device="cuda")
    ct = torch.full_like(ut, 9.0)

    def tail(x):
        above = np.nonzero(x.cpu().numpy() > 0.99)[0]
        return float(1.0 - uu[above[0]]) if len(above) else 0.0

    out["qs_tail_chi9_xi_gt_0.99"] = {"exact": tail(api.qed_exact_sample(0, torch.tensor([9.0], dtype=torch.float64,
                                                                                          device="cuda"), ut)),
                                      "mlp": tail(mlp.sample(0, ct, ut)),
                                      "table256_f32": tail(api.qed_table_sample(tabs, 0, api.QED_F32, ct, ut))}
    out["params_bytes_bf16_per_network"] = 2 * 4417
    out["table_bytes_fp32_256x256_per_process"] = 2 * 256 * 256 * 4
    # The sampler kernel's roofline: its GELUs take 128 tanh.approx.f32 per sample
    # on the special-function units (the largest stall is that queue), measured
    # against a kernel of nothing but tanh chains; the tensor cores' share beside it.
    probe = max((api.qed_probe_tanh(ctas_per_sm=c) for c in (4, 8)), key=lambda r: r["tanh_per_s"])
    rate = min(out["qs_mlp_samples_per_s"], out["bw_mlp_samples_per_s"])
    ach = TANH_PER_SAMPLE * rate
    peaks_ = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    bf16 = float(peaks_.get("bf16_tflops", 1900.0)) * 1e12
    out["roofline"] = {"bound": "alu", "kernel": "mlp_sample_tc_kernel", "unit": "tanh/s", "achieved": ach,
                       "peak": probe["tanh_per_s"], "frac": round(ach / probe["tanh_per_s"], 4),
                       "peak_kind": "measured: qed_probe_tanh (dependent tanh.approx.f32 chains) on this GPU",
                       "tanh_per_sample": TANH_PER_SAMPLE, "samples_per_s": rate,
                       "tensor_flop_per_sample": TC_FLOP_PER_SAMPLE,
                       "tensor_frac_of_bf16_peak": round(TC_FLOP_PER_SAMPLE * rate / bf16, 4)}
    return out


# The paper's kernel timings (Table tab:comp, quoted for context): ms to apply one
# kernel to all 10^8 particles of the §4 distribution, FP64 / FP32, on a Quadro GV100 (CUDA)
PAPER_GV100_MS = {"bw_evol": (14.52, 7.43), "bw_prod": (29.94, 15.70), "qs_evol": (14.62, 7.39),
                  "qs_em": (26.88, 14.15)}


def paper_table_leg(api, tabs, n=100_000_000, reps=5, precs=None):
    """Table tab:comp of the paper on this GPU: each of its four kernels applied to
    all n particles of the §4 distribution (one species), FP64 and FP32.  Evolution:
    qed_evolve_optical_depth with dt = 10 (a few particles fire).  Production /
    emission: every particle fires (its optical depth set below zero and evolved
    once, which lists all of them with their chi), then qed_generate_pairs /
    qed_generate_photons runs on all n; before each repetition the state the
    event kernel changed is restored and the destinations emptied (outside the
    CUDA events, which bracket the call alone)."""
    import torch

    from paper_2110_00256_gb300 import workloads
    out = {"workload": "%g particles of the paper's benchmark distribution (one species per kernel), every "
                       "kernel applied to all of them; production/emission: every particle fires" % n,
           "gb300_ms": {}, "paper_gv100_cuda_ms": {k: {"f64": v[0], "f32": v[1]} for k, v in PAPER_GV100_MS.items()}}

    def timed(fn, before=None):
        ms = []
        for r in range(reps + 1):
            if before:
                before()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            if r:  # the first call is a warm-up
                ms.append(a.elapsed_time(b))
        return round(sorted(ms)[len(ms) // 2], 4)

    for prec, key in ((api.QED_F64, "f64"), (api.QED_F32, "f32")):
        if precs is not None and prec not in precs:
            continue
        dt_ = torch.float64 if prec == api.QED_F64 else torch.float32
        for proc, name in ((api.QED_PROC_QS, "qs"), (api.QED_PROC_BW, "bw")):
            sp = api.SpeciesBuffers(n, prec)
            d = workloads.paper_benchmark_torch(n, 31 + proc, 0, dtype=dt_)
            for c, v in d.items():
                sp.arrays[c][:n].copy_(v)
            del d
            sp.count.fill_(n)
            fire = api.FireBuffers(n)
            out["gb300_ms"].setdefault(name + "_evol", {})[key] = timed(
                lambda: api.qed_evolve_optical_depth(tabs, proc, sp, DT, fire))
            # every particle fires: the event kernel then runs on all n
            sp.arrays["tau"][:n].fill_(-1.0)
            sp.arrays["tau_c"][:n].zero_()
            api.qed_evolve_optical_depth(tabs, proc, sp, DT, fire)
            torch.cuda.synchronize()
            assert fire.n() == n
            changed = ("px", "py", "pz", "tau", "tau_c") if proc == api.QED_PROC_QS else ("tau", "tau_c", "weight")
            saved = {c: sp.arrays[c][:n].clone() for c in changed}
            if proc == api.QED_PROC_QS:
                dst = api.SpeciesBuffers(n, prec)

                def restore():
                    for c in changed:
                        sp.arrays[c][:n].copy_(saved[c])
                    dst.count.zero_()
                out["gb300_ms"].setdefault("qs_em", {})[key] = timed(
                    lambda: api.qed_generate_photons(tabs, sp, dst, fire, SEED, 7), restore)
                made = dst.n()
            else:
                ele, pos = api.SpeciesBuffers(n, prec), api.SpeciesBuffers(n, prec)

                def restore():
                    for c in changed:
                        sp.arrays[c][:n].copy_(saved[c])
                    ele.count.zero_()
                    pos.count.zero_()
                out["gb300_ms"].setdefault("bw_prod", {})[key] = timed(
                    lambda: api.qed_generate_pairs(tabs, sp, ele, pos, fire, SEED, 7), restore)
                made = ele.n()
                del ele, pos
            out.setdefault("secondaries_per_call", {})[name + "_" + key] = made
            del sp, fire, saved
            if proc == api.QED_PROC_QS:
                del dst
            torch.cuda.empty_cache()
    out["speedup_vs_gv100"] = {k: {p: round(out["paper_gv100_cuda_ms"][k][p] / v * n / 1e8, 1)
                                   for p, v in d_.items()} for k, d_ in out["gb300_ms"].items()}
    return out


E2E_IN = ("px", "py", "pz", "ex", "ey", "ez", "bx", "by", "bz", "tau", "tau_c")
E2E_OUT = ("px", "py", "pz", "tau", "tau_c")


def e2e_host_buffers(capacity):
    """Pinned host buffers of the end-to-end leg, made once at the start of the
    run (outside every timed region)."""
    import torch
    return {k: ({c: torch.empty(capacity, dtype=torch.float32, pin_memory=True) for c in E2E_IN},
                {c: torch.empty(capacity, dtype=torch.float32, pin_memory=True) for c in E2E_OUT})
            for k in ("electrons", "photons")}


def e2e_leg(api, t, bufs, fire, steps, ws, pinned):
    """Same metric through the C ABI with host buffers: every step copies the
    inputs host -> device from pinned memory, runs the substep, and copies the
    updated optical depths and momenta back.  Two device buffer sets and three
    streams overlap step s's copy-in with step s-1's substep and copy-out (the
    host link runs both directions at once); the timed region spans every copy
    of every step."""
    import torch
    names_in, names_out = E2E_IN, E2E_OUT
    host, out = {}, {}
    for k in ("electrons", "photons"):
        n = int(bufs[k].count.item())
        host[k] = {c: pinned[k][0][c][:n] for c in names_in}
        for c in names_in:
            host[k][c].copy_(bufs[k].arrays[c][:n])
        out[k] = {c: pinned[k][1][c][:n] for c in names_out}
    counts_h = torch.zeros(3, dtype=torch.int64).pin_memory()
    # the second buffer set: ids and weights as in the first (the inputs do not carry them)
    sets = [(bufs, fire)]
    b2 = {k: api.SpeciesBuffers(bufs[k].capacity, api.QED_F32) for k in ("electrons", "positrons", "photons")}
    for k in ("electrons", "photons"):
        b2[k].arrays["id"].copy_(bufs[k].arrays["id"])
        b2[k].arrays["weight"].copy_(bufs[k].arrays["weight"])
    sets.append((b2, [api.FireBuffers(b2[k].capacity) for k in ("electrons", "positrons", "photons")]))
    calls = [api.SubstepCall(t, b["electrons"], b["positrons"], b["photons"], f, DT, SEED) for b, f in sets]
    s_in, s_comp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in sets]
    ev_comp = [torch.cuda.Event() for _ in sets]
    ev_out = [None for _ in sets]
    bi = sum(v.numel() * v.element_size() for d in host.values() for v in d.values())
    bo = sum(v.numel() * v.element_size() for d in out.values() for v in d.values()) + counts_h.numel() * 8
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_step = counts(bufs)
    # warm-up, untimed: one pass of every copy in both directions through both
    # buffer sets (the first transfers from newly pinned pages run at a third of
    # the link's rate)
    for b, _ in sets:
        for k in host:
            n = host[k]["px"].numel()
            for c in names_in:
                b[k].arrays[c][:n].copy_(host[k][c], non_blocking=True)
            for c in names_out:
                out[k][c].copy_(b[k].arrays[c][:n], non_blocking=True)
    barrier(ws)
    torch.cuda.synchronize()
    t0.record(s_in)
    for s in range(steps):
        j = s % 2
        b, _ = sets[j]
        with torch.cuda.stream(s_in):
            if ev_out[j] is not None:
                s_in.wait_event(ev_out[j])
            for k in host:
                n = host[k]["px"].numel()
                for c in names_in:
                    b[k].arrays[c][:n].copy_(host[k][c], non_blocking=True)
                b[k].count.fill_(n)
            b["positrons"].count.zero_()
            ev_in[j].record(s_in)
        s_comp.wait_event(ev_in[j])
        calls[j](10_000 + s, s_comp)
        ev_comp[j].record(s_comp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_comp[j])
            for k in host:
                n = host[k]["px"].numel()
                for c in names_out:
                    out[k][c].copy_(b[k].arrays[c][:n], non_blocking=True)
            counts_h[0:1].copy_(b["electrons"].count, non_blocking=True)
            counts_h[1:2].copy_(b["positrons"].count, non_blocking=True)
            counts_h[2:3].copy_(b["photons"].count, non_blocking=True)
            ev_out[j] = torch.cuda.Event()
            ev_out[j].record(s_out)
    s_out.wait_stream(s_in)
    s_out.wait_stream(s_comp)
    t1.record(s_out)
    torch.cuda.synchronize()
    barrier(ws)
    ms = t0.elapsed_time(t1)
    del host, out, sets, b2
    return ms, n_step, bi, bo


def batched_leg(api, tabs, ws, steps=10, warmup=3):
    """The batched substep (qed_substep_batched) on the many-patch workload:
    64 patches of round(10^(3+4U)) particles (seed 7; sum ~7e7), half
    electrons, half photons, the §4 distribution with its stored fields; CUDA
    events around each step and around its evolution launch."""
    import torch

    from paper_2110_00256_gb300 import workloads
    sizes = workloads.patch_counts(64, 7)
    patches, off = [], 0
    for i, c in enumerate(sizes):
        c = int(c)
        p = {}
        for k, m, s in (("electrons", c // 2, 1), ("photons", c - c // 2, 2)):
            b = api.SpeciesBuffers(m + max(256, m // 20), api.QED_F32)
            d = workloads.paper_benchmark_torch(m, SEED + 100 * i + s, off, dtype=torch.float32)
            for col, v in d.items():
                b.arrays[col][:m].copy_(v)
            del d
            b.count.fill_(m)
            off += m
            p[k] = b
        p["positrons"] = api.SpeciesBuffers(max(256, c // 20), api.QED_F32)
        p["fire"] = [api.FireBuffers(p[k].capacity) for k in ("electrons", "positrons", "photons")]
        patches.append(p)
    b = api.Batch(patches, api.QED_F32)
    stats = api.Stats()
    opts = api.make_opts(stats=stats)
    for s in range(warmup):
        api.qed_substep_batched(tabs, b, DT, SEED, s, opts)
    torch.cuda.synchronize()
    live = sum(int(p[k].count.item()) for p in patches for k in ("electrons", "positrons", "photons"))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    st = torch.cuda.current_stream()
    for a, e in evs:
        a.record(st), e.record(st)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0 = stats.as_dict()["evolved"]
    barrier(ws)
    torch.cuda.synchronize()
    t0.record(st)
    for s in range(steps):
        opts.evolve_begin, opts.evolve_end = evs[s][0].cuda_event, evs[s][1].cuda_event
        api.qed_substep_batched(tabs, b, DT, SEED, warmup + s, opts)
    t1.record(st)
    torch.cuda.synchronize()
    ms = max_over_ranks(ws, t0.elapsed_time(t1))
    evolved = stats.as_dict()["evolved"] - ev0
    ev_ms = sum(a.elapsed_time(e) for a, e in evs) / steps
    gbs = BYTES_F32 * (evolved / steps) / (ev_ms * 1e-3) / 1e9
    hbm, which = peaks()
    # the same steps with the direct-load kernel (16-byte loads into registers), for comparison
    od = api.make_opts(stats=stats, evolve_pipeline=api.QED_EVOLVE_DIRECT)
    dms, evd0 = [], stats.as_dict()["evolved"]
    for s in range(steps):
        od.evolve_begin, od.evolve_end = evs[s][0].cuda_event, evs[s][1].cuda_event
        api.qed_substep_batched(tabs, b, DT, SEED, warmup + steps + s, od)
        torch.cuda.synchronize()
        dms.append(evs[s][0].elapsed_time(evs[s][1]))
    out = {"value": sum_over_ranks(ws, evolved) / (ms * 1e-3), "unit": UNIT, "patches": len(patches),
           "particles": live, "ms_per_step": ms / steps, "launches_per_step": 4, "evolve_ms": round(ev_ms, 4),
           "evolve_hbm_gbs": round(gbs, 1), "evolve_frac": round(gbs / hbm, 4), "peak_kind": which,
           "direct_loads_evolve_hbm_gbs": round(BYTES_F32 * ((stats.as_dict()["evolved"] - evd0) / steps) /
                                                (sum(dms) / steps * 1e-3) / 1e9, 1),
           "workload": "64 patches, counts round(10^(3+4U)) (seed 7), half e-, half photons, paper §4 distribution, "
                       "FP32, stored fields"}
    del patches, b
    torch.cuda.empty_cache()
    return out


def subsample_step(api, tabs, bufs, fire, step, m=500_000):
    """One substep of the headline state with every (n/m)-th electron and photon
    copied to the host before and after, and the firing lists mapped to them."""
    import numpy as np
    import torch
    out = {"pre": {}, "post": {}, "fire": {}, "step": step, "n_particles": 0}
    sel = {}
    for k in ("electrons", "photons"):
        n = int(bufs[k].count.item())
        stride = max(1, n // m)
        idx = torch.arange(0, stride * min(m, n), stride, device="cuda")
        sel[k] = (idx, stride)
        out["n_particles"] += n
        out["pre"][k] = {c: bufs[k].arrays[c].index_select(0, idx).cpu().numpy()
                         for c in ("px", "py", "pz", "ex", "ey", "ez", "bx", "by", "bz", "tau", "tau_c")}
        out["pre"][k]["id"] = bufs[k].arrays["id"].index_select(0, idx).cpu().numpy().view(np.uint64)
    api.SubstepCall(tabs, bufs["electrons"], bufs["positrons"], bufs["photons"], fire, DT, SEED)(step)
    torch.cuda.synchronize()
    for k, j in (("electrons", 0), ("photons", 2)):
        idx, stride = sel[k]
        out["post"][k] = {c: bufs[k].arrays[c].index_select(0, idx).cpu().numpy() for c in ("tau", "tau_c")}
        nf = int(fire[j].count.item())
        fi = fire[j].idx[:nf].cpu().numpy()
        fc = fire[j].chi[:nf].cpu().numpy()
        keep = (fi % stride == 0) & (fi // stride < idx.numel())
        out["fire"][k] = ((fi[keep] // stride).astype(np.int64), fc[keep])
    return out


def chi_for_inputs(d, photon):
    """chi of the unscaled synthetic particles (§2 definition, FP64 numpy), only
    to rescale their fields so that chi follows the workload's distribution."""
    import numpy as np
    p = np.stack([d["px"], d["py"], d["pz"]], 1)
    E = np.stack([d["ex"], d["ey"], d["ez"]], 1)
    B = np.stack([d["bx"], d["by"], d["bz"]], 1)
    p2 = np.sum(p * p, 1)
    en = np.sqrt(p2) if photon else np.sqrt(1.0 + p2)
    f = en[:, None] * E + np.cross(p, B)
    s = np.sum(f * f, 1) - np.sum(p * E, 1) ** 2
    return np.sqrt(np.maximum(s, 0.0))


def longrun_leg(api, tabs, ws, rank, steps=1000, chunk=100, n=1_000_000, extra=4_000_000):
    """The full QS + BW workload over many steps: 1e6 electrons + 1e6 photons,
    §4 momenta, Gaussian field components rescaled per particle so that chi is
    log-uniform in [1e-3, 1e2], tables 256 / 256x256, dt = 10, 1000 steps,
    secondaries appended to buffers of 4e6 per species; FP32 and FP64.  One
    patch through qed_substep_batched, 100 steps per CUDA graph (device step
    counter), the particle-steps counted on the device (QED_STAT_EVOLVED)."""
    import torch

    from paper_2110_00256_gb300 import workloads
    host = {}
    for k, seed, off in (("electrons", 101, 0), ("photons", 102, 10 ** 12)):
        d = workloads.gaussian_fields(n, seed + 1000 * rank, 1e-3, 1e2, id_offset=off + rank * 10 ** 10)
        d = workloads.rescale_fields(d, chi_for_inputs(d, k == "photons"))
        d.pop("chi_target")
        host[k] = d
    out = {}
    for name, prec in (("fp32", api.QED_F32), ("fp64", api.QED_F64)):
        patch = {"electrons": api.SpeciesBuffers(n + extra, prec).set(host["electrons"]),
                 "positrons": api.SpeciesBuffers(extra, prec),
                 "photons": api.SpeciesBuffers(n + extra, prec).set(host["photons"])}
        patch["fire"] = [api.FireBuffers(patch[k].capacity) for k in ("electrons", "positrons", "photons")]
        b = api.Batch([patch], prec)
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):  # dt = 0: loads the kernels, changes no particle
            api.qed_substep_batched(tabs, b, 0.0, SEED, 0, api.make_opts(), stream=stream)
        stats = api.Stats()
        d_step = torch.zeros(1, dtype=torch.int64, device="cuda")
        opts = api.make_opts(stats=stats, d_step=d_step)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            with torch.cuda.graph(g, stream=stream):
                for _ in range(chunk):
                    api.qed_substep_batched(tabs, b, DT, SEED, 0, opts, stream=stream)
        d_step.zero_()
        stats.t.zero_()
        n0 = sum(int(patch[k].count.item()) for k in ("electrons", "positrons", "photons"))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(ws)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(steps // chunk):
                g.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(ws, e0.elapsed_time(e1))
        st = stats.as_dict()
        n1 = sum(int(patch[k].count.item()) for k in ("electrons", "positrons", "photons"))
        out[name] = {"value": sum_over_ranks(ws, st["evolved"]) / (ms * 1e-3), "unit": UNIT,
                     "ms_per_step": ms / steps, "steps": steps, "particles_start": n0, "particles_end": n1,
                     "qs_events": st["qs_events"], "bw_events": st["bw_events"], "pairs": st["pairs"],
                     "dropped_capacity": st["dropped_capacity"], "wait_timeout": st["wait_timeout"]}
        del g, b, patch
        torch.cuda.empty_cache()
    out["workload"] = ("1e6 e- + 1e6 photons, p from §4, Gaussian E, B rescaled so chi is log-uniform in "
                       "[1e-3, 1e2], tables 256 / 256x256, dt = 10, 1000 steps, 4e6 secondaries per species")
    return out


def schwinger_leg(api, ws):
    """Schwinger pairs per cell (qed_schwinger_pairs) on 1e8 FP32 cells: fields
    of PIC strength (components N(0, 1e-3) E_s: the rate underflows, the FP32
    pre-check skips the FP64 evaluation) and near-critical ones (N(0, 0.025)
    E_s: every cell through the FP64 rate); cell volume (2.6e4 hbar/(m_e c))^3
    (10 nm), dt = 1e3 hbar/(m_e c^2), pairs of weight 1."""
    import torch
    n = 100_000_000
    g = torch.Generator(device="cuda")
    g.manual_seed(17)
    out = {}
    for name, sigma in (("pic_fields", 1e-3), ("near_critical", 0.025)):
        f = {k: torch.randn(n, generator=g, device="cuda", dtype=torch.float32) * sigma
             for k in ("ex", "ey", "ez", "bx", "by", "bz")}
        e = api.SpeciesBuffers(4_000_000, api.QED_F32)
        p = api.SpeciesBuffers(4_000_000, api.QED_F32)
        st = api.Stats()
        ms = []
        for rep in range(4):
            e.count.zero_(), p.count.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            api.qed_schwinger_pairs(f, 1.7e13, 1e3, 1.0, 5, rep, e, p, stats=st)
            b.record()
            torch.cuda.synchronize()
            if rep:
                ms.append(a.elapsed_time(b))
        m = sorted(ms)[len(ms) // 2]
        out[name] = {"cells_per_s": n / (m * 1e-3), "ms": round(m, 4), "hbm_gbs": round(24 * n / (m * 1e-3) / 1e9, 1),
                     "pairs_per_launch": st.as_dict()["schwinger_pairs"] / 4}
        del f, e, p
        torch.cuda.empty_cache()
    return out


_ORACLE_TIMING = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import oracle
from paper_2110_00256_gb300 import workloads
ot = oracle.tables()
m = {m}
sp = {{"electrons": workloads.paper_benchmark(m, 11, 0), "photons": workloads.paper_benchmark(m, 12, 10 ** 12),
      "positrons": workloads.paper_benchmark(0, 13, 2 * 10 ** 12)}}
steps, t0 = 0, time.perf_counter()
while True:
    out = oracle.substep(ot, sp, dt={dt}, seed={seed}, step=steps)
    sp = {{k: {{c: out[k][c] for c in sp[k]}} for k in sp}}
    steps += 1
    if time.perf_counter() - t0 > {seconds}:
        break
print(json.dumps({{"steps": steps, "seconds": time.perf_counter() - t0}}))
"""


def _time_oracle(m: int, seconds: float, threads: int) -> dict:
    """The oracle's substep on 2m particles of the §4 distribution, in a child
    process with `threads` OpenMP threads, for about `seconds`."""
    code = _ORACLE_TIMING.format(root=ROOT, m=m, dt=DT, seed=SEED, seconds=seconds)
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": 2 * m * d["steps"] / d["seconds"], "steps": d["steps"], "seconds": round(d["seconds"], 1)}


def cpu_baseline(seconds=12.0, check=None):
    """The FP64 oracle on the host cores, on a bounded sample of the workload:
    all cores and one core, each in its own process; and, when `check` holds a
    GPU substep of a subsample of the headline workload, its error statement."""
    cores = os.cpu_count() or 1
    m = 250_000
    allc = _time_oracle(m, seconds, cores)
    one = _time_oracle(20_000, seconds / 2, 1)
    out = {"value": allc["value"], "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
           "sample": f"{2 * m} particles (paper §4 distribution, 256/256x256 FP64 oracle tables), {allc['steps']} "
                     f"substeps, {allc['seconds']} s wall; evolution OpenMP-parallel over particles, events serial",
           "one_core": {"value": one["value"], "unit": UNIT, "cores": 1,
                        "sample": f"40000 particles, {one['steps']} substeps, {one['seconds']} s wall"}}
    if check is not None:
        out["error_vs_oracle"] = error_vs_oracle(**check)
    return out


def error_vs_oracle(pre: dict, post: dict, fire: dict, step: int, n_particles: int) -> dict:
    """The FP32 substep's error against the FP64 oracle on a subsample of the
    headline workload (the oracle started from the GPU's pre-step state):
    optical depths of the particles that did not fire against the rounding bound
    of the FP32 evaluation, chi of the firing ones, and the firing decisions
    that differ with their margin m = |tau_new| / tau_old."""
    import numpy as np

    import oracle
    ot = oracle.tables()
    res = {"particles": 0, "max_tau_err_over_bound": 0.0, "max_rel_tau_err": 0.0, "max_rel_chi_err_firing": 0.0,
           "events_checked": 0, "decisions_differing": 0, "max_margin_of_differing": 0.0}
    for name, proc in (("electrons", 0), ("photons", 1)):
        h = pre[name]
        n = len(h["id"])
        res["particles"] += n
        tau_old = h["tau"].astype(np.float64) - h["tau_c"].astype(np.float64)
        inp = {c: h[c].astype(np.float64) for c in ("px", "py", "pz", "ex", "ey", "ez", "bx", "by", "bz")}
        inp["tau"] = tau_old
        tn, chi, rate, f = oracle.evolve(proc, ot, inp, DT)
        p2 = inp["px"] ** 2 + inp["py"] ** 2 + inp["pz"] ** 2
        en = np.sqrt(p2) if proc else np.sqrt(1.0 + p2)
        S = en * np.sqrt(inp["ex"] ** 2 + inp["ey"] ** 2 + inp["ez"] ** 2) + \
            np.sqrt(p2) * np.sqrt(inp["bx"] ** 2 + inp["by"] ** 2 + inp["bz"] ** 2)
        dchi = 1e-5 * S + 16 * 2.0 ** -53 * S * S / np.maximum(chi, 1e-300)
        r_hi = ot.rates(proc, chi + dchi, en)
        r_lo = ot.rates(proc, np.maximum(chi - dchi, 0.0), en)
        bound = 1e-5 * np.abs(tau_old) + DT * (np.maximum(np.abs(r_hi - rate), np.abs(r_lo - rate)) + 1e-5 * rate)
        gf = np.zeros(n, dtype=bool)
        gf[fire[name][0]] = True
        quiet = ~gf & ~f & np.isfinite(tn)  # (photons removed earlier keep tau = +inf and take no decision)
        t_gpu = post[name]["tau"].astype(np.float64) - post[name]["tau_c"].astype(np.float64)
        err = np.abs(t_gpu[quiet] - tn[quiet])
        res["max_tau_err_over_bound"] = max(res["max_tau_err_over_bound"],
                                            float(np.max(err / (bound[quiet] + 1e-300), initial=0.0)))
        res["max_rel_tau_err"] = max(res["max_rel_tau_err"],
                                     float(np.max(err / np.maximum(np.abs(tn[quiet]), 1e-30), initial=0.0)))
        both = gf & f
        idx, chig = fire[name]
        sel = both[idx]
        if sel.any():
            res["max_rel_chi_err_firing"] = max(res["max_rel_chi_err_firing"],
                                                float(np.max(np.abs(chig[sel] - chi[idx[sel]]) / chi[idx[sel]])))
        res["events_checked"] += int(both.sum())
        diff = np.nonzero(gf != f)[0]
        res["decisions_differing"] += int(len(diff))
        if len(diff):
            res["max_margin_of_differing"] = max(res["max_margin_of_differing"],
                                                 float(np.max(np.abs(tn[diff]) / np.abs(tau_old[diff]))))
    res["sample"] = (f"{res['particles']} particles (every {n_particles // max(res['particles'], 1)}-th of the "
                     f"headline's 1e8) through one FP32 substep, step {step}")
    return res


def cpu_model() -> str:
    """The host CPU as lscpu names it (model and architecture)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        info = dict(line.split(":", 1) for line in out.splitlines() if ":" in line)
        name = info.get("Model name", "").strip() or info.get("Vendor ID", "").strip()
        return f"{name} ({info.get('Architecture', '').strip()}, {info.get('CPU(s)', '').strip()} CPUs)"
    except Exception:
        return "unknown"


def gpu_main(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2110_00256_gb300 import api, build, workloads
    if rank == 0 or ws == 1:
        build.build()
    barrier(ws)

    t_gen0 = time.perf_counter()
    tabs = api.qed_tables_generate(api.table_params())
    gen_ms = (time.perf_counter() - t_gen0) * 1e3

    n = args.n
    extra = max(4_000_000, n // 25)
    pinned = e2e_host_buffers(n + extra) if not args.no_e2e else None
    bufs, fire = make_species(api, workloads, api.QED_F32, n, extra, SEED, rank)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    r = time_substep(api, tabs, bufs, fire, args.steps, args.warmup, ws)
    clk = clocks.stop(r["t0_host"], r["t1_host"])

    ms_max = max_over_ranks(ws, r["ms"])
    total = sum_over_ranks(ws, r["n_before"] * args.steps)
    value = total / (ms_max * 1e-3)
    ev = r["evolve_ms"]
    ev_mean = sum(ev) / len(ev)
    hbm, which = peaks()
    ach = BYTES_F32 * r["n_before"] / (ev_mean * 1e-3) / 1e9
    traffic_bpp = traffic_record()
    roofline = {"bound": "hbm", "kernel": "evolve_bulk_kernel<15,2,1,4>", "achieved": round(ach, 1), "peak": hbm,
                "unit": "GB/s", "frac": round(ach / hbm, 4), "peak_kind": which,
                "traffic": (traffic_bpp * r["n_before"]) if traffic_bpp else None,
                "algorithmic_bytes": BYTES_F32 * r["n_before"], "evolve_ms": round(ev_mean, 4),
                "frac_of_8TBs": round(ach / 8000.0, 4)}

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
              "config": headline_config(n, ws), "table_generation_ms": round(gen_ms, 1),
              "roofline": roofline,
              "gpu_launches": 4 * args.steps,  # zero3, evolution, the three event lists, clamp_all
              "events_per_step": {k: v / (args.warmup + args.steps) for k, v in r["stats"].items()
                                  if v and k != "compacted"},
              "removed_dropped_before_timing": r["stats"].get("compacted", 0)}
    if clk:
        result["clocks"] = clk

    # the evolution kernel's variants on the same workload (include/qed.h, QED_EVOLVE_*)
    variants = {}
    for name, shape in (("direct_loads_4cta", (api.QED_EVOLVE_DIRECT, 0, 4)),
                        ("direct_loads_3cta", (api.QED_EVOLVE_DIRECT, 0, 3)),
                        ("bulk_8w_4stages", (api.QED_EVOLVE_BULK, 0, 0)),
                        ("bulk_16w_2stages", (api.QED_EVOLVE_BULK, 512, 0)),
                        ("bulk_8w_2stages_2cta", (api.QED_EVOLVE_BULK, 0, 2))):
        rv = time_substep(api, tabs, bufs, fire, 6, 2, ws, step0=500, shape=shape)
        evm = sum(rv["evolve_ms"]) / len(rv["evolve_ms"])
        variants[name] = {"evolve_ms": round(evm, 4), "hbm_gbs": round(BYTES_F32 * rv["n_before"] / (evm * 1e-3) / 1e9, 1),
                          "wait_timeout": rv["stats"].get("wait_timeout", 0)}
    result["evolve_variants"] = variants

    # one more substep of the same state, kept for the error statement against
    # the oracle (cpu_baseline leg): a subsample of 1e6 particles, every n/5e5-th
    # electron and photon, before and after the step, with the firing lists
    check = None
    if rank == 0 and not args.no_cpu_baseline:
        check = subsample_step(api, tabs, bufs, fire, 2000)

    if not args.no_e2e:
        k = max(4, min(args.steps, 8))
        ms, n_step, bi, bo = e2e_leg(api, tabs, bufs, fire, k, ws, pinned)
        ms = max_over_ranks(ws, ms)
        result["e2e"] = {"value": sum_over_ranks(ws, n_step * k) / (ms * 1e-3), "unit": UNIT,
                         "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "steps": k,
                         "ms_per_step": ms / k}

    # FP64 table path beside it (same workload, FP64 SoA)
    if not args.no_fp64:
        del bufs, fire
        torch.cuda.empty_cache()
        b64, f64 = make_species(api, workloads, api.QED_F64, n, extra, SEED, rank)
        r64 = time_substep(api, tabs, b64, f64, max(3, args.steps // 4), 2, ws)
        ms64 = max_over_ranks(ws, r64["ms"])
        tot64 = sum_over_ranks(ws, r64["n_before"] * max(3, args.steps // 4))
        ev64 = sum(r64["evolve_ms"]) / len(r64["evolve_ms"])
        ach64 = BYTES_F64 * r64["n_before"] / (ev64 * 1e-3) / 1e9
        result["paths"] = {"fp64_table": {"value": tot64 / (ms64 * 1e-3), "unit": UNIT,
                                          "ms_per_step": ms64 / max(3, args.steps // 4),
                                          "evolve_ms": round(ev64, 4), "hbm_gbs": round(ach64, 1),
                                          "hbm_frac": round(ach64 / hbm, 4)}}
        # the FP64 pipe's peak, measured by a kernel of nothing but FMA chains
        probe = api.qed_probe_fp64_fma()
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        mhz = clk["sm_mhz"] if clk else 2070.0
        result["paths"]["fp64_table"]["fp64_fma_probe"] = {
            "fma_per_s": probe["fma_per_s"], "per_sm_per_clock": round(probe["fma_per_s"] / (sms * mhz * 1e6), 3),
            "clock_mhz_assumed": mhz, "ms": round(probe["ms"], 3)}
        ipp = profile_record("evolve_kernel_fp64_insts.txt", "fp64_inst_per_particle")
        if ipp:
            peak64 = probe["fma_per_s"]
            ach_i = ipp * r64["n_before"] / (ev64 * 1e-3)
            result["paths"]["fp64_table"]["roofline"] = {
                "bound": "alu", "kernel": "evolve_kernel<double,2,4,3>", "unit": "FP64 instructions/s",
                "achieved": ach_i, "peak": peak64, "frac": round(ach_i / peak64, 4),
                "peak_kind": "measured: qed_probe_fp64_fma (dependent DFMA chains) on this GPU",
                "fp64_inst_per_particle": ipp}
        bufs, fire = b64, f64
        del b64, f64
        torch.cuda.empty_cache()
        bufs, fire = make_species(api, workloads, api.QED_F32, n, extra, SEED, rank)

    if not args.no_mlp:
        result.setdefault("paths", {})["fp32_mlp"] = mlp_leg(api, tabs, bufs, fire, args, ws)

    if not args.no_paper_table:
        result["paper_table"] = paper_table_leg(api, tabs, n=args.paper_table_n)

    if not args.no_cascade:
        del bufs, fire
        torch.cuda.empty_cache()
        from paper_2110_00256_gb300 import cascade, workloads
        # memory of the full-scale cascade: per electron of the start, buffers for 1.1 electrons,
        # 0.1 positrons and PHOTONS photons (68 B each in FP32 with positions and ids), firing lists
        # (16 B per entry; a quarter of the photons' capacity) and the compaction scratch
        photons_per_e, fire_frac = 36.0, 0.25
        n_e = float(workloads.patch_counts(64, 7).sum()) * args.cascade_scale
        need = n_e * ((1.2 + photons_per_e) * 68 + (1.2 + fire_frac * photons_per_e) * 16) + \
            16 * photons_per_e * float(workloads.patch_counts(64, 7).max()) * args.cascade_scale
        free = torch.cuda.mem_get_info()[0]
        scale = args.cascade_scale if need < 0.85 * free else 0.1
        c = cascade.run(tabs, steps=args.cascade_steps, scale=scale, photon_factor=photons_per_e,
                        fire_fraction=fire_frac)
        torch.cuda.empty_cache()
        cs = cascade.run(tabs, steps=args.cascade_steps, scale=0.1, fused=False)
        result["cascade"] = {"value": c["value"], "unit": UNIT, "steps": c["steps"], "patches": c["patches"],
                             "electrons_start": c["electrons"], "particles_end": c["n_end"],
                             "particle_steps": c["particle_steps"], "memory_gb": c["memory_gb"],
                             "memory_needed_estimate_gb": round(need / 1e9, 1), "free_gb": round(free / 1e9, 1),
                             "ms": round(c["ms"], 3), "launches_per_step": c["launches_per_step"],
                             "graph": "all steps in one CUDA graph, step counter on the device",
                             "push": "fused into the evolution (qed_push_substep_batched)",
                             "compaction": "removed photons dropped every %d steps (qed_compact_species)"
                                           % c["compact_every"],
                             "separate_push_at_0.1_scale": {"value": cs["value"], "ms": round(cs["ms"], 3),
                                                            "launches_per_step": cs["launches_per_step"],
                                                            "tuned_evolve": cs["tuned"]},
                             "events": c["stats"],
                             "workload": "64 patches, counts round(10^(3+4U)) x %g (seed 7), e- beam gamma 2000 +-5%% "
                                         "vs a0=100 linear plane wave (0.8 um), dt = T_L/200, photons < 2 m_e c^2 "
                                         "discarded" % scale}

    if not args.no_cascade:
        result["batched"] = batched_leg(api, tabs, ws)

    if not args.no_schwinger:
        result.setdefault("paths", {})["schwinger"] = schwinger_leg(api, ws)

    if not args.no_longrun:
        result.setdefault("paths", {})["full_qs_bw_1000_steps"] = longrun_leg(api, tabs, ws, rank)

    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(check=check)
        if "error_vs_oracle" in result["cpu_baseline"]:  # reported beside the headline it qualifies
            result["error_vs_oracle"] = result["cpu_baseline"].pop("error_vs_oracle")
    if rank == 0:
        print(json.dumps(result), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------------------------------
# reference leg: the oracle, timed on the host cores
# ----------------------------------------------------------------------------------------
def reference_main(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2110_00256_gb300 import workloads
    ot = oracle.tables()
    m = 100_000  # particles per species per step: the bounded sample
    sp = {"electrons": workloads.paper_benchmark(m, 11, 0), "photons": workloads.paper_benchmark(m, 12, 10 ** 12),
          "positrons": workloads.paper_benchmark(0, 13, 2 * 10 ** 12)}
    for s in range(args.warmup):
        out = oracle.substep(ot, sp, dt=DT, seed=SEED, step=s)
        sp = {k: {c: out[k][c] for c in sp[k]} for k in sp}
    n_proc = 0
    t0 = time.perf_counter()
    for s in range(args.steps):
        n_proc += sum(len(sp[k]["px"]) for k in sp)
        out = oracle.substep(ot, sp, dt=DT, seed=SEED, step=args.warmup + s)
        sp = {k: {c: out[k][c] for c in sp[k]} for k in sp}
    el = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    v = n_proc / el
    sample = f"{2 * m} particles per step of the same distribution (FP64 oracle, 256/256x256 oracle tables)"
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": headline_config(args.n, ws),
                      "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                                       "cpu": cpu_model(), "sample": sample},
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        reference_main(a)
    else:
        gpu_main(a)
