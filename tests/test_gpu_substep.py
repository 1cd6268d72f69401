"""GPU parity of the whole substep (evolution of electrons, positrons, photons;
pair production; photon emission; appended secondaries) against the FP64
oracle from identical seeded state, FP64 and FP32; capacity overflow; the
photon keep-threshold; CUDA-graph capture; and the 10^8-particle FP32 workload
checked on a sampled subset of particles."""
import numpy as np
import pytest

import oracle
from helpers import (FIELDS, as_f64, check_substep_by_event, compare_states as _compare, gpu_tables,
                     margin_ids as _margin_ids, sort_by_id, tau_bound, tau_eff)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPECIES = ("electrons", "positrons", "photons")


@pytest.fixture(scope="module")
def api():
    from paper_2110_00256_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def tabs(api, oracle_tables_256):
    return oracle_tables_256, gpu_tables(api, oracle_tables_256)


def _inputs(n, seed, tau_scale=2e-4, n_pos=None):
    from paper_2110_00256_gb300 import workloads
    d = {"electrons": workloads.paper_benchmark(n, seed, 0),
         "positrons": workloads.paper_benchmark(n if n_pos is None else n_pos, seed + 1, 10 ** 12),
         "photons": workloads.paper_benchmark(n, seed + 2, 2 * 10 ** 12)}
    for v in d.values():
        v["tau"] *= tau_scale
    return d


def _run_gpu(api, t, host, prec, dt, seed, step, extra=3.0, threshold=0.0, caps=None, cuts=(0.0, 0.0)):
    bufs, fire = {}, []
    for k in SPECIES:
        n = len(host[k]["px"])
        cap = caps[k] if caps else int(n * extra) + 64
        b = api.SpeciesBuffers(cap, prec)
        if n:
            b.set(host[k])
        bufs[k] = b
        fire.append(api.FireBuffers(cap))
    stats = api.Stats()
    api.qed_substep(t, bufs["electrons"], bufs["positrons"], bufs["photons"], dt, seed, step, fire,
                    photon_threshold=threshold, stats=stats, qs_chi_cut=cuts[0], bw_chi_cut=cuts[1])
    torch.cuda.synchronize()
    return {k: bufs[k].to_host() for k in SPECIES}, stats.as_dict(), fire


def test_substep_fp64_parity(api, tabs):
    ot, t = tabs
    host = _inputs(100_000, 11)
    h64 = {k: as_f64(v, np.float64) for k, v in host.items()}
    got, st, _ = _run_gpu(api, t, host, api.QED_F64, dt=10.0, seed=99, step=3)
    ref = oracle.substep(ot, h64, dt=10.0, seed=99, step=3)
    assert st["qs_events"] > 100 and st["pairs"] > 100
    assert st["dropped_capacity"] == 0 and st["nonfinite"] == 0
    assert ref["n_new"]["photons"] == st["photons_kept"]
    assert ref["n_new"]["electrons"] == st["pairs"]
    excl = _margin_ids(ot, h64, 10.0, 1e-12, 99, 3)
    assert len(excl) <= 9
    _compare(got, ref, False, 1e-12, exclude=excl)


def test_substep_chi_cuts_fp64_parity(api, tabs):
    """With chi cut-offs for both processes, particles below them keep their
    optical depth bit for bit and never fire; the rest matches the oracle."""
    ot, t = tabs
    cuts = (15.0, 20.0)
    host = _inputs(60_000, 13)
    h64 = {k: as_f64(v, np.float64) for k, v in host.items()}
    got, st, _ = _run_gpu(api, t, host, api.QED_F64, dt=10.0, seed=98, step=4, cuts=cuts)
    ref = oracle.substep(ot, h64, dt=10.0, seed=98, step=4, qs_chi_cut=cuts[0], bw_chi_cut=cuts[1])
    assert st["qs_events"] > 100 and st["pairs"] > 10 and st["dropped_capacity"] == 0
    for k, proc in (("electrons", 0), ("positrons", 0), ("photons", 1)):
        _, chi, _, f = oracle.evolve(proc, ot, h64[k], 10.0, cuts[proc])
        below = chi < cuts[proc] * (1 - 1e-9)
        assert 0.2 < below.mean() < 0.9 and not f[below].any()
        g = got[k]
        n = len(h64[k]["id"])
        assert np.array_equal(g["id"][:n], h64[k]["id"])
        assert np.array_equal(g["tau"][:n][below], h64[k]["tau"][below])
    excl = _margin_ids(ot, h64, 10.0, 1e-12, 98, 4, cuts)
    _compare(got, ref, False, 1e-12, exclude=excl)


def test_substep_fp32_parity(api, tabs):
    ot, t = tabs
    host = _inputs(50_000, 21)
    h32 = {k: as_f64(v, np.float32) for k, v in host.items()}
    got, st, fire = _run_gpu(api, t, host, api.QED_F32, dt=10.0, seed=7, step=1)
    fl = {k: (f.idx[:f.n()].cpu().numpy(), f.chi[:f.n()].cpu().numpy()) for k, f in zip(SPECIES, fire)}
    rep = check_substep_by_event(ot, h32, got, fl, 10.0, 7, 1)
    assert rep["events"] > 200
    assert st["dropped_capacity"] == 0 and st["nonfinite"] == 0
    print("fp32 substep:", rep)


@pytest.mark.parametrize("prec_name", ["f64", "f32"])
def test_substep_every_particle_fires(api, tabs, prec_name):
    """Optical depths of order 1e-12, so that nearly every particle fires (as
    in the paper's per-kernel benchmark of emission and pair production): 4e4
    emissions and 2e4 pair productions in one step, checked event by event
    against the oracle: the chi of the firing list, every sample by its backward
    error at the GPU's chi, energy and direction of the products, the optical
    depths drawn for parents and children, fields and weights copied.  (With
    every particle firing, the small-chi ones included, the FP64 chi of many
    events differ from the oracle's within the cancellation bound of a
    difference of squares, and a sampled xi inherits that; a forward
    comparison of the products would measure the chi, not the sampling.)"""
    ot, t = tabs
    host = _inputs(20_000, 41, tau_scale=1e-12)
    prec = api.QED_F64 if prec_name == "f64" else api.QED_F32
    hp = {k: as_f64(v, np.float64 if prec_name == "f64" else np.float32) for k, v in host.items()}
    got, st, fire = _run_gpu(api, t, host, prec, dt=10.0, seed=5, step=2, extra=4.0)
    fl = {k: (f.idx[:f.n()].cpu().numpy(), f.chi[:f.n()].cpu().numpy()) for k, f in zip(SPECIES, fire)}
    rep = check_substep_by_event(ot, hp, got, fl, 10.0, 5, 2, fp64=prec_name == "f64")
    print(f"{prec_name} all-fire substep:", rep)
    assert rep["events"] > 55_000
    assert st["qs_events"] > 35_000 and st["pairs"] > 15_000
    assert st["dropped_capacity"] == 0 and st["nonfinite"] == 0


def test_substep_fp64_config1_with_events(api):
    """The 10^4-electron FP64 case (static B = 0.01 along z, gamma = 10^(2 + 2U),
    isotropic, 64-point tables) with dt = 10 instead of 1e-3, so that photons
    are emitted (~370 emissions over the 100 steps; the photons' chi stays far
    below pair production's): every step of the whole substep against the
    oracle run from the GPU's own pre-step state (decisions within the error
    bound excluded)."""
    from paper_2110_00256_gb300 import workloads
    ot = oracle.tables(qs_n_chi=64, qs_n_xi=64, bw_n_chi=64, bw_n_xi=64)
    t = gpu_tables(api, ot)
    beam = workloads.isotropic_beam(10_000, 0)
    empty = {k: v[:0] for k, v in beam.items()}
    bufs = {"electrons": api.SpeciesBuffers(20_000, api.QED_F64).set(beam),
            "positrons": api.SpeciesBuffers(10_000, api.QED_F64),
            "photons": api.SpeciesBuffers(20_000, api.QED_F64)}
    fire = [api.FireBuffers(20_000) for _ in SPECIES]
    events = 0
    for step in range(100):
        pre = {k: bufs[k].to_host() for k in SPECIES}
        pre = {k: {kk: (v.astype(np.uint64) if kk == "id" else v) for kk, v in pre[k].items()
                   if kk in empty} for k in SPECIES}
        stats = api.Stats()
        api.qed_substep(t, bufs["electrons"], bufs["positrons"], bufs["photons"], 10.0, 11, step, fire,
                        stats=stats)
        torch.cuda.synchronize()
        ref = oracle.substep(ot, pre, dt=10.0, seed=11, step=step)
        got = {k: bufs[k].to_host() for k in SPECIES}
        excl = _margin_ids(ot, pre, 10.0, 1e-12, 11, step)
        _compare(got, ref, False, 1e-12, exclude=excl)
        st = stats.as_dict()
        events += st["qs_events"] + st["bw_events"]
    print("config-1 beam with dt = 10: events over 100 steps", events)
    assert events > 100


def test_energy_conservation_and_threshold(api, tabs):
    ot, t = tabs
    host = _inputs(50_000, 31)
    got, st, _ = _run_gpu(api, t, host, api.QED_F64, dt=10.0, seed=3, step=0, threshold=0.0)

    def energy(s):
        e = 0.0
        for k in ("electrons", "positrons"):
            d = s[k]
            e += np.sum(d["weight"] * np.sqrt(1 + d["px"] ** 2 + d["py"] ** 2 + d["pz"] ** 2))
        d = s["photons"]
        return e + np.sum(d["weight"] * np.sqrt(d["px"] ** 2 + d["py"] ** 2 + d["pz"] ** 2))

    h64 = {k: as_f64(v, np.float64) for k, v in host.items()}
    assert energy(got) == pytest.approx(energy(h64), rel=1e-12)
    # with the keep-threshold (§5) photons below 2 m_e c^2 are discarded, leptons still recoil
    got2, st2, _ = _run_gpu(api, t, host, api.QED_F64, dt=10.0, seed=3, step=0, threshold=2.0)
    ref2 = oracle.substep(ot, h64, dt=10.0, seed=3, step=0, photon_threshold=2.0)
    assert st2["photons_discarded"] > 0
    assert st2["photons_kept"] + st2["photons_discarded"] == st2["qs_events"]
    assert len(got2["photons"]["px"]) == len(ref2["photons"]["px"])


def test_capacity_overflow_leaves_events_for_next_step(api, tabs):
    ot, t = tabs
    n = 20_000
    host = _inputs(n, 41, tau_scale=1e-3)
    caps = {"electrons": n + 5, "positrons": n + 5, "photons": n + 7}
    got, st, _ = _run_gpu(api, t, host, api.QED_F64, dt=10.0, seed=5, step=0, caps=caps)
    for k in SPECIES:
        assert len(got[k]["px"]) <= caps[k]
    assert st["dropped_capacity"] > 0
    # every event either ran or left its parent untouched with tau < 0
    h64 = {k: as_f64(v, np.float64) for k, v in host.items()}
    ref = oracle.substep(ot, h64, dt=10.0, seed=5, step=0)
    fired_e = ref["fire"]["electrons"].sum()
    e = sort_by_id(got["electrons"])
    e0 = e["id"] < n
    still_neg = (e["tau"][e0] < 0).sum()
    assert st["qs_events"] + st["dropped_capacity"] >= fired_e
    assert still_neg > 0
    # placeholders written into partially reserved slots are removed particles
    for k in ("electrons", "positrons"):
        d = got[k]
        dead = d["id"] == np.uint64(0xFFFFFFFFFFFFFFFF)
        assert np.all(d["weight"][dead] == 0) and np.all(np.isinf(d["tau"][dead]))


def test_substep_graph_capture_matches_eager(api, tabs):
    ot, t = tabs
    host = _inputs(30_000, 51)
    eager, _, _ = _run_gpu(api, t, host, api.QED_F32, dt=10.0, seed=8, step=4)
    bufs, fire = {}, []
    for k in SPECIES:
        b = api.SpeciesBuffers(3 * 30_000 + 64, api.QED_F32).set(host[k])
        bufs[k] = b
        fire.append(api.FireBuffers(3 * 30_000 + 64))
    call = api.SubstepCall(t, bufs["electrons"], bufs["positrons"], bufs["photons"], fire, 10.0, 8)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            call(4, stream=s)
    g.replay()
    torch.cuda.synchronize()
    for k in SPECIES:
        a, b = sort_by_id(eager[k]), sort_by_id(bufs[k].to_host())
        assert np.array_equal(a["id"], b["id"])
        for c in ("px", "py", "pz", "tau", "tau_c"):
            assert np.array_equal(a[c], b[c]), (k, c)


def test_full_size_fp32_workload_sampled(api, tabs):
    """10^8 particles (5e7 electrons + 5e7 photons, the paper's §4 distribution),
    one FP32 substep in the benchmark's launch configuration; 2e5 sampled
    particles are recomputed by the oracle from their pre-step state."""
    from paper_2110_00256_gb300 import workloads
    ot, t = tabs
    n = 50_000_000
    dev = {"electrons": workloads.paper_benchmark_torch(n, 1, 0),
           "photons": workloads.paper_benchmark_torch(n, 2, 2 * 10 ** 12)}
    extra = 2_000_000
    bufs = {}
    for k, d in dev.items():
        b = api.SpeciesBuffers(n + extra, api.QED_F32)
        for c, v in d.items():
            b.arrays[c][:n].copy_(v)
        b.count.fill_(n)
        bufs[k] = b
    bufs["positrons"] = api.SpeciesBuffers(extra, api.QED_F32)
    del dev
    fire = [api.FireBuffers(bufs[k].capacity) for k in SPECIES]
    idx = workloads.subsample_ids(n, 200_000, 5)
    ti = torch.as_tensor(idx, device="cuda")
    pre = {k: {c: bufs[k].arrays[c][ti].cpu().numpy() for c in FIELDS + ("tau", "tau_c", "weight", "id")}
           for k in ("electrons", "photons")}
    stats = api.Stats()
    api.qed_substep(t, bufs["electrons"], bufs["positrons"], bufs["photons"], 10.0, 77, 0, fire, stats=stats)
    torch.cuda.synchronize()
    st = stats.as_dict()
    assert st["nonfinite"] == 0 and st["dropped_capacity"] == 0 and st["fire_overflow"] == 0
    assert st["qs_events"] > 0 and st["pairs"] > 0
    for k, proc in (("electrons", 0), ("photons", 1)):
        p = {c: v.astype(np.float64) if c != "id" else v.view(np.uint64) for c, v in pre[k].items()}
        tau_new, chi, rate, f = oracle.evolve(proc, ot, p, 10.0)
        bound = tau_bound(ot, proc, p, chi, rate, 10.0, 1e-5)
        post_tau = bufs[k].arrays["tau"][ti].cpu().double().numpy() - bufs[k].arrays["tau_c"][ti].cpu().double().numpy()
        fl = fire[0 if k == "electrons" else 2]
        gpu_fired = np.isin(idx, fl.idx[:fl.n()].cpu().numpy())
        assert np.all(np.abs(tau_new[gpu_fired != f]) <= bound[gpu_fired != f])
        quiet = ~f & ~gpu_fired
        assert np.all(np.abs(post_tau[quiet] - tau_new[quiet]) <= bound[quiet]), k
        assert f.sum() > 0


@pytest.mark.parametrize("variant", [(2, 0, 0), (2, 512, 0), (2, 0, 2), (1, 0, 3)],
                         ids=["bulk8w4s", "bulk16w2s", "bulk8w2sx2", "direct3cta"])
def test_evolution_variants_equal_direct_loads(api, tabs, variant):
    """Every variant of the evolution kernel (bulk copies into shared memory,
    three CTAs per SM) gives the same bits as the default direct loads (four
    CTAs per SM): the same particles fire with the same chi, and every particle
    (secondaries included) ends identical.  Sizes give full tiles, a ragged
    tail, and a species smaller than one tile.  Every destination has room for
    every event (which events run when one fills up depends on the order of the
    firing list)."""
    _, t = tabs
    pipe_v, threads, ctas = variant
    host = _inputs(600_003, 41, n_pos=1000)  # more tiles than the grid has CTAs
    host["photons"] = _inputs(70_001, 42)["photons"]
    out = {}
    for key, (pipe, th, ct) in (("ref", (api.QED_EVOLVE_DIRECT, 0, 0)), ("var", (pipe_v, threads, ctas))):
        bufs, fire = {}, []
        for k in SPECIES:
            n = len(host[k]["px"])
            b = api.SpeciesBuffers(n + 700_000, api.QED_F32)
            b.set(host[k])
            bufs[k] = b
            fire.append(api.FireBuffers(b.capacity))
        stats = api.Stats()
        api.qed_substep(t, bufs["electrons"], bufs["positrons"], bufs["photons"], 10.0, 5, 2, fire, stats=stats,
                        pipeline=pipe, threads=th, ctas_per_sm=ct)
        torch.cuda.synchronize()
        fl = []
        for f in fire:
            i, c = f.idx[:f.n()].cpu().numpy(), f.chi[:f.n()].cpu().numpy()
            o = np.argsort(i)
            fl.append((i[o], c[o]))
        out[key] = ({k: sort_by_id(bufs[k].to_host()) for k in SPECIES}, stats.as_dict(), fl)
    (da, sa, fa), (db, sb, fb) = out["ref"], out["var"]
    assert sa == sb and sb["wait_timeout"] == 0 and sb["dropped_capacity"] == 0
    assert sb["qs_events"] > 100 and sb["pairs"] > 10
    for (ia, ca), (ib, cb) in zip(fa, fb):
        assert np.array_equal(ia, ib) and np.array_equal(ca, cb)
    for k in SPECIES:
        for c in da[k]:
            assert np.array_equal(da[k][c], db[k][c]), (k, c)


def test_full_size_batched_workload_sampled(api, tabs):
    """The many-patch workload at full size (64 patches of round(10^(3+4U))
    particles, seed 7: 6.4e7 in all, half electrons, half photons), one FP32
    batched substep in the benchmark's configuration (the bulk-copy evolution
    over device-resident segments); 2000 sampled particles of each of 8 patches
    are recomputed by the oracle from their pre-step state."""
    from paper_2110_00256_gb300 import workloads
    ot, t = tabs
    sizes = workloads.patch_counts(64, 7)
    patches, picks, off = [], [], 0
    order = np.argsort(sizes)[::-1]
    sampled = set(order[:4].tolist()) | set(order[30:34].tolist())  # the largest and some mid-sized
    for i, c in enumerate(sizes):
        c = int(c)
        p = {}
        for k, m, s in (("electrons", c // 2, 1), ("photons", c - c // 2, 2)):
            b = api.SpeciesBuffers(m + max(256, m // 20), api.QED_F32)
            d = workloads.paper_benchmark_torch(m, 100 * i + s, off, dtype=torch.float32)
            for col, v in d.items():
                b.arrays[col][:m].copy_(v)
            del d
            b.count.fill_(m)
            off += m
            p[k] = b
        p["positrons"] = api.SpeciesBuffers(max(256, c // 20), api.QED_F32)
        p["fire"] = [api.FireBuffers(p[k].capacity) for k in SPECIES]
        patches.append(p)
        if i in sampled:
            for k, proc in (("electrons", 0), ("photons", 1)):
                n = int(p[k].count.item())
                idx = workloads.subsample_ids(n, min(n, 2000), 11 + i)
                ti = torch.as_tensor(idx, device="cuda")
                pre = {col: p[k].arrays[col][ti].cpu().numpy() for col in FIELDS + ("tau", "tau_c", "weight", "id")}
                picks.append((i, k, proc, idx, ti, pre))
    b = api.Batch(patches, api.QED_F32)
    stats = api.Stats()
    api.qed_substep_batched(t, b, 10.0, 77, 0, api.make_opts(stats=stats))
    torch.cuda.synchronize()
    st = stats.as_dict()
    assert st["nonfinite"] == 0 and st["dropped_capacity"] == 0 and st["fire_overflow"] == 0
    assert st["evolved"] == int(sizes.sum()) and st["qs_events"] > 0
    fired_total = 0
    for i, k, proc, idx, ti, pre in picks:
        p = {c: v.astype(np.float64) if c != "id" else v.view(np.uint64) for c, v in pre.items()}
        tau_new, chi, rate, f = oracle.evolve(proc, ot, p, 10.0)
        bound = tau_bound(ot, proc, p, chi, rate, 10.0, 1e-5)
        arr = patches[i][k].arrays
        post_tau = arr["tau"][ti].cpu().double().numpy() - arr["tau_c"][ti].cpu().double().numpy()
        fl = patches[i]["fire"][0 if k == "electrons" else 2]
        gpu_fired = np.isin(idx, fl.idx[:fl.n()].cpu().numpy())
        assert np.all(np.abs(tau_new[gpu_fired != f]) <= bound[gpu_fired != f]), (i, k)
        quiet = ~f & ~gpu_fired
        assert np.all(np.abs(post_tau[quiet] - tau_new[quiet]) <= bound[quiet]), (i, k)
        fired_total += int(f.sum())
    assert fired_total > 0
