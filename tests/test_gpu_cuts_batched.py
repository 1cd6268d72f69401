"""The chi cut-offs of both processes and the photon keep-threshold (§5: what
a PIC code such as WarpX applies around the substep) through the many-patch
paths: qed_substep_batched and qed_push_substep_batched, eager and replayed
from a CUDA graph, must leave every patch exactly as qed_substep (or the
separate push + substep) leaves it with the same options, and must match the
oracle's substep with the same cut-offs and threshold (FP64, element by
element, decisions within the error bound of a cut or of zero excluded)."""
import math

import numpy as np
import pytest

import oracle
from helpers import as_f64, compare_states, gpu_tables, margin_ids

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPECIES = ("electrons", "positrons", "photons")
CUTS = (15.0, 20.0)      # chi below which leptons do not emit / photons do not decay
THRESHOLD = 150.0        # photons with gamma_g below this (m_e c^2) are not kept
DT = 10.0


@pytest.fixture(scope="module")
def api():
    from paper_2110_00256_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def tabs(api, oracle_tables_256):
    return oracle_tables_256, gpu_tables(api, oracle_tables_256)


def _host_patches(sizes, seed, tau_scale=3e-4, positions=False):
    from paper_2110_00256_gb300 import workloads
    out = []
    r = np.random.default_rng(seed)
    for i, n in enumerate(sizes):
        d = {}
        for j, k in enumerate(SPECIES):
            m = n if k != "positrons" else n // 3
            h = workloads.paper_benchmark(m, seed + 10 * i + j, (3 * i + j) * 10 ** 9)
            h["tau"] *= tau_scale
            if positions:
                h.update(x=r.uniform(0, 50.0, m), y=r.uniform(-1, 1, m), z=r.uniform(-1, 1, m))
            d[k] = h
        out.append(d)
    return out


def _device_patches(api, host, prec, positions=False):
    # room for every event: which events run when a destination fills up depends
    # on the order of the firing lists, which differs between launch forms
    out = []
    for h in host:
        p = {}
        big = 8 * max(len(h[k]["px"]) for k in SPECIES) + 64
        for k in SPECIES:
            n = len(h[k]["px"])
            b = api.SpeciesBuffers(n + big, prec, positions=positions)
            if n:
                b.set(h[k])
            p[k] = b
        p["fire"] = [api.FireBuffers(p[k].capacity) for k in SPECIES]
        out.append(p)
    return out


def _sorted(b):
    h = b.to_host()
    o = np.argsort(h["id"], kind="stable")
    return {k: v[o] for k, v in h.items()}


def _assert_same(pa, pb):
    for k in SPECIES:
        a, b = _sorted(pa[k]), _sorted(pb[k])
        assert np.array_equal(a["id"], b["id"]), k
        for c in a:
            assert np.array_equal(a[c], b[c]), (k, c)


def _opts(api, stats, cuts=CUTS, **kw):
    return api.make_opts(photon_threshold=THRESHOLD, stats=stats, qs_chi_cut=cuts[0], bw_chi_cut=cuts[1], **kw)


@pytest.mark.parametrize("prec_name", ["f32", "f64"])
def test_batched_cuts_equal_per_patch_eager_and_graph(api, tabs, prec_name):
    """Three steps: per-patch qed_substep, one qed_substep_batched per step,
    and the same three steps captured in one graph (device step counter)."""
    _, t = tabs
    prec = api.QED_F32 if prec_name == "f32" else api.QED_F64
    sizes = [1, 900, 5003, 0, 20000, 37, 4096]
    host = _host_patches(sizes, 5)
    ref, bat, gra = (_device_patches(api, host, prec) for _ in range(3))
    s_ref, s_bat, s_gra = api.Stats(), api.Stats(), api.Stats()
    b = api.Batch(bat, prec)
    steps = 3
    for s in range(steps):
        for p in ref:
            api.qed_substep(t, p["electrons"], p["positrons"], p["photons"], DT, 41, s, p["fire"],
                            photon_threshold=THRESHOLD, stats=s_ref, qs_chi_cut=CUTS[0], bw_chi_cut=CUTS[1])
        api.qed_substep_batched(t, b, DT, 41, s, _opts(api, s_bat))
    torch.cuda.synchronize()
    # the graph: warm-up call outside the capture on a throwaway batch (dt = 0 changes nothing)
    d_step = torch.zeros(1, dtype=torch.int64, device="cuda")
    bg = api.Batch(gra, prec)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        api.qed_substep_batched(t, bg, 0.0, 41, 0, _opts(api, None), stream=stream)
    torch.cuda.synchronize()
    for p in gra:  # the dt = 0 call fired nothing, but give the graph the same starting state
        for f in p["fire"]:
            f.count.zero_()
    og = _opts(api, s_gra, d_step=d_step)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            for _ in range(steps):
                api.qed_substep_batched(t, bg, DT, 41, 0, og, stream=stream)
    d_step.zero_()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        g.replay()
    torch.cuda.synchronize()
    assert int(d_step.item()) == steps
    sr, sb, sg = s_ref.as_dict(), s_bat.as_dict(), s_gra.as_dict()
    sb.pop("evolved"), sg.pop("evolved"), sr.pop("evolved")
    assert sr == sb == sg
    assert sr["qs_events"] > 100 and sr["pairs"] > 10 and sr["photons_discarded"] > 10
    assert sr["photons_kept"] > 10 and sr["dropped_capacity"] == 0
    for pa, pb, pc in zip(ref, bat, gra):
        _assert_same(pa, pb)
        _assert_same(pa, pc)


def test_batched_cuts_match_oracle_fp64(api, tabs):
    """One batched FP64 step with both cut-offs and the threshold, every patch
    against oracle.substep with the same options."""
    ot, t = tabs
    sizes = [3000, 17, 12000, 1]
    host = _host_patches(sizes, 9)
    dev = _device_patches(api, host, api.QED_F64)
    st = api.Stats()
    api.qed_substep_batched(t, api.Batch(dev, api.QED_F64), DT, 77, 2, _opts(api, st))
    torch.cuda.synchronize()
    s = st.as_dict()
    assert s["qs_events"] > 50 and s["pairs"] > 5 and s["photons_discarded"] > 5
    n_below = 0
    for h, p in zip(host, dev):
        h64 = {k: as_f64(v, np.float64) for k, v in h.items()}
        ref = oracle.substep(ot, h64, dt=DT, seed=77, step=2, photon_threshold=THRESHOLD,
                             qs_chi_cut=CUTS[0], bw_chi_cut=CUTS[1])
        got = {k: p[k].to_host() for k in SPECIES}
        for k, proc in (("electrons", 0), ("positrons", 0), ("photons", 1)):
            n = len(h64[k]["id"])
            if not n:
                continue
            _, chi, _, _ = oracle.evolve(proc, ot, h64[k], DT, CUTS[proc])
            below = chi < CUTS[proc] * (1 - 1e-9)
            n_below += int(below.sum())
            # below the cut: the optical depth is kept bit for bit
            assert np.array_equal(got[k]["tau"][:n][below], h64[k]["tau"][below])
            assert not ref["fire"][k][below].any()
        excl = margin_ids(ot, h64, DT, 1e-12, 77, 2, CUTS)
        compare_states(got, ref, False, 1e-12, exclude=excl)
    assert n_below > 1000


OMEGA = 2.0 * math.pi * 2.426e-12 / 0.8e-6  # hbar omega / (m_e c^2) of a 0.8 um wave: 3.03e-6
E0 = 100.0 * OMEGA                            # a0 = 100
WAVE_CUTS = (0.6, 0.4)                        # chi ~ 0.1 .. 3 for these particles in this wave


def test_fused_push_substep_cuts_equal_separate_and_oracle(api, tabs):
    """qed_push_substep_batched with the cut-offs and threshold equals
    qed_push_batched + qed_substep_batched bit for bit over four steps; the
    separate form's substep, from its pushed state, matches the oracle (FP64)."""
    ot, t = tabs
    prec = api.QED_F64
    sizes = [2500, 0, 9000, 3]
    host = _host_patches(sizes, 13, positions=True)
    r = np.random.default_rng(2)
    for h in host:  # the wave supplies the fields: start from zero stored fields, spread over one wavelength
        for d in h.values():
            for c in ("ex", "ey", "ez", "bx", "by", "bz"):
                d[c] = np.zeros(len(d["px"]))
            d["x"] = r.uniform(0.0, 2.0 * math.pi / OMEGA, len(d["px"]))
    sep, fus = _device_patches(api, host, prec, True), _device_patches(api, host, prec, True)
    bs, bf = api.Batch(sep, prec), api.Batch(fus, prec)
    w = api.plane_wave(E0, OMEGA, 0.3, False)
    ss, sf = api.Stats(), api.Stats()
    for k in range(4):
        api.qed_push_batched(bs, w, 1.0, 1.0e4, k)
        if k == 3:  # the pushed state before the last substep: the oracle's input
            torch.cuda.synchronize()
            pre = [{kk: p[kk].to_host() for kk in SPECIES} for p in sep]
        api.qed_substep_batched(t, bs, 1.0e4, 23, k, _opts(api, ss, WAVE_CUTS))
        api.qed_push_substep_batched(t, bf, w, 1.0, 1.0e4, 23, k, _opts(api, sf, WAVE_CUTS), store_fields=True)
    torch.cuda.synchronize()
    a, b = ss.as_dict(), sf.as_dict()
    assert a == b and a["dropped_capacity"] == 0
    assert a["qs_events"] > 100 and a["photons_discarded"] > 10
    for pa, pb in zip(sep, fus):
        _assert_same(pa, pb)
    cols = ("px", "py", "pz", "ex", "ey", "ez", "bx", "by", "bz", "tau", "weight", "id")
    n_below, n_above = [0, 0], [0, 0]
    for h, p in zip(pre, sep):
        h64 = {k: {c: (v[c] if c == "id" else v[c].astype(np.float64)) for c in cols} for k, v in h.items()}
        if not sum(len(v["id"]) for v in h64.values()):
            continue
        ref = oracle.substep(ot, h64, dt=1.0e4, seed=23, step=3, photon_threshold=THRESHOLD,
                             qs_chi_cut=WAVE_CUTS[0], bw_chi_cut=WAVE_CUTS[1])
        for k, proc in (("electrons", 0), ("positrons", 0), ("photons", 1)):
            if len(h64[k]["id"]):
                chi = oracle.evolve(proc, ot, h64[k], 1.0e4, WAVE_CUTS[proc])[1]
                n_below[proc] += int((chi < WAVE_CUTS[proc]).sum())
                n_above[proc] += int((chi >= WAVE_CUTS[proc]).sum())
        got = {k: {c: v for c, v in p[k].to_host().items() if c in cols} for k in SPECIES}
        excl = margin_ids(ot, h64, 1.0e4, 1e-12, 23, 3, WAVE_CUTS)
        compare_states(got, ref, False, 1e-12, exclude=excl)
    # both sides of both cut-offs are populated
    assert min(n_below) > 100 and min(n_above) > 100, (n_below, n_above)
