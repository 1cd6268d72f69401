"""The plane-wave push on the GPU against its FP64 reference (oracle/pusher.py),
the batched push against per-species pushes, and a short cascade (push +
substep, graph-captured with a device step counter) that keeps the total
light-front momentum sum(gamma - d p_x) of the plane wave's invariant."""
import math

import numpy as np
import pytest

from oracle import pusher as opush

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E0, OMEGA = 3.0328877982211224e-4, 3.0328877982211224e-6  # a0 = 100 at 0.8 um
DT = 2 * math.pi / OMEGA / 200


@pytest.fixture(scope="module")
def api():
    from paper_2110_00256_gb300 import api as a
    return a


def _species(api, n, prec, seed, photons=False):
    r = np.random.default_rng(seed)
    sp = api.SpeciesBuffers(n, prec, positions=True)
    p = r.normal(0, 300, (n, 3))
    p[:, 0] += 2000.0
    x = r.uniform(0, 2 * math.pi / OMEGA, n)
    sp.set({"px": p[:, 0], "py": p[:, 1], "pz": p[:, 2], "x": x, "y": r.uniform(-10, 10, n),
            "z": r.uniform(-10, 10, n), "tau": r.exponential(1.0, n), "weight": np.ones(n),
            "id": np.arange(n, dtype=np.uint64) + seed * 10 ** 6})
    return sp


@pytest.mark.parametrize("charge", [-1.0, 1.0, 0.0])
@pytest.mark.parametrize("circular", [False, True])
def test_push_fp64_matches_oracle(api, charge, circular):
    n = 3000
    sp = _species(api, n, api.QED_F64, 5)
    h = sp.to_host()
    pos = np.stack([h["x"], h["y"], h["z"]], 1)
    p = np.stack([h["px"], h["py"], h["pz"]], 1)
    w = api.plane_wave(E0, OMEGA, 0.3, circular)
    t = 0.0
    for step in range(40):
        api.qed_push_plane_wave(sp, charge, w, t, DT)
        E, B, p, pos = opush.push(pos, p, charge, t, DT, E0, OMEGA, 0.3, circular)
        t += DT
    torch.cuda.synchronize()
    g = sp.to_host()
    scale = np.linalg.norm(p, axis=1)
    for i, c in enumerate(("px", "py", "pz")):
        assert np.all(np.abs(g[c] - p[:, i]) <= 1e-10 * scale), c
    for i, c in enumerate(("x", "y", "z")):
        assert np.allclose(g[c], pos[:, i], rtol=1e-12, atol=1e-6), c
    for i, c in enumerate(("ex", "ey", "ez")):
        assert np.allclose(g[c], E[:, i], rtol=0, atol=1e-9 * E0), c
    for i, c in enumerate(("bx", "by", "bz")):
        assert np.allclose(g[c], B[:, i], rtol=0, atol=1e-9 * E0), c


def test_push_fp32_one_step(api):
    n = 5000
    sp = _species(api, n, api.QED_F32, 6)
    h = {k: v.astype(np.float64) for k, v in sp.to_host().items() if k != "id"}
    pos = np.stack([h["x"], h["y"], h["z"]], 1)
    p = np.stack([h["px"], h["py"], h["pz"]], 1)
    w = api.plane_wave(E0, OMEGA)
    api.qed_push_plane_wave(sp, -1.0, w, 123.0 * DT, DT)
    torch.cuda.synchronize()
    E, B, p2, pos2 = opush.push(pos, p, -1.0, 123.0 * DT, DT, E0, OMEGA)
    g = sp.to_host()
    scale = np.linalg.norm(p, axis=1)
    for i, c in enumerate(("px", "py", "pz")):
        assert np.all(np.abs(g[c] - p2[:, i]) <= 1e-5 * scale), c


def test_batched_push_equals_single(api):
    sizes = [10, 3000, 0, 777]
    pa, pb = [], []
    for i, n in enumerate(sizes):
        for lst in (pa, pb):
            d = {"electrons": _species(api, max(n, 1), api.QED_F32, 10 + i),
                 "positrons": _species(api, max(n // 2, 1), api.QED_F32, 20 + i),
                 "photons": _species(api, max(n, 1), api.QED_F32, 30 + i)}
            if n == 0:
                for k in d:
                    d[k].count.zero_()
            d["fire"] = [api.FireBuffers(d[k].capacity) for k in ("electrons", "positrons", "photons")]
            lst.append(d)
    w = api.plane_wave(E0, OMEGA, 0.1, True)
    b = api.Batch(pb, api.QED_F32)
    api.qed_push_batched(b, w, 5.0, DT, 7)
    for d in pa:
        for k, q in (("electrons", -1.0), ("positrons", 1.0), ("photons", 0.0)):
            api.qed_push_plane_wave(d[k], q, w, 5.0 + 7 * DT, DT)
    torch.cuda.synchronize()
    for da, db in zip(pa, pb):
        for k in ("electrons", "positrons", "photons"):
            a, bb = da[k].to_host(), db[k].to_host()
            for c in ("px", "py", "pz", "x", "y", "z", "ex", "ey", "bz"):
                assert np.array_equal(a[c], bb[c]), (k, c)


def test_cascade_conserves_light_front_momentum(api):
    """Electrons (gamma ~ 2000) against the a0 = 100 wave for one period: they
    emit many photons; push + substep keep sum(gamma + p_x) (wave along -x) up to
    the ultra-relativistic approximation of the emission (O(1/gamma^2))."""
    tabs = api.qed_tables_generate(api.table_params(qs_n_chi=128, qs_n_xi=128, bw_n_chi=128, bw_n_xi=128))
    n = 20000
    patches = []
    r = np.random.default_rng(3)
    for i in range(4):
        e = api.SpeciesBuffers(n + 4000, api.QED_F64, positions=True)
        gam = 2000.0 * (1 + 0.05 * (2 * r.uniform(size=n) - 1))
        e.set({"px": np.sqrt(gam ** 2 - 1), "py": np.zeros(n), "pz": np.zeros(n),
               "x": r.uniform(0, 2 * math.pi / OMEGA, n), "y": np.zeros(n), "z": np.zeros(n),
               "tau": r.exponential(1.0, n), "weight": np.ones(n), "id": np.arange(n, dtype=np.uint64) + i * 10 ** 7})
        pos = api.SpeciesBuffers(4000, api.QED_F64, positions=True)
        ph = api.SpeciesBuffers(40 * n, api.QED_F64, positions=True)
        patches.append({"electrons": e, "positrons": pos, "photons": ph,
                        "fire": [api.FireBuffers(e.capacity), api.FireBuffers(pos.capacity),
                                 api.FireBuffers(ph.capacity)]})

    def light_front():
        tot = 0.0
        for d in patches:
            for k in ("electrons", "positrons"):
                h = d[k].to_host()
                tot += np.sum(h["weight"] * (np.sqrt(1 + h["px"] ** 2 + h["py"] ** 2 + h["pz"] ** 2) + h["px"]))
            h = d["photons"].to_host()
            tot += np.sum(h["weight"] * (np.sqrt(h["px"] ** 2 + h["py"] ** 2 + h["pz"] ** 2) + h["px"]))
        return tot

    lf0 = light_front()
    b = api.Batch(patches, api.QED_F64)
    w = api.plane_wave(E0, OMEGA)
    d_step = torch.zeros(1, dtype=torch.int64, device="cuda")
    stats = api.Stats()
    opts = api.make_opts(stats=stats, d_step=d_step)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):  # first calls outside the capture
        api.qed_push_batched(b, w, 0.0, 0.0, 0, stream=stream)
        api.qed_substep_batched(tabs, b, 0.0, 1, 0, api.make_opts(), stream=stream)
    torch.cuda.synchronize()
    steps = 200
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            for _ in range(steps):
                api.qed_push_batched(b, w, 0.0, DT, 0, d_step, stream=stream)
                api.qed_substep_batched(tabs, b, DT, 1, 0, opts, stream=stream)
    with torch.cuda.stream(stream):
        g.replay()
    torch.cuda.synchronize()
    s = stats.as_dict()
    assert int(d_step.item()) == steps
    assert s["qs_events"] > 4 * n and s["dropped_capacity"] == 0 and s["nonfinite"] == 0
    lf1 = light_front()
    assert lf1 == pytest.approx(lf0, rel=1e-3), (lf0, lf1, s)


@pytest.mark.parametrize("charge", [-1.0, 1.0, 0.0])
def test_push_stored_fields_fp64_matches_oracle(api, charge):
    """Boris push in the fields stored with the particles (here random, a
    different field per particle), 30 steps, against oracle/pusher.boris; the
    fields are left untouched."""
    n = 4000
    r = np.random.default_rng(8)
    sp = _species(api, n, api.QED_F64, 9)
    E = r.uniform(-1e-3, 1e-3, (n, 3))
    B = r.uniform(-1e-3, 1e-3, (n, 3))
    h = sp.to_host()
    h.update({c: E[:, i] for i, c in enumerate(("ex", "ey", "ez"))})
    h.update({c: B[:, i] for i, c in enumerate(("bx", "by", "bz"))})
    sp.set(h)
    pos = np.stack([h["x"], h["y"], h["z"]], 1)
    p = np.stack([h["px"], h["py"], h["pz"]], 1)
    dt = 500.0
    for _ in range(30):
        api.qed_push_stored_fields(sp, charge, dt)
        if charge == 0:
            v = p / np.linalg.norm(p, axis=1, keepdims=True)
        else:
            p = opush.boris(p, E, B, charge, dt)
            v = p / np.sqrt(1 + np.sum(p * p, axis=1, keepdims=True))
        pos = pos + v * dt
    torch.cuda.synchronize()
    g = sp.to_host()
    scale = np.linalg.norm(p, axis=1)
    for i, c in enumerate(("px", "py", "pz")):
        assert np.all(np.abs(g[c] - p[:, i]) <= 1e-11 * scale), c
    for i, c in enumerate(("x", "y", "z")):
        assert np.allclose(g[c], pos[:, i], rtol=1e-12, atol=1e-6), c
    for i, c in enumerate(("ex", "ey", "ez")):
        assert np.array_equal(g[c], E[:, i]), c
    for i, c in enumerate(("bx", "by", "bz")):
        assert np.array_equal(g[c], B[:, i]), c


def _wave_patches(api, prec, sizes, seed):
    from paper_2110_00256_gb300 import workloads
    out = []
    r = np.random.default_rng(seed)
    for i, n in enumerate(sizes):
        d = {}
        for j, (k, m) in enumerate((("electrons", n), ("positrons", n // 3), ("photons", n))):
            h = workloads.paper_benchmark(m, seed + 10 * i + j, (3 * i + j) * 10 ** 9)
            for c in ("ex", "ey", "ez", "bx", "by", "bz"):
                h[c] = np.zeros(m)
            h.update(x=r.uniform(0, 2 * math.pi / OMEGA, m), y=r.uniform(-1, 1, m), z=r.uniform(-1, 1, m))
            # room for every event (which events run when a destination fills up
            # depends on the order of the firing lists)
            b = api.SpeciesBuffers(m + 8 * n + 64, prec, positions=True)
            if m:
                b.set(h)
            d[k] = b
        d["fire"] = [api.FireBuffers(d[k].capacity) for k in ("electrons", "positrons", "photons")]
        out.append(d)
    return out


@pytest.mark.parametrize("store_fields", [False, True])
@pytest.mark.parametrize("prec_name", ["f32", "f64"])
def test_fused_push_substep_equals_separate(api, prec_name, store_fields):
    """qed_push_substep_batched (push fused into the evolution) against
    qed_push_batched + qed_substep_batched, 12 steps of a circularly polarised
    a0 = 100 wave on patches of uneven size: every particle ends with the same
    bits (the fields too when the fused call stores them)."""
    prec = api.QED_F32 if prec_name == "f32" else api.QED_F64
    tabs = api.qed_tables_generate(api.table_params(qs_n_chi=128, qs_n_xi=128, bw_n_chi=128, bw_n_xi=128))
    sizes = [1, 700, 5003, 0, 20000, 33]
    sep, fus = _wave_patches(api, prec, sizes, 4), _wave_patches(api, prec, sizes, 4)
    bs, bf = api.Batch(sep, prec), api.Batch(fus, prec)
    w = api.plane_wave(E0, OMEGA, 0.2, True)
    ss, sf = api.Stats(), api.Stats()
    for k in range(12):
        api.qed_push_batched(bs, w, 3.0, DT, k)
        api.qed_substep_batched(tabs, bs, DT, 17, k, api.make_opts(stats=ss))
        api.qed_push_substep_batched(tabs, bf, w, 3.0, DT, 17, k, api.make_opts(stats=sf), store_fields=store_fields)
    torch.cuda.synchronize()
    assert ss.as_dict()["dropped_capacity"] == 0 and sf.as_dict()["dropped_capacity"] == 0
    assert ss.as_dict() == sf.as_dict() and sf.as_dict()["qs_events"] > 1000
    cols = ("px", "py", "pz", "x", "y", "z", "tau", "tau_c", "weight", "id")
    if store_fields:
        cols += ("ex", "ey", "ez", "bx", "by", "bz")
    for a, b in zip(sep, fus):
        for k in ("electrons", "positrons", "photons"):
            ha, hb = a[k].to_host(), b[k].to_host()
            oa, ob = np.argsort(ha["id"], kind="stable"), np.argsort(hb["id"], kind="stable")
            for c in cols:
                if c in ha:
                    assert np.array_equal(ha[c][oa], hb[c][ob]), (k, c)
