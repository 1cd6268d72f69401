"""Many patches in one sequence of launches (qed_substep_batched): every patch
ends exactly as qed_substep leaves it when run on that patch alone; the
launch-shape tuner leaves the particles untouched; and 20 steps captured in one
CUDA graph with a device step counter equal 20 eager steps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPECIES = ("electrons", "positrons", "photons")


@pytest.fixture(scope="module")
def api():
    from paper_2110_00256_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def tables(api):
    return api.qed_tables_generate(api.table_params(qs_n_chi=128, qs_n_xi=128, bw_n_chi=128, bw_n_xi=128))


def _host_patches(sizes, seed, tau_scale=3e-4):
    from paper_2110_00256_gb300 import workloads
    out = []
    for i, n in enumerate(sizes):
        d = {}
        for j, k in enumerate(SPECIES):
            m = n if k != "positrons" else n // 3
            h = workloads.paper_benchmark(m, seed + 10 * i + j, (3 * i + j) * 10 ** 9)
            h["tau"] *= tau_scale
            d[k] = h
        out.append(d)
    return out


def _device_patches(api, host, prec):
    out = []
    for h in host:
        p = {}
        for k in SPECIES:
            n = len(h[k]["px"])
            b = api.SpeciesBuffers(2 * n + 40, prec)
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


@pytest.mark.parametrize("prec_name", ["f32", "f64"])
def test_batched_equals_per_patch(api, tables, prec_name):
    prec = api.QED_F32 if prec_name == "f32" else api.QED_F64
    sizes = [1, 100, 1000, 5003, 33, 0, 20000, 777, 4096, 2]
    host = _host_patches(sizes, 7)
    ref = _device_patches(api, host, prec)
    bat = _device_patches(api, host, prec)
    s_ref, s_bat = api.Stats(), api.Stats()
    for p in ref:
        api.qed_substep(tables, p["electrons"], p["positrons"], p["photons"], 10.0, 3, 5, p["fire"], stats=s_ref)
    b = api.Batch(bat, prec)
    api.qed_substep_batched(tables, b, 10.0, 3, 5, api.make_opts(stats=s_bat))
    torch.cuda.synchronize()
    ref_stats, bat_stats = s_ref.as_dict(), s_bat.as_dict()
    # the batched call also counts the particles it evolved: every live particle once
    live = sum(len(h[k]["px"]) for h in host for k in SPECIES)
    assert ref_stats.pop("evolved") == 0 and bat_stats.pop("evolved") == live
    assert ref_stats == bat_stats
    assert bat_stats["qs_events"] > 0 and bat_stats["pairs"] > 0
    for pa, pb in zip(ref, bat):
        _assert_same(pa, pb)


def test_tuner_leaves_particles_untouched(api, tables):
    host = _host_patches([3000, 50, 12000], 11)
    bat = _device_patches(api, host, api.QED_F32)
    before = [{k: _sorted(p[k]) for k in SPECIES} for p in bat]
    b = api.Batch(bat, api.QED_F32)
    res = api.qed_tune_evolve(tables, b)
    torch.cuda.synchronize()
    # the default bulk-copy kernel (0, 0) or a direct-load shape
    assert (res["threads"], res["ctas_per_sm"]) == (0, 0) or \
        (res["threads"] in (128, 256, 512) and 1 <= res["ctas_per_sm"] <= 6)
    assert res["ms"] > 0
    for p, bf in zip(bat, before):
        for k in SPECIES:
            a = _sorted(p[k])
            for c in a:
                assert np.array_equal(a[c], bf[k][c]), (k, c)
    for p in bat:
        assert all(f.n() == 0 for f in p["fire"])


def test_graph_of_many_steps_equals_eager(api, tables):
    rng = np.random.default_rng(3)
    sizes = list((10 ** rng.uniform(1, 3.5, 12)).astype(int))
    # optical depths at their natural scale: over 20 steps a few percent fire,
    # so no destination fills up (the order of dropped events is not reproducible)
    host = _host_patches(sizes, 21, tau_scale=0.05)
    eager = _device_patches(api, host, api.QED_F32)
    graph = _device_patches(api, host, api.QED_F32)
    be, bg = api.Batch(eager, api.QED_F32), api.Batch(graph, api.QED_F32)
    steps = 20
    se = api.Stats()
    live_sum = 0
    for s in range(steps):
        # photons that decayed into pairs stay in the arrays (weight 0, tau = +inf) and are not counted
        live_sum += sum(int(p[k].count.item()) for p in eager for k in SPECIES) - se.as_dict()["pairs"]
        api.qed_substep_batched(tables, be, 10.0, 9, s, api.make_opts(stats=se))
    torch.cuda.synchronize()
    # the population grows with the photons and pairs appended; the counter follows it step by step
    assert se.as_dict()["pairs"] > 0
    assert se.as_dict()["evolved"] == live_sum > steps * sum(len(h[k]["px"]) for h in host for k in SPECIES)
    d_step = torch.zeros(1, dtype=torch.int64, device="cuda")
    sg = api.Stats()
    opts = api.make_opts(d_step=d_step, stats=sg)
    stream = torch.cuda.Stream()
    # first call outside the capture (sets the kernels' shared-memory limits)
    with torch.cuda.stream(stream):
        api.qed_substep_batched(tables, bg, 0.0, 9, 0, api.make_opts(), stream=stream)
    torch.cuda.synchronize()
    bg2 = api.Batch(graph, api.QED_F32)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            for _ in range(steps):
                api.qed_substep_batched(tables, bg2, 10.0, 9, 0, opts, stream=stream)
    # the dt = 0 warm-up call fired nothing and left the optical depths' values; replay the graph
    d_step.zero_()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        g.replay()
    torch.cuda.synchronize()
    assert int(d_step.item()) == steps
    assert sg.as_dict() == se.as_dict()
    for p in eager:
        for k in SPECIES:
            assert not np.any(_sorted(p[k])["id"] == np.uint64(0xFFFFFFFFFFFFFFFF))
    for pa, pb in zip(eager, graph):
        for k in SPECIES:
            a, b = _sorted(pa[k]), _sorted(pb[k])
            assert np.array_equal(a["id"], b["id"]), k
            for c in ("px", "py", "pz", "weight"):
                assert np.array_equal(a[c], b[c]), (k, c)
            ta = a["tau"].astype(np.float64) - a["tau_c"]
            tb = b["tau"].astype(np.float64) - b["tau_c"]
            fin = np.isfinite(ta)
            assert np.array_equal(fin, np.isfinite(tb))
            assert np.allclose(ta[fin], tb[fin], rtol=1e-6, atol=1e-12)


def test_batched_bulk_equals_direct_loads(api, tables):
    """The batched evolution's default for FP32 (bulk copies through shared
    memory, tiles of 1920 particles) against the direct-load kernel on patches
    of many tiles with ragged tails: the same bits, the same events."""
    sizes = [300_001, 1921, 1919, 0, 77_777, 5]
    host = _host_patches(sizes, 31, tau_scale=0.05)
    a = _device_patches(api, host, api.QED_F32)
    b = _device_patches(api, host, api.QED_F32)
    ba, bb = api.Batch(a, api.QED_F32), api.Batch(b, api.QED_F32)
    sa, sb = api.Stats(), api.Stats()
    for s in range(3):
        api.qed_substep_batched(tables, ba, 10.0, 4, s, api.make_opts(stats=sa))
        api.qed_substep_batched(tables, bb, 10.0, 4, s, api.make_opts(stats=sb, evolve_pipeline=api.QED_EVOLVE_DIRECT))
    torch.cuda.synchronize()
    assert sa.as_dict() == sb.as_dict() and sa.as_dict()["qs_events"] > 100
    assert sa.as_dict()["dropped_capacity"] == 0
    for pa, pb in zip(a, b):
        _assert_same(pa, pb)


def test_maximum_patch_count(api, tables):
    """QED_MAX_PATCHES patches (3072 segments: the largest shared-memory prefix
    of the batched kernels) of a few particles each: the bulk-copy evolution
    equals the direct-load one, every particle is counted once, and a second
    batch of the same patches one over the maximum is refused."""
    from paper_2110_00256_gb300 import _lib
    n_max = _lib.QED_MAX_PATCHES
    rng = np.random.default_rng(5)
    sizes = list(rng.integers(0, 9, n_max))
    host = _host_patches(sizes, 41, tau_scale=0.05)
    a = _device_patches(api, host, api.QED_F32)
    b = _device_patches(api, host, api.QED_F32)
    ba, bb = api.Batch(a, api.QED_F32), api.Batch(b, api.QED_F32)
    sa, sb = api.Stats(), api.Stats()
    api.qed_substep_batched(tables, ba, 10.0, 6, 0, api.make_opts(stats=sa))
    api.qed_substep_batched(tables, bb, 10.0, 6, 0, api.make_opts(stats=sb, evolve_pipeline=api.QED_EVOLVE_DIRECT))
    torch.cuda.synchronize()
    live = sum(len(h[k]["px"]) for h in host for k in SPECIES)
    assert sa.as_dict() == sb.as_dict() and sa.as_dict()["evolved"] == live
    for pa, pb in zip(a, b):
        _assert_same(pa, pb)
    with pytest.raises(api.QedError):
        api.Batch(a + a[:1], api.QED_F32)
