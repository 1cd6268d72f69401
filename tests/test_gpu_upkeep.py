"""Species upkeep and the device error word, through the C ABI:

* qed_species_energy against numpy's sum of w E (leptons gamma, photons |p|);
  a substep leaves the sum over the three species unchanged (§2.1, §2.2);
* qed_compact_species against a numpy model of the same placement (live
  particles at [n', n) fill the removed slots in [0, n') in order), bit for
  bit, on sizes around the 2048-particle tile, with positions, all removed,
  none removed, FP32 and FP64, eager and replayed from a CUDA graph;
* the bounded waits of the bulk-copy evolution: with a limit of a few cycles
  the handshake waits run out, QED_STAT_WAIT_TIMEOUT counts the CTAs and
  qed_device_status returns QED_ERR_TIMEOUT; the next call with the default
  limit is correct again (the GPU context is intact);
* qed_device_status for non-finite inputs (QED_ERR_NUMERIC) and full
  destinations (QED_ERR_CAPACITY), with no statistics array passed.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPECIES = ("electrons", "positrons", "photons")
COLS = ("px", "py", "pz", "ex", "ey", "ez", "bx", "by", "bz", "tau", "tau_c", "weight", "id")


@pytest.fixture(scope="module")
def api():
    from paper_2110_00256_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def tables(api):
    return api.qed_tables_generate(api.table_params(qs_n_chi=128, qs_n_xi=128, bw_n_chi=128, bw_n_xi=128))


def _bench(n, seed, off=0, tau_scale=1.0):
    from paper_2110_00256_gb300 import workloads
    d = workloads.paper_benchmark(n, seed, off)
    d["tau"] *= tau_scale
    return d


# ---------------------------------------------------------------------------------------
# energy
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec_name", ["f32", "f64"])
def test_species_energy_matches_numpy(api, prec_name):
    prec = api.QED_F32 if prec_name == "f32" else api.QED_F64
    dt = np.float32 if prec_name == "f32" else np.float64
    for n in (0, 1, 1000, 300_001):
        d = _bench(n, 3 + n)
        w = np.random.default_rng(n).uniform(0, 2, n)
        w[::7] = 0.0
        d["weight"] = w
        b = api.SpeciesBuffers(n + 10, prec).set(d)
        h = {k: np.asarray(v, dtype=dt).astype(np.float64) for k, v in d.items() if k != "id"}
        p2 = h["px"] ** 2 + h["py"] ** 2 + h["pz"] ** 2
        for photon in (False, True):
            got = api.qed_species_energy(b, photon).cpu().numpy()
            want = np.sum(h["weight"] * np.sqrt(p2 if photon else 1.0 + p2))
            assert got[0] == pytest.approx(want, rel=1e-12, abs=1e-300)
            assert got[1] == np.count_nonzero(h["weight"])


def test_substep_conserves_total_energy(api, tables):
    bufs = {}
    for j, k in enumerate(SPECIES):
        n = 0 if k == "positrons" else 200_000
        bufs[k] = api.SpeciesBuffers(3 * 200_000, api.QED_F64)
        if n:
            bufs[k].set(_bench(n, 40 + j, j * 10 ** 12, tau_scale=3e-4))
    fire = [api.FireBuffers(bufs[k].capacity) for k in SPECIES]
    st = api.Stats()

    def total():
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        for k in SPECIES:
            api.qed_species_energy(bufs[k], k == "photons", out)
        return float(out[0].item())

    e0 = total()
    for s in range(3):
        api.qed_substep(tables, bufs["electrons"], bufs["positrons"], bufs["photons"], 10.0, 5, s, fire, stats=st)
    e1 = total()
    assert st.as_dict()["qs_events"] > 1000 and st.as_dict()["pairs"] > 100
    assert abs(e1 / e0 - 1.0) < 1e-13


# ---------------------------------------------------------------------------------------
# compaction
# ---------------------------------------------------------------------------------------
def _compact_model(h, n):
    """The placement qed_compact_species promises (include/qed.h)."""
    rm = (h["weight"][:n] == 0) & np.isposinf(h["tau"][:n])
    r = int(rm.sum())
    np_ = n - r
    holes = np.nonzero(rm[:np_])[0]
    movers = np.nonzero(~rm[np_:])[0] + np_
    assert len(holes) == len(movers)
    out = {k: v[:n].copy() for k, v in h.items()}
    for k in out:
        out[k][holes] = h[k][movers]
        out[k] = out[k][:np_]
    return out, r


def _with_removed(n, seed, frac, prec, positions, where="anywhere"):
    d = _bench(n, seed)
    r = np.random.default_rng(seed)
    if where == "tail":
        rm = np.zeros(n, dtype=bool)
        rm[n - int(frac * n):] = True
    else:
        rm = r.uniform(size=n) < frac
    d["weight"] = np.where(rm, 0.0, d["weight"])
    d["tau"] = np.where(rm, np.inf, d["tau"])
    # a weight-0 particle with a finite optical depth is not removed
    keep0 = (~rm) & (r.uniform(size=n) < 0.01)
    d["weight"][keep0] = 0.0
    if positions:
        d.update(x=r.normal(size=n), y=r.normal(size=n), z=r.normal(size=n))
    return d


@pytest.mark.parametrize("prec_name", ["f32", "f64"])
def test_compaction_matches_model(api, prec_name):
    prec = api.QED_F32 if prec_name == "f32" else api.QED_F64
    cases = [(0, 0.3, "anywhere", False), (1, 1.0, "anywhere", False), (2047, 0.3, "anywhere", True),
             (2048, 0.5, "anywhere", False), (2049, 0.02, "anywhere", True), (100_003, 0.2, "anywhere", True),
             (100_003, 0.0, "anywhere", False), (50_000, 1.0, "anywhere", False), (70_001, 0.3, "tail", True),
             (333_333, 0.01, "anywhere", True)]
    for n, frac, where, pos in cases:
        d = _with_removed(n, 11 + n, frac, prec, pos, where)
        b = api.SpeciesBuffers(n + 4097, prec, positions=pos)
        if n:
            b.set(d)
        h = b.to_host()
        want, r = _compact_model(h, n)
        st = api.Stats()
        work = api.CompactWork(b.capacity)
        work.t.fill_(-7)  # the call must not depend on the scratch's contents
        api.qed_compact_species(b, work, st)
        got = b.to_host()
        assert b.n() == n - r, (n, frac)
        assert st.as_dict()["compacted"] == r
        for k in want:
            assert np.array_equal(got[k], want[k]), (n, frac, where, k)


def test_compaction_in_a_graph_and_scratch_size(api):
    n = 40_000
    d = _with_removed(n, 5, 0.25, api.QED_F32, True)
    a = api.SpeciesBuffers(n + 100, api.QED_F32, positions=True).set(d)
    b = api.SpeciesBuffers(n + 100, api.QED_F32, positions=True).set(d)
    wa, wb = api.CompactWork(a.capacity), api.CompactWork(b.capacity)
    api.qed_compact_species(a, wa)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            api.qed_compact_species(b, wb, stream=stream)
    g.replay()
    torch.cuda.synchronize()
    ha, hb = a.to_host(), b.to_host()
    assert a.n() == b.n() < n
    for k in ha:
        assert np.array_equal(ha[k], hb[k]), k
    # a second replay finds nothing to remove
    g.replay()
    torch.cuda.synchronize()
    assert b.n() == a.n()
    # scratch one entry short of QED_COMPACT_WORK(capacity): refused before anything runs
    work = api.CompactWork(a.capacity)
    work.t = work.t[:-1]
    with pytest.raises(api.QedError):
        api.qed_compact_species(a, work)


# ---------------------------------------------------------------------------------------
# bounded waits and the device error word
# ---------------------------------------------------------------------------------------
def _three(api, n, prec, seed):
    bufs = {}
    for j, k in enumerate(SPECIES):
        m = n if k != "positrons" else n // 4
        bufs[k] = api.SpeciesBuffers(3 * n + 64, prec).set(_bench(m, seed + j, j * 10 ** 12, tau_scale=3e-4))
    return bufs, [api.FireBuffers(bufs[k].capacity) for k in SPECIES]


def _same(a, b):
    for k in SPECIES:
        ha, hb = a[k].to_host(), b[k].to_host()
        oa, ob = np.argsort(ha["id"], kind="stable"), np.argsort(hb["id"], kind="stable")
        for c in ha:
            if not np.array_equal(ha[c][oa], hb[c][ob]):
                return False
    return True


def test_wait_limit_runs_out_and_is_reported(api, tables):
    from paper_2110_00256_gb300 import _lib
    api.qed_device_status(clear=True)
    n = 200_000  # ~100 tiles of the bulk-copy evolution
    ref, fr = _three(api, n, api.QED_F32, 70)
    short, fs = _three(api, n, api.QED_F32, 70)
    again, fa = _three(api, n, api.QED_F32, 70)
    s_ref, s_short = api.Stats(), api.Stats()
    api.qed_substep(tables, ref["electrons"], ref["positrons"], ref["photons"], 10.0, 3, 0, fr, stats=s_ref)
    assert api.qed_device_status() == (_lib.QED_OK, 0)
    # a limit of 8 cycles: the consumers' first wait for a tile's copies runs out
    call = api.SubstepCall(tables, short["electrons"], short["positrons"], short["photons"], fs, 10.0, 3,
                           stats=s_short)
    call.opts.wait_limit_cycles = 8
    call(0)
    status, word = api.qed_device_status()
    assert s_short.as_dict()["wait_timeout"] > 0
    assert status == 5 and word & _lib.QED_EW_WAIT_TIMEOUT  # QED_ERR_TIMEOUT
    assert not _same(ref, short)  # the CTAs that gave up evolved nothing
    # cleared: the same call with the default limit is correct again
    assert api.qed_device_status() == (_lib.QED_OK, 0)
    api.qed_substep(tables, again["electrons"], again["positrons"], again["photons"], 10.0, 3, 0, fa,
                    stats=api.Stats())
    assert api.qed_device_status() == (_lib.QED_OK, 0)
    assert _same(ref, again)

    # the batched evolution's waits
    pb, fb = _three(api, 60_000, api.QED_F32, 90)
    pc, fc = _three(api, 60_000, api.QED_F32, 90)
    b_short = api.Batch([dict(pb, fire=fb)], api.QED_F32)
    b_ok = api.Batch([dict(pc, fire=fc)], api.QED_F32)
    sb = api.Stats()
    api.qed_substep_batched(tables, b_short, 10.0, 3, 0, api.make_opts(stats=sb, wait_limit_cycles=8))
    status, word = api.qed_device_status()
    assert status == 5 and word & _lib.QED_EW_WAIT_TIMEOUT and sb.as_dict()["wait_timeout"] > 0
    api.qed_substep_batched(tables, b_ok, 10.0, 3, 0, api.make_opts(stats=api.Stats()))
    assert api.qed_device_status() == (_lib.QED_OK, 0)


def test_device_status_numeric_and_capacity(api, tables):
    from paper_2110_00256_gb300 import _lib
    api.qed_device_status(clear=True)
    bufs, fire = _three(api, 5000, api.QED_F64, 50)
    px = bufs["electrons"]["px"]
    px[17] = float("nan")
    api.qed_substep(tables, bufs["electrons"], bufs["positrons"], bufs["photons"], 10.0, 3, 0, fire)
    status, word = api.qed_device_status()
    assert status == 4 and word == _lib.QED_EW_NONFINITE  # QED_ERR_NUMERIC
    # photons with no room: emission events are left for the next step
    e = api.SpeciesBuffers(6000, api.QED_F64).set(_bench(5000, 51, 0, tau_scale=3e-4))
    p = api.SpeciesBuffers(10, api.QED_F64)
    g = api.SpeciesBuffers(5, api.QED_F64)
    fire = [api.FireBuffers(x.capacity) for x in (e, p, g)]
    api.qed_substep(tables, e, p, g, 10.0, 3, 0, fire)
    status, word = api.qed_device_status(clear=False)
    assert status == 3 and word & _lib.QED_EW_CAPACITY  # QED_ERR_CAPACITY
    assert api.qed_device_status()[1] == word  # read again, then cleared
    assert api.qed_device_status() == (_lib.QED_OK, 0)
