"""Schwinger pair production on the GPU (qed_schwinger_pairs) against the
oracle: the same number of pairs in every cell (inversion and normal-
approximation branches), the same ids and optical depths, pairs at rest with
their cell's fields and position; capacity limits drop whole pairs only."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2110_00256_gb300 import api as a
    return a


def _cells(n, seed, dtype):
    r = np.random.default_rng(seed)
    f = {k: r.normal(0, 0.12, n).astype(dtype) for k in ("ex", "ey", "ez", "bx", "by", "bz")}
    pos = {k: r.uniform(-5, 5, n).astype(dtype) for k in ("x", "y", "z")}
    return f, pos


def _run(api, prec, f, pos, dv, dt, weight, seed, step, cap):
    td = torch.float32 if prec == api.QED_F32 else torch.float64
    df = {k: torch.as_tensor(v, device="cuda", dtype=td) for k, v in f.items()}
    dp = {k: torch.as_tensor(v, device="cuda", dtype=td) for k, v in pos.items()}
    e = api.SpeciesBuffers(cap, prec, positions=True)
    p = api.SpeciesBuffers(cap, prec, positions=True)
    stats = api.Stats()
    api.qed_schwinger_pairs(df, dv, dt, weight, seed, step, e, p, stats=stats, positions=dp)
    torch.cuda.synchronize()
    return e.to_host(), p.to_host(), stats.as_dict()


@pytest.mark.parametrize("prec_name", ["f32", "f64"])
@pytest.mark.parametrize("dv", [1e5, 3e7])  # means below 20 only; up to ~5e3 (normal branch) in the strongest cells
def test_schwinger_matches_oracle(api, prec_name, dv):
    prec = api.QED_F32 if prec_name == "f32" else api.QED_F64
    dtype = np.float32 if prec_name == "f32" else np.float64
    f, pos = _cells(20_003, 7, dtype)
    ref = oracle.schwinger({k: v.astype(np.float64) for k, v in f.items()}, dv, 10.0, 1.0, 21, 5)
    total = int(ref["count"].sum())
    assert total > 300
    if dv > 1e6:
        assert ref["lambda"].max() > 100
    e, p, st = _run(api, prec, f, pos, dv, 10.0, 1.0, 21, 5, total + 1000)
    assert st["schwinger_pairs"] == total and st["dropped_capacity"] == 0
    for h, ids, taus in ((e, ref["e_id"], ref["e_tau"]), (p, ref["p_id"], ref["p_tau"])):
        o = np.argsort(h["id"])
        r = np.argsort(ids)
        assert np.array_equal(h["id"][o], ids[r])
        cell = ref["cell"][r]
        tau = h["tau"][o].astype(np.float64) - h["tau_c"][o]
        assert np.allclose(tau, taus[r], rtol=1e-12 if prec_name == "f64" else 1e-9, atol=0)
        for c in ("px", "py", "pz"):
            assert not h[c].any()
        for c in ("ex", "ey", "ez", "bx", "by", "bz"):
            assert np.array_equal(h[c][o], f[c][cell])
        for c in ("x", "y", "z"):
            assert np.array_equal(h[c][o], pos[c][cell])
        assert np.all(h["weight"] == 1.0)


def test_schwinger_capacity_drops_whole_pairs(api):
    f, pos = _cells(20_003, 8, np.float32)
    ref = oracle.schwinger({k: v.astype(np.float64) for k, v in f.items()}, 3e7, 10.0, 1.0, 3, 0)
    total = int(ref["count"].sum())
    cap = total // 3
    e, p, st = _run(api, api.QED_F32, f, pos, 3e7, 10.0, 1.0, 3, 0, cap)
    assert len(e["id"]) == cap and len(p["id"]) == cap
    assert st["schwinger_pairs"] + st["dropped_capacity"] == total
    live_e = set(e["id"][e["weight"] > 0].tolist())
    live_p = set(p["id"][p["weight"] > 0].tolist())
    assert len(live_e) == st["schwinger_pairs"] == len(live_p)
    pairs = dict(zip(ref["e_id"].tolist(), ref["p_id"].tolist()))
    assert {pairs[i] for i in live_e} == live_p  # no half pairs


@pytest.mark.parametrize("prec_name", ["f64", "f32"])
def test_schwinger_weak_and_strong_field_mix(api, prec_name):
    """cells around the FP64 underflow of exp(-pi/eps) (eps = 0.0042) and
    magnetic-dominated cells: the GPU skips only cells whose rate is exactly
    zero (FP32: through both FP32 bounds of the streamed kernel), and counts
    equal the oracle's"""
    r = np.random.default_rng(9)
    n = 30_000
    dtype = np.float64 if prec_name == "f64" else np.float32
    scale = np.exp(r.uniform(np.log(1e-3), np.log(0.5), n))
    f = {k: (r.normal(0, 1, n) * scale).astype(dtype) for k in ("ex", "ey", "ez")}
    f.update({k: (r.normal(0, 1, n) * scale * r.uniform(0, 30, n)).astype(dtype) for k in ("bx", "by", "bz")})
    pos = {k: np.zeros(n, dtype=dtype) for k in ("x", "y", "z")}
    ref = oracle.schwinger({k: v.astype(np.float64) for k, v in f.items()}, 500.0, 10.0, 1.0, 5, 1)
    total = int(ref["count"].sum())
    assert total > 50
    prec = api.QED_F64 if prec_name == "f64" else api.QED_F32
    e, p, st = _run(api, prec, f, pos, 500.0, 10.0, 1.0, 5, 1, total + 100)
    assert st["schwinger_pairs"] == total
    assert np.array_equal(np.sort(e["id"]), np.sort(ref["e_id"]))


def test_full_size_schwinger_sampled(api):
    """1e8 FP32 cells (the benchmark's size; fields N(0, 0.12) E_s, so that a
    few percent of the cells make pairs) through the streamed kernel; for 3000
    sampled cells the oracle's count and pair ids from the cell's own fields
    and index.  Cells carry their index in (x, y), which the pairs inherit."""
    from paper_2110_00256_gb300 import workloads
    n = 100_000_000
    g = torch.Generator(device="cuda")
    g.manual_seed(23)
    f = {k: torch.randn(n, generator=g, device="cuda", dtype=torch.float32) * 0.12
         for k in ("ex", "ey", "ez", "bx", "by", "bz")}
    cell = torch.arange(n, device="cuda")
    pos = {"x": torch.div(cell, 16384, rounding_mode="floor").float(), "y": (cell % 16384).float(),
           "z": torch.zeros(n, device="cuda")}
    del cell
    e = api.SpeciesBuffers(3_000_000, api.QED_F32, positions=True)
    p = api.SpeciesBuffers(3_000_000, api.QED_F32, positions=True)
    stats = api.Stats()
    dv, dt, w, seed, step = 5e4, 10.0, 1.0, 21, 5  # ~1e6 pairs in all
    api.qed_schwinger_pairs(f, dv, dt, w, seed, step, e, p, stats=stats, positions=pos)
    torch.cuda.synchronize()
    st = stats.as_dict()
    assert st["dropped_capacity"] == 0 and st["schwinger_pairs"] > 100_000
    idx = workloads.subsample_ids(n, 3000, 9)
    ti = torch.as_tensor(idx, device="cuda")
    fh = {k: v[ti].cpu().numpy().astype(np.float64) for k, v in f.items()}
    del f, pos
    eh = e.to_host()
    gpu_cell = eh["x"].astype(np.int64) * 16384 + eh["y"].astype(np.int64)
    sel = np.isin(gpu_cell, idx)
    got = dict(zip(*np.unique(gpu_cell[sel], return_counts=True)))
    want_ids, made = set(), 0
    for j, c in enumerate(idx.tolist()):
        lam = oracle.schwinger_rate([fh[k][j] for k in ("ex", "ey", "ez")], [fh[k][j] for k in ("bx", "by", "bz")]) \
            * dv * dt / w
        k = oracle.poisson(lam, seed, c, step)
        assert got.get(c, 0) == k, (c, lam, k, got.get(c, 0))
        made += k
        want_ids.update(oracle.schwinger_pair_ids(seed, c, step, i)[0] for i in range(k))
    assert made > 10
    assert set(eh["id"][sel].tolist()) == want_ids
