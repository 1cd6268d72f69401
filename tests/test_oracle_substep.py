"""Pins of the oracle's substep: Philox against an independent implementation,
table lookups against their definition at grid points and outside the range,
inverse-CDF sampling against the exact distribution (KS) and against the
paper's printed table-resolution claims, the optical-depth method against the
direct per-step decay probability (§2.1), and energy conservation of the
products (§2.1, §2.2)."""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table_resolution.json")


# ---------------------------------------------------------------------------------------
# Philox4x32-10
# ---------------------------------------------------------------------------------------
_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl

@triton.jit
def k(seed, c0p, c1p, c2p, c3p, o0, o1, o2, o3, N: tl.constexpr):
    i = tl.arange(0, N)
    a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i), tl.load(c3p + i))
    tl.store(o0 + i, a); tl.store(o1 + i, b); tl.store(o2 + i, c); tl.store(o3 + i, d)

cfg = json.loads(sys.argv[1])
cs = [torch.tensor(c, dtype=torch.uint32) for c in cfg["ctr"]]
outs = [torch.zeros(len(cfg["ctr"][0]), dtype=torch.uint32) for _ in range(4)]
k[(1,)](cfg["seed"], *cs, *outs, N=len(cfg["ctr"][0]))
print(json.dumps([o.tolist() for o in outs]))
"""


def test_philox_matches_triton_reference():
    """Triton's Philox4x32-10 (its own Python source, run by its CPU interpreter)
    is an implementation independent of the oracle's C code."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(3)
    n = 8
    ctr = [[int(v) for v in rng.integers(0, 2 ** 32, n, dtype=np.uint64)] for _ in range(4)]
    ctr[0][0] = ctr[1][0] = ctr[2][0] = ctr[3][0] = 0
    ctr[0][1] = ctr[1][1] = ctr[2][1] = ctr[3][1] = 0xFFFFFFFF
    seed = 0x1234567890ABCDEF
    res = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT, json.dumps({"seed": seed, "ctr": ctr})],
                         capture_output=True, text=True, timeout=600)
    if res.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + res.stderr[-300:])
    ref = json.loads(res.stdout.strip().splitlines()[-1])
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in range(n):
        got = oracle.philox([ctr[i][j] for i in range(4)], key)
        assert [int(v) for v in got] == [ref[i][j] for i in range(4)]


def test_uniform_and_tau_distribution():
    stats = pytest.importorskip("scipy.stats")
    ids = np.arange(20000, dtype=np.uint64) * 7919 + 11
    u = np.array([oracle.uniform(5, int(i), 3, 0, 0) for i in ids])
    u2 = np.array([oracle.uniform(5, int(i), 3, 0, 1) for i in ids])
    assert np.all(u > 0) and np.all(u < 1)
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    assert stats.kstest(u2, "uniform").pvalue > 1e-4
    assert abs(np.corrcoef(u, u2)[0, 1]) < 0.05
    tau = oracle.init_tau(ids, 5, 0)
    assert stats.kstest(tau, "expon").pvalue > 1e-4
    # purposes give different streams
    assert oracle.uniform(5, 1, 3, 0) != oracle.uniform(5, 1, 3, 1)


# ---------------------------------------------------------------------------------------
# lookups
# ---------------------------------------------------------------------------------------
def test_lookup_at_grid_points_and_outside(oracle_tables_small):
    t = oracle_tables_small
    p = t.params
    l0, l1, N = math.log(p["qs_chi_min"]), math.log(p["qs_chi_max"]), p["qs_n_chi"]
    for n in (1, 10, 33, 62):
        chi = math.exp(l0 + n * (l1 - l0) / (N - 1))
        assert t.qs_G(chi) == pytest.approx(math.exp(t.qs_lnG[n]), rel=1e-13)
    # QS: clamp outside the range, zero at chi == 0
    assert t.qs_G(1e-7) == pytest.approx(math.exp(t.qs_lnG[0]), rel=1e-15)
    assert t.qs_G(1e6) == pytest.approx(math.exp(t.qs_lnG[-1]), rel=1e-15)
    assert t.qs_G(0.0) == 0.0
    # BW: asymptotes outside
    assert t.bw_T(1e-3) == pytest.approx(oracle.bw_T_small(1e-3), rel=1e-15)
    assert t.bw_T(1e5) == pytest.approx(oracle.bw_T_large(1e5), rel=1e-15)
    # log-log interpolation: exact for a power law between two nodes
    n = 20
    a = math.exp(l0 + n * (l1 - l0) / (N - 1))
    b = math.exp(l0 + (n + 1) * (l1 - l0) / (N - 1))
    mid = math.sqrt(a * b)
    assert t.qs_G(mid) == pytest.approx(math.sqrt(math.exp(t.qs_lnG[n] + t.qs_lnG[n + 1])), rel=1e-13)


def test_table_asymptote_jumps_are_small(oracle_tables_256):
    # the out-of-table BW asymptotes join the table within a few percent at both ends
    t = oracle_tables_256
    lo, hi = t.params["bw_chi_min"], t.params["bw_chi_max"]
    assert t.bw_T(lo * (1 - 1e-12)) / t.bw_T(lo) == pytest.approx(1.0, abs=0.01)
    assert t.bw_T(hi * (1 + 1e-12)) / t.bw_T(hi) == pytest.approx(1.0, abs=0.03)


# ---------------------------------------------------------------------------------------
# inverse-CDF sampling
# ---------------------------------------------------------------------------------------
def _ks_against(cdf_sorted, samples):
    x = np.sort(samples)
    n = x.size
    F = cdf_sorted(x)
    return max(np.max(np.arange(1, n + 1) / n - F), np.max(F - np.arange(0, n) / n))


@pytest.mark.parametrize("chi", (0.05, 2.0, 80.0))
def test_qs_sampling_ks(oracle_tables_256, chi):
    t = oracle_tables_256
    n = 3000
    r = (np.arange(n) + 0.5) / n  # stratified: KS then measures table error only
    xi = np.array([t.qs_sample_xi(chi, v) for v in r])
    assert np.all((xi > 0) & (xi <= 1))
    # stratified r: the KS distance is the table's own error (plus 1/2n); at 256
    # points it peaks (~2e-3 at chi = 80) in the xi -> 1 tail, where the
    # log-spaced xi grid is coarsest in xi
    d = _ks_against(lambda v: oracle.qs_cdf_sorted(chi, v), xi)
    assert d < 4e-3


@pytest.mark.parametrize("chig", (0.5, 5.0, 200.0))
def test_bw_sampling_ks(oracle_tables_256, chig):
    t = oracle_tables_256
    n = 2000
    r = (np.arange(n) + 0.5) / n
    out = [t.bw_sample_xi(chig, v) for v in r]
    xi_minus = np.array([x if e else 1 - x for x, e in out])
    is_el = np.array([e for _, e in out])
    assert is_el.sum() == n // 2
    d = _ks_against(lambda v: oracle.bw_cdf_sorted(chig, v), xi_minus)
    assert d < 2e-3


def _load_claims():
    with open(GOLDEN) as f:
        return {c["id"]: c for c in json.load(f)["claims"]}


def test_paper_claim_1d_resolution():
    claims = _load_claims()
    c = claims["qs_G_32"]
    t = oracle.tables(qs_n_chi=c["n"], qs_n_xi=c["n"], bw_n_chi=c["n"], bw_n_xi=c["n"])
    chis = np.geomspace(*c["chi_range"], 41)[1:-1] * 1.013
    err = max(abs(t.qs_G(x) / oracle.qs_G(x) - 1) for x in chis)
    assert err < c["max_rel_err"]
    c = claims["bw_T_128"]
    t = oracle.tables(qs_n_chi=c["n"], qs_n_xi=c["n"], bw_n_chi=c["n"], bw_n_xi=c["n"])
    chis = np.geomspace(*c["chi_range"], 41)[1:-1] * 1.013
    err = max(abs(t.bw_T(x) / oracle.bw_T(x) - 1) for x in chis)
    assert err < c["max_rel_err"]


def _density_error(t, proc, chi, r):
    if proc == "qs":
        xi = np.array([t.qs_sample_xi(chi, v) for v in r])
        G = oracle.qs_G(chi)
        pdf = np.array([oracle.qs_S(chi, x) / x / G for x in xi])
    else:
        xi = np.array([t.bw_sample_xi(chi, v)[0] for v in r])
        norm = oracle.bw_T(chi) * math.pi * math.sqrt(3.0) * chi
        pdf = np.array([oracle.bw_bracket(chi, x) / norm for x in xi])
    drdxi = np.gradient(r, xi)
    return np.abs(drdxi / pdf - 1.0)[1:-1]


@pytest.mark.parametrize("cid,proc", (("bw_P_128", "bw"), ("qs_P_128", "qs")))
def test_paper_claim_2d_resolution(cid, proc):
    c = _load_claims()[cid]
    t = oracle.tables(qs_n_chi=c["n"], qs_n_xi=c["n"], bw_n_chi=c["n"], bw_n_xi=c["n"])
    r = np.linspace(*c["r_range"], 300)
    for chi in c["chi"]:
        e = _density_error(t, proc, chi, r)
        val = e.max() if c["metric"] == "max" else np.percentile(e, 95)
        assert val < c["max_rel_err"], (chi, val)


# ---------------------------------------------------------------------------------------
# optical-depth method == direct per-step decay probability (§2.1)
# ---------------------------------------------------------------------------------------
def test_optical_depth_equals_direct_method(oracle_tables_small):
    t = oracle_tables_small
    n, steps, dt = 40000, 12, 3000.0
    ids = np.arange(n, dtype=np.uint64) + 1000
    st = dict(px=np.full(n, 500.0), py=np.zeros(n), pz=np.zeros(n), ex=np.zeros(n), ey=np.zeros(n),
              ez=np.zeros(n), bx=np.zeros(n), by=np.zeros(n), bz=np.full(n, 2e-3),
              tau=oracle.init_tau(ids, 9, 0))
    _, chi, rate, _ = oracle.evolve(oracle.QS, t, st, dt)
    p = 1.0 - math.exp(-rate[0] * dt)
    assert 0.01 < p < 0.2
    counts = []
    for s in range(steps):
        tau, _, _, fire = oracle.evolve(oracle.QS, t, st, dt)
        for i in np.nonzero(fire)[0]:
            tau[i] = oracle.tau_draw(9, int(ids[i]), s, oracle.PURPOSE_TAU_RESET)
        st["tau"] = tau
        counts.append(int(fire.sum()))
    counts = np.array(counts)
    # each step is Binomial(n, p) by memorylessness
    z = (counts - n * p) / math.sqrt(n * p * (1 - p))
    assert np.all(np.abs(z) < 4.5)
    assert abs(z.sum() / math.sqrt(steps)) < 4.0


# ---------------------------------------------------------------------------------------
# products: energy conservation and collinearity
# ---------------------------------------------------------------------------------------
def test_qs_products_conserve_energy(oracle_tables_small):
    t = oracle_tables_small
    rng = np.random.default_rng(1)
    m = 500
    p = rng.normal(size=(m, 3)) * 300
    chi = 10 ** rng.uniform(-3, 3, m)
    ids = rng.integers(0, 2 ** 62, m, dtype=np.uint64)
    ev = oracle.qs_events(t, p, chi, ids, 4, 17)
    gam = np.sqrt(1 + (p ** 2).sum(1))
    gl = np.sqrt(1 + ev["lep_px"] ** 2 + ev["lep_py"] ** 2 + ev["lep_pz"] ** 2)
    gph = np.sqrt(ev["ph_px"] ** 2 + ev["ph_py"] ** 2 + ev["ph_pz"] ** 2)
    assert np.allclose(gl + gph, gam, rtol=1e-12, atol=0)
    assert np.all(gph <= gam - 1 + 1e-9 * gam)
    assert np.all((ev["xi"] > 0) & (ev["xi"] <= 1))
    cross = np.cross(p, np.stack([ev["ph_px"], ev["ph_py"], ev["ph_pz"]], 1))
    assert np.all(np.linalg.norm(cross, axis=1) <= 1e-12 * np.linalg.norm(p, axis=1) * (gph + 1))
    assert np.all(ev["lep_tau"] > 0) and np.all(ev["ph_tau"] > 0)
    # threshold (§5): photons below it are not kept
    ev2 = oracle.qs_events(t, p, chi, ids, 4, 17, threshold=2.0)
    assert np.array_equal(ev2["keep"], gph >= 2.0)


def test_bw_products_conserve_energy(oracle_tables_small):
    t = oracle_tables_small
    rng = np.random.default_rng(2)
    m = 500
    p = rng.normal(size=(m, 3)) * 300
    p[0] = (1.5, 0, 0)  # below the pair threshold gamma_g <= 2
    chi = 10 ** rng.uniform(-1.5, 3, m)
    ids = rng.integers(0, 2 ** 62, m, dtype=np.uint64)
    ev = oracle.bw_events(t, p, chi, ids, 4, 17)
    gg = np.linalg.norm(p, axis=1)
    ge = np.sqrt(1 + ev["el_px"] ** 2 + ev["el_py"] ** 2 + ev["el_pz"] ** 2)
    gp = np.sqrt(1 + ev["po_px"] ** 2 + ev["po_py"] ** 2 + ev["po_pz"] ** 2)
    made = ev["made"]
    assert not made[0] and made[1:].all()
    assert np.allclose((ge + gp)[made], gg[made], rtol=1e-12, atol=0)
    assert np.all(ev["xi_minus"] >= 0) and np.all(ev["xi_minus"] <= 1)
    assert np.all(ev["el_id"] != ev["po_id"])


def test_substep_conserves_energy_and_bookkeeping(oracle_tables_small):
    t = oracle_tables_small
    rng = np.random.default_rng(4)
    n = 3000

    def species(kind, seed_off):
        r = np.random.default_rng(seed_off)
        d = {k: r.uniform(-1, 1, n) * s for k, s in (("px", 2000), ("py", 2000), ("pz", 2000),
                                                       ("ex", 0.01), ("ey", 0.01), ("ez", 0.01),
                                                       ("bx", 0.01), ("by", 0.01), ("bz", 0.01))}
        d["id"] = np.arange(n, dtype=np.uint64) + seed_off * 10 ** 9
        d["tau"] = r.exponential(size=n) * 1e-3  # near threshold: many events
        d["weight"] = np.ones(n)
        return d

    sp = {"electrons": species("e", 1), "positrons": species("p", 2), "photons": species("g", 3)}

    def energy(s):
        e = 0.0
        for name in ("electrons", "positrons"):
            d = s[name]
            e += np.sum(d["weight"] * np.sqrt(1 + d["px"] ** 2 + d["py"] ** 2 + d["pz"] ** 2))
        d = s["photons"]
        e += np.sum(d["weight"] * np.sqrt(d["px"] ** 2 + d["py"] ** 2 + d["pz"] ** 2))
        return e

    out = oracle.substep(t, sp, dt=10.0, seed=1, step=0)
    fired = {k: int(v.sum()) for k, v in out["fire"].items()}
    assert all(v > 10 for v in fired.values())
    assert energy(out) == pytest.approx(energy(sp), rel=1e-12)
    assert out["n_new"]["photons"] == fired["electrons"] + fired["positrons"]
    assert out["n_new"]["electrons"] == out["n_new"]["positrons"] == fired["photons"]
    assert len(out["electrons"]["px"]) == n + fired["photons"]
    # fired photons are removed (weight 0, tau = +inf); others keep their weight
    ph = out["photons"]
    assert np.all(ph["weight"][:n][out["fire"]["photons"]] == 0)
    assert np.all(np.isinf(ph["tau"][:n][out["fire"]["photons"]]))
    # every optical depth left is positive
    for name in ("electrons", "positrons", "photons"):
        assert np.all(out[name]["tau"] > 0)


def test_chi_cut_special_cases(oracle_tables_small):
    """A chi cut-off of 0 changes nothing; one above every particle's chi
    freezes every optical depth; in between, exactly the particles below it
    are frozen and the rest evolve as without a cut."""
    from paper_2110_00256_gb300 import workloads
    ot = oracle_tables_small
    h = {k: np.asarray(v, dtype=np.float64) if k != "id" else v
         for k, v in workloads.paper_benchmark(5000, 3, 0).items()}
    h["tau"] = h["tau"] * 1e-3
    t0, chi0, r0, f0 = oracle.evolve(0, ot, h, 10.0)
    t1, chi1, r1, f1 = oracle.evolve(0, ot, h, 10.0, 0.0)
    assert np.array_equal(t0, t1) and np.array_equal(f0, f1) and f0.any()
    t2, _, r2, f2 = oracle.evolve(0, ot, h, 10.0, 10 * chi0.max())
    assert np.array_equal(t2, h["tau"]) and not f2.any() and not r2.any()
    cut = np.median(chi0)
    t3, _, r3, f3 = oracle.evolve(0, ot, h, 10.0, cut)
    lo = chi0 < cut
    assert np.array_equal(t3[lo], h["tau"][lo]) and not f3[lo].any()
    assert np.array_equal(t3[~lo], t0[~lo]) and np.array_equal(f3[~lo], f0[~lo]) and np.array_equal(r3[~lo], r0[~lo])
