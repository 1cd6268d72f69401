"""What the learned sampler gains over the 2-D tables it replaces (§3.1, §3.2),
judged against the oracle's exact distributions (oracle.qs_cdf / bw_cdf: FP64
quadrature of the spectra, no table):

* the exact inverse CDF on the GPU (qed_exact_sample, the training targets)
  against the oracle's CDF: P(chi, xi) = U to 1e-9;
* the networks, trained on 10^7 exact samples by the library's own kernels,
  against the oracle's CDF in 5 chi bins of each table range, beside the
  256 x 256 FP32 tables on the same draws: the KS distance of every bin
  stays below a stated bound (0.005), the largest sup |P - U| of a single chi
  below 0.003, and in the two highest-chi bins
  the QS network's is under half the table's (the table's last log-spaced
  xi interval, below);
* the hard-photon tail at chi = 9, where the 256-point log-spaced xi grid puts
  its last interval at [0.897, 1] and the table's log-log interpolation spreads
  the hardest emissions across it: P(xi > 0.99) is 1.1e-6 exactly, ~1.4e-3
  from the table; the network must be within 1e-4 of the exact value, closer
  than the table at xi > 0.95 as well, and its parameters must take under 1/25
  of the table's memory.

The KS distance of a sampler at fixed chi is sup_U |P(chi, xi(chi, U)) - U|
(the sampler is monotone in U), evaluated on 500 stratified U; a bin pools four
chi values spread over it (the mixture's KS against the pooled U).  The oracle's
CDFs run in a pool of processes started with spawn.
"""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BINS = 5
CHI_PER_BIN = 4
NU = 500
# (measured with the present training, which gives the same bits run after run: pooled
# 0.002 / 0.002, worst chi 0.001 / 0.0008)
KS_BOUND = {0: 0.005, 1: 0.005}
WORST_CHI_BOUND = {0: 0.003, 1: 0.003}


@pytest.fixture(scope="module")
def api():
    from paper_2110_00256_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def tables(api):
    return api.qed_tables_generate(api.table_params())


@pytest.fixture(scope="module")
def trained(api, tables):
    from paper_2110_00256_gb300 import surrogate
    m = api.Mlp(tables, seed=3)
    reps = {p: surrogate.train(m, tables, p, n_samples=10_000_000) for p in (0, 1)}
    return m, reps


def _cdf(proc, chi, xs):
    o = np.argsort(xs)
    f = (oracle.qs_cdf_sorted if proc == 0 else oracle.bw_cdf_sorted)(chi, xs[o])
    out = np.empty_like(f)
    out[o] = f
    return out


def _cdf_job(args):
    return _cdf(*args)


@pytest.fixture(scope="module")
def pool():
    import multiprocessing as mp
    import os
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as p:
        yield p


@pytest.mark.parametrize("proc,chis", [(0, (1e-3, 0.05, 2.0, 80.0, 900.0)), (1, (0.02, 0.5, 5.0, 200.0, 1e3))])
def test_exact_sampler_matches_oracle_cdf(api, pool, proc, chis):
    u = (torch.arange(NU, dtype=torch.float64, device="cuda") + 0.5) / NU
    u = torch.cat([u, torch.tensor([1e-12, 1e-6, 1 - 1e-6], dtype=torch.float64, device="cuda")])
    k = u.numel()
    xi = api.qed_exact_sample(proc, torch.tensor(chis, dtype=torch.float64, device="cuda"), u.repeat(len(chis)))
    xi = xi.cpu().numpy().reshape(len(chis), k)
    uu = u.cpu().numpy()
    fs = pool.map(_cdf_job, [(proc, c, xi[i]) for i, c in enumerate(chis)])
    for i, c in enumerate(chis):
        assert np.all(np.diff(xi[i][:NU]) >= 0)  # monotone in U
        err = np.abs(fs[i] - uu)
        assert err.max() < 1e-9, (c, err.max(), uu[np.argmax(err)])


def _bin_chis(tables, proc):
    ax = tables.params.qs if proc == 0 else tables.params.bw
    lo, hi = math.log(ax.chi_min), math.log(ax.chi_max)
    out = []
    for b in range(BINS):
        t = (b + (np.arange(CHI_PER_BIN) + 0.5) / CHI_PER_BIN) / BINS
        out.append(np.exp(lo + (hi - lo) * t))
    return out


def _ks_bins(proc, chis_per_bin, sample, pool):
    """Per bin: the mixture KS of the pooled P(chi, xi) against the pooled U,
    and the worst per-chi sup |P - U|."""
    u = (np.arange(NU) + 0.5) / NU
    jobs = [(proc, c, sample(np.full(NU, c), u)) for chis in chis_per_bin for c in chis]
    vs = iter(pool.map(_cdf_job, jobs))
    res = []
    for chis in chis_per_bin:
        v_all, u_all, worst = [], [], 0.0
        for c in chis:
            v = next(vs)
            worst = max(worst, float(np.max(np.abs(v - u))))
            v_all.append(v)
            u_all.append(u)
        v_all, u_all = np.sort(np.concatenate(v_all)), np.sort(np.concatenate(u_all))
        grid = np.concatenate([v_all, u_all])
        ks = np.max(np.abs(np.searchsorted(v_all, grid, side="right") - np.searchsorted(u_all, grid, side="right")))
        res.append((ks / len(v_all), worst))
    return res


@pytest.mark.parametrize("proc", [0, 1])
def test_network_ks_per_chi_bin(api, tables, trained, pool, proc):
    m, reps = trained

    def net(chi, u):
        return m.sample(proc, torch.tensor(chi, device="cuda"), torch.tensor(u, device="cuda")).cpu().numpy()

    def tab(chi, u):
        return api.qed_table_sample(tables, proc, api.QED_F32, torch.tensor(chi, device="cuda"),
                                    torch.tensor(u, device="cuda")).cpu().numpy()

    chis = _bin_chis(tables, proc)
    rn, rt = _ks_bins(proc, chis, net, pool), _ks_bins(proc, chis, tab, pool)
    print(f"proc {proc}: network KS per bin {[round(a, 5) for a, _ in rn]} (worst chi {[round(b, 5) for _, b in rn]})")
    print(f"         256x256 FP32 table   {[round(a, 5) for a, _ in rt]} (worst chi {[round(b, 5) for _, b in rt]})")
    print(f"         training: {reps[proc]['seconds']:.1f} s, final loss {reps[proc]['final_loss']:.3e}")
    assert max(a for a, _ in rn) <= KS_BOUND[proc]
    assert max(b for _, b in rn) <= WORST_CHI_BOUND[proc]
    if proc == 0:  # where the table's hard end is coarse, the network is the better sampler
        assert all(rn[i][1] < 0.5 * rt[i][1] for i in (BINS - 2, BINS - 1))


def test_network_tail_and_memory_against_table(api, tables, trained):
    m, _ = trained
    chi, q = 9.0, 0.99
    exact = 1.0 - oracle.qs_cdf(chi, q)
    assert 3e-7 < exact < 3e-6  # ~1.1e-6
    # the tail P(xi > q) = 1 - U* with U* the smallest U mapped above q (both samplers are monotone in U)
    u = np.concatenate([np.linspace(0.5, 1 - 1e-3, 20000), 1 - np.logspace(-3, -12, 20000)])
    ut = torch.tensor(u, dtype=torch.float64, device="cuda")
    ct = torch.full_like(ut, chi)

    def tail(x):
        above = np.nonzero(x > q)[0]
        return float(1.0 - u[above[0]]) if len(above) else 0.0

    x_net = m.sample(0, ct, ut).cpu().numpy()
    x_tab = api.qed_table_sample(tables, 0, api.QED_F32, ct, ut).cpu().numpy()
    p_net, p_tab = tail(x_net), tail(x_tab)
    print(f"P(xi > {q} | chi = {chi}): exact {exact:.3e}, network {p_net:.3e}, 256x256 table {p_tab:.3e}")
    assert abs(p_tab - exact) > 5e-4  # the table's known excess
    assert abs(p_net - exact) <= 1e-4
    q = 0.95
    exact = 1.0 - oracle.qs_cdf(chi, q)
    p_net, p_tab = tail(x_net), tail(x_tab)
    print(f"P(xi > {q} | chi = {chi}): exact {exact:.3e}, network {p_net:.3e}, 256x256 table {p_tab:.3e}")
    assert abs(p_net - exact) < 0.5 * abs(p_tab - exact)
    # memory: two networks' bf16 parameters against one process's FP32 table with its column differences
    from paper_2110_00256_gb300 import _lib
    net_bytes = 2 * 2 * _lib.QED_MLP_PARAMS
    table_bytes = 2 * 256 * 256 * 4
    assert net_bytes * 25 < table_bytes
